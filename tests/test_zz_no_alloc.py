"""The allocation-free forward projector against the handle-based one.

roi_recon_forward_local_noalloc serves callers that cannot allocate device memory
(their memory belongs to a fixed budget owned by a framework allocator or a server,
or their loop cannot take cudaMalloc's implicit synchronisation); its scratch is a
fixed array inside the library.  This file is collected last so that a run stopping
at the first failure has already run every other test."""
import numpy as np
import pytest

import paper_1604_02292_gb300 as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5  # the relative L2 bar of the FP32 projector tests


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _noalloc(N, na, nd, region, x, stride):
    g = R.Geometry(N, na, nd, None, R.ROI_F32)
    y = torch.full((na, stride), float("nan"), dtype=torch.float32, device="cuda")
    s, msg = R.roi_recon_forward_local_noalloc(g, R.Region(*region), x.data_ptr(), y.data_ptr(),
                                               torch.cuda.current_stream().cuda_stream)
    assert s == R.ROI_OK, msg
    return y


def test_noalloc_forward_matches_handle_twice_in_a_row():
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs CUDA")
    cases = [(128, 64, 128, (63.5, 63.5, 16.0, 8.0), 1),
             (256, 200, 256, (128.0, 100.0, 50.0, 20.0), 2)]
    for N, na, nd, region, seed in cases:
        rr = R.RoiRecon(N, na, nd)
        pl = rr.plan(region)
        x = torch.from_numpy(np.random.default_rng(seed).random((pl.box[3], pl.box[2])).astype(np.float32)).cuda()
        ref = rr.forward_local(region, x).cpu().numpy()
        got = _noalloc(N, na, nd, region, x, pl.window_stride).cpu().numpy()
        assert np.isfinite(got).all()
        assert _rel(got, ref) <= TOL
        rr.close()


def test_noalloc_rejects_oversize_and_custom_angles():
    g = R.Geometry(8192, 64, 4096, None, R.ROI_F32)
    x = torch.zeros(1, device="cuda")
    s, msg = R.roi_recon_forward_local_noalloc(g, R.Region(4096.0, 4096.0, 2000.0, 100.0), x.data_ptr(),
                                               x.data_ptr(), 0)
    assert s == R.ROI_EINVAL and "limit" in msg
    ang = np.zeros(4)
    g2 = R.Geometry(64, 4, 64, ang.ctypes.data_as(R.ctypes.POINTER(R.ctypes.c_double)), R.ROI_F32)
    s, msg = R.roi_recon_forward_local_noalloc(g2, R.Region(32.0, 32.0, 4.0, 1.0), x.data_ptr(), x.data_ptr(), 0)
    assert s == R.ROI_EINVAL
