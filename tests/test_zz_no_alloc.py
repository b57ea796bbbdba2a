"""The allocation-free forward projector against the handle-based one.

roi_recon_forward_local_noalloc serves callers that cannot allocate device memory
(their memory belongs to a fixed budget owned by a framework allocator or a server,
or their loop cannot take cudaMalloc's implicit synchronisation); its scratch is a
fixed array inside the library, shared by every call.  It runs the same kernel on the
same host plan as roi_recon_forward_local, so the two agree bit for bit.  This file is
collected last so that a run stopping at the first failure has already run every other
test."""
import numpy as np
import pytest

import paper_1604_02292_gb300 as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs CUDA")


def _noalloc(N, na, nd, region, x, y):
    g = R.Geometry(N, na, nd, None, R.ROI_F32, R.ROI_F32)
    s, msg = R.roi_recon_forward_local_noalloc(g, R.Region(*region), x.data_ptr(), y.data_ptr(),
                                               torch.cuda.current_stream().cuda_stream)
    assert s == R.ROI_OK, msg


# (N, n_angles, n_det, region, seed): a small box, a large one (more angles than one chunk of
# the ray table), the small one again, a clipped box at the grid edge, the large one again
CASES = [(128, 64, 128, (63.5, 63.5, 16.0, 8.0), 1),
         (256, 400, 256, (128.0, 100.0, 50.0, 20.0), 2),
         (128, 64, 128, (63.5, 63.5, 16.0, 8.0), 1),
         (192, 333, 200, (5.0, 180.0, 30.0, 12.0), 3),
         (256, 400, 256, (128.0, 100.0, 50.0, 20.0), 4)]


def test_noalloc_forward_equals_handle_in_any_order():
    """Each call's y (filled with NaN beforehand) equals forward_local's bit for bit, whatever
    the previous call left in the shared scratch (a larger box, more angles)."""
    _need_gpu()
    for N, na, nd, region, seed in CASES:
        rr = R.RoiRecon(N, na, nd)
        pl = rr.plan(region)
        x = torch.from_numpy(np.random.default_rng(seed).random((pl.box[3], pl.box[2])).astype(np.float32)).cuda()
        ref = rr.forward_local(region, x).cpu().numpy()
        for _ in range(2):  # twice in a row
            y = torch.full((na, pl.window_stride), float("nan"), dtype=torch.float32, device="cuda")
            _noalloc(N, na, nd, region, x, y)
            got = y.cpu().numpy()
            assert np.isfinite(got).all()
            assert np.array_equal(got, ref), (N, na, region)
        rr.close()


def test_noalloc_leaves_device_memory_unchanged():
    """After a first call (which may load the module holding the scratch array), further
    calls change the device's free memory by nothing."""
    _need_gpu()
    N, na, nd, region = 256, 400, 256, (128.0, 100.0, 50.0, 20.0)
    pl = R.plan(N, na, nd, region)
    x = torch.rand((pl.box[3], pl.box[2]), dtype=torch.float32, device="cuda")
    y = torch.empty((na, pl.window_stride), dtype=torch.float32, device="cuda")
    _noalloc(N, na, nd, region, x, y)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        _noalloc(N, na, nd, region, x, y)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_oversize_and_custom_angles():
    _need_gpu()
    g = R.Geometry(8192, 64, 4096, None, R.ROI_F32, R.ROI_F32)
    x = torch.zeros(1, device="cuda")
    s, msg = R.roi_recon_forward_local_noalloc(g, R.Region(4096.0, 4096.0, 2000.0, 100.0), x.data_ptr(),
                                               x.data_ptr(), 0)
    assert s == R.ROI_EINVAL and "limit" in msg
    ang = np.zeros(4)
    g2 = R.Geometry(64, 4, 64, ang.ctypes.data_as(R.ctypes.POINTER(R.ctypes.c_double)), R.ROI_F32, R.ROI_F32)
    s, msg = R.roi_recon_forward_local_noalloc(g2, R.Region(32.0, 32.0, 4.0, 1.0), x.data_ptr(), x.data_ptr(), 0)
    assert s == R.ROI_EINVAL
    g3 = R.Geometry(64, 4, 64, None, R.ROI_F32, R.ROI_BF16)
    s, msg = R.roi_recon_forward_local_noalloc(g3, R.Region(32.0, 32.0, 4.0, 1.0), x.data_ptr(), x.data_ptr(), 0)
    assert s == R.ROI_EINVAL
