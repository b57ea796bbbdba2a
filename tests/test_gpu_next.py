"""Truncated projection data with constant padding (Sec. 5.6) and tiled reconstructions
(Sec. 5.5), through the C ABI, against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import paper_1604_02292_gb300 as R
from paper_1604_02292_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, NA, ND = 128, 64, 128


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.fixture(scope="module")
def sino():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    ph = synth.random_phantom(N, 10, texture=False, seed=81)
    return synth.poisson_noise(synth.analytic_sinogram(ph, NA, ND), 1e4, seed=82).astype(np.float32)


def test_truncated_data_with_constant_padding(sino):
    nm = 64
    off = (ND - nm) // 2
    pt = np.ascontiguousarray(sino[:, off:off + nm])
    g = oracle.Geometry(N, NA, ND)
    padded = np.pad(pt.astype(np.float64), ((0, 0), (off, off)), mode="edge")
    rr = R.RoiRecon(N, NA, ND)
    rr.set_sinogram_truncated(torch.from_numpy(pt).cuda())
    xg = torch.empty((N, N), device="cuda")
    rr.fbp(xg)
    xg = xg.cpu().numpy()
    assert rel_l2(xg, oracle.fov(g, oracle.fbp(g, padded))) <= 1e-5
    # padding reduces the truncation error inside the measured disk (against the full data)
    full = oracle.fbp(g, sino.astype(np.float64))
    zero = oracle.fbp(g, np.pad(pt.astype(np.float64), ((0, 0), (off, off))))
    jj, ii = np.meshgrid(np.arange(N) - (N - 1) / 2, (N - 1) / 2 - np.arange(N))
    m = jj ** 2 + ii ** 2 <= (nm / 2 - 2) ** 2
    assert rel_l2(xg[m], full[m]) < rel_l2(zero[m], full[m])
    # the paper's method on the padded data
    n = 20
    rr.filter_prepare(n)
    region = (63.5, 63.5, 16.0, 8.0)
    out, _ = rr.solve_local(region, R.ROI_FILTER_SIRT, iters=n)
    x, _ = oracle.filter_solve(g, padded, region, n)
    assert rel_l2(out.cpu().numpy(), x) <= 1e-4


def test_truncated_argument_errors(sino):
    rr = R.RoiRecon(N, NA, ND)
    for nm in (0, 63, ND + 2):
        pt = torch.zeros((NA, max(nm, 1)), device="cuda")
        assert R.roi_recon_set_sinogram_truncated(rr.h, pt.data_ptr(), R.ROI_F32, 1, nm) == R.ROI_EINVAL


def test_tiles_are_the_batched_boxes_pasted(sino):
    g = oracle.Geometry(N, NA, ND)
    rr = R.RoiRecon(N, NA, ND)
    rr.set_sinogram(torch.from_numpy(sino).cuda())
    rr.fbp()
    tile, margin = 32, 8
    prm = dict(reg=R.ROI_SIRT_NONNEG, iters=20)
    out = rr.solve_tiled(tile, margin, prm).cpu().numpy()
    nt = N // tile
    regions = [(tj * tile + 0.5 * (tile - 1), ti * tile + 0.5 * (tile - 1), tile / 2, margin)
               for ti in range(nt) for tj in range(nt)]
    outs, infos = rr.solve_batch(regions, [prm] * len(regions))
    rr.sync()
    ref = np.zeros((N, N), np.float32)
    for k, (o, inf) in enumerate(zip(outs, infos)):
        ti, tj = divmod(k, nt)
        b = o.cpu().numpy()
        ty, tx = ti * tile - inf.box_y0, tj * tile - inf.box_x0
        ref[ti * tile:(ti + 1) * tile, tj * tile:(tj + 1) * tile] = b[ty:ty + tile, tx:tx + tile]
    assert np.array_equal(out, ref)
    # one tile against the oracle
    k = 1 * nt + 2
    region = regions[k]
    box = oracle.roi_box(N, *region)
    x, _, _, _ = oracle.solve_local(g, sino.astype(np.float64), region, "sirt", iters=20)
    ti, tj = divmod(k, nt)
    tx, ty = tj * tile - box[0], ti * tile - box[1]
    assert rel_l2(out[ti * tile:(ti + 1) * tile, tj * tile:(tj + 1) * tile], x[ty:ty + tile, tx:tx + tile]) <= 1e-4


def test_tiling_argument_errors(sino):
    rr = R.RoiRecon(N, NA, ND)
    rr.set_sinogram(torch.from_numpy(sino).cuda())
    rr.fbp()
    for tile in (0, 3, 48):
        with pytest.raises(R.RoiError) as e:
            rr.solve_tiled(tile, 4, dict(iters=2))
        assert e.value.status == R.ROI_EINVAL
