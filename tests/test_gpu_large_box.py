"""Single-region solves of boxes too large for the single-launch solver (padded image above
a block's shared memory, sides above about 216 px).  roi_recon_solve_local runs them in the
whole-region solver as one cooperative team of every co-resident block, with the exterior
step p' = (p - W x_fbp) + W_L x_fbp (Eq. locouter); ROI_OPT_SINGLE_LAUNCH = 0 keeps the
launch-per-operator path.  Checked: both paths against the oracle (SIRT and CP-TV), the
team result equal bit for bit to roi_recon_solve_batch's for the same region (alone and in
a mix), and the resumable state kept only by the launch-per-operator path."""
import numpy as np
import pytest

import oracle
import paper_1604_02292_gb300 as R
from paper_1604_02292_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, NA, ND = 512, 120, 520
SOLVE_TOL = 1e-4   # whole solves, as in the float32 parity tests
REGIONS = [(256.0, 250.0, 110.0, 20.0),   # box 260 x 260
           (120.0, 400.0, 100.0, 40.0)]   # box 260 x 252, clipped at the left and bottom edges


@pytest.fixture(scope="module")
def data():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    ph = synth.random_phantom(N, 25, texture=True, seed=71)
    p = synth.poisson_noise(synth.analytic_sinogram(ph, NA, ND), 1e4, seed=72).astype(np.float32)
    rr = R.RoiRecon(N, NA, ND)
    rr.set_sinogram(torch.from_numpy(p).cuda())
    rr.fbp()
    g = oracle.Geometry(N, NA, ND)
    xf = oracle.fbp(g, p.astype(np.float64))
    return p, rr, g, xf


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


CASES = [(0, dict(reg=R.ROI_SIRT_NONNEG, iters=40)),
         (1, dict(reg=R.ROI_TV_CP, iters=30, lam=0.02)),
         (0, dict(reg=R.ROI_SIRT_NONNEG, iters=25, weighting=1))]


@pytest.mark.parametrize("single", [1, 0])
@pytest.mark.parametrize("k,prm", CASES)
def test_large_box_matches_oracle(data, k, prm, single):
    p, rr, g, xf = data
    region = REGIONS[k]
    assert max(rr.plan(region).box[2:]) > 216
    box = oracle.roi_box(N, *region)
    pp = oracle.exterior(g, box, p.astype(np.float64), xf)
    if prm["reg"] == R.ROI_SIRT_NONNEG:
        x = oracle.sirt(g, box, pp, prm["iters"], weighting=prm.get("weighting", 0))
    else:
        x = oracle.cp_tv(g, box, pp, prm["iters"], prm["lam"], precond=1)
    rr.set_option(R.ROI_OPT_SINGLE_LAUNCH, single)
    try:
        out, info = rr.solve_local(region, **prm)
    finally:
        rr.set_option(R.ROI_OPT_SINGLE_LAUNCH, 1)
    assert (info.box_x0, info.box_y0, info.box_w, info.box_h) == box
    assert info.iters_done == prm["iters"]
    err = _rel(out.cpu().numpy(), x)
    assert err <= SOLVE_TOL, err


def test_large_box_equals_batch(data):
    """The team of all blocks gives the same bits as solve_batch (a team of 16 blocks for one
    region, one block per region in a batch of many)."""
    _, rr, _, _ = data
    prms = [dict(reg=R.ROI_TV_CP, iters=20, lam=0.01), dict(reg=R.ROI_SIRT_NONNEG, iters=20)]
    for region, prm in zip(REGIONS, prms):
        alone, _ = rr.solve_local(region, **prm)
        one, _ = rr.solve_batch([region], [prm])
        many_regions = [region] + [(40.0 + (37 * i) % 430, 40.0 + (53 * i) % 430, 20.0, 10.0) for i in range(80)]
        many, _ = rr.solve_batch(many_regions, [prm] * len(many_regions))
        a = alone.cpu().numpy()
        assert np.array_equal(a, one[0].cpu().numpy())
        assert np.array_equal(a, many[0].cpu().numpy())


def test_large_box_host_output_and_state(data):
    """Host output through the team path; its solve keeps no resumable state (refused with a
    message), while the launch-per-operator path keeps one."""
    _, rr, _, _ = data
    region = REGIONS[0]
    prm = dict(reg=R.ROI_TV_CP, iters=10, lam=0.02)
    dev, _ = rr.solve_local(region, **prm)
    pl = rr.plan(region)
    host = np.empty((pl.box[3], pl.box[2]), np.float32)
    rr.solve_local(region, out=host, **prm)
    assert np.array_equal(host, dev.cpu().numpy())
    with pytest.raises(R.RoiError) as ei:
        rr.state()
    assert "whole-region" in str(ei.value)
    rr.set_option(R.ROI_OPT_SINGLE_LAUNCH, 0)
    try:
        rr.solve_local(region, **prm)
        st = rr.state()
        assert st is not None
    finally:
        rr.set_option(R.ROI_OPT_SINGLE_LAUNCH, 1)


def test_large_box_serving_geometry_equals_batch():
    """Radius 128 and 256 px (boxes 384 and 768) on the 2048 x 2048 / 180-angle serving
    geometry: solve_local (team of all blocks, band-streamed images) equals solve_batch."""
    from paper_1604_02292_gb300 import workloads as WL

    w = WL.SERVING["roi_serve_2048"]
    rr = R.RoiRecon(*w.geometry())
    rr.set_sinogram(torch.from_numpy(WL.sinogram(w, 0)).cuda())
    rr.fbp()
    c = (w.N - 1) / 2.0
    for r, prm in ((128.0, dict(reg=R.ROI_SIRT_NONNEG, iters=15)), (256.0, dict(reg=R.ROI_TV_CP, iters=10, lam=0.01))):
        region = (c + 100.0, c - 150.0, r, r / 2.0)
        alone, _ = rr.solve_local(region, **prm)
        one, _ = rr.solve_batch([region], [prm])
        assert np.array_equal(alone.cpu().numpy(), one[0].cpu().numpy())
        assert np.isfinite(alone.cpu().numpy()).all()
    rr.close()
