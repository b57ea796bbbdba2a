"""Phase B tile shapes of the whole-region solvers and their autotuner (batching tier,
Sec. 5.5: many independent local solves).

Every shape (16 x 16, 8 x 8, 16 x 8 pixels per warp) gives whole solves within the float32
solve tolerance of the FP64 oracle.  Shapes group a pixel's angles into partial sums the
same way (chunks of 16 angles) but anchor the fixed-point window coordinate at their own
tile corners, so different shapes agree to rounding only; with one shape, a region's result
is bit-identical whether a single block or a team solves it, batched or served.  The
autotuner picks one shape per box-size class, and batches then use exactly those shapes."""
import numpy as np
import pytest

import oracle
import paper_1604_02292_gb300 as R
from paper_1604_02292_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, NA, ND = 256, 96, 272
SOLVE_TOL = 1e-4
# boxes 48 and 90 (class 0), 100 x 180 (class 1, clipped at the left edge), 240 (class 2, band-streamed)
REGIONS = [((128.0, 128.0, 16.0, 8.0), dict(reg=R.ROI_SIRT_NONNEG, iters=20)),
           ((60.0, 180.0, 30.0, 15.0), dict(reg=R.ROI_TV_CP, iters=20, lam=0.02)),
           ((10.0, 120.0, 60.0, 30.0), dict(reg=R.ROI_SIRT_NONNEG, iters=15, weighting=1)),
           ((128.0, 128.0, 80.0, 40.0), dict(reg=R.ROI_TV_CP, iters=10, lam=0.01))]


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.fixture(scope="module")
def data():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    ph = synth.random_phantom(N, 20, texture=True, seed=91)
    p = synth.poisson_noise(synth.analytic_sinogram(ph, NA, ND), 2e4, seed=92).astype(np.float32)
    g = oracle.Geometry(N, NA, ND)
    xf = oracle.fbp(g, p.astype(np.float64))
    exp = []
    for region, prm in REGIONS:
        box = oracle.roi_box(N, *region)
        pp = oracle.exterior(g, box, p.astype(np.float64), xf)
        if prm["reg"] == R.ROI_SIRT_NONNEG:
            exp.append(oracle.sirt(g, box, pp, prm["iters"], weighting=prm.get("weighting", 0)))
        else:
            exp.append(oracle.cp_tv(g, box, pp, prm["iters"], prm["lam"], precond=1))
    rr = R.RoiRecon(N, NA, ND)
    rr.set_sinogram(torch.from_numpy(p).cuda())
    rr.fbp()
    return rr, exp


def _batch(rr, shape, regions=None):
    rr.set_option(R.ROI_OPT_TILE_SHAPE, shape)
    try:
        regions = regions or [r for r, _ in REGIONS]
        params = [REGIONS[k % len(REGIONS)][1] for k in range(len(regions))]
        outs, _ = rr.solve_batch(regions, params)
        rr.sync()
        return [o.cpu().numpy() for o in outs]
    finally:
        rr.set_option(R.ROI_OPT_TILE_SHAPE, -1)


@pytest.mark.parametrize("shape", sorted(R.TILE_SHAPES))
def test_every_shape_matches_oracle(data, shape):
    rr, exp = data
    outs = _batch(rr, shape)
    for k, (o, x) in enumerate(zip(outs, exp)):
        err = rel_l2(o, x)
        assert err <= SOLVE_TOL, (shape, k, err)


@pytest.mark.parametrize("shape", sorted(R.TILE_SHAPES))
def test_shape_is_bit_identical_across_units(data, shape):
    """With one shape: a team per region (few regions), one block per region (in a batch of
    many) and the server's units give the same bits."""
    rr, _ = data
    teams = _batch(rr, shape)                                   # 4 regions: teams of blocks
    mix = [r for r, _ in REGIONS] + [(40.0 + (37 * i) % 170, 40.0 + (53 * i) % 170, 12.0, 6.0)
                                     for i in range(160)]
    singles = _batch(rr, shape, mix)[:len(REGIONS)]            # one block per region
    for a, b in zip(teams, singles):
        assert np.array_equal(a, b)
    rr.set_option(R.ROI_OPT_TILE_SHAPE, shape)
    try:
        with R.Server(team_blocks=4, teams=8, large_side=100) as s:
            s.add(rr)
            ids = {s.submit(0, r, p): k for k, (r, p) in enumerate(REGIONS)}
            s.drain(120000.0)
            for c in s.poll():
                assert c["status"] == R.ROI_OK
                k = ids[c["id"]]
                assert np.array_equal(s.take(c["id"], (c["box"][3], c["box"][2])), teams[k]), k
    finally:
        rr.set_option(R.ROI_OPT_TILE_SHAPE, -1)


def test_shapes_differ_only_by_rounding(data):
    rr, _ = data
    base = _batch(rr, 0)
    for shape in (1, 2):
        for a, b in zip(_batch(rr, shape), base):
            assert rel_l2(a, b) <= 1e-5


def test_autotune_picks_a_shape_per_class_and_batches_use_it(data):
    rr, _ = data
    shapes, ms = rr.autotune(regions_per_class=48, iters=4)
    assert len(shapes) == 3 and all(s in R.TILE_SHAPES for s in shapes)
    assert rr.tile_shapes == shapes
    for c in range(3):  # every class fits this grid (box sides up to 256)
        assert all(t > 0 for t in ms[c]), ms
        assert ms[c][shapes[c]] == min(ms[c])
    # a batch under the tuned table equals, region by region, the batch forced to its class's shape
    tuned = _batch(rr, -1)
    side_class = [0, 0, 1, 2]  # the four boxes: 48, 90, 100 x 180 (clipped), 240
    for k, (region, _) in enumerate(REGIONS):
        w, h = rr.plan(region).box[2:]
        side = max(w, h)
        c = 0 if side <= 96 else (1 if side <= 216 else 2)
        assert c == side_class[k], (k, side)
        assert np.array_equal(tuned[k], _batch(rr, shapes[c])[k])
    # a handle created later with the same geometry starts from the tuned table
    other = R.RoiRecon(N, NA, ND)
    assert other.tile_shapes == shapes
    other.close()
    rr.tile_shapes = [0, 0, 0]
    assert rr.tile_shapes == [0, 0, 0]
    with pytest.raises(R.RoiError):
        rr.tile_shapes = [0, 3, 0]
    # team sizes of few-region batches: one of the candidates per class, the fastest measured
    caps, cms = rr.team_caps, rr.team_caps_ms()
    for c in range(3):
        assert caps[c] in R.TEAM_CAPS
        assert all(t > 0 for t in cms[c]), cms
        assert cms[c][R.TEAM_CAPS.index(caps[c])] == min(cms[c])
    rr.team_caps = [16, 16, 16]
    with pytest.raises(R.RoiError):
        rr.team_caps = [16, 0, 16]


def test_few_region_batch_is_bit_identical_for_every_team_size(data):
    """A batch of fewer regions than half the blocks runs on teams; the team size (the
    handle's team table) changes the time, never the bits."""
    rr, exp = data
    regions = [r for r, _ in REGIONS]
    params = [p for _, p in REGIONS]
    keep = rr.team_caps
    try:
        res = []
        for cap in R.TEAM_CAPS + (1, 38):
            rr.team_caps = [cap] * 3
            outs, _ = rr.solve_batch(regions, params)
            rr.sync()
            res.append([o.cpu().numpy() for o in outs])
        for other in res[1:]:
            for a, b in zip(res[0], other):
                assert np.array_equal(a, b)
        for o, x in zip(res[0], exp):
            assert rel_l2(o, x) <= SOLVE_TOL
    finally:
        rr.team_caps = keep


@pytest.mark.parametrize("shape", sorted(R.TILE_SHAPES))
def test_lone_large_box_team_path_per_shape(shape):
    """solve_local of a box beyond the single-launch solver (one team of every block, phase B
    cooperative over (tile, chunk) items) equals solve_batch's team of 16 for each shape."""
    from paper_1604_02292_gb300 import workloads as WL

    w = WL.WORKLOADS["roi_cptv_1024"]
    rr = R.RoiRecon(*w.geometry())
    rr.set_sinogram(torch.from_numpy(WL.sinogram(w, 0)).cuda())
    rr.fbp()
    rr.set_option(R.ROI_OPT_TILE_SHAPE, shape)
    for region, prm in (((500.0, 520.0, 90.0, 45.0), dict(reg=R.ROI_TV_CP, iters=8, lam=0.01)),
                        ((300.0, 700.0, 150.0, 75.0), dict(reg=R.ROI_SIRT_NONNEG, iters=6))):
        alone, _ = rr.solve_local(region, **prm)
        one, _ = rr.solve_batch([region], [prm])
        assert np.array_equal(alone.cpu().numpy(), one[0].cpu().numpy())
    rr.close()
