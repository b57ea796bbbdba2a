"""Batched local solves (roi_recon_solve_batch) against the FP64 oracle and against the
single-region path; a region's result must not depend on the rest of the batch."""
import numpy as np
import pytest

import oracle
import paper_1604_02292_gb300 as R
from paper_1604_02292_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SOLVE_TOL = 1e-4
N, NA, ND = 256, 96, 272


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    ph = synth.random_phantom(N, 20, texture=True, seed=31)
    p = synth.poisson_noise(synth.analytic_sinogram(ph, NA, ND), 2e4, seed=32).astype(np.float32)
    g = oracle.Geometry(N, NA, ND)
    xf = oracle.fbp(g, p.astype(np.float64))
    rr = R.RoiRecon(N, NA, ND)
    rr.set_sinogram(torch.from_numpy(p).cuda())
    rr.fbp()
    return rr, p, g, xf


# (region, params): sizes from 24 to 300 px, boxes clipped at the edges, both solvers
CASES = [
    ((128.0, 128.0, 16.0, 8.0), dict(reg=R.ROI_SIRT_NONNEG, iters=40)),
    ((40.0, 200.0, 24.0, 12.0), dict(reg=R.ROI_TV_CP, iters=40, lam=0.02)),
    ((10.0, 10.0, 20.0, 10.0), dict(reg=R.ROI_TV_CP, iters=30, lam=0.05)),           # clipped corner
    ((200.0, 90.0, 33.3, 10.0), dict(reg=R.ROI_SIRT_NONNEG, iters=30, weighting=1)),
    ((128.0, 120.0, 60.0, 30.0), dict(reg=R.ROI_TV_CP, iters=25, lam=0.01)),         # 180 x 180 box
    ((130.0, 128.0, 100.0, 50.0), dict(reg=R.ROI_SIRT_NONNEG, iters=20)),            # box > shared memory
    ((250.0, 5.0, 7.0, 3.0), dict(reg=R.ROI_SIRT_NONNEG, iters=40)),                 # small, clipped
    ((90.0, 170.0, 40.0, 20.0), dict(reg=R.ROI_TV_CP, iters=30, lam=0.1, crop_disk=1)),
]


def _oracle_case(g, p, xf, region, prm):
    box = oracle.roi_box(N, *region)
    pp = oracle.exterior(g, box, p.astype(np.float64), xf)
    if prm["reg"] == R.ROI_SIRT_NONNEG:
        x = oracle.sirt(g, box, pp, prm["iters"], weighting=prm.get("weighting", 0))
    else:
        x = oracle.cp_tv(g, box, pp, prm["iters"], prm["lam"], precond=1)
    if prm.get("crop_disk"):
        ii, jj = np.meshgrid(np.arange(box[3]) + box[1], np.arange(box[2]) + box[0], indexing="ij")
        x = np.where((jj - region[0]) ** 2 + (ii - region[1]) ** 2 <= region[2] ** 2, x, 0.0)
    return x, box


@pytest.fixture(scope="module")
def batch_result(setup):
    rr, p, g, xf = setup
    outs, infos = rr.solve_batch([c[0] for c in CASES], [c[1] for c in CASES])
    rr.sync()
    return [o.cpu().numpy() for o in outs], infos


@pytest.mark.parametrize("i", range(len(CASES)))
def test_batch_matches_oracle(setup, batch_result, i):
    rr, p, g, xf = setup
    outs, infos = batch_result
    region, prm = CASES[i]
    x, box = _oracle_case(g, p, xf, region, prm)
    info = infos[i]
    assert (info.box_x0, info.box_y0, info.box_w, info.box_h) == box
    assert rel_l2(outs[i], x) <= SOLVE_TOL


def test_batch_agrees_with_single_region_path(setup, batch_result):
    rr, p, g, xf = setup
    outs, _ = batch_result
    for i in (1, 4, 5):
        region, prm = CASES[i]
        single, _ = rr.solve_local(region, prm["reg"], iters=prm["iters"], lam=prm.get("lam", 0.0),
                                   weighting=prm.get("weighting", 0), crop_disk=prm.get("crop_disk", 0))
        assert rel_l2(outs[i], single.cpu().numpy()) <= 1e-5


def test_result_alone_equals_result_in_the_mix(setup, batch_result):
    """Bit-identical: each region solved alone (a batch of one) and inside a shuffled batch
    with repeats."""
    rr, p, g, xf = setup
    outs, _ = batch_result
    for i in (0, 2, 5):
        alone, _ = rr.solve_batch([CASES[i][0]], [CASES[i][1]])
        assert np.array_equal(alone[0].cpu().numpy(), outs[i])
    order = [5, 3, 0, 7, 1, 6, 2, 4, 0, 3]
    mixed, _ = rr.solve_batch([CASES[k][0] for k in order], [CASES[k][1] for k in order])
    rr.sync()
    for pos, k in enumerate(order):
        assert np.array_equal(mixed[pos].cpu().numpy(), outs[k]), (pos, k)


def test_host_outputs_equal_device_outputs(setup, batch_result):
    rr, p, g, xf = setup
    outs, _ = batch_result
    host = [np.empty_like(o) for o in outs]
    rr.solve_batch([c[0] for c in CASES], [c[1] for c in CASES], outs=host)
    for a, b in zip(host, outs):
        assert np.array_equal(a, b)


def test_batch_argument_errors(setup):
    rr = setup[0]
    with pytest.raises(R.RoiError) as e:
        rr.solve_batch([(128.0, 128.0, 16.0, 8.0), (900.0, 900.0, 5.0, 1.0)], dict(iters=5))
    assert e.value.status == R.ROI_EINVAL and "region 1" in str(e.value)
    regs = (R.Region * 1)(R.Region(128.0, 128.0, 16.0, 8.0))
    prms = (R.SolveParams * 1)(R.SolveParams(R.ROI_TV_CP, 0.01, 5, 0, 0, 0, 0))
    out = torch.empty((48, 48), device="cuda")
    ptrs = (R.ctypes.c_void_p * 1)(out.data_ptr())
    assert R.roi_recon_solve_batch(rr.h, regs, prms, ptrs, 1) == R.ROI_EINVAL
    fresh = R.RoiRecon(N, NA, ND)
    with pytest.raises(R.RoiError) as e:
        fresh.solve_batch([(128.0, 128.0, 16.0, 8.0)], dict(iters=5))
    assert e.value.status == R.ROI_ESTATE


BATCH_SUBSET, BATCH_SUBSET_ITERS = 32, 8


def test_batch_geometry_2048_subset_per_result(capsys):
    """The 2048 x 2048 / 180-angle batching workload: a seeded subset of 32 of its regions
    (radii 16..128 px, SIRT and CP-TV) solved in one batch, every result against the oracle
    (one relative L2 error per result; BATCH_SUBSET_ITERS iterations, because the oracle's
    exterior step and iterations at this size take about a second each per region on the
    host cores); every result finite, SIRT results nonnegative."""
    from paper_1604_02292_gb300 import workloads as WL

    w = WL.BATCHES["roi_batch_2048"]
    items = WL.batch_regions(w, seed=0, count=BATCH_SUBSET)
    items = [(r, dict(prm, iters=BATCH_SUBSET_ITERS)) for r, prm in items]
    p = WL.sinogram(w, 0)
    rr = R.RoiRecon(*w.geometry())
    rr.set_sinogram(torch.from_numpy(p).cuda())
    rr.fbp()
    outs, infos = rr.solve_batch([r for r, _ in items], [prm for _, prm in items])
    rr.sync()
    outs = [o.cpu().numpy() for o in outs]
    g = oracle.Geometry(*w.geometry())
    xf = oracle.fbp(g, p.astype(np.float64))
    errs = []
    for k, ((region, prm), o) in enumerate(zip(items, outs)):
        assert np.isfinite(o).all()
        if prm["reg"] == R.ROI_SIRT_NONNEG:
            assert (o >= 0).all()
        box = oracle.roi_box(w.N, *region)
        assert (infos[k].box_x0, infos[k].box_y0, infos[k].box_w, infos[k].box_h) == box
        pp = oracle.exterior(g, box, p.astype(np.float64), xf)
        if prm["reg"] == R.ROI_SIRT_NONNEG:
            x = oracle.sirt(g, box, pp, prm["iters"])
        else:
            x = oracle.cp_tv(g, box, pp, prm["iters"], prm["lam"], precond=1)
        errs.append(rel_l2(o, x))
    with capsys.disabled():
        print(f"\nbatch 2048 subset: {len(errs)} results, relative L2 per result: "
              + " ".join(f"{e:.1e}" for e in errs))
    assert max(errs) <= SOLVE_TOL, errs
