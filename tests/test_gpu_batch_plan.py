"""Batch plans (roi_recon_batch_plan_*): a batch planned once and replayed as one captured
CUDA graph (Sec. 5.5: many independent local solves in one persistent launch).  A plan's
results equal roi_recon_solve_batch's bit for bit -- for a batch of one block per region and
for a few-region batch on cooperative teams -- on the sinogram it was planned on and, after
set_sinogram + fbp, on a new sinogram of the same geometry; they match the FP64 oracle."""
import numpy as np
import pytest

import oracle
import paper_1604_02292_gb300 as R
from paper_1604_02292_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, NA, ND = 256, 96, 272
SOLVE_TOL = 1e-4

FEW = [((128.0, 128.0, 16.0, 8.0), dict(reg=R.ROI_SIRT_NONNEG, iters=30)),
       ((40.0, 200.0, 24.0, 12.0), dict(reg=R.ROI_TV_CP, iters=30, lam=0.02)),
       ((130.0, 128.0, 100.0, 50.0), dict(reg=R.ROI_SIRT_NONNEG, iters=12)),   # band-streamed box
       ((10.0, 10.0, 20.0, 10.0), dict(reg=R.ROI_TV_CP, iters=20, lam=0.05))]     # clipped corner


def _many():
    regs = [(20.0 + (37 * i) % 216, 20.0 + (53 * i) % 216, 8.0 + (i % 7), 4.0) for i in range(160)]
    prms = [dict(reg=R.ROI_SIRT_NONNEG, iters=15) if i % 2 else dict(reg=R.ROI_TV_CP, iters=15, lam=0.02)
            for i in range(160)]
    return list(zip(regs, prms))


def _sino(seed):
    ph = synth.random_phantom(N, 20, texture=True, seed=seed)
    return synth.poisson_noise(synth.analytic_sinogram(ph, NA, ND), 2e4, seed=seed + 1).astype(np.float32)


@pytest.fixture(scope="module")
def rr():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    h = R.RoiRecon(N, NA, ND)
    h.set_sinogram(torch.from_numpy(_sino(41)).cuda())
    h.fbp()
    yield h
    h.close()


def _batch(rr, cases):
    outs, _ = rr.solve_batch([r for r, _ in cases], [p for _, p in cases])
    rr.sync()
    return [o.cpu().numpy() for o in outs]


@pytest.mark.parametrize("name", ["few_regions_on_teams", "one_block_per_region"])
def test_plan_equals_solve_batch_on_this_and_a_new_sinogram(rr, name):
    cases = FEW if name == "few_regions_on_teams" else _many()
    plan = rr.batch_plan([r for r, _ in cases], [p for _, p in cases])
    try:
        for k in range(2):  # replayed twice: the same bits
            got = [o.cpu().numpy() for o in plan.launch()]
            rr.sync()
            for a, b in zip(got, _batch(rr, cases)):
                assert np.array_equal(a, b), k
        # a new sinogram of the same geometry: the plan solves it without being rebuilt
        rr.set_sinogram(torch.from_numpy(_sino(43)).cuda())
        rr.fbp()
        got = [o.cpu().numpy() for o in plan.launch()]
        rr.sync()
        ref = _batch(rr, cases)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
        if name == "few_regions_on_teams":  # against the oracle on the new sinogram
            p = _sino(43).astype(np.float64)
            g = oracle.Geometry(N, NA, ND)
            xf = oracle.fbp(g, p)
            for (region, prm), x in zip(cases, got):
                box = oracle.roi_box(N, *region)
                pp = oracle.exterior(g, box, p, xf)
                if prm["reg"] == R.ROI_SIRT_NONNEG:
                    xo = oracle.sirt(g, box, pp, prm["iters"])
                else:
                    xo = oracle.cp_tv(g, box, pp, prm["iters"], prm["lam"], precond=1)
                err = np.linalg.norm(x - xo) / np.linalg.norm(xo)
                assert err <= SOLVE_TOL, err
    finally:
        plan.close()
        rr.set_sinogram(torch.from_numpy(_sino(41)).cuda())
        rr.fbp()


def test_plan_arguments_and_state(rr):
    region, _ = FEW[0]
    with pytest.raises(R.RoiError):  # the paper's filter method is not taken by plans
        rr.batch_plan([region], [dict(reg=R.ROI_FILTER_SIRT, iters=5)])
    fresh = R.RoiRecon(N, NA, ND)
    fresh.set_sinogram(torch.from_numpy(_sino(41)).cuda())
    with pytest.raises(R.RoiError):  # no FBP yet
        fresh.batch_plan([region], [dict(reg=R.ROI_SIRT_NONNEG, iters=5)])
    fresh.fbp()
    plan = fresh.batch_plan([region], [dict(reg=R.ROI_SIRT_NONNEG, iters=5)])
    assert R.roi_recon_batch_plan_launch(rr.h, plan.h) == R.ROI_EINVAL  # a plan of another handle
    plan.launch()
    fresh.sync()
    fresh.close()  # destroys the plan with the handle
    plan.h = None
