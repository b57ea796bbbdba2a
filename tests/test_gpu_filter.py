"""The paper's own local method (Sec. 3) on the GPU against the FP64 oracle: the filters of
Alg. filtcalc, the disc grey value, and whole ROI_FILTER_SIRT solves (Alg. method with
x >= 0, disc added back) for several regions of one prepared sinogram."""
import numpy as np
import pytest

import oracle
import paper_1604_02292_gb300 as R
from paper_1604_02292_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FILTER_TOL = 1e-5   # filters: float projections, double accumulation of W q_k
SOLVE_TOL = 1e-4    # whole solves, as for the other solvers


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("nd", [64, 65])
def test_filters_match_oracle(nd):
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    N, na, n = 64, 48, 20
    ph = synth.random_phantom(N, 6, texture=False, seed=71)
    p = synth.analytic_sinogram(ph, na, nd).astype(np.float32)
    rr = R.RoiRecon(N, na, nd)
    rr.set_sinogram(torch.from_numpy(p).cuda())
    rr.filter_prepare(n)
    u, gv = rr.filters(n)
    g = oracle.Geometry(N, na, nd)
    uo = oracle.filtcalc(g, n)
    u = u.cpu().numpy()
    for k in (0, 4, n - 1):
        assert rel_l2(u[k], uo[k]) <= FILTER_TOL, k
    go, _, _ = oracle.disc(g, p.astype(np.float64))
    assert abs(gv - go) <= 1e-6 * abs(go)


@pytest.fixture(scope="module")
def prepared():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    N, na, nd, n = 128, 64, 128, 50
    ph = synth.random_phantom(N, 10, texture=False, seed=72)
    p = synth.poisson_noise(synth.analytic_sinogram(ph, na, nd), 1e4, seed=73).astype(np.float32)
    rr = R.RoiRecon(N, na, nd)
    rr.set_sinogram(torch.from_numpy(p).cuda())
    rr.filter_prepare(n)
    g = oracle.Geometry(N, na, nd)
    return rr, p, g, oracle.filtcalc(g, n), n


@pytest.mark.parametrize("region", [(64.0, 64.0, 16.0, 8.0), (30.5, 90.2, 12.0, 6.0), (120.0, 4.0, 10.0, 5.0),
                                    (64.0, 60.0, 40.0, 20.0)])
def test_filter_solve_matches_oracle(prepared, region):
    rr, p, g, uo, n = prepared
    out, info = rr.solve_local(region, R.ROI_FILTER_SIRT, iters=n)
    x, box = oracle.filter_solve(g, p.astype(np.float64), region, n, u=uo)
    assert (info.box_x0, info.box_y0, info.box_w, info.box_h) == box
    assert rel_l2(out.cpu().numpy(), x) <= SOLVE_TOL
    assert (out.cpu().numpy() >= 0).all()


def test_fewer_iterations_reuse_the_prepared_filters(prepared):
    rr, p, g, uo, n = prepared
    region = (64.0, 64.0, 16.0, 8.0)
    out, _ = rr.solve_local(region, R.ROI_FILTER_SIRT, iters=7)
    x, _ = oracle.filter_solve(g, p.astype(np.float64), region, 7, u=uo)
    assert rel_l2(out.cpu().numpy(), x) <= SOLVE_TOL


def test_filter_state_errors(prepared):
    rr, p, g, uo, n = prepared
    with pytest.raises(R.RoiError) as e:
        rr.solve_local((64.0, 64.0, 16.0, 8.0), R.ROI_FILTER_SIRT, iters=n + 1)
    assert e.value.status == R.ROI_ESTATE
    fresh = R.RoiRecon(128, 64, 128)
    with pytest.raises(R.RoiError) as e:
        fresh.filter_prepare(10)
    assert e.value.status == R.ROI_ESTATE
    fresh.set_sinogram(torch.from_numpy(p).cuda())
    with pytest.raises(R.RoiError) as e:
        fresh.solve_local((64.0, 64.0, 16.0, 8.0), R.ROI_FILTER_SIRT, iters=5)
    assert e.value.status == R.ROI_ESTATE
    with pytest.raises(R.RoiError) as e:
        fresh.filter_prepare(0)
    assert e.value.status == R.ROI_EINVAL


def test_batched_and_served_filter_solves(prepared):
    """The paper's method in the whole-region solvers (one block or a team per region):
    batched and served results are identical to each other, agree with the one-launch-per-
    operator path to rounding and with the oracle within the solve tolerance."""
    rr, p, g, uo, n = prepared
    regions = [(64.0, 64.0, 16.0, 8.0), (30.5, 90.2, 12.0, 6.0), (64.0, 60.0, 40.0, 20.0)]
    prm = dict(reg=R.ROI_FILTER_SIRT, iters=n)
    outs, infos = rr.solve_batch(regions, [prm] * len(regions))
    rr.sync()
    with R.Server(team_blocks=4, teams=8, large_side=100) as s:
        s.add(rr)
        ids = {s.submit(0, r, prm): k for k, r in enumerate(regions)}
        s.drain(120000.0)
        served = {}
        for c in s.poll():
            assert c["status"] == R.ROI_OK
            served[ids[c["id"]]] = s.take(c["id"], (c["box"][3], c["box"][2]))
    for k, region in enumerate(regions):
        b = outs[k].cpu().numpy()
        assert np.array_equal(b, served[k]), k
        single, _ = rr.solve_local(region, R.ROI_FILTER_SIRT, iters=n)
        assert rel_l2(b, single.cpu().numpy()) <= 1e-5
        x, _ = oracle.filter_solve(g, p.astype(np.float64), region, n, u=uo)
        assert rel_l2(b, x) <= SOLVE_TOL


@pytest.mark.parametrize("region,lam", [((64.0, 64.0, 16.0, 8.0), 300.0), ((30.5, 90.2, 12.0, 6.0), 800.0),
                                        ((64.0, 60.0, 40.0, 20.0), 300.0)])
def test_fista_tv_matches_oracle(prepared, region, lam):
    """Alg. methodfista (ROI_FILTER_TV): FISTA with the filtered SIRT step and an FGP TV prox."""
    rr, p, g, uo, n = prepared
    iters, nf = 20, 25
    out, _ = rr.solve_local(region, R.ROI_FILTER_TV, iters=iters, lam=lam, inner_iters=nf)
    x, box = oracle.filter_fista_solve(g, p.astype(np.float64), region, iters, lam, n_fgp=nf, u=uo)
    assert rel_l2(out.cpu().numpy(), x) <= SOLVE_TOL


def test_fista_tv_batched_equals_served(prepared):
    rr, p, g, uo, n = prepared
    regions = [(64.0, 64.0, 16.0, 8.0), (90.0, 40.0, 20.0, 10.0)]
    prm = dict(reg=R.ROI_FILTER_TV, iters=10, lam=300.0)
    outs, _ = rr.solve_batch(regions, [prm] * len(regions))
    rr.sync()
    with R.Server(teams=0) as s:
        s.add(rr)
        ids = {s.submit(0, r, prm): k for k, r in enumerate(regions)}
        s.drain(120000.0)
        for c in s.poll():
            assert c["status"] == R.ROI_OK
            got = s.take(c["id"], (c["box"][3], c["box"][2]))
            assert np.array_equal(got, outs[ids[c["id"]]].cpu().numpy())


@pytest.mark.parametrize("region,lam", [((64.0, 64.0, 16.0, 8.0), 400.0), ((64.0, 60.0, 40.0, 20.0), 200.0),
                                        ((3.0, 70.0, 9.0, 4.0), 400.0)])
def test_haar_ista_matches_oracle(prepared, region, lam):
    """Alg. method with the Haar-ISTA prior of Eq. sirtista (ROI_FILTER_ISTA)."""
    rr, p, g, uo, n = prepared
    iters = 20
    out, _ = rr.solve_local(region, R.ROI_FILTER_ISTA, iters=iters, lam=lam)
    x, box = oracle.filter_ista_solve(g, p.astype(np.float64), region, iters, lam, u=uo)
    assert out.shape == x.shape
    assert rel_l2(out.cpu().numpy(), x) <= SOLVE_TOL
