"""The ROI server (roi_server_*): served results against the FP64 oracle, equality with
the batched solver, identity alone vs in the mix and across unit pools, admission by
memory budget, idle exit and relaunch, and argument errors."""
import ctypes
import random
import time

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
def sinos():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    g = oracle.Geometry(N, NA, ND)
    out = []
    for seed in (41, 42):
        ph = synth.random_phantom(N, 20, texture=True, seed=seed)
        p = synth.poisson_noise(synth.analytic_sinogram(ph, NA, ND), 2e4, seed=seed + 100).astype(np.float32)
        rr = R.RoiRecon(N, NA, ND)
        rr.set_sinogram(torch.from_numpy(p).cuda())
        rr.fbp()
        out.append((rr, p, oracle.fbp(g, p.astype(np.float64))))
    return g, out


# (sino, region, params): boxes from 16 to 300 px, clipped ones, both solvers
CASES = [
    (0, (128.0, 128.0, 16.0, 8.0), dict(reg=R.ROI_SIRT_NONNEG, iters=30)),
    (1, (40.0, 200.0, 24.0, 12.0), dict(reg=R.ROI_TV_CP, iters=30, lam=0.02)),
    (0, (10.0, 10.0, 20.0, 10.0), dict(reg=R.ROI_TV_CP, iters=25, lam=0.05)),
    (1, (200.0, 90.0, 33.3, 10.0), dict(reg=R.ROI_SIRT_NONNEG, iters=25, weighting=1)),
    (0, (128.0, 120.0, 60.0, 30.0), dict(reg=R.ROI_TV_CP, iters=20, lam=0.01)),
    (1, (130.0, 128.0, 100.0, 50.0), dict(reg=R.ROI_SIRT_NONNEG, iters=15)),
    (0, (250.0, 5.0, 7.0, 3.0), dict(reg=R.ROI_SIRT_NONNEG, iters=30)),
    (1, (90.0, 170.0, 40.0, 20.0), dict(reg=R.ROI_TV_CP, iters=25, lam=0.1, crop_disk=1)),
]


def serve_all(server, cases, shuffle_seed=None):
    """Submit all cases at once; returns {case index: result} (and repeats appended)."""
    order = list(range(len(cases)))
    if shuffle_seed is not None:
        rng = random.Random(shuffle_seed)
        order = order + order[: len(order) // 2]
        rng.shuffle(order)
    ids = {}
    for k in order:
        sino, region, prm = cases[k]
        ids.setdefault(server.submit(sino, region, prm), k)
    server.drain(120000.0)
    res = {}
    for c in server.poll():
        assert c["status"] == R.ROI_OK
        x0, y0, w, h = c["box"]
        res.setdefault(ids[c["id"]], []).append(server.take(c["id"], (h, w)))
    assert sum(len(v) for v in res.values()) == len(order)
    return res


def make_server(sinos, **kw):
    s = R.Server(**kw)
    for rr, _, _ in sinos[1]:
        s.add(rr)
    return s


@pytest.fixture(scope="module")
def served(sinos):
    with make_server(sinos, team_blocks=4, teams=8, large_side=100) as s:
        res = serve_all(s, CASES)
        st = s.stats()
    return {k: v[0] for k, v in res.items()}, st


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
    return x


@pytest.mark.parametrize("i", range(len(CASES)))
def test_served_matches_oracle(sinos, served, i):
    g, S = sinos
    sino, region, prm = CASES[i]
    _, p, xf = S[sino]
    x = _oracle_case(g, p, xf, region, prm)
    assert served[0][i].shape == x.shape
    assert rel_l2(served[0][i], x) <= SOLVE_TOL


def test_both_pools_were_used(served):
    st = served[1]
    assert st["teams"] == 8 and st["team_blocks"] == 4 and st["single_units"] == st["blocks"] - 32
    assert st["completed"] == len(CASES) and st["failed"] == 0
    assert st["device_in_use"] == 0 and st["host_in_use"] == 0


def test_served_equals_batched(sinos, served):
    """Same exterior form and per-ray / per-tile arithmetic as roi_recon_solve_batch."""
    for sino in (0, 1):
        rr = sinos[1][sino][0]
        ks = [k for k, c in enumerate(CASES) if c[0] == sino]
        outs, _ = rr.solve_batch([CASES[k][1] for k in ks], [CASES[k][2] for k in ks])
        rr.sync()
        for k, o in zip(ks, outs):
            assert np.array_equal(o.cpu().numpy(), served[0][k]), k


def test_alone_equals_in_the_mix(sinos, served):
    with make_server(sinos, team_blocks=4, teams=8, large_side=100) as s:
        for k in (0, 4, 5):
            alone = serve_all(s, [CASES[k]])[0][0]
            assert np.array_equal(alone, served[0][k]), k
        mixed = serve_all(s, CASES, shuffle_seed=7)
    for k, outs in mixed.items():
        for o in outs:
            assert np.array_equal(o, served[0][k]), k


def test_single_blocks_and_teams_agree(sinos, served):
    with make_server(sinos, team_blocks=8, teams=6, large_side=1) as s:  # everything to teams
        res = serve_all(s, CASES)
        assert s.stats()["teams"] == 6
    for k, outs in res.items():
        assert np.array_equal(outs[0], served[0][k]), k
    with make_server(sinos, teams=0) as s:  # everything to single blocks
        res = serve_all(s, CASES)
        assert s.stats()["teams"] == 0
    for k, outs in res.items():
        assert np.array_equal(outs[0], served[0][k]), k


def test_admission_by_memory_budget(sinos, served):
    sides = [R.server_footprint(N, NA, ND, c[1]) for c in CASES]
    big = max(d for d, _, _ in sides)
    budget = int(big * 2.5)
    with make_server(sinos, device_bytes=budget, team_blocks=4, teams=8, large_side=100) as s:
        res = serve_all(s, CASES + CASES)
        st = s.stats()
    assert st["device_peak"] <= budget
    assert st["completed"] == 2 * len(CASES)
    for k, outs in res.items():
        for o in outs:
            assert np.array_equal(o, served[0][k % len(CASES)])
    with make_server(sinos, device_bytes=big // 2) as s:
        with pytest.raises(R.RoiError) as e:
            s.submit(1, CASES[5][1], CASES[5][2])
        assert e.value.status == R.ROI_ENOMEM


def test_idle_exit_and_relaunch(sinos, served):
    with make_server(sinos, idle_us=500) as s:
        a = serve_all(s, [CASES[0]])[0][0]
        time.sleep(0.2)  # the kernel leaves after 0.5 ms without work
        b = serve_all(s, [CASES[0]])[0][0]
        st = s.stats()
    assert st["kernel_launches"] >= 2
    assert np.array_equal(a, served[0][0]) and np.array_equal(b, served[0][0])


def test_progress_without_thread(sinos, served):
    with make_server(sinos, start=False) as s:
        rid = s.submit(0, CASES[6][1], CASES[6][2])
        s.drain(60000.0)  # runs the progress engine itself
        c = s.poll()
        assert [x["id"] for x in c] == [rid]
        assert c[0]["t_submit_ms"] <= c[0]["t_publish_ms"] <= c[0]["t_done_ms"]
        x0, y0, w, h = c[0]["box"]
        assert np.array_equal(s.take(rid, (h, w)), served[0][6])


def test_server_argument_errors(sinos):
    g, S = sinos
    with make_server(sinos) as s:
        with pytest.raises(R.RoiError) as e:
            s.submit(5, CASES[0][1], CASES[0][2])
        assert e.value.status == R.ROI_EINVAL
        with pytest.raises(R.RoiError) as e:
            s.submit(0, (900.0, 900.0, 5.0, 1.0), CASES[0][2])
        assert e.value.status == R.ROI_EINVAL
        prm = R.SolveParams(R.ROI_TV_CP, 0.01, 5, 0, 0, 0, 0)  # CP without the diagonal steps
        st, _ = R.roi_server_submit(s.s, 0, R.Region(128.0, 128.0, 16.0, 8.0), prm)
        assert st == R.ROI_EINVAL
        rid = s.submit(0, CASES[0][1], CASES[0][2])
        with pytest.raises(R.RoiError) as e:  # sinograms only before the first submit
            s.add(S[0][0])
        assert e.value.status == R.ROI_ESTATE
        s.drain()
        s.poll()
        s.take(rid, (48, 48))
        with pytest.raises(R.RoiError) as e:
            s.take(rid, (48, 48))
        assert e.value.status == R.ROI_EINVAL
    fresh = R.RoiRecon(N, NA, ND)
    with R.Server() as s:
        with pytest.raises(R.RoiError) as e:
            s.add(fresh)  # no FBP yet
        assert e.value.status == R.ROI_ESTATE


def test_small_requests_spill_to_idle_teams(sinos):
    """With the teams idle a small-box request is admitted to the team pool (unless
    no_spill); its result is the same bits as through the single-block pool."""
    sino, region, prm = CASES[0]  # 48-px box, below large_side
    got = {}
    for ns in (0, 1):
        with make_server(sinos, team_blocks=4, teams=8, large_side=100, no_spill=ns) as s:
            rid = s.submit(sino, region, prm)
            s.drain(120000.0)
            (c,) = s.poll()
            assert c["status"] == R.ROI_OK
            assert c["pool"] == (0 if ns else 1)
            got[ns] = s.take(rid, (c["box"][3], c["box"][2]))
    assert np.array_equal(got[0], got[1])


def test_solo_launch_and_leaving_it(sinos):
    """A lone request on an idle server runs solo (one team of all blocks); when the work
    queued behind it exceeds solo_queue_ms (here 1 ms of estimated whole-GPU time), the solo
    launch finishes the request it holds and leaves, and the queue is served by the
    configured pools.  Every result equals the batched solver's."""
    long_req = (1, (130.0, 128.0, 100.0, 50.0), dict(reg=R.ROI_SIRT_NONNEG, iters=200))
    reqs = [long_req] + [CASES[k % len(CASES)] for k in range(12)]
    with make_server(sinos, team_blocks=4, teams=8, large_side=100, start=False, solo_queue_ms=1) as s:
        ids = [s.submit(*reqs[0])]
        s.progress()  # solo launch with the lone request
        ids += [s.submit(*r) for r in reqs[1:]]
        s.progress()  # twelve wait behind it: the solo launch is asked to leave
        s.drain(300000.0)
        comp = {c["id"]: c for c in s.poll()}
        got = []
        for rid in ids:
            c = comp[rid]
            assert c["status"] == R.ROI_OK
            got.append(s.take(rid, (c["box"][3], c["box"][2])))
        assert comp[ids[0]]["pool"] == 1
        assert s.stats()["kernel_launches"] >= 2
    for (sino, region, prm), g in zip(reqs, got):
        rr = sinos[1][sino][0]
        outs, _ = rr.solve_batch([region], [prm])
        rr.sync()
        assert np.array_equal(outs[0].cpu().numpy(), g)


def test_destroy_with_requests_outstanding(sinos):
    s = make_server(sinos, device_bytes=8 << 20)
    for k in range(24):
        s.submit(k % 2, CASES[k % len(CASES)][1], CASES[k % len(CASES)][2])
    t0 = time.time()
    s.close()
    assert time.time() - t0 < 60.0


def test_serving_geometry_2048_sampled():
    """Two 2048 x 2048 / 180-angle sinograms, request radii from 16 to 256 px (boxes up to
    768 px, served by teams): every result equals the batched solver's; the two smallest
    and the largest are compared with the oracle."""
    from paper_1604_02292_gb300 import workloads as WL

    w = WL.SERVING["roi_serve_2048"]
    reqs = WL.serve_requests(w, seed=0, count=6, radii=(16.0, 24.0, 64.0, 130.0, 200.0, 256.0))
    reqs = [(sino % 2, reg, dict(prm, iters=8)) for sino, reg, prm in reqs]
    recons, sinos_np = [], []
    for k in range(2):
        p = WL.sinogram(w, k)
        rr = R.RoiRecon(*w.geometry())
        rr.set_sinogram(torch.from_numpy(p).cuda())
        rr.fbp()
        recons.append(rr)
        sinos_np.append(p)
    with R.Server(team_blocks=8, teams=12, large_side=320, no_spill=1) as s:
        for rr in recons:
            s.add(rr)
        ids = {s.submit(sino, reg, prm): k for k, (sino, reg, prm) in enumerate(reqs)}
        s.drain(300000.0)
        served = {}
        for c in s.poll():
            assert c["status"] == R.ROI_OK
            x0, y0, bw, bh = c["box"]
            served[ids[c["id"]]] = s.take(c["id"], (bh, bw))
            assert (c["pool"] == 1) == (max(bw, bh) >= 320)
    for k, (sino, reg, prm) in enumerate(reqs):
        outs, _ = recons[sino].solve_batch([reg], [prm])
        assert np.array_equal(outs[0].cpu().numpy(), served[k]), k
    g = oracle.Geometry(*w.geometry())
    xfs = {}
    for k in (0, 1, 5):
        sino, reg, prm = reqs[k]
        if sino not in xfs:
            xfs[sino] = oracle.fbp(g, sinos_np[sino].astype(np.float64))
        xf = xfs[sino]
        box = oracle.roi_box(w.N, *reg)
        pp = oracle.exterior(g, box, sinos_np[sino].astype(np.float64), xf)
        if prm["reg"] == R.ROI_SIRT_NONNEG:
            x = oracle.sirt(g, box, pp, prm["iters"])
        else:
            x = oracle.cp_tv(g, box, pp, prm["iters"], prm["lam"], precond=1)
        assert rel_l2(served[k], x) <= SOLVE_TOL, k
