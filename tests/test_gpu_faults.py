"""Failure detection on the GPU without faulting it: a barrier wait that can never
complete (a participant that is never launched) runs out after a short limit, the host
reads ROI_ETIMEOUT, and the handle and the CUDA context stay usable for the next solve --
the grid barrier of the single-launch solver, the team barriers of batched solves and of
large boxes, and the team barriers and mailboxes of the serving kernel (whose server keeps
serving).  Also: cancellation of queued requests, and allocation failures injected on the
host (every allocation of handle creation, of a first batch and of server creation)."""
import time

import numpy as np
import pytest

import paper_1604_02292_gb300 as R
from paper_1604_02292_gb300 import workloads as WL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_barrier_wait_times_out_and_handle_recovers():
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs CUDA")
    w = WL.WORKLOADS["roi_sirt_128"]
    p = WL.sinogram(w, 0)
    region = WL.region(w, seed=0)
    rr = R.RoiRecon(*w.geometry())
    rr.set_sinogram(torch.from_numpy(p).cuda())
    rr.fbp()
    ref, _ = rr.solve_local(region, R.ROI_TV_CP, iters=30, lam=0.01)
    rr.sync()
    ref = ref.cpu().numpy()

    rr.set_option(R.ROI_OPT_WAIT_LIMIT_US, 20000)      # 20 ms
    rr.set_option(R.ROI_OPT_TEST_ABSENT_BLOCKS, 1)     # the barrier waits for one block never launched
    rr.solve_local(region, R.ROI_TV_CP, iters=30, lam=0.01)
    with pytest.raises(R.RoiError) as e:
        rr.sync()
    assert e.value.status == R.ROI_ETIMEOUT
    # host output makes solve_local synchronise and report the timeout itself
    host = np.empty_like(ref)
    with pytest.raises(R.RoiError) as e:
        rr.solve_local(region, R.ROI_TV_CP, iters=30, lam=0.01, out=host)
    assert e.value.status == R.ROI_ETIMEOUT

    rr.set_option(R.ROI_OPT_TEST_ABSENT_BLOCKS, 0)
    again, _ = rr.solve_local(region, R.ROI_TV_CP, iters=30, lam=0.01)
    rr.sync()
    assert np.array_equal(again.cpu().numpy(), ref)
    torch.cuda.synchronize()


def test_option_arguments_are_checked():
    w = WL.WORKLOADS["roi_sirt_128"]
    rr = R.RoiRecon(*w.geometry())
    for opt, val in [(R.ROI_OPT_WAIT_LIMIT_US, 0), (R.ROI_OPT_TEST_ABSENT_BLOCKS, -1), (17, 1)]:
        with pytest.raises(R.RoiError) as e:
            rr.set_option(opt, val)
        assert e.value.status == R.ROI_EINVAL


# ---- team barriers and mailboxes of the batched, large-box and serving kernels -------------

def _handle_128():
    w = WL.WORKLOADS["roi_sirt_128"]
    rr = R.RoiRecon(*w.geometry())
    rr.set_sinogram(torch.from_numpy(WL.sinogram(w, 0)).cuda())
    rr.fbp()
    return rr


BATCH_REGIONS = [(50.0, 60.0, 16.0, 8.0), (80.0, 70.0, 12.0, 6.0)]
BATCH_PARAMS = [dict(reg=R.ROI_TV_CP, iters=20, lam=0.01), dict(reg=R.ROI_SIRT_NONNEG, iters=20)]


def test_batch_team_barrier_times_out_and_recovers():
    """Two regions run as teams of blocks (k_batch_team); a team barrier that waits for a
    block never launched gives up after 20 ms, the host reads ROI_ETIMEOUT, and the next
    batch on the same handle gives the reference bits."""
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs CUDA")
    rr = _handle_128()
    ref, _ = rr.solve_batch(BATCH_REGIONS, BATCH_PARAMS)
    rr.sync()
    ref = [o.cpu().numpy() for o in ref]
    rr.set_option(R.ROI_OPT_WAIT_LIMIT_US, 20000)
    rr.set_option(R.ROI_OPT_TEST_ABSENT_BLOCKS, 1)
    rr.solve_batch(BATCH_REGIONS, BATCH_PARAMS)
    with pytest.raises(R.RoiError) as e:
        rr.sync()
    assert e.value.status == R.ROI_ETIMEOUT
    rr.set_option(R.ROI_OPT_TEST_ABSENT_BLOCKS, 0)
    again, _ = rr.solve_batch(BATCH_REGIONS, BATCH_PARAMS)
    rr.sync()
    for a, b in zip(again, ref):
        assert np.array_equal(a.cpu().numpy(), b)
    rr.close()


def test_large_box_team_barrier_times_out_and_recovers():
    """A box too large for the single-launch solver runs as one team of every block; its
    barrier runs out the same way and the handle recovers."""
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs CUDA")
    w = WL.WORKLOADS["roi_cptv_1024"]
    rr = R.RoiRecon(*w.geometry())
    rr.set_sinogram(torch.from_numpy(WL.sinogram(w, 0)).cuda())
    rr.fbp()
    region = (500.0, 520.0, 120.0, 20.0)  # box 280 x 280
    ref, _ = rr.solve_local(region, R.ROI_SIRT_NONNEG, iters=10)
    rr.sync()
    ref = ref.cpu().numpy()
    rr.set_option(R.ROI_OPT_WAIT_LIMIT_US, 20000)
    rr.set_option(R.ROI_OPT_TEST_ABSENT_BLOCKS, 1)
    host = np.empty_like(ref)
    with pytest.raises(R.RoiError) as e:
        rr.solve_local(region, R.ROI_SIRT_NONNEG, iters=10, out=host)
    assert e.value.status == R.ROI_ETIMEOUT
    rr.set_option(R.ROI_OPT_TEST_ABSENT_BLOCKS, 0)
    again, _ = rr.solve_local(region, R.ROI_SIRT_NONNEG, iters=10)
    rr.sync()
    assert np.array_equal(again.cpu().numpy(), ref)
    rr.close()


def test_server_team_barrier_times_out_and_server_keeps_serving():
    """Requests claimed by teams whose barrier waits for an absent block complete with
    ROI_ETIMEOUT; with the option cleared the same server serves the same requests again,
    equal to the batched solver's bits."""
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs CUDA")
    rr = _handle_128()
    ref, _ = rr.solve_batch(BATCH_REGIONS, BATCH_PARAMS)
    ref = [o.cpu().numpy() for o in ref]
    with R.Server(team_blocks=4, teams=8, large_side=1, no_spill=1, start=False) as s:
        s.add(rr)
        s.set_option(R.ROI_OPT_WAIT_LIMIT_US, 20000)
        s.set_option(R.ROI_OPT_TEST_ABSENT_BLOCKS, 1)
        ids = [s.submit(0, r, p) for r, p in zip(BATCH_REGIONS, BATCH_PARAMS)]
        s.drain(60000.0)
        done = {c["id"]: c for c in s.poll()}
        assert sorted(done) == sorted(ids)
        for i in ids:
            assert done[i]["status"] == R.ROI_ETIMEOUT
            with pytest.raises(R.RoiError) as e:
                s.take(i, (done[i]["box"][3], done[i]["box"][2]))
            assert e.value.status == R.ROI_ETIMEOUT
        s.set_option(R.ROI_OPT_TEST_ABSENT_BLOCKS, 0)
        ids = [s.submit(0, r, p) for r, p in zip(BATCH_REGIONS, BATCH_PARAMS)]
        s.drain(60000.0)
        done = {c["id"]: c for c in s.poll()}
        for k, i in enumerate(ids):
            assert done[i]["status"] == R.ROI_OK
            assert np.array_equal(s.take(i, (done[i]["box"][3], done[i]["box"][2])), ref[k])
    rr.close()


def test_server_mailbox_wait_times_out_and_server_keeps_serving():
    """Team leaders that never claim (test option -1): their members' mailbox waits give up,
    the kernel leaves and progress reports ROI_ETIMEOUT; the queued request stays queued and
    is served once the option is cleared."""
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs CUDA")
    rr = _handle_128()
    ref, _ = rr.solve_batch(BATCH_REGIONS[:1], BATCH_PARAMS[:1])
    ref = ref[0].cpu().numpy()
    with R.Server(team_blocks=4, teams=8, large_side=1, no_spill=1, start=False) as s:
        s.add(rr)
        s.set_option(R.ROI_OPT_WAIT_LIMIT_US, 20000)
        s.set_option(R.ROI_OPT_TEST_ABSENT_BLOCKS, -1)
        rid = s.submit(0, BATCH_REGIONS[0], BATCH_PARAMS[0])
        seen = False
        t0 = time.monotonic()
        while not seen and time.monotonic() - t0 < 30.0:
            try:
                s.progress()
            except R.RoiError as e:
                assert e.status == R.ROI_ETIMEOUT
                seen = True
            time.sleep(0.002)
        assert seen
        assert s.stats()["completed"] == 0
        s.set_option(R.ROI_OPT_TEST_ABSENT_BLOCKS, 0)
        s.drain(60000.0)
        (c,) = s.poll()
        assert c["id"] == rid and c["status"] == R.ROI_OK
        assert np.array_equal(s.take(rid, (c["box"][3], c["box"][2])), ref)
    rr.close()


def test_server_cancel():
    """A queued request is cancelled (completion ROI_ECANCELED, take returns it); one already
    on the device is not (ROI_EBUSY); the others are served."""
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs CUDA")
    rr = _handle_128()
    ref, _ = rr.solve_batch(BATCH_REGIONS, BATCH_PARAMS)
    ref = [o.cpu().numpy() for o in ref]
    with R.Server(team_blocks=4, teams=8, start=False) as s:
        s.add(rr)
        a = s.submit(0, BATCH_REGIONS[0], BATCH_PARAMS[0])
        b = s.submit(0, BATCH_REGIONS[1], BATCH_PARAMS[1])
        s.cancel(b)
        with pytest.raises(R.RoiError) as e:
            s.cancel(b)
        assert e.value.status == R.ROI_EINVAL  # completed (cancelled) already
        s.progress()                           # a is admitted and published
        with pytest.raises(R.RoiError) as e:
            s.cancel(a)
        assert e.value.status == R.ROI_EBUSY
        s.drain(60000.0)
        done = {c["id"]: c for c in s.poll()}
        assert done[b]["status"] == R.ROI_ECANCELED and done[a]["status"] == R.ROI_OK
        with pytest.raises(R.RoiError) as e:
            s.take(b, (1, 1))
        assert e.value.status == R.ROI_ECANCELED
        assert np.array_equal(s.take(a, (done[a]["box"][3], done[a]["box"][2])), ref[0])
        st = s.stats()
        assert st["cancelled"] == 1 and st["completed"] == 1 and st["failed"] == 0
        with pytest.raises(R.RoiError) as e:
            s.cancel(12345)
        assert e.value.status == R.ROI_EINVAL
    rr.close()


# ---- injected allocation failures (host side) ------------------------------------------------

def test_injected_allocation_failures_leave_handles_usable():
    """Every device / page-locked allocation of roi_recon_create, of a first solve_batch and of
    roi_server_create fails in turn (roi_recon_test_fail_alloc): the call returns ROI_ENOMEM,
    and the same handle (or a new server) then works and gives the reference bits."""
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs CUDA")
    w = WL.WORKLOADS["roi_sirt_128"]
    g, _keep = R._geometry(*w.geometry())
    p = torch.from_numpy(WL.sinogram(w, 0)).cuda()
    rr = _handle_128()
    ref, _ = rr.solve_batch(BATCH_REGIONS, BATCH_PARAMS)
    ref = [o.cpu().numpy() for o in ref]
    rr.close()
    try:
        # roi_recon_create
        n_create = 0
        for nth in range(1, 64):
            R.roi_recon_test_fail_alloc(nth)
            st, h = R.roi_recon_create(g, 0)
            R.roi_recon_test_fail_alloc(0)  # disarm: the countdown may not have run out
            if st == R.ROI_OK:
                R.roi_recon_destroy(h)
                break
            assert st == R.ROI_ENOMEM and not h
            n_create += 1
        assert n_create >= 5
        # the first solve_batch of a handle
        n_batch = 0
        for nth in range(1, 64):
            r2 = R.RoiRecon(*w.geometry())
            r2.set_sinogram(p)
            r2.fbp()
            R.roi_recon_test_fail_alloc(nth)
            try:
                r2.solve_batch(BATCH_REGIONS, BATCH_PARAMS)
                ok = True
            except R.RoiError as e:
                assert e.status == R.ROI_ENOMEM
                ok = False
                n_batch += 1
            R.roi_recon_test_fail_alloc(0)
            outs, _ = r2.solve_batch(BATCH_REGIONS, BATCH_PARAMS)  # the handle still works
            r2.sync()
            for a, b in zip(outs, ref):
                assert np.array_equal(a.cpu().numpy(), b)
            r2.close()
            if ok:
                break
        assert n_batch >= 3
        # roi_server_create
        n_srv = 0
        for nth in range(1, 32):
            R.roi_recon_test_fail_alloc(nth)
            try:
                srv = R.Server(start=False)
            except R.RoiError as e:
                assert e.status == R.ROI_ENOMEM
                n_srv += 1
                continue
            R.roi_recon_test_fail_alloc(0)
            srv.close()
            break
        assert n_srv >= 3
    finally:
        R.roi_recon_test_fail_alloc(0)
