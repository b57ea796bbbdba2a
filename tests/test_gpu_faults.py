"""Failure detection on the GPU without faulting it: a grid-barrier wait of the
single-launch solver that can never complete (a participant that is never launched)
runs out after a short limit, the host reads ROI_ETIMEOUT, and the handle and the
CUDA context stay usable for the next solve."""
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
