"""Checkpoint / resume of single-region solves through the C ABI: a solve split into two
calls through an exported iterate state is bit-identical to the uninterrupted solve (the
single-launch path and the one-launch-per-operator path; SIRT with scalar and row/column
weights; CP with diagonal and scalar steps), with the state in host or device memory; a state
that does not match the call, or a handle without one, is refused."""
import numpy as np
import pytest

import paper_1604_02292_gb300 as R
from paper_1604_02292_gb300 import workloads as WL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REGION = (64.0, 60.0, 16.0, 8.0)


@pytest.fixture(scope="module")
def rr():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    w = WL.WORKLOADS["roi_sirt_128"]
    r = R.RoiRecon(*w.geometry())
    r.set_sinogram(torch.from_numpy(WL.sinogram(w, 0)).cuda())
    r.fbp()
    return r


CASES = [
    (dict(reg=R.ROI_SIRT_NONNEG), 1),
    (dict(reg=R.ROI_SIRT_NONNEG, weighting=1), 1),
    (dict(reg=R.ROI_TV_CP, lam=0.02), 1),
    (dict(reg=R.ROI_TV_CP, lam=0.02, precond=0), 1),
    (dict(reg=R.ROI_SIRT_NONNEG), 0),
    (dict(reg=R.ROI_TV_CP, lam=0.02), 0),
]


@pytest.mark.parametrize("on_device", [False, True])
@pytest.mark.parametrize("prm,single", CASES)
def test_split_solve_is_bit_identical(rr, prm, single, on_device):
    rr.set_option(R.ROI_OPT_SINGLE_LAUNCH, single)
    try:
        full, _ = rr.solve_local(REGION, iters=30, **prm)
        full = full.cpu().numpy()
        rr.solve_local(REGION, iters=18, **prm)
        st = rr.state(on_device=on_device)
        out, info = rr.solve_local(REGION, iters=12, resume=st, **prm)
        assert info.iters_done == 30
        assert np.array_equal(out.cpu().numpy(), full)
        # the state after a resumed solve continues the same way
        st2 = rr.state()
        out2, info2 = rr.solve_local(REGION, iters=5, resume=st2, **prm)
        assert info2.iters_done == 35
        ref, _ = rr.solve_local(REGION, iters=35, **prm)
        assert np.array_equal(out2.cpu().numpy(), ref.cpu().numpy())
    finally:
        rr.set_option(R.ROI_OPT_SINGLE_LAUNCH, 1)


def test_state_size_and_layout(rr):
    rr.solve_local(REGION, R.ROI_SIRT_NONNEG, iters=4)
    pl = rr.plan(REGION)
    n_img = pl.box[2] * pl.box[3]
    assert rr.state().nbytes == 64 + 4 * n_img
    x, _ = rr.solve_local(REGION, R.ROI_TV_CP, iters=4, lam=0.02)
    st = rr.state()
    assert st.nbytes == 64 + 4 * (4 * n_img + rr.n_angles * pl.window_stride)
    assert bytes(st[:8]) == b"ROISTAT1"
    # the first array is x itself
    assert np.array_equal(st[64:64 + 4 * n_img].view(np.float32).reshape(pl.box[3], pl.box[2]), x.cpu().numpy())


def test_state_errors(rr):
    fresh = R.RoiRecon(128, 64, 128)
    with pytest.raises(R.RoiError) as e:
        fresh.state()
    assert e.value.status == R.ROI_ESTATE
    rr.solve_local(REGION, R.ROI_TV_CP, iters=5, lam=0.02)
    st = rr.state()
    bad = [
        dict(region=(40.0, 40.0, 10.0, 5.0), reg=R.ROI_TV_CP, lam=0.02),  # another box
        dict(region=REGION, reg=R.ROI_TV_CP, lam=0.05),                  # another lambda
        dict(region=REGION, reg=R.ROI_TV_CP, lam=0.02, precond=0),       # another step rule
        dict(region=REGION, reg=R.ROI_SIRT_NONNEG),                      # another regularizer
    ]
    for b in bad:
        region = b.pop("region")
        with pytest.raises(R.RoiError) as e:
            rr.solve_local(region, iters=3, resume=st, **b)
        assert e.value.status == R.ROI_EINVAL, b
    with pytest.raises(R.RoiError) as e:  # truncated
        rr.solve_local(REGION, R.ROI_TV_CP, iters=3, lam=0.02, resume=st[:100].copy())
    assert e.value.status == R.ROI_EINVAL
    garbage = st.copy()
    garbage[:8] = 0
    with pytest.raises(R.RoiError) as e:
        rr.solve_local(REGION, R.ROI_TV_CP, iters=3, lam=0.02, resume=garbage)
    assert e.value.status == R.ROI_EINVAL
    # other uses of the solver buffers end the state
    rr.solve_local(REGION, R.ROI_TV_CP, iters=5, lam=0.02)
    pl = rr.plan(REGION)
    rr.forward_local(REGION, torch.zeros((pl.box[3], pl.box[2]), dtype=torch.float32, device="cuda"))
    with pytest.raises(R.RoiError) as e:
        rr.state()
    assert e.value.status == R.ROI_ESTATE
    rr.solve_local(REGION, R.ROI_TV_CP, iters=5, lam=0.02, eval_objective=1)
    with pytest.raises(R.RoiError) as e:
        rr.state()
    assert e.value.status == R.ROI_ESTATE
