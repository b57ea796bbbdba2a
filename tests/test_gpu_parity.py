"""GPU parity: the CUDA library, called through its C ABI, against the FP64 oracle.

Tolerances (relative L2 over all compared values):
  * single operators (W_L, W_L^T, ramp filter, FBP, exterior subtraction): 1e-5,
    the FP32 projector bar; observed values are a few 1e-7;
  * adjoint identity of the GPU pair: 1e-6 of ||W x|| ||y||, the scale of <W x, y>;
  * whole local solves (SIRT 200, CP-TV up to 500 iterations): 1e-4.  Each
    iteration adds FP32 rounding of about 1e-7 relative and the iterations are
    non-expansive, so after k iterations the error stays below k * 1e-7 plus the
    input differences (5e-5 for k = 500).
Every input is drawn from fixed seeds and rounded to float32 before it is given
to both sides, so both see identical data.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import paper_1604_02292_gb300 as R
from paper_1604_02292_gb300 import synth
from paper_1604_02292_gb300 import workloads as WL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OP_TOL = 1e-5
SOLVE_TOL = 1e-4


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    err = float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))
    _record(err)
    return err


def _record(err):
    """Append the measured error to $PARITY_LOG (JSON lines) when set."""
    path = os.environ.get("PARITY_LOG")
    if path:
        test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
        with open(path, "a") as f:
            f.write(json.dumps({"test": test, "rel_l2": err}) + "\n")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    R.lib()
    yield
    torch.cuda.synchronize()


# geometry cases: (N, n_angles, n_det, region)
GEOMS = [
    (128, 64, 128, (63.5, 63.5, 16.0, 8.0)),        # the 128 x 128 workload, centred
    (128, 64, 128, WL.region(WL.WORKLOADS["roi_sirt_128"], seed=0)),
    (96, 37, 150, (10.0, 50.0, 12.0, 4.0)),          # box clipped at the left edge, 37 angles (ragged chunk)
    (100, 45, 80, (70.3, 33.7, 20.0, 5.0)),          # detector narrower than the grid, odd box
    (256, 200, 256, (128.0, 100.0, 50.0, 20.0)),    # 140 x 140 box: 4 tiles + ragged tail
    (64, 1, 64, (32.0, 32.0, 10.0, 2.0)),            # single angle
    (64, 16, 64, (0.5, 0.5, 0.5, 0.0)),              # 2 x 2 box in the corner
    (192, 90, 200, (96.0, 96.0, 60.0, 30.0)),        # box = whole grid (180 of 192)
]


def _window_of(full, pl):
    """Extract the per-angle windows of a full oracle sinogram into [na][stride]."""
    na = full.shape[0]
    out = np.zeros((na, pl.window_stride))
    for a in range(na):
        w = pl.width[a]
        out[a, :w] = full[a, pl.d0[a]:pl.d0[a] + w]
    return out


def _full_of(win, pl, nd):
    na = win.shape[0]
    out = np.zeros((na, nd))
    for a in range(na):
        w = pl.width[a]
        out[a, pl.d0[a]:pl.d0[a] + w] = win[a, :w]
    return out


@pytest.mark.parametrize("N,na,nd,region", GEOMS)
def test_forward_local_matches_oracle(N, na, nd, region):
    rr = R.RoiRecon(N, na, nd)
    pl = rr.plan(region)
    x0, y0, w, h = pl.box
    x = np.random.default_rng(1).random((h, w)).astype(np.float32)
    y = rr.forward_local(region, torch.from_numpy(x).cuda()).cpu().numpy()
    g = oracle.Geometry(N, na, nd)
    full = oracle.forward(g, x.astype(np.float64), rect=pl.box)
    exp = _window_of(full, pl)
    assert rel_l2(y, exp) <= OP_TOL
    for a in range(na):
        assert (y[a, pl.width[a]:] == 0).all()


@pytest.mark.parametrize("N,na,nd,region", GEOMS)
def test_back_local_matches_oracle(N, na, nd, region):
    rr = R.RoiRecon(N, na, nd)
    pl = rr.plan(region)
    x0, y0, w, h = pl.box
    win = np.random.default_rng(2).random((na, pl.window_stride)).astype(np.float32)
    for a in range(na):
        win[a, pl.width[a]:] = 0.0
    xg = rr.back_local(region, torch.from_numpy(win).cuda()).cpu().numpy()
    g = oracle.Geometry(N, na, nd)
    exp = oracle.back(g, _full_of(win.astype(np.float64), pl, nd), rect=pl.box)
    assert rel_l2(xg, exp) <= OP_TOL


@pytest.mark.parametrize("N,na,nd,region", GEOMS[:5])
def test_gpu_pair_is_adjoint(N, na, nd, region):
    rr = R.RoiRecon(N, na, nd)
    pl = rr.plan(region)
    x0, y0, w, h = pl.box
    rng = np.random.default_rng(3)
    x = rng.standard_normal((h, w)).astype(np.float32)
    win = rng.standard_normal((na, pl.window_stride)).astype(np.float32)
    for a in range(na):
        win[a, pl.width[a]:] = 0.0
    wx = rr.forward_local(region, torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    wty = rr.back_local(region, torch.from_numpy(win).cuda()).cpu().numpy().astype(np.float64)
    lhs = float((wx * win).sum())
    rhs = float((x.astype(np.float64) * wty).sum())
    # zero-mean data make <Wx, y> a sum with cancellation: compare against its scale
    # |<Wx, y>| <= ||Wx|| ||y|| (Cauchy-Schwarz)
    scale = float(np.linalg.norm(wx) * np.linalg.norm(win))
    assert abs(lhs - rhs) <= 1e-6 * scale


def _workload_data(name, seed=0):
    w = WL.WORKLOADS[name]
    return w, WL.sinogram(w, seed)


@pytest.mark.parametrize("N,na,nd", [(128, 64, 128), (100, 37, 257), (64, 8, 33)])
def test_ramp_filter_matches_oracle(N, na, nd):
    p = np.random.default_rng(4).random((na, nd)).astype(np.float32)
    rr = R.RoiRecon(N, na, nd)
    rr.set_sinogram(torch.from_numpy(p).cuda())
    q = rr.ramp_filter().cpu().numpy()
    exp = oracle.ramp(oracle.Geometry(N, na, nd), p.astype(np.float64))
    assert rel_l2(q, exp) <= OP_TOL


def test_fbp_matches_oracle_128():
    w, p = _workload_data("roi_sirt_128")
    rr = R.RoiRecon(*w.geometry())
    rr.set_sinogram(torch.from_numpy(p).cuda())
    out = torch.empty((w.N, w.N), dtype=torch.float32, device="cuda")
    rr.fbp(out)
    g = oracle.Geometry(*w.geometry())
    exp = oracle.fov(g, oracle.fbp(g, p.astype(np.float64)))  # the cached image: inside the field of view
    assert rel_l2(out.cpu().numpy(), exp) <= OP_TOL


@pytest.mark.parametrize("centred", [True, False])
def test_exterior_matches_oracle_128(centred):
    w, p = _workload_data("roi_sirt_128")
    region = WL.region(w, seed=0, centred=centred)
    rr = R.RoiRecon(*w.geometry())
    rr.set_sinogram(torch.from_numpy(p).cuda())
    rr.fbp()
    pl = rr.plan(region)
    win = torch.zeros((w.n_angles, pl.window_stride), dtype=torch.float32, device="cuda")
    d0 = rr.reproject_exterior(region, win)
    assert list(d0) == pl.d0
    g = oracle.Geometry(*w.geometry())
    xf = oracle.fbp(g, p.astype(np.float64))
    exp = _window_of(oracle.exterior(g, pl.box, p.astype(np.float64), xf), pl)
    assert rel_l2(win.cpu().numpy(), exp) <= OP_TOL


def _oracle_pipeline(w, p, region, reg, iters, lam=0.0, weighting=0, precond=1):
    g = oracle.Geometry(*w.geometry())
    return oracle.solve_local(g, p.astype(np.float64), region, reg=reg, iters=iters, lam=lam,
                              weighting=weighting, precond=precond)


PATHS = [1, 0]  # ROI_OPT_SINGLE_LAUNCH: one cooperative launch per solve, or one launch per operator


@pytest.mark.parametrize("single", PATHS)
@pytest.mark.parametrize("centred", [True, False])
def test_sirt_pipeline_128(centred, single):
    """The whole 128 x 128 workload: Ram-Lak FBP, exterior subtraction, 200 nonneg SIRT."""
    w, p = _workload_data("roi_sirt_128")
    region = WL.region(w, seed=0, centred=centred)
    rr = R.RoiRecon(*w.geometry())
    rr.set_option(R.ROI_OPT_SINGLE_LAUNCH, single)
    rr.set_sinogram(torch.from_numpy(p).cuda())
    rr.fbp()
    out, info = rr.solve_local(region, R.ROI_SIRT_NONNEG, iters=w.iters)
    x, box, _, _ = _oracle_pipeline(w, p, region, "sirt", w.iters)
    assert (info.box_x0, info.box_y0, info.box_w, info.box_h) == box
    got = out.cpu().numpy()
    assert (got >= 0).all()
    assert rel_l2(got, x) <= SOLVE_TOL


@pytest.mark.parametrize("single", PATHS)
def test_sirt_weighted_pipeline_128(single):
    w, p = _workload_data("roi_sirt_128", seed=1)
    region = WL.region(w, seed=1)
    rr = R.RoiRecon(*w.geometry())
    rr.set_option(R.ROI_OPT_SINGLE_LAUNCH, single)
    rr.set_sinogram(torch.from_numpy(p).cuda())
    rr.fbp()
    out, _ = rr.solve_local(region, R.ROI_SIRT_NONNEG, iters=50, weighting=1)
    x, _, _, _ = _oracle_pipeline(w, p, region, "sirt", 50, weighting=1)
    assert rel_l2(out.cpu().numpy(), x) <= SOLVE_TOL


@pytest.mark.parametrize("single", PATHS)
@pytest.mark.parametrize("lam", [0.0, 0.01, 0.5])
def test_cp_tv_pipeline_128(lam, single):
    w, p = _workload_data("roi_sirt_128", seed=2)
    region = WL.region(w, seed=2)
    rr = R.RoiRecon(*w.geometry())
    rr.set_option(R.ROI_OPT_SINGLE_LAUNCH, single)
    rr.set_sinogram(torch.from_numpy(p).cuda())
    rr.fbp()
    out, info = rr.solve_local(region, R.ROI_TV_CP, iters=150, lam=lam, eval_objective=1)
    x, box, pp, _ = _oracle_pipeline(w, p, region, "tv", 150, lam=lam)
    assert rel_l2(out.cpu().numpy(), x) <= SOLVE_TOL
    fo = oracle.objective(oracle.Geometry(*w.geometry()), box, pp, x, lam)
    assert abs(info.objective - fo) <= 1e-4 * abs(fo)


@pytest.mark.parametrize("single", PATHS)
def test_cp_tv_scalar_steps_128(single):
    """precond = 0: steps 0.99/||K|| from 100 power iterations on the device."""
    w, p = _workload_data("roi_sirt_128", seed=3)
    region = WL.region(w, seed=3)
    rr = R.RoiRecon(*w.geometry())
    rr.set_option(R.ROI_OPT_SINGLE_LAUNCH, single)
    rr.set_sinogram(torch.from_numpy(p).cuda())
    rr.fbp()
    out, info = rr.solve_local(region, R.ROI_TV_CP, iters=100, lam=0.05, precond=0)
    g = oracle.Geometry(*w.geometry())
    box = oracle.roi_box(w.N, *region)
    L = oracle.power_norm(g, box, 100)
    assert abs(info.step_L - L) <= 1e-4 * L
    x, _, _, _ = _oracle_pipeline(w, p, region, "tv", 100, lam=0.05, precond=0)
    assert rel_l2(out.cpu().numpy(), x) <= SOLVE_TOL


def test_host_buffers_and_determinism():
    """Host sinogram in, host result out; repeated solves are bit-identical."""
    w, p = _workload_data("roi_sirt_128", seed=4)
    region = WL.region(w, seed=4)
    rr = R.RoiRecon(*w.geometry())
    rr.set_sinogram(p)
    rr.fbp()
    torch.cuda.synchronize()
    pl = rr.plan(region)
    host = np.empty((pl.box[3], pl.box[2]), np.float32)
    rr.solve_local(region, R.ROI_TV_CP, iters=40, lam=0.01, out=host)
    d1, _ = rr.solve_local(region, R.ROI_TV_CP, iters=40, lam=0.01)
    d2, _ = rr.solve_local(region, R.ROI_TV_CP, iters=40, lam=0.01)
    a, b = d1.cpu().numpy(), d2.cpu().numpy()
    assert np.array_equal(a, b)
    assert np.array_equal(host, a)


def test_crop_disk_and_zero_iterations():
    w, p = _workload_data("roi_sirt_128")
    region = (64.0, 60.0, 16.0, 8.0)
    rr = R.RoiRecon(*w.geometry())
    rr.set_sinogram(torch.from_numpy(p).cuda())
    rr.fbp()
    z, _ = rr.solve_local(region, R.ROI_SIRT_NONNEG, iters=0)
    assert (z.cpu().numpy() == 0).all()
    full, _ = rr.solve_local(region, R.ROI_SIRT_NONNEG, iters=20)
    crop, info = rr.solve_local(region, R.ROI_SIRT_NONNEG, iters=20, crop_disk=1)
    full, crop = full.cpu().numpy(), crop.cpu().numpy()
    ii, jj = np.meshgrid(np.arange(info.box_h) + info.box_y0, np.arange(info.box_w) + info.box_x0, indexing="ij")
    inside = (jj - region[0]) ** 2 + (ii - region[1]) ** 2 <= region[2] ** 2
    assert np.array_equal(crop[inside], full[inside])
    assert (crop[~inside] == 0).all()


def test_call_order_and_argument_errors():
    w = WL.WORKLOADS["roi_sirt_128"]
    rr = R.RoiRecon(*w.geometry())
    with pytest.raises(R.RoiError) as e:
        rr.fbp()
    assert e.value.status == R.ROI_ESTATE
    rr.set_sinogram(torch.zeros((w.n_angles, w.n_det), device="cuda"))
    with pytest.raises(R.RoiError) as e:
        rr.solve_local((64.0, 64.0, 16.0, 8.0))
    assert e.value.status == R.ROI_ESTATE
    rr.fbp()
    for bad in [dict(iters=-1), dict(lam=-1.0, reg=R.ROI_TV_CP), dict(reg=7)]:
        with pytest.raises(R.RoiError) as e:
            rr.solve_local((64.0, 64.0, 16.0, 8.0), **bad)
        assert e.value.status == R.ROI_EINVAL
    with pytest.raises(R.RoiError) as e:
        rr.solve_local((900.0, 900.0, 16.0, 8.0))
    assert e.value.status == R.ROI_EINVAL
    # the handle still works after errors
    out, _ = rr.solve_local((64.0, 64.0, 16.0, 8.0), iters=3)
    assert torch.isfinite(out).all()


def test_zero_sinogram_gives_zero_image():
    w = WL.WORKLOADS["roi_sirt_128"]
    rr = R.RoiRecon(*w.geometry())
    rr.set_sinogram(torch.zeros((w.n_angles, w.n_det), device="cuda"))
    rr.fbp()
    for reg in (R.ROI_SIRT_NONNEG, R.ROI_TV_CP):
        out, _ = rr.solve_local((64.0, 64.0, 16.0, 8.0), reg, iters=10, lam=0.01)
        assert (out.cpu().numpy() == 0).all()


# ---------------------------------------------------------------- full-size workload

@pytest.fixture(scope="module")
def big():
    w, p = _workload_data("roi_cptv_1024")
    g = oracle.Geometry(*w.geometry())
    xf = oracle.fbp(g, p.astype(np.float64))
    return w, p, g, xf


def test_fbp_full_size_1024(big):
    w, p, g, xf = big
    rr = R.RoiRecon(*w.geometry())
    rr.set_sinogram(torch.from_numpy(p).cuda())
    out = torch.empty((w.N, w.N), dtype=torch.float32, device="cuda")
    rr.fbp(out)
    assert rel_l2(out.cpu().numpy(), oracle.fov(g, xf)) <= OP_TOL


@pytest.mark.parametrize("single", PATHS)
def test_cp_tv_full_size_1024(big, single):
    """The 1024 x 1024 workload as the benchmark runs it: FBP, exterior subtraction and
    500 preconditioned Chambolle-Pock iterations on the 192 x 192 box, all outputs compared."""
    w, p, g, xf = big
    region = WL.region(w, seed=0)
    rr = R.RoiRecon(*w.geometry())
    rr.set_option(R.ROI_OPT_SINGLE_LAUNCH, single)
    rr.set_sinogram(torch.from_numpy(p).cuda())
    rr.fbp()
    pl = rr.plan(region)
    win = torch.zeros((w.n_angles, pl.window_stride), dtype=torch.float32, device="cuda")
    rr.reproject_exterior(region, win)
    pp = oracle.exterior(g, pl.box, p.astype(np.float64), xf)
    assert rel_l2(win.cpu().numpy(), _window_of(pp, pl)) <= OP_TOL
    out, info = rr.solve_local(region, R.ROI_TV_CP, iters=w.iters, lam=w.lam, eval_objective=1)
    x = oracle.cp_tv(g, pl.box, pp, w.iters, w.lam, precond=1)
    assert rel_l2(out.cpu().numpy(), x) <= SOLVE_TOL
    fo = oracle.objective(g, pl.box, pp, x, w.lam)
    assert abs(info.objective - fo) <= 1e-4 * abs(fo)


@pytest.mark.parametrize("reg,N,na,nd,region", [
    (R.ROI_TV_CP, 256, 200, 256, (128.0, 100.0, 50.0, 20.0)),     # 140 x 140 box, ragged tiles
    (R.ROI_SIRT_NONNEG, 96, 37, 150, (10.0, 50.0, 12.0, 4.0)),    # clipped box, odd angle count
    (R.ROI_TV_CP, 192, 90, 200, (96.0, 96.0, 60.0, 30.0)),        # 180 x 180 box
])
def test_single_launch_matches_multi_launch(reg, N, na, nd, region):
    """The cooperative single-launch solver and the per-operator launches agree to rounding."""
    p = np.random.default_rng(9).random((na, nd)).astype(np.float32) * 50
    outs = []
    for single in (1, 0):
        rr = R.RoiRecon(N, na, nd)
        rr.set_option(R.ROI_OPT_SINGLE_LAUNCH, single)
        rr.set_sinogram(torch.from_numpy(p).cuda())
        rr.fbp()
        out, _ = rr.solve_local(region, reg, iters=60, lam=0.02)
        rr.sync()
        outs.append(out.cpu().numpy())
    assert rel_l2(outs[0], outs[1]) <= 1e-5
