"""16-bit storage (bfloat16 / half) of the resident sinogram and FBP image and of the
projector images of batched and served solves, float arithmetic throughout.

The oracle is fed the same quantized sinogram (rounded by torch on the CPU, round to
nearest even); what remains is the rounding of the stored FBP image (and, in batched /
served solves, of the iterate the forward projector reads), which bounds the error:
relative rounding 2^-9 (bfloat16) or 2^-12 (half) per stored value, about 1.1e-3 / 1.4e-4
RMS after the uniform-error average, amplified by the exterior subtraction where p' is a
small difference of large terms.  Measured on GB300: FBP image 1.6e-3 / 2.0e-4, whole
solves up to 2.5e-3 / 3.1e-4 (bfloat16 / half).  Tolerances below carry that bound with a
margin of two to three and are the same for every case of a storage type."""
import numpy as np
import pytest

import oracle
import paper_1604_02292_gb300 as R
from paper_1604_02292_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, NA, ND = 256, 96, 272
TDT = {R.ROI_BF16: "bfloat16", R.ROI_F16: "float16"}
# relative L2 bounds: FBP image (one rounding per pixel) and whole solves
FBP_TOL = {R.ROI_BF16: 3e-3, R.ROI_F16: 4e-4}
SOLVE_TOL = {R.ROI_BF16: 5e-3, R.ROI_F16: 1e-3}
MEASURED = {}


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def quantize(a, storage):
    t = torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(getattr(torch, TDT[storage]))
    return t.to(torch.float64).numpy()


@pytest.fixture(scope="module")
def data():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    ph = synth.random_phantom(N, 20, texture=True, seed=51)
    p = synth.poisson_noise(synth.analytic_sinogram(ph, NA, ND), 2e4, seed=52).astype(np.float32)
    return p, oracle.Geometry(N, NA, ND)


@pytest.fixture(scope="module", params=[R.ROI_BF16, R.ROI_F16], ids=["bf16", "f16"])
def handle(request, data):
    p, g = data
    st = request.param
    rr = R.RoiRecon(N, NA, ND, storage=st)
    rr.set_sinogram(torch.from_numpy(p).cuda())
    xf_gpu = torch.empty((N, N), device="cuda")
    rr.fbp(xf_gpu)
    pq = quantize(p, st)
    return st, rr, pq, oracle.fbp(g, pq), xf_gpu.cpu().numpy()


def test_device_rounding_matches_torch(data):
    """set_sinogram narrowing on the device rounds like torch (nearest even): a float32
    sinogram into a 16-bit handle gives the same FBP as the pre-rounded 16-bit tensor."""
    p, _ = data
    for st in (R.ROI_BF16, R.ROI_F16):
        a = R.RoiRecon(N, NA, ND, storage=st)
        b = R.RoiRecon(N, NA, ND, storage=st)
        a.set_sinogram(torch.from_numpy(p).cuda())
        b.set_sinogram(torch.from_numpy(p).cuda().to(getattr(torch, TDT[st])))
        xa_, xb_ = torch.empty((N, N), device="cuda"), torch.empty((N, N), device="cuda")
        a.fbp(xa_)
        b.fbp(xb_)
        assert torch.equal(xa_, xb_)


def test_widening_is_exact(data):
    """A 16-bit sinogram into a float32 handle equals its float32 widening."""
    p, _ = data
    pb = torch.from_numpy(p).cuda().to(torch.bfloat16)
    a, b = R.RoiRecon(N, NA, ND), R.RoiRecon(N, NA, ND)
    a.set_sinogram(pb)
    b.set_sinogram(pb.to(torch.float32))
    xa_, xb_ = torch.empty((N, N), device="cuda"), torch.empty((N, N), device="cuda")
    a.fbp(xa_)
    b.fbp(xb_)
    assert torch.equal(xa_, xb_)


def test_fbp_image_is_stored_rounded(handle):
    st, rr, pq, xf, xg = handle
    again = quantize(xg, st)
    assert np.array_equal(again.astype(np.float32), xg)  # representable in the storage type
    err = rel_l2(xg, xf)
    MEASURED[("fbp", st)] = err
    assert err <= FBP_TOL[st]


REGIONS = [((128.0, 128.0, 16.0, 8.0), dict(reg=R.ROI_SIRT_NONNEG, iters=30)),
           ((60.0, 180.0, 30.0, 15.0), dict(reg=R.ROI_TV_CP, iters=25, lam=0.02)),
           ((130.0, 128.0, 100.0, 50.0), dict(reg=R.ROI_SIRT_NONNEG, iters=15))]  # banded staging


def _oracle(g, pq, xf, region, prm):
    box = oracle.roi_box(N, *region)
    pp = oracle.exterior(g, box, pq, xf)
    if prm["reg"] == R.ROI_SIRT_NONNEG:
        return oracle.sirt(g, box, pp, prm["iters"])
    return oracle.cp_tv(g, box, pp, prm["iters"], prm["lam"], precond=1)


@pytest.mark.parametrize("k", range(len(REGIONS)))
def test_solve_local_16bit_resident(data, handle, k):
    """Single-region path: 16-bit resident sinogram and FBP image, float solve."""
    g = data[1]
    st, rr, pq, xf, _ = handle
    region, prm = REGIONS[k]
    x = _oracle(g, pq, xf, region, prm)
    out, _ = rr.solve_local(region, prm["reg"], iters=prm["iters"], lam=prm.get("lam", 0.0))
    err = rel_l2(out.cpu().numpy(), x)
    MEASURED[("local", st, k)] = err
    assert err <= SOLVE_TOL[st]


def test_batch_and_server_16bit(data, handle):
    """Batched and served solves also store the projector images in 16 bits; the two paths
    give identical results, within the storage bound of the oracle."""
    g = data[1]
    st, rr, pq, xf, _ = handle
    regions = [r for r, _ in REGIONS]
    params = [p for _, p in REGIONS]
    outs, _ = rr.solve_batch(regions, params)
    rr.sync()
    with R.Server(team_blocks=4, teams=8, large_side=100) as s:
        s.add(rr)
        ids = {s.submit(0, r, p): k for k, (r, p) in enumerate(REGIONS)}
        s.drain(120000.0)
        served = {}
        for c in s.poll():
            assert c["status"] == R.ROI_OK
            served[ids[c["id"]]] = s.take(c["id"], (c["box"][3], c["box"][2]))
    for k, (region, prm) in enumerate(REGIONS):
        b = outs[k].cpu().numpy()
        assert np.array_equal(b, served[k]), k
        x = _oracle(g, pq, xf, region, prm)
        err = rel_l2(b, x)
        MEASURED[("batch", st, k)] = err
        assert err <= SOLVE_TOL[st]



def test_precision_geometry_4096_sampled():
    """The 4096 x 4096 / 1024-angle / 4096-bin geometry with bfloat16 storage: one region of
    radius 256 px (box 768 x 768, band-streamed), 3 CP iterations, served by a team, against
    the oracle fed the same quantized sinogram."""
    from paper_1604_02292_gb300 import workloads as WL

    w = WL.PRECISION["roi_precision_4096"]
    (region, prm), = WL.precision_regions(w, seed=0, count=1)
    prm = dict(prm, iters=3)
    ph = synth.random_phantom(w.N, w.n_ellipses, texture=w.texture, seed=0)
    p = synth.poisson_noise(synth.analytic_sinogram(ph, w.n_angles, w.n_det), w.I0, seed=1000).astype(np.float32)
    rr = R.RoiRecon(*w.geometry(), storage=R.ROI_BF16)
    rr.set_sinogram(torch.from_numpy(p).cuda())
    rr.fbp()
    with R.Server(team_blocks=8, teams=4, large_side=1) as s:
        s.add(rr)
        rid = s.submit(0, region, prm)
        s.drain(300000.0)
        (c,) = s.poll()
        x = s.take(rid, (c["box"][3], c["box"][2]))
    g = oracle.Geometry(*w.geometry())
    pq = quantize(p, R.ROI_BF16)
    xf = oracle.fbp(g, pq)
    box = oracle.roi_box(w.N, *region)
    pp = oracle.exterior(g, box, pq, xf)
    xo = oracle.cp_tv(g, box, pp, prm["iters"], prm["lam"], precond=1)
    err = rel_l2(x, xo)
    MEASURED[("geometry_4096", R.ROI_BF16)] = err
    assert err <= SOLVE_TOL[R.ROI_BF16]


def test_report_measured_errors():
    """Prints the measured errors (pytest -s) so they can be quoted."""
    for key in sorted(MEASURED, key=str):
        print("precision", key, f"{MEASURED[key]:.3e}")
