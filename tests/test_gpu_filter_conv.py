"""The filtered sinograms of the paper's own method (Sec. 3.1, Eq. sirtapp: iteration k of
Alg. method uses C_{u_k} p) through roi_recon_filter_conv, on the tensor cores (tcgen05,
kind::tf32 with head/remainder operand splits) and on the FMA pipe, against the oracle's
plain double-precision convolution (orc_filter_conv) on seeded random filters and rows.

Tolerance, derived from the arithmetic: an output is a sum of K = 2 N_d - 1 products (fewer
nonzero).  Summed in fp32 in any order, with each addition rounded to nearest or truncated,
its error is at most about K * 2^-23 * sum |u||p| (first-order bound of recursive
summation, truncation doubling the unit roundoff); the tensor-core path adds the split
errors, the omitted lo*lo product and the tf32 truncation of lo, each below 2^-20 |u||p|
per product.  The element bound used is (K * 2^-23 + 2^-19) * sum |u||p|, and the relative
L2 error of a whole result, where the rounding errors average out, must stay below 1e-5.
"""
import numpy as np
import pytest

import oracle
import paper_1604_02292_gb300 as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (angles, detector bins, filters): ragged bins (not a multiple of 8 or of a 128-bin tile),
# a last pass with one tile, filters not a multiple of 16, two filter blocks (n > 256), one
# bin, and the full-size detector of the 1024-pixel workloads
SHAPES = [(3, 64, 5), (5, 100, 17), (4, 257, 40), (2, 300, 260), (2, 1, 3), (3, 1024, 24), (1, 131, 1)]


def _case(na, nd, n, seed):
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((n, na, 2 * nd - 1)).astype(np.float32)
    p = rng.standard_normal((na, nd)).astype(np.float32)
    return u, p


def _oracle(na, nd, u, p):
    g = oracle.Geometry(max(nd, 1), na, nd)
    ud = u.astype(np.float64)
    pd = p.astype(np.float64)
    exp = np.stack([oracle.filter_conv(g, ud[k], pd) for k in range(u.shape[0])])
    bound = np.stack([oracle.filter_conv(g, np.abs(ud[k]), np.abs(pd)) for k in range(u.shape[0])])
    return exp, bound


def _gpu(na, nd, u, p, path):
    rr = R.RoiRecon(max(nd, 1), na, nd)
    try:
        rr.set_option(R.ROI_OPT_FILTER_CONV, path)
        out = rr.filter_conv(torch.from_numpy(u).cuda(), torch.from_numpy(p).cuda())
        torch.cuda.synchronize()
        return out.cpu().numpy().astype(np.float64)
    finally:
        rr.close()


def _check(got, exp, bound, nd):
    k_terms = 2 * nd - 1
    tol = k_terms * 2.0 ** -23 + 2.0 ** -19
    err = np.abs(got - exp)
    worst = float(np.max(err / np.maximum(bound, 1e-30)))
    assert worst <= tol, (worst, tol)
    rel = float(np.linalg.norm(got - exp) / max(np.linalg.norm(exp), 1e-30))
    assert rel <= 1e-5, rel
    return worst, rel


@pytest.mark.parametrize("path", [0, 1], ids=["tensor_cores", "fma"])
@pytest.mark.parametrize("na,nd,n", SHAPES)
def test_filter_conv_matches_oracle(na, nd, n, path):
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    u, p = _case(na, nd, n, seed=1000 + 7 * nd + n)
    exp, bound = _oracle(na, nd, u, p)
    got = _gpu(na, nd, u, p, path)
    worst, rel = _check(got, exp, bound, nd)
    print(f"filter_conv na={na} nd={nd} n={n} path={path}: max err / sum|u||p| {worst:.2e}, rel L2 {rel:.2e}")


def test_detector_too_wide_for_shared_memory_takes_the_fma_pipe():
    """A row of 3000 bins with 100 filters leaves no room for two stages of the filter bank:
    the operator runs on the FMA pipe and still matches the oracle."""
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    na, nd, n = 1, 3000, 100
    u, p = _case(na, nd, n, seed=77)
    exp, bound = _oracle(na, nd, u, p)
    _check(_gpu(na, nd, u, p, 0), exp, bound, nd)


def test_tensor_core_and_fma_paths_agree_through_filter_prepare():
    """filter_prepare's filtered sinograms on either path give the same ROI_FILTER_SIRT solve
    to float rounding (1e-5) on one prepared sinogram."""
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_1604_02292_gb300 import synth

    N, na, nd, n = 128, 64, 128, 40
    ph = synth.random_phantom(N, 10, texture=False, seed=72)
    p = synth.poisson_noise(synth.analytic_sinogram(ph, na, nd), 1e4, seed=73).astype(np.float32)
    res = []
    for path in (0, 1):
        rr = R.RoiRecon(N, na, nd)
        rr.set_option(R.ROI_OPT_FILTER_CONV, path)
        rr.set_sinogram(torch.from_numpy(p).cuda())
        rr.filter_prepare(n)
        out, _ = rr.solve_local((64.0, 60.0, 24.0, 12.0), R.ROI_FILTER_SIRT, iters=n)
        res.append(out.cpu().numpy().astype(np.float64))
        rr.close()
    rel = np.linalg.norm(res[0] - res[1]) / np.linalg.norm(res[1])
    assert rel <= 1e-5, rel


def test_filter_conv_rejects_bad_arguments():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    rr = R.RoiRecon(16, 4, 16)
    assert R.roi_recon_filter_conv(rr.h, 0, 1, 1, 1) == R.ROI_EINVAL
    assert R.roi_recon_filter_conv(rr.h, 2, 0, 1, 1) == R.ROI_EINVAL
    assert R.roi_recon_set_option(rr.h, R.ROI_OPT_FILTER_CONV, 2) == R.ROI_EINVAL
    rr.close()


def test_tensor_core_waits_run_out_and_the_handle_recovers():
    """Failure detection without a fault: with ROI_OPT_TEST_ABSENT_BLOCKS the stage barriers
    wait for 16 bytes that no copy delivers, the bounded waits (20 ms here) run out, the call
    returns ROI_ETIMEOUT, and the same handle then computes the right result."""
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    na, nd, n = 4, 257, 40
    u, p = _case(na, nd, n, seed=5)
    exp, bound = _oracle(na, nd, u, p)
    rr = R.RoiRecon(nd, na, nd)
    ud, pd = torch.from_numpy(u).cuda(), torch.from_numpy(p).cuda()
    out = torch.empty((n, na, nd), dtype=torch.float32, device="cuda")
    rr.set_option(R.ROI_OPT_WAIT_LIMIT_US, 20000)
    rr.set_option(R.ROI_OPT_TEST_ABSENT_BLOCKS, 1)
    st = R.roi_recon_filter_conv(rr.h, n, ud.data_ptr(), pd.data_ptr(), out.data_ptr())
    assert st == R.ROI_ETIMEOUT, st
    rr.set_option(R.ROI_OPT_TEST_ABSENT_BLOCKS, 0)
    got = rr.filter_conv(ud, pd)
    torch.cuda.synchronize()
    _check(got.cpu().numpy().astype(np.float64), exp, bound, nd)
    rr.close()


def test_full_size_filter_workload_sampled_filters():
    """The 1024 filter workload's full launch (256 angles, 1024 bins, 200 filters: 152 blocks,
    four tap groups per stage, two stages) on seeded random filters and rows; the oracle
    computes four of the 200 filtered sinograms whole (first, last and two inside)."""
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    na, nd, n = 256, 1024, 200
    u, p = _case(na, nd, n, seed=2024)
    rr = R.RoiRecon(1024, na, nd)
    got = rr.filter_conv(torch.from_numpy(u).cuda(), torch.from_numpy(p).cuda())
    torch.cuda.synchronize()
    rr.close()
    g = oracle.Geometry(1024, na, nd)
    pd = p.astype(np.float64)
    for k in (0, 57, 133, 199):
        exp = oracle.filter_conv(g, u[k].astype(np.float64), pd)
        bound = oracle.filter_conv(g, np.abs(u[k]).astype(np.float64), np.abs(pd))
        worst, rel = _check(got[k].cpu().numpy().astype(np.float64)[None], exp[None], bound[None], nd)
        print(f"filter_conv full size, filter {k}: max err / sum|u||p| {worst:.2e}, rel L2 {rel:.2e}")
