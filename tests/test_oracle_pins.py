"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed-form
line integrals, special angles where Joseph's method reduces to exact column or
row sums, an explicit system matrix built by a different formulation, the
transpose relation, Eq. locouter, the closed form Eq. sirtfull2, least-squares
and TV minimisers computed by independent algorithms, and textbook identities
of the Ram-Lak filter and of FBP.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1604_02292_gb300 import synth


def _centres(N):
    jj = np.arange(N) - (N - 1) / 2.0
    ii = (N - 1) / 2.0 - np.arange(N)
    return np.meshgrid(jj, ii)


def _hat_matrix(N, na, nd, rect=None):
    """Explicit W on the pixels of ``rect`` built from the hat form of Joseph's
    interpolation: at each row (or column) sample the weight of pixel j is
    max(0, 1 - |u - j|) / |cos| -- no floor(), no tap pairs (a different
    formulation from the oracle's stepping loop)."""
    x0, y0, w, h = rect or (0, 0, N, N)
    th = np.arange(na) * math.pi / na
    W = np.zeros((na * nd, w * h))
    half = (N - 1) / 2.0
    for a in range(na):
        c, s = math.cos(th[a]), math.sin(th[a])
        row = abs(c) >= abs(s) - 1e-12
        for d in range(nd):
            t = d - (nd - 1) / 2.0
            for i in range(y0, y0 + h):
                for j in range(x0, x0 + w):
                    if row:
                        u = (t - (half - i) * s) / c + half
                        wt = max(0.0, 1.0 - abs(u - j)) / abs(c)
                    else:
                        v = half - (t - (j - half) * c) / s
                        wt = max(0.0, 1.0 - abs(v - i)) / abs(s)
                    W[a * nd + d, (i - y0) * w + (j - x0)] = wt
    return W


def _oracle_matrix(g, rect=None):
    x0, y0, w, h = rect or (0, 0, g.N, g.N)
    cols = []
    for k in range(w * h):
        e = np.zeros(w * h)
        e[k] = 1.0
        cols.append(oracle.forward(g, e, rect=(x0, y0, w, h)).ravel())
    return np.stack(cols, 1)


# --------------------------------------------------------------------------- W


def test_theta_zero_is_column_sums():
    """At theta = 0 with n_det = N every ray passes through a column of pixel centres."""
    N = 32
    g = oracle.Geometry(N, 4, N)
    x = np.random.default_rng(0).random((N, N))
    p = oracle.forward(g, x)
    np.testing.assert_allclose(p[0], x.sum(0), rtol=0, atol=1e-12)


def test_theta_half_pi_is_row_sums():
    """At theta = pi/2 bin d lies on the row of centre y = t_d, i.e. row N-1-d."""
    N = 32
    g = oracle.Geometry(N, 4, N)
    x = np.random.default_rng(1).random((N, N))
    p = oracle.forward(g, x)
    np.testing.assert_allclose(p[2], x.sum(1)[::-1], rtol=0, atol=1e-12)


def test_gaussian_blob_line_integrals():
    """A smooth image sampled on the grid projects to its closed-form line integrals
    (discretisation error O(h^2); checks the 1/|cos| weight, the angle and detector origin)."""
    N, na, nd = 64, 32, 64
    g = oracle.Geometry(N, na, nd)
    X, Y = _centres(N)
    sig, x0, y0 = 4.0, 5.3, -7.1
    img = np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / (2 * sig**2))
    p = oracle.forward(g, img)
    z = np.zeros(0)
    ph = synth.Phantom(z, z, z, z, z, z, np.array([x0]), np.array([y0]), np.array([sig]), np.array([1.0]))
    pa = synth.analytic_sinogram(ph, na, nd)
    assert np.linalg.norm(p - pa) / np.linalg.norm(pa) < 1e-2


def test_ellipse_phantom_line_integrals():
    """Supersampled ellipse phantom vs analytic ellipse integrals (edge discretisation)."""
    ph = synth.random_phantom(128, 10, seed=0)
    g = oracle.Geometry(128, 64, 128)
    p = oracle.forward(g, synth.rasterize(ph, 128))
    pa = synth.analytic_sinogram(ph, 64, 128)
    assert np.linalg.norm(p - pa) / np.linalg.norm(pa) < 1.5e-2


def test_explicit_matrix_matches_hat_formulation():
    N, na, nd = 16, 12, 20
    g = oracle.Geometry(N, na, nd)
    np.testing.assert_allclose(_oracle_matrix(g), _hat_matrix(N, na, nd), rtol=0, atol=1e-13)


def test_explicit_matrix_matches_hat_formulation_on_box():
    N, na, nd = 16, 12, 16
    rect = (3, 5, 7, 6)
    g = oracle.Geometry(N, na, nd)
    np.testing.assert_allclose(_oracle_matrix(g, rect), _hat_matrix(N, na, nd, rect), rtol=0, atol=1e-13)


# ------------------------------------------------------------------------- W^T


@pytest.mark.parametrize("rect", [None, (2, 3, 9, 7)])
def test_backprojector_is_transpose_16(rect):
    """W^T built row by row from unit sinograms equals the transpose of W (16 x 16)."""
    N, na, nd = 16, 12, 20
    g = oracle.Geometry(N, na, nd)
    W = _oracle_matrix(g, rect)
    x0, y0, w, h = rect or (0, 0, N, N)
    rows = []
    for r in range(na * nd):
        e = np.zeros(na * nd)
        e[r] = 1.0
        rows.append(oracle.back(g, e, rect=(x0, y0, w, h)).ravel())
    WT = np.stack(rows, 1)  # column r = W^T e_r
    np.testing.assert_allclose(WT, W.T, rtol=0, atol=1e-13)


@pytest.mark.parametrize("N,na,nd,rect,hole", [
    (128, 64, 128, None, None),
    (128, 64, 160, (40, 24, 48, 48), None),
    (128, 90, 128, None, (40, 24, 48, 48)),
    (100, 37, 131, (0, 70, 33, 30), None),
])
def test_adjoint_identity(N, na, nd, rect, hole):
    """<W x, y> = <x, W^T y> to 1e-12 (full grid, ROI box, outer operator)."""
    g = oracle.Geometry(N, na, nd)
    rng = np.random.default_rng(7)
    x0, y0, w, h = rect or (0, 0, N, N)
    x = rng.standard_normal((h, w))
    if hole is not None:
        hx, hy, hw, hh = hole
        x[hy - y0:hy - y0 + hh, hx - x0:hx - x0 + hw] = 0.0
    y = rng.standard_normal((na, nd))
    lhs = float((oracle.forward(g, x, rect=rect, hole=hole) * y).sum())
    rhs = float((x * oracle.back(g, y, rect=rect, hole=hole)).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_local_plus_outer_is_full():
    """Eq. locouter: W = W_L + W_F."""
    N, na, nd = 96, 48, 120
    g = oracle.Geometry(N, na, nd)
    box = (30, 17, 40, 40)
    x = np.random.default_rng(3).random((N, N))
    full = oracle.forward(g, x)
    loc = oracle.forward(g, x[17:57, 30:70], rect=box)
    out = oracle.forward(g, x, hole=box)
    np.testing.assert_allclose(loc + out, full, rtol=0, atol=1e-11)


# ------------------------------------------------------------------- filter/FBP


def test_ramlak_impulse_response():
    """Ram-Lak taps (Kak & Slaney): h[0] = 1/4, h[odd k] = -1/(pi k)^2, h[even k] = 0, x pi/N_theta."""
    na, nd = 4, 33
    g = oracle.Geometry(8, na, nd)
    p = np.zeros((na, nd))
    p[:, 16] = 1.0
    q = oracle.ramp(g, p)
    k = np.arange(nd) - 16
    h = np.where(k == 0, 0.25, np.where(k % 2 == 0, 0.0, -1.0 / (np.pi * np.maximum(np.abs(k), 1)) ** 2))
    np.testing.assert_allclose(q, np.tile(h * np.pi / na, (na, 1)), rtol=0, atol=1e-15)


def test_ramlak_taps_sum_to_zero_tail():
    """sum_k h[k] = 0, so a constant row filters to minus the tail beyond the detector."""
    na, nd = 2, 401
    g = oracle.Geometry(8, na, nd)
    q = oracle.ramp(g, np.ones((na, nd)))
    centre = q[0, 200] * na / np.pi
    # sum over odd m >= 1 of 1/m^2 is pi^2/8, so the part beyond |k| = 200 is
    # 2/pi^2 (pi^2/8 - sum_{odd m <= 199} 1/m^2)
    tail = 2.0 / np.pi**2 * (np.pi**2 / 8.0 - sum(1.0 / m**2 for m in range(1, 200, 2)))
    assert abs(centre - tail) < 1e-14


def test_fbp_of_disc_recovers_density():
    """FBP of the analytic sinogram of a unit-density disc is ~1 inside and ~0 far outside."""
    N, na, nd = 128, 256, 128
    R = 40.0
    z = np.zeros(0)
    ph = synth.Phantom(np.array([0.0]), np.array([0.0]), np.array([R]), np.array([R]), np.array([0.0]),
                       np.array([1.0]), z, z, z, z)
    g = oracle.Geometry(N, na, nd)
    x = oracle.fbp(g, synth.analytic_sinogram(ph, na, nd))
    X, Y = _centres(N)
    r = np.hypot(X, Y)
    assert abs(x[r < 30].mean() - 1.0) < 0.01
    assert x[r < 30].std() < 0.02
    assert abs(x[(r > 48) & (r < 60)].mean()) < 0.02


# ------------------------------------------------------------------------ SIRT


def test_sirt_closed_form():
    """Eq. sirtfull2: x^n = alpha [sum_{k<n} A^k] W^T p with A = I - alpha W^T W, x^0 = 0."""
    N, na, nd = 16, 10, 18
    box = (4, 3, 8, 9)
    g = oracle.Geometry(N, na, nd)
    W = _hat_matrix(N, na, nd, box)
    rng = np.random.default_rng(11)
    p = rng.random(na * nd)
    alpha = 1.0 / (na * nd)
    n = 25
    A = np.eye(W.shape[1]) - alpha * W.T @ W
    S = np.zeros_like(A)
    Ak = np.eye(W.shape[1])
    for _ in range(n):
        S += Ak
        Ak = Ak @ A
    expect = alpha * S @ W.T @ p
    got = oracle.sirt(g, box, p, n, alpha=alpha, nonneg=0)
    np.testing.assert_allclose(got.ravel(), expect, rtol=1e-12, atol=1e-14)


def test_sirt_converges_to_pinv_solution():
    """From x^0 = 0 with 0 < alpha < 2/||W||^2 SIRT tends to the minimum-norm LS solution."""
    N, na, nd = 8, 4, 10          # rank-deficient: 40 rays, 64 pixels, rank 35
    box = (0, 0, 8, 8)
    g = oracle.Geometry(N, na, nd)
    W = _hat_matrix(N, na, nd)
    assert np.linalg.matrix_rank(W) < min(W.shape)
    rng = np.random.default_rng(5)
    p = rng.random(na * nd)
    alpha = 1.5 / np.linalg.norm(W, 2) ** 2
    got = oracle.sirt(g, box, p, 40000, alpha=alpha, nonneg=0)
    expect = np.linalg.pinv(W, rcond=1e-10) @ p
    assert np.linalg.norm(got.ravel() - expect) / np.linalg.norm(expect) < 1e-6


def test_nonneg_sirt_recovers_consistent_nonneg_image():
    N, na, nd = 6, 12, 8
    g = oracle.Geometry(N, na, nd)
    W = _hat_matrix(N, na, nd)
    assert np.linalg.matrix_rank(W) == N * N
    xt = np.random.default_rng(9).random(N * N)
    xt[::5] = 0.0
    p = W @ xt
    alpha = 1.5 / np.linalg.norm(W, 2) ** 2
    got = oracle.sirt(g, (0, 0, N, N), p, 40000, alpha=alpha, nonneg=1)
    assert np.abs(got.ravel() - xt).max() < 1e-6


def test_nonneg_clamp_is_active():
    """Eq. sirtbox with l = 0: no negative pixel survives, and data that pull pixels negative get clamped."""
    N, na, nd = 16, 8, 16
    g = oracle.Geometry(N, na, nd)
    p = -np.random.default_rng(2).random((na, nd))
    x = oracle.sirt(g, (0, 0, N, N), p, 5, nonneg=1)
    assert (x == 0.0).all()


def test_local_exactness_with_true_exterior():
    """Noise-free p = W x_true and the true exterior p' = p - W_F x_true make W_L x = p'
    consistent; local SIRT then converges to x_true on the local part."""
    N, na, nd = 24, 16, 32
    g = oracle.Geometry(N, na, nd)
    box = (9, 9, 6, 6)
    xt = np.random.default_rng(4).random((N, N))
    p = oracle.forward(g, xt)
    pp = p - oracle.forward(g, xt, hole=box)
    W = _hat_matrix(N, na, nd, box)
    assert np.linalg.matrix_rank(W) == 36
    alpha = 1.5 / np.linalg.norm(W, 2) ** 2
    got = oracle.sirt(g, box, pp, 40000, alpha=alpha, nonneg=1)
    np.testing.assert_allclose(got, xt[9:15, 9:15], atol=1e-6)


def test_sirt_weighted_matches_explicit():
    """Weighted SIRT x <- x + C W^T R (p - W x), R = 1/(W 1), C = 1/(W^T 1), in matrix form."""
    N, na, nd = 12, 8, 14
    box = (2, 1, 7, 9)
    g = oracle.Geometry(N, na, nd)
    W = _hat_matrix(N, na, nd, box)
    rs, cs = W.sum(1), W.sum(0)
    R = np.where(rs > 1e-3, 1.0 / np.where(rs > 0, rs, 1.0), 0.0)
    C = np.where(cs > 1e-3, 1.0 / np.where(cs > 0, cs, 1.0), 0.0)
    p = np.random.default_rng(8).random(na * nd)
    x = np.zeros(W.shape[1])
    for _ in range(30):
        x = x + C * (W.T @ (R * (p - W @ x)))
    got = oracle.sirt(g, box, p, 30, weighting=1, nonneg=0)
    np.testing.assert_allclose(got.ravel(), x, rtol=1e-11, atol=1e-12)


# -------------------------------------------------------------------------- TV


def test_grad_div_adjoint():
    """div = -grad^T: <grad x, v> = -<x, div v> (pins the boundary handling)."""
    rng = np.random.default_rng(12)
    x = rng.standard_normal((9, 13))
    vx, vy = rng.standard_normal((2, 9, 13))
    gx, gy = oracle.grad(x)
    assert (gx[:, -1] == 0).all() and (gy[-1, :] == 0).all()
    lhs = (gx * vx).sum() + (gy * vy).sum()
    rhs = -(x * oracle.div(vx, vy)).sum()
    # vx in the last column / vy in the last row meet a zero difference; they are not in grad's range
    vx2, vy2 = vx.copy(), vy.copy()
    vx2[:, -1] = 0
    vy2[-1, :] = 0
    rhs2 = -(x * oracle.div(vx2, vy2)).sum()
    assert abs(lhs - rhs2) < 1e-12
    assert abs(rhs - rhs2) < 1e-12


def test_objective_tv_of_ramp():
    """TV of x_ij = j on an h x w box is h (w - 1) (unit horizontal differences)."""
    N, na, nd = 16, 4, 16
    g = oracle.Geometry(N, na, nd)
    box = (2, 2, 10, 7)
    x = np.tile(np.arange(10.0), (7, 1))
    pp = oracle.forward(g, x, rect=box)
    assert abs(oracle.objective(g, box, pp, x, 1.0) - 7 * 9) < 1e-9
    assert abs(oracle.objective(g, box, pp, x, 0.0)) < 1e-20


def test_power_norm_matches_svd():
    N, na, nd = 10, 8, 12
    box = (1, 2, 7, 6)
    g = oracle.Geometry(N, na, nd)
    W = _hat_matrix(N, na, nd, box)
    h, w = 6, 7
    D = []
    for k in range(w * h):
        e = np.zeros((h, w))
        e.flat[k] = 1
        gx, gy = oracle.grad(e)
        D.append(np.concatenate([gx.ravel(), gy.ravel()]))
    K = np.vstack([W, np.array(D).T])
    L = oracle.power_norm(g, box, 500)
    assert abs(L - np.linalg.norm(K, 2)) < 1e-8 * L


def test_cp_lambda_zero_is_least_squares():
    N, na, nd = 8, 12, 10
    box = (0, 0, 8, 8)
    g = oracle.Geometry(N, na, nd)
    W = _hat_matrix(N, na, nd)
    assert np.linalg.matrix_rank(W) == 64
    p = np.random.default_rng(13).random(na * nd)
    expect = np.linalg.lstsq(W, p, rcond=None)[0]
    for precond in (1, 0):
        got = oracle.cp_tv(g, box, p, 30000, 0.0, precond=precond)
        assert np.linalg.norm(got.ravel() - expect) / np.linalg.norm(expect) < 1e-6, precond


def _admm_tv(W, p, lam, h, w, iters=30000, rho=1.0):
    """Independent TV solver: ADMM on min ||Wx - p||^2 + lam sum_ij |(Dx)_ij|_2 with an exact
    linear solve for x and group soft-thresholding for z = Dx."""
    n = h * w
    Dx = np.zeros((n, n))
    Dy = np.zeros((n, n))
    for i in range(h):
        for j in range(w):
            k = i * w + j
            if j < w - 1:
                Dx[k, k], Dx[k, k + 1] = -1.0, 1.0
            if i < h - 1:
                Dy[k, k], Dy[k, k + w] = -1.0, 1.0
    D = np.vstack([Dx, Dy])
    M = np.linalg.inv(2 * W.T @ W + rho * D.T @ D)
    b = 2 * W.T @ p
    z = np.zeros(2 * n)
    y = np.zeros(2 * n)
    x = np.zeros(n)
    for _ in range(iters):
        x = M @ (b + rho * D.T @ (z - y))
        q = D @ x + y
        qx, qy = q[:n], q[n:]
        m = np.hypot(qx, qy)
        sc = np.where(m > lam / rho, 1.0 - (lam / rho) / np.where(m > 0, m, 1.0), 0.0)
        z = np.concatenate([qx * sc, qy * sc])
        y = y + D @ x - z
    return x


def test_cp_tv_matches_independent_admm():
    """Preconditioned CP and an ADMM solver reach the same TV minimiser (objective to 1e-8)."""
    N, na, nd = 8, 10, 10
    box = (0, 0, 8, 8)
    g = oracle.Geometry(N, na, nd)
    W = _hat_matrix(N, na, nd)
    rng = np.random.default_rng(14)
    xt = (rng.random((8, 8)) > 0.5).astype(float)
    p = W @ xt.ravel() + 0.05 * rng.standard_normal(na * nd)
    lam = 0.5
    xa = _admm_tv(W, p, lam, 8, 8)
    xc = oracle.cp_tv(g, box, p, 40000, lam, precond=1)
    fa = oracle.objective(g, box, p, xa.reshape(8, 8), lam)
    fc = oracle.objective(g, box, p, xc, lam)
    assert abs(fa - fc) <= 1e-8 * fa
    assert np.abs(xc.ravel() - xa).max() < 1e-4


# ------------------------------------------------------------------- pipeline


def _fov_mask(N, nd):
    """Field of view by direct distance: pixel centre within min(N, N_d)/2 of the axis."""
    jj, ii = _centres(N)
    return np.hypot(jj, ii) <= min(N, nd) / 2.0


@pytest.mark.parametrize("N,nd", [(64, 64), (64, 80), (63, 50)])
def test_exterior_is_p_minus_outer_projection(N, nd):
    """Eq. locouter on the global reconstruction inside its field of view:
    p - p' + W_L (x_V on the box) = W x_V with x_V = M_V x_fbp."""
    na = 32
    g = oracle.Geometry(N, na, nd)
    box = oracle.roi_box(N, 30.0, 34.0, 8, 4)
    xf = np.random.default_rng(6).random((N, N))
    p = np.random.default_rng(7).random((na, nd))
    pp = oracle.exterior(g, box, p, xf)
    xv = np.where(_fov_mask(N, nd), xf, 0.0)
    x0, y0, w, h = box
    np.testing.assert_allclose(p - pp + oracle.forward(g, xv[y0:y0 + h, x0:x0 + w], rect=box),
                               oracle.forward(g, xv), rtol=0, atol=1e-11)


def test_fov_restriction():
    """The field of view: the disc of diameter min(N, N_d) on the rotation axis.  An image
    outside it reprojects to nothing in the exterior step (p' = p); inside it, the exterior
    step is the plain p - W M_F x; the pixel count of the disc is the lattice-point count of
    a brute-force enumeration."""
    for N, nd in [(16, 16), (16, 12), (15, 40), (7, 7)]:
        g = oracle.Geometry(N, 8, nd)
        m = _fov_mask(N, nd)
        count = sum(1 for i in range(N) for j in range(N)
                    if (2 * j - (N - 1)) ** 2 + ((N - 1) - 2 * i) ** 2 <= min(N, nd) ** 2)
        assert int(m.sum()) == count
        x = np.random.default_rng(N + nd).random((N, N)) + 0.5
        xv = oracle.fov(g, x)
        assert np.array_equal(xv != 0.0, m)
        p = np.random.default_rng(3).random((8, nd))
        box = (N // 3, N // 3, 3, 2)
        outside = np.where(m, 0.0, x)
        assert np.array_equal(oracle.exterior(g, box, p, outside), p)
        inside = np.where(m, x, 0.0)
        np.testing.assert_allclose(oracle.exterior(g, box, p, inside),
                                   p - oracle.forward(g, inside, hole=box), rtol=0, atol=1e-12)


def test_roi_box_rule():
    assert oracle.roi_box(128, 64.0, 64.0, 16, 8) == (40, 40, 48, 48)
    assert oracle.roi_box(128, 63.5, 20.0, 16, 8) == (40, 0, 48, 44)
    assert oracle.roi_box(128, 10.2, 120.7, 16.5, 0) == (0, 104, 27, 24)


def _grad_matrix(h, w):
    n = h * w
    Dx = np.zeros((n, n))
    Dy = np.zeros((n, n))
    for i in range(h):
        for j in range(w):
            k = i * w + j
            if j < w - 1:
                Dx[k, k], Dx[k, k + 1] = -1.0, 1.0
            if i < h - 1:
                Dy[k, k], Dy[k, k + w] = -1.0, 1.0
    return Dx, Dy


@pytest.mark.parametrize("lam,precond", [(0.0, 1), (0.3, 1), (0.3, 0)])
def test_cp_first_iterations_explicit_matrices(lam, precond):
    """Brute force on a tiny box: Chambolle-Pock with explicit K = [W_L; Dx; Dy], the
    diagonal steps sigma_i = 1/sum_j |K_ij|, tau_j = 1/sum_i |K_ij| (Pock & Chambolle 2011)
    or scalar steps 0.99/||K||, and over-relaxation xbar = 2x+ - x, for 1..6 iterations."""
    N, na, nd = 12, 9, 14
    box = (3, 2, 6, 5)
    h, w = 5, 6
    g = oracle.Geometry(N, na, nd)
    W = _hat_matrix(N, na, nd, box)
    Dx, Dy = _grad_matrix(h, w)
    K = np.vstack([W, Dx, Dy])
    p = np.random.default_rng(21).random(na * nd)
    if precond:
        rs = W.sum(1)
        su = np.where(rs > 1e-6, 1.0 / np.where(rs > 0, rs, 1.0), 0.0)
        sv = 0.5
        tau = 1.0 / np.abs(K).sum(0)
    else:
        L = np.linalg.norm(K, 2)
        su = np.full(na * nd, 0.99 / L)
        sv = 0.99 / L
        tau = np.full(h * w, 0.99 / L)
    x = np.zeros(h * w)
    xb = x.copy()
    u = np.zeros(na * nd)
    vx = np.zeros(h * w)
    vy = np.zeros(h * w)
    for it in range(1, 7):
        u = (u + su * (W @ xb - p)) / (1.0 + su / 2.0)
        ax, ay = vx + sv * (Dx @ xb), vy + sv * (Dy @ xb)
        m = np.hypot(ax, ay)
        sc = np.where(m > lam, lam / np.where(m > 0, m, 1.0), 1.0)
        vx, vy = ax * sc, ay * sc
        xn = x - tau * (W.T @ u + Dx.T @ vx + Dy.T @ vy)
        xb = 2.0 * xn - x
        x = xn
        got = oracle.cp_tv(g, box, p, it, lam, precond=precond, L=None if precond else oracle.power_norm(g, box, 2000))
        np.testing.assert_allclose(got.ravel(), x, rtol=1e-9, atol=1e-12)
