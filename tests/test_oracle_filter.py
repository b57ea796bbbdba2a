"""Pins of the oracle's version of the paper's own local method (Sec. 3): the filters of
Alg. filtcalc against matrix powers of an explicit system matrix, the filter convolution
against numpy's, the disc grey value against its least-squares definition, Alg. method
against the same recursion written with explicit matrices, and the approximation of SIRT
by FBP with the computed filter (Eq. sfbp) on a consistent problem."""
import math

import numpy as np
import pytest

import oracle
from paper_1604_02292_gb300 import synth
from test_oracle_pins import _hat_matrix


def _impulse(N):
    """The unit impulse at the grid centre, shared by the four central pixels when N is even."""
    c = np.zeros((N, N))
    if N % 2:
        c[N // 2, N // 2] = 1.0
    else:
        m = N // 2
        c[m - 1:m + 1, m - 1:m + 1] = 0.25
    return c.ravel()


def _filter_matrix(N, na, nd):
    """Projection onto the integer offsets -(nd-1) .. nd-1: bins on the integers for odd nd;
    for even nd, bins on the half-integers, adjacent pairs averaged."""
    if nd % 2:
        return _hat_matrix(N, na, 2 * nd - 1)
    H = _hat_matrix(N, na, 2 * nd).reshape(na, 2 * nd, N * N)
    return (0.5 * (H[:, :-1] + H[:, 1:])).reshape(na * (2 * nd - 1), N * N)


@pytest.mark.parametrize("N,nd", [(7, 10), (8, 11), (8, 10)])
def test_filters_are_projected_sums_of_matrix_powers(N, nd):
    na, n = 5, 6
    g = oracle.Geometry(N, na, nd)
    alpha = 1.0 / (na * nd)
    W = _hat_matrix(N, na, nd)
    Wp = _filter_matrix(N, na, nd)
    A = np.eye(N * N) - alpha * W.T @ W
    u = oracle.filtcalc(g, n)
    c0 = _impulse(N)
    for k in range(1, n + 1):
        qk = sum(np.linalg.matrix_power(A, j) @ c0 for j in range(k))
        uk = alpha * (Wp @ qk)
        assert np.allclose(u[k - 1].ravel(), uk, rtol=0, atol=1e-13 * max(1.0, np.abs(uk).max()))


@pytest.mark.parametrize("nd", [20, 21])
def test_filter_is_symmetric_about_the_axis(nd):
    """The impulse is centred on the rotation axis, so each filter row is even in m."""
    g = oracle.Geometry(16, 8, nd)
    u = oracle.filtcalc(g, 4)
    assert np.allclose(u, u[:, :, ::-1], atol=1e-15)


def test_filter_conv_is_linear_convolution():
    rng = np.random.default_rng(3)
    na, nd = 4, 11
    g = oracle.Geometry(8, na, nd)
    uk = rng.normal(size=(na, 2 * nd - 1))
    p = rng.normal(size=(na, nd))
    out = oracle.filter_conv(g, uk, p)
    for a in range(na):
        full = np.convolve(p[a], uk[a])
        assert np.allclose(out[a], full[nd - 1:2 * nd - 1], atol=1e-13)


def test_disc_grey_value_is_the_least_squares_fit_of_the_dc_components():
    N, na, nd = 24, 10, 30
    g = oracle.Geometry(N, na, nd)
    jj, ii = np.meshgrid(np.arange(N) - (N - 1) / 2, (N - 1) / 2 - np.arange(N))
    D = (jj ** 2 + ii ** 2 <= (N / 2) ** 2).astype(float)
    WD = oracle.forward(g, D)
    # exact disc data: the fit recovers the grey value and leaves nothing
    gv, pd, Do = oracle.disc(g, 0.7 * WD)
    assert np.array_equal(Do, D)
    assert abs(gv - 0.7) < 1e-12 and np.abs(pd).max() < 1e-10
    # general data: the derivative of sum_a (P_a - g T_a)^2 vanishes at g
    rng = np.random.default_rng(4)
    p = rng.uniform(0, 5, size=(na, nd))
    gv, pd, _ = oracle.disc(g, p)
    P, T = p.sum(1), WD.sum(1)
    assert abs(np.dot(T, P - gv * T)) < 1e-9 * np.dot(T, T)
    assert np.allclose(pd, p - gv * WD, atol=1e-12)


def _method_matrix(N, na, nd, box, p, u, n, alpha, shift, lo, hi):
    W = _hat_matrix(N, na, nd, rect=box)
    x0, y0, w, h = box
    y = np.zeros(w * h)
    x = np.zeros(w * h)
    sh = shift.ravel()
    for k in range(1, n + 1):
        cp = np.stack([np.convolve(p[a], u[k - 1, a])[nd - 1:2 * nd - 1] for a in range(na)]).ravel()
        xs = W.T @ cp
        s = xs + y - alpha * (W.T @ (W @ y))
        x = np.clip(s + sh, lo, hi) - sh
        y = x - xs
    return (x + sh).reshape(h, w)


@pytest.mark.parametrize("lo,hi", [(0.0, np.inf), (-np.inf, np.inf), (0.02, 0.3)])
def test_local_method_matches_explicit_recursion(lo, hi):
    N, na, nd, n = 10, 6, 13, 5
    g = oracle.Geometry(N, na, nd)
    alpha = 1.0 / (na * nd)
    rng = np.random.default_rng(5)
    x_true = rng.uniform(0, 1, size=(N, N))
    p = oracle.forward(g, x_true) + 0.01 * rng.normal(size=(na, nd))
    u = oracle.filtcalc(g, n)
    box = (2, 3, 5, 4)
    shift = rng.uniform(-0.1, 0.1, size=(4, 5))
    got = oracle.filter_method(g, box, p, u, shift=shift, lo=lo, hi=hi)
    ref = _method_matrix(N, na, nd, box, p, u, n, alpha, shift, lo, hi)
    assert np.allclose(got, ref, atol=1e-12)


def test_unconstrained_method_is_local_fbp_with_the_last_filter():
    """With no prior (d = 0) y stays 0 and x^n = W_L^T C_{u_n} p (Eq. locsirtapp)."""
    N, na, nd, n = 12, 8, 15, 4
    g = oracle.Geometry(N, na, nd)
    rng = np.random.default_rng(6)
    p = rng.normal(size=(na, nd))
    u = oracle.filtcalc(g, n)
    box = (3, 2, 6, 7)
    x = oracle.filter_method(g, box, p, u, lo=-np.inf, hi=np.inf)
    ref = oracle.back(g, oracle.filter_conv(g, u[n - 1], p), rect=box)
    assert np.allclose(x, ref, atol=1e-13)


@pytest.mark.parametrize("N,nd", [(64, 64), (64, 65)])
def test_filtered_backprojection_approximates_sirt(N, nd):
    """Eq. sfbp: FBP with the filter u_n approximates n unconstrained SIRT iterations on the
    whole grid.  It is an approximation (W^T W is only nearly shift-invariant; measured
    8-11 % relative L2 inside the disk at these sizes), so the bound is loose; a filter
    sampled half a bin off, or scaled wrongly, gives 30 % and more."""
    na, n = 96, 100
    g = oracle.Geometry(N, na, nd)
    ph = synth.random_phantom(N, 8, texture=False, seed=8)
    p = synth.analytic_sinogram(ph, na, nd)
    u = oracle.filtcalc(g, n)
    x_f = oracle.back(g, oracle.filter_conv(g, u[n - 1], p))
    x_s = oracle.sirt(g, (0, 0, N, N), p, n, nonneg=0)
    jj, ii = np.meshgrid(np.arange(N) - (N - 1) / 2, (N - 1) / 2 - np.arange(N))
    m = jj ** 2 + ii ** 2 <= (N / 2 - 2) ** 2
    rel = np.linalg.norm((x_f - x_s)[m]) / np.linalg.norm(x_s[m])
    assert rel < 0.15, rel
