"""Pins of the oracle's FGP (TV denoising by the fast gradient projection) and of Alg.
methodfista (the paper's method with FISTA and TV): FGP against an independent ADMM solver
of the same denoising problem and against its first iterations written with explicit
difference matrices; Alg. methodfista against the same recursion written with explicit
matrices and a numpy FGP."""
import math

import numpy as np
import pytest

import oracle
from test_oracle_pins import _admm_tv, _grad_matrix, _hat_matrix


def _tv(x):
    gx = np.zeros_like(x)
    gy = np.zeros_like(x)
    gx[:, :-1] = x[:, 1:] - x[:, :-1]
    gy[:-1, :] = x[1:, :] - x[:-1, :]
    return float(np.hypot(gx, gy).sum())


def test_fgp_solves_tv_denoising():
    """FGP's fixed point minimises ||x - z||^2 + 2 lam TV(x): same objective as ADMM."""
    rng = np.random.default_rng(11)
    h, w, lam = 6, 7, 0.15
    z = rng.uniform(0, 1, size=(h, w))
    x = oracle.fgp(z, lam, 4000)
    xa = _admm_tv(np.eye(h * w), z.ravel(), 2 * lam, h, w, iters=20000).reshape(h, w)
    f = lambda v: float(np.sum((v - z) ** 2) + 2 * lam * _tv(v))
    assert abs(f(x) - f(xa)) <= 1e-8 * f(xa)
    assert np.abs(x - xa).max() < 1e-4


def _fgp_matrix(z, lam, iters):
    """The same iteration with explicit difference matrices (grad = [Dx; Dy], div = -grad^T)."""
    h, w = z.shape
    Dx, Dy = _grad_matrix(h, w)
    zf = z.ravel()
    n = h * w
    vx = np.zeros(n)
    vy = np.zeros(n)
    rx = np.zeros(n)
    ry = np.zeros(n)
    t = 1.0
    for _ in range(iters):
        x = zf - lam * (Dx.T @ rx + Dy.T @ ry)
        ax = rx + (Dx @ x) / (8 * lam)
        ay = ry + (Dy @ x) / (8 * lam)
        m = np.maximum(1.0, np.hypot(ax, ay))
        ax, ay = ax / m, ay / m
        tn = 0.5 * (1 + math.sqrt(1 + 4 * t * t))
        rx = ax + (t - 1) / tn * (ax - vx)
        ry = ay + (t - 1) / tn * (ay - vy)
        vx, vy, t = ax, ay, tn
    return (zf - lam * (Dx.T @ vx + Dy.T @ vy)).reshape(h, w)


@pytest.mark.parametrize("iters", [1, 2, 7])
def test_fgp_iterations_match_explicit_matrices(iters):
    rng = np.random.default_rng(12)
    z = rng.uniform(-1, 1, size=(5, 6))
    assert np.allclose(oracle.fgp(z, 0.3, iters), _fgp_matrix(z, 0.3, iters), atol=1e-13)


def test_fgp_without_regularisation_is_identity():
    z = np.random.default_rng(13).normal(size=(4, 5))
    assert np.array_equal(oracle.fgp(z, 0.0, 10), z)


def test_local_fista_matches_explicit_recursion():
    N, na, nd, n, nf, lam = 10, 6, 13, 5, 6, 40.0
    g = oracle.Geometry(N, na, nd)
    alpha = 1.0 / (na * nd)
    rng = np.random.default_rng(14)
    p = oracle.forward(g, rng.uniform(0, 1, size=(N, N))) + 0.01 * rng.normal(size=(na, nd))
    u = oracle.filtcalc(g, n)
    box = (2, 3, 5, 4)
    shift = rng.uniform(-0.1, 0.1, size=(4, 5))
    got = oracle.filter_fista(g, box, p, u, lam, n_fgp=nf, shift=shift)
    W = _hat_matrix(N, na, nd, rect=box)
    xl = np.zeros(20)
    xprev = np.zeros(20)
    t = 1.0
    for k in range(1, n + 1):
        cp = np.stack([np.convolve(p[a], u[k - 1, a])[nd - 1:2 * nd - 1] for a in range(na)]).ravel()
        xs = W.T @ cp
        z = xs + xl - alpha * (W.T @ (W @ xl)) + shift.ravel()
        xk = _fgp_matrix(z.reshape(4, 5), 0.5 * alpha * lam, nf).ravel() - shift.ravel()
        tn = 0.5 * (1 + math.sqrt(1 + 4 * t * t))
        r = xk + (t - 1) / tn * (xk - xprev)
        xl = r - xs
        xprev, t = xk, tn
    ref = (xprev + shift.ravel()).reshape(4, 5)
    assert np.allclose(got, ref, atol=1e-12)
