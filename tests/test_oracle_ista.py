"""Pins of the oracle's Haar-wavelet ISTA inside the paper's method (Eq. sirtista with the
recursion of Alg. method): the Haar decomposition against closed forms and an independent
matrix construction, its orthogonality, and the whole recursion against explicit matrices."""
import math

import numpy as np
import pytest

import oracle
from test_oracle_pins import _hat_matrix


def _split_matrix(L):
    """Pair sums / differences over sqrt(2), sums first, an odd last entry carried as a sum."""
    S = np.zeros((L, L))
    m, c = L // 2, (L + 1) // 2
    s = 1 / math.sqrt(2)
    for j in range(m):
        S[j, 2 * j], S[j, 2 * j + 1] = s, s
        S[c + j, 2 * j], S[c + j, 2 * j + 1] = s, -s
    if L % 2:
        S[m, L - 1] = 1.0
    return S


def _haar_matrix_apply(x, levels=32):
    c = x.copy()
    h, w = c.shape
    hl, wl, n = h, w, 0
    while n < levels and hl >= 2 and wl >= 2:
        blk = c[:hl, :wl]
        c[:hl, :wl] = _split_matrix(hl) @ blk @ _split_matrix(wl).T
        hl, wl, n = (hl + 1) // 2, (wl + 1) // 2, n + 1
    return c


@pytest.mark.parametrize("shape", [(8, 8), (7, 10), (5, 3), (1, 6), (12, 9)])
def test_haar_matches_matrix_construction_and_is_orthogonal(shape):
    rng = np.random.default_rng(21)
    x = rng.normal(size=shape)
    c = oracle.haar(x)
    assert np.allclose(c, _haar_matrix_apply(x), atol=1e-13)
    assert abs(np.linalg.norm(c) - np.linalg.norm(x)) < 1e-12
    assert np.allclose(oracle.haar_inv(c), x, atol=1e-13)


def test_haar_two_by_two_closed_form():
    # one level: mean-like and difference coefficients of [[a, b], [c, d]]
    a, b, c, d = 1.0, 2.0, 3.0, 4.0
    got = oracle.haar(np.array([[a, b], [c, d]]))
    ref = np.array([[a + b + c + d, a - b + c - d], [a + b - c - d, a - b - c + d]]) / 2
    assert np.allclose(got, ref, atol=1e-15)


def test_haar_level_limit():
    x = np.random.default_rng(22).normal(size=(16, 16))
    assert np.allclose(oracle.haar(x, levels=1), _haar_matrix_apply(x, levels=1), atol=1e-13)


def test_local_ista_matches_explicit_recursion():
    N, na, nd, n, lam = 10, 6, 13, 5, 60.0
    g = oracle.Geometry(N, na, nd)
    alpha = 1.0 / (na * nd)
    rng = np.random.default_rng(23)
    p = oracle.forward(g, rng.uniform(0, 1, size=(N, N))) + 0.01 * rng.normal(size=(na, nd))
    u = oracle.filtcalc(g, n)
    box = (2, 3, 5, 4)
    shift = rng.uniform(-0.1, 0.1, size=(4, 5))
    got = oracle.filter_ista(g, box, p, u, lam, shift=shift)
    W = _hat_matrix(N, na, nd, rect=box)
    tau = 0.5 * alpha * lam
    y = np.zeros(20)
    x = np.zeros(20)
    for k in range(1, n + 1):
        cp = np.stack([np.convolve(p[a], u[k - 1, a])[nd - 1:2 * nd - 1] for a in range(na)]).ravel()
        xs = W.T @ cp
        z = (xs + y - alpha * (W.T @ (W @ y)) + shift.ravel()).reshape(4, 5)
        c = _haar_matrix_apply(z)
        c = np.sign(c) * np.maximum(np.abs(c) - tau, 0.0)
        # inverse of an orthogonal transform: apply the transposed steps in reverse order
        hl, wl, blocks = 4, 5, []
        while hl >= 2 and wl >= 2:
            blocks.append((hl, wl))
            hl, wl = (hl + 1) // 2, (wl + 1) // 2
        for hl, wl in reversed(blocks):
            c[:hl, :wl] = _split_matrix(hl).T @ c[:hl, :wl] @ _split_matrix(wl)
        x = c.ravel() - shift.ravel()
        y = x - xs
    assert np.allclose(got, (x + shift.ravel()).reshape(4, 5), atol=1e-12)
