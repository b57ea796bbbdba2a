"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module draws phantoms and measurement noise. It holds none of the
reconstruction arithmetic (no projector, filter or solver): it produces the
sinogram ``p`` and a ground-truth image that both the CUDA library and the CPU
oracle receive as plain arrays.

Geometry conventions (parallel beam, single rotation axis; paper Sec. 2.1):

* image: ``N x N`` pixels, pixel (i, j) = (row from the top, column) has its
  centre at world coordinates ``(j - (N-1)/2, (N-1)/2 - i)``;
* detector: ``n_det`` unit-width bins with centres ``t_d = d - (n_det-1)/2``;
* angles: ``theta_a = a * pi / n_angles`` (``[0, pi)``);
* a ray at angle theta and offset t is the line ``x cos(theta) + y sin(theta) = t``.

Phantoms are sums of ellipses and Gaussian blobs whose line integrals are known in
closed form, so the sinogram is computed analytically rather than by projecting a
pixel image (no inverse crime).  This stands in for the paper's high-resolution
phantom that is resampled to the detector (Sec. 4); the paper's own phantoms and
its experimental data set are not used.

Noise follows the paper's description (Sec. 4): line integrals are mapped to
photon counts with the largest count equal to ``I0``, each count is redrawn from a
Poisson distribution with that mean, and the counts are mapped back.  The
attenuation scale the paper leaves open is ``mu = 1 / max(p)``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Phantom",
    "default_angles",
    "random_phantom",
    "analytic_sinogram",
    "rasterize",
    "poisson_noise",
    "random_roi_centre",
]


def default_angles(n_angles: int) -> np.ndarray:
    """Equally spaced angles ``a*pi/n_angles`` in ``[0, pi)`` (float64)."""
    return np.arange(n_angles, dtype=np.float64) * (math.pi / n_angles)


@dataclasses.dataclass
class Phantom:
    """Analytic phantom: additive ellipses and Gaussian blobs (world units = pixels)."""

    # ellipses: centre (x0, y0), semi-axes (a, b), rotation phi of the a-axis, density rho
    ex0: np.ndarray
    ey0: np.ndarray
    ea: np.ndarray
    eb: np.ndarray
    ephi: np.ndarray
    erho: np.ndarray
    # Gaussian blobs: centre, standard deviation, peak value
    bx0: np.ndarray
    by0: np.ndarray
    bsig: np.ndarray
    brho: np.ndarray


def random_phantom(N: int, n_ellipses: int, texture: bool = False, seed: int = 0) -> Phantom:
    """Random ellipse phantom sized for an ``N x N`` grid.

    Semi-axes are U[5, 40] px at N = 128 and scale with N/128; each ellipse's
    centre is uniform in the disk of radius ``N/2 - max(a, b)`` so that every
    ellipse stays inside the inscribed disk (and hence inside the detector's
    field of view when ``n_det >= N``); rotation U[0, pi); density U[0, 1].
    With ``texture`` True, N/2 Gaussian blobs with sigma U[1, 3] px and peak
    U[0, 0.05] are added (fine texture of about 5 % contrast).
    """
    rng = np.random.default_rng(seed)
    scale = N / 128.0
    a = rng.uniform(5.0, 40.0, n_ellipses) * scale
    b = rng.uniform(5.0, 40.0, n_ellipses) * scale
    rmax = N / 2.0 - np.maximum(a, b)
    rmax = np.maximum(rmax, 0.0)
    rad = rmax * np.sqrt(rng.uniform(0.0, 1.0, n_ellipses))
    ang = rng.uniform(0.0, 2.0 * math.pi, n_ellipses)
    ex0 = rad * np.cos(ang)
    ey0 = rad * np.sin(ang)
    phi = rng.uniform(0.0, math.pi, n_ellipses)
    rho = rng.uniform(0.0, 1.0, n_ellipses)
    if texture:
        nb = N // 2
        sig = rng.uniform(1.0, 3.0, nb)
        brad = (N / 2.0 - 3.0 * sig) * np.sqrt(rng.uniform(0.0, 1.0, nb))
        bang = rng.uniform(0.0, 2.0 * math.pi, nb)
        bx0 = brad * np.cos(bang)
        by0 = brad * np.sin(bang)
        brho = rng.uniform(0.0, 0.05, nb)
    else:
        sig = bx0 = by0 = brho = np.zeros(0)
    return Phantom(ex0, ey0, a, b, phi, rho, bx0, by0, sig, brho)


def analytic_sinogram(ph: Phantom, n_angles: int, n_det: int, angles=None) -> np.ndarray:
    """Exact line integrals of the phantom, float64 ``[n_angles][n_det]``.

    Ellipse (textbook): with ``a2(theta) = A^2 cos^2(theta-phi) + B^2 sin^2(theta-phi)``
    and ``t' = t - x0 cos(theta) - y0 sin(theta)``, the integral is
    ``2 rho A B sqrt(a2 - t'^2) / a2`` for ``t'^2 <= a2`` and 0 otherwise.
    Gaussian blob: ``rho sqrt(2 pi) sigma exp(-t'^2 / (2 sigma^2))``.
    """
    th = default_angles(n_angles) if angles is None else np.asarray(angles, np.float64)
    t = np.arange(n_det, dtype=np.float64) - (n_det - 1) / 2.0
    c = np.cos(th)[:, None]
    s = np.sin(th)[:, None]
    p = np.zeros((th.size, n_det), np.float64)
    for k in range(ph.ea.size):
        tp = t[None, :] - ph.ex0[k] * c - ph.ey0[k] * s
        a2 = (ph.ea[k] * np.cos(th - ph.ephi[k])) ** 2 + (ph.eb[k] * np.sin(th - ph.ephi[k])) ** 2
        a2 = a2[:, None]
        inside = tp * tp <= a2
        val = 2.0 * ph.erho[k] * ph.ea[k] * ph.eb[k] * np.sqrt(np.where(inside, a2 - tp * tp, 0.0)) / a2
        p += np.where(inside, val, 0.0)
    for k in range(ph.bsig.size):
        tp = t[None, :] - ph.bx0[k] * c - ph.by0[k] * s
        p += ph.brho[k] * math.sqrt(2.0 * math.pi) * ph.bsig[k] * np.exp(-tp * tp / (2.0 * ph.bsig[k] ** 2))
    return p


def rasterize(ph: Phantom, N: int, supersample: int = 4) -> np.ndarray:
    """Ground-truth ``N x N`` image: the phantom averaged over ``supersample^2`` points per pixel."""
    ss = supersample
    off = (np.arange(ss) + 0.5) / ss - 0.5
    img = np.zeros((N, N), np.float64)
    jj = np.arange(N, dtype=np.float64) - (N - 1) / 2.0
    ii = (N - 1) / 2.0 - np.arange(N, dtype=np.float64)
    for oy in off:
        for ox in off:
            X = (jj + ox)[None, :]
            Y = (ii - oy)[:, None]
            acc = np.zeros((N, N))
            for k in range(ph.ea.size):
                dx = X - ph.ex0[k]
                dy = Y - ph.ey0[k]
                cp, sp = math.cos(ph.ephi[k]), math.sin(ph.ephi[k])
                u = dx * cp + dy * sp
                v = -dx * sp + dy * cp
                acc += np.where((u / ph.ea[k]) ** 2 + (v / ph.eb[k]) ** 2 <= 1.0, ph.erho[k], 0.0)
            for k in range(ph.bsig.size):
                r2 = (X - ph.bx0[k]) ** 2 + (Y - ph.by0[k]) ** 2
                acc += ph.brho[k] * np.exp(-r2 / (2.0 * ph.bsig[k] ** 2))
            img += acc
    return img / (ss * ss)


def poisson_noise(p: np.ndarray, I0: float, seed: int = 0) -> np.ndarray:
    """Poisson-noisy line integrals (paper Sec. 4 noise model).

    Counts ``c ~ Poisson(I0 exp(-mu p))`` with ``mu = 1/max(p)`` (so the largest
    expected count, at p = 0, is I0), then ``p_noisy = -ln(max(c, 1)/I0)/mu``.
    ``I0 <= 0`` returns a copy of ``p`` (noise-free).
    """
    p = np.asarray(p, np.float64)
    if I0 <= 0:
        return p.copy()
    pmax = float(p.max())
    mu = 1.0 / pmax if pmax > 0 else 1.0
    rng = np.random.default_rng(seed)
    counts = rng.poisson(I0 * np.exp(-mu * p)).astype(np.float64)
    return -np.log(np.maximum(counts, 1.0) / I0) / mu


def random_roi_centre(N: int, radius: float, margin: float, seed: int = 0):
    """Seeded ROI centre (column, row) in pixel-index units whose extended box lies inside the grid."""
    rng = np.random.default_rng(seed)
    R = math.ceil(radius + margin)
    lo = R
    hi = N - R
    if hi <= lo:
        return ((N - 1) / 2.0, (N - 1) / 2.0)
    return (float(rng.integers(lo, hi + 1)), float(rng.integers(lo, hi + 1)))
