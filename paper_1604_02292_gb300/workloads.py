"""Named synthetic workloads shaped like the paper's experiments (sizes only).

Each workload fixes the geometry, the phantom recipe, the noise level, the region
and the solver settings.  Inputs are drawn by ``synth`` from fixed seeds; the
paper's own phantoms and its experimental data are not used (they stand in for
them with the same grid sizes, detector counts, angle counts and noise model).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import synth


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    N: int
    n_angles: int
    n_det: int
    n_ellipses: int
    texture: bool
    I0: float
    radius: float
    margin: float
    reg: str            # "sirt" or "tv"
    iters: int
    lam: float = 0.0

    def geometry(self):
        return self.N, self.n_angles, self.n_det


WORKLOADS = {
    # 128 x 128, 64 angles in [0, pi), 128 unit bins, 10 ellipses, I0 = 1e4,
    # ROI radius 16 px + margin 8 px, Ram-Lak FBP then 200 nonnegative SIRT iterations
    "roi_sirt_128": Workload("roi_sirt_128", 128, 64, 128, 10, False, 1e4, 16.0, 8.0, "sirt", 200),
    # 1024 x 1024, 256 angles, 1024 bins, 50 ellipses + fine texture, I0 = 5e3,
    # ROI radius 64 px + margin 32 px, Chambolle-Pock TV lambda = 0.01, 500 iterations
    "roi_cptv_1024": Workload("roi_cptv_1024", 1024, 256, 1024, 50, True, 5e3, 64.0, 32.0, "tv", 500, 0.01),
    # the paper's own method on the 1024 geometry: ROI radius 64 px + margin 32 px, 200
    # iterations of nonnegative SIRT approximated by filtered backprojections (Sec. 3)
    "roi_filter_1024": Workload("roi_filter_1024", 1024, 256, 1024, 50, True, 5e3, 64.0, 32.0, "filter", 200),
    # tiling (Sec. 5.5) on the 1024 geometry: 64 tiles of 128 x 128 (radius 64 px), margin 16 px
    # (1/8 of the tile side, Sec. 3.3), the paper's method with x >= 0, 200 iterations, against
    # 200 nonnegative SIRT iterations on the whole grid
    "roi_tile_1024": Workload("roi_tile_1024", 1024, 256, 1024, 50, True, 5e3, 64.0, 16.0, "tile", 200),
}


@dataclasses.dataclass(frozen=True)
class BatchWorkload:
    """Many regions over one sinogram: centres on a jittered grid of cells, radii uniform,
    margin = radius / 2, SIRT or TV by a seeded coin."""
    name: str
    N: int
    n_angles: int
    n_det: int
    n_ellipses: int
    I0: float
    grid: int             # cells per side
    r_lo: float
    r_hi: float
    iters: int
    lam: float

    def geometry(self):
        return self.N, self.n_angles, self.n_det


BATCHES = {
    # 2048 x 2048, 180 angles, 2048 bins, 50 ellipses (noise-free); 4096 regions with centres
    # on a jittered 64 x 64 grid of 32 px cells, radius U[16, 128], margin r/2, SIRT/TV 50/50,
    # 200 iterations
    "roi_batch_2048": BatchWorkload("roi_batch_2048", 2048, 180, 2048, 50, 0.0, 64, 16.0, 128.0, 200, 0.01),
}


def batch_regions(w: BatchWorkload, seed: int = 0, count: int | None = None):
    """[(region, params)] for the batch: params dicts as taken by RoiRecon.solve_batch."""
    rng = np.random.default_rng(seed + 3000)
    cell = w.N / w.grid
    out = []
    for i in range(w.grid):
        for j in range(w.grid):
            cx = (j + 0.5) * cell + rng.uniform(-cell / 4, cell / 4)
            cy = (i + 0.5) * cell + rng.uniform(-cell / 4, cell / 4)
            r = float(rng.uniform(w.r_lo, w.r_hi))
            tv = bool(rng.integers(0, 2))
            prm = dict(reg=1 if tv else 0, iters=w.iters, lam=w.lam if tv else 0.0)
            out.append(((float(cx), float(cy), r, r / 2.0), prm))
    if count is not None:
        idx = rng.permutation(len(out))[:count]
        out = [out[k] for k in sorted(idx)]
    return out


def sinogram(w, seed: int = 0, noise: bool = True) -> np.ndarray:
    """Analytic sinogram of the seeded phantom, float32 [n_angles][n_det], with the
    workload's Poisson noise (noise=False: the noise-free line integrals)."""
    ph = synth.random_phantom(w.N, w.n_ellipses, texture=getattr(w, "texture", False), seed=seed)
    p = synth.analytic_sinogram(ph, w.n_angles, w.n_det)
    if noise:
        p = synth.poisson_noise(p, w.I0, seed=seed + 1000)
    return p.astype(np.float32)


def region(w: Workload, seed: int = 0, centred: bool = False):
    """(cx, cy, radius, margin); the extended box lies inside the grid."""
    if centred:
        c = (w.N - 1) / 2.0
        return (c, c, w.radius, w.margin)
    cx, cy = synth.random_roi_centre(w.N, w.radius, w.margin, seed=seed + 2000)
    return (cx, cy, w.radius, w.margin)


def box_side(w: Workload) -> int:
    return 2 * math.ceil(w.radius + w.margin)


@dataclasses.dataclass(frozen=True)
class ServeWorkload:
    """ROI requests over resident sinograms: Poisson arrivals, radius log-uniform, margin
    r / 2, centre uniform in the disk where the ROI lies inside the object, SIRT or TV by a
    seeded coin."""
    name: str
    N: int
    n_angles: int
    n_det: int
    n_ellipses: int
    I0: float
    n_sinos: int
    rate: float           # requests per second
    r_lo: float
    r_hi: float
    iters: int
    lam: float

    def geometry(self):
        return self.N, self.n_angles, self.n_det


SERVING = {
    # 8 resident 2048 x 2048 / 180-angle / 2048-bin sinograms (50 ellipses, noise-free);
    # requests at 2000 / s, radius log-uniform in [16, 256] px, margin r/2, SIRT/TV 50/50,
    # 200 iterations
    "roi_serve_2048": ServeWorkload("roi_serve_2048", 2048, 180, 2048, 50, 0.0, 8, 2000.0, 16.0, 256.0, 200, 0.01),
}


def serve_requests(w: ServeWorkload, seed: int = 0, count: int = 256, radii=None):
    """[(sino, region, params)] in arrival order; radii overrides the drawn radii."""
    rng = np.random.default_rng(seed + 5000)
    out = []
    for i in range(count):
        r = float(radii[i]) if radii is not None else float(np.exp(rng.uniform(math.log(w.r_lo), math.log(w.r_hi))))
        rho = (w.N / 2.0 - r) * math.sqrt(rng.uniform(0.0, 1.0))
        phi = rng.uniform(0.0, 2.0 * math.pi)
        c = (w.N - 1) / 2.0
        cx, cy = c + rho * math.cos(phi), c + rho * math.sin(phi)
        tv = bool(rng.integers(0, 2))
        prm = dict(reg=1 if tv else 0, iters=w.iters, lam=w.lam if tv else 0.0)
        out.append((int(rng.integers(0, w.n_sinos)), (cx, cy, r, r / 2.0), prm))
    return out


def arrivals(w: ServeWorkload, seed: int = 0, count: int = 256, rate: float | None = None) -> np.ndarray:
    """Poisson arrival times in seconds from 0 (exponential gaps at `rate`, default w.rate)."""
    rng = np.random.default_rng(seed + 6000)
    gaps = rng.exponential(1.0 / (rate or w.rate), size=count)
    gaps[0] = 0.0
    return np.cumsum(gaps)


@dataclasses.dataclass(frozen=True)
class PrecisionWorkload:
    """Large regions on a large grid with 16-bit storage: ROI centres uniform in the disk
    where the ROI lies inside the object, fixed radius and margin, TV by Chambolle-Pock."""
    name: str
    N: int
    n_angles: int
    n_det: int
    n_ellipses: int
    texture: bool
    I0: float
    count: int
    radius: float
    margin: float
    iters: int
    lam: float

    def geometry(self):
        return self.N, self.n_angles, self.n_det


PRECISION = {
    # 4096 x 4096, 1024 angles, 4096 bins, 50 ellipses, I0 = 1e3; 256 regions of radius 256 px,
    # margin 128 px (box 768 x 768), CP-TV lambda = 0.01, 200 iterations
    "roi_precision_4096": PrecisionWorkload("roi_precision_4096", 4096, 1024, 4096, 50, False, 1e3, 256, 256.0,
                                            128.0, 200, 0.01),
}


def precision_regions(w: PrecisionWorkload, seed: int = 0, count: int | None = None):
    """[(region, params)] of the precision workload (the first `count`)."""
    rng = np.random.default_rng(seed + 7000)
    out = []
    c = (w.N - 1) / 2.0
    for _ in range(w.count if count is None else count):
        rho = (w.N / 2.0 - w.radius) * math.sqrt(rng.uniform(0.0, 1.0))
        phi = rng.uniform(0.0, 2.0 * math.pi)
        out.append(((c + rho * math.cos(phi), c + rho * math.sin(phi), w.radius, w.margin),
                    dict(reg=1, iters=w.iters, lam=w.lam)))
    return out
