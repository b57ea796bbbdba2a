"""FP64 CPU oracle for local ROI reconstruction -- TEST INFRASTRUCTURE ONLY.

Thin ctypes binding over ``roi_oracle.c`` (plain C, FP64).  Only the tests, the
smoke check and the benchmark's CPU-baseline leg may import this package; the
CUDA library and its Python binding never do.  Nothing here is shared with the
CUDA path.

The C source states which passage of Pelt & Batenburg (arXiv 1604.02292) each
function follows.  ``build()`` compiles it with gcc (``-O2 -fopenmp
-ffp-contract=off``, so x86 and Arm hosts round identically); the library is
compiled on first use if missing or older than its source.

All images are float64 row-major ``[h][w]`` on a rectangle ``(x0, y0, w, h)`` of
the ``N x N`` grid; sinograms are float64 ``[n_angles][n_det]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "roi_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_lib/liboracle.so`` (gcc, FP64, OpenMP)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i7 = [_I] * 4
            lib.orc_forward.argtypes = [_I, _I, _I, _D] + i7 + [_D] + i7 + [_D]
            lib.orc_back.argtypes = [_I, _I, _I, _D] + i7 + i7 + [_D, _D]
            lib.orc_ramp.argtypes = [_I, _I, _D, _D]
            lib.orc_fbp.argtypes = [_I, _I, _I, _D, _D, _D]
            lib.orc_exterior.argtypes = [_I, _I, _I, _D] + i7 + [_D, _D, _D]
            lib.orc_fov.argtypes = [_I, _I, _D]
            lib.orc_rowcol_sums.argtypes = [_I, _I, _I, _D] + i7 + [_D, _D]
            lib.orc_sirt.argtypes = [_I, _I, _I, _D] + i7 + [_D, _I, ctypes.c_double, _I, _I, _D]
            lib.orc_cp.argtypes = [_I, _I, _I, _D] + i7 + [_D, _I, ctypes.c_double, _I, ctypes.c_double, _D]
            lib.orc_objective.argtypes = [_I, _I, _I, _D] + i7 + [_D, _D, ctypes.c_double]
            lib.orc_objective.restype = ctypes.c_double
            lib.orc_power_norm.argtypes = [_I, _I, _I, _D] + i7 + [_I]
            lib.orc_power_norm.restype = ctypes.c_double
            lib.orc_filtcalc.argtypes = [_I, _I, _I, _D, _I, ctypes.c_double, _D]
            lib.orc_filter_conv.argtypes = [_I, _I, _D, _D, _D]
            lib.orc_disc.argtypes = [_I, _I, _I, _D, _D, _D, _D]
            lib.orc_disc.restype = ctypes.c_double
            lib.orc_filter_method.argtypes = [_I, _I, _I, _D] + i7 + [_D, _I, ctypes.c_double, _D, _D,
                                                                      ctypes.c_double, ctypes.c_double, _D]
            lib.orc_fgp.argtypes = [_I, _I, _D, ctypes.c_double, _I, _D]
            lib.orc_filter_fista.argtypes = [_I, _I, _I, _D] + i7 + [_D, _I, ctypes.c_double, _D, _D,
                                                                     ctypes.c_double, _I, _D]
            lib.orc_haar.argtypes = [_I, _I, _I, _D, _D]
            lib.orc_haar_inv.argtypes = [_I, _I, _I, _D, _D]
            lib.orc_filter_ista.argtypes = [_I, _I, _I, _D] + i7 + [_D, _I, ctypes.c_double, _D, _D,
                                                                    ctypes.c_double, _I, _D]
            lib.orc_grad.argtypes = [_I, _I, _D, _D, _D]
            lib.orc_div.argtypes = [_I, _I, _D, _D, _D]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Geometry:
    """Parallel-beam geometry: N x N grid, n_det unit bins, angles in radians."""

    def __init__(self, N: int, n_angles: int, n_det: int, angles=None):
        self.N, self.na, self.nd = int(N), int(n_angles), int(n_det)
        if angles is None:
            angles = np.arange(self.na, dtype=np.float64) * (np.pi / self.na)
        self.angles = _f64(angles)
        assert self.angles.shape == (self.na,)

    def _g(self):
        return (self.N, self.na, self.nd, _p(self.angles))


def _rect(r):
    if r is None:
        return (0, 0, 0, 0)
    x0, y0, w, h = (int(v) for v in r)
    return (x0, y0, w, h)


def forward(g: Geometry, img, rect=None, hole=None) -> np.ndarray:
    """W applied to an image given on ``rect`` (whole grid if None), pixels in ``hole`` zeroed."""
    rect = (0, 0, g.N, g.N) if rect is None else _rect(rect)
    img = _f64(img).reshape(rect[3], rect[2])
    out = np.empty((g.na, g.nd), np.float64)
    _load().orc_forward(*g._g(), *rect, _p(img), *_rect(hole), _p(out))
    return out


def back(g: Geometry, sino, rect=None, hole=None) -> np.ndarray:
    """W^T evaluated on the pixels of ``rect`` (whole grid if None); pixels in ``hole`` are 0."""
    rect = (0, 0, g.N, g.N) if rect is None else _rect(rect)
    sino = _f64(sino).reshape(g.na, g.nd)
    out = np.empty((rect[3], rect[2]), np.float64)
    _load().orc_back(*g._g(), *rect, *_rect(hole), _p(sino), _p(out))
    return out


def ramp(g: Geometry, p) -> np.ndarray:
    """Ram-Lak row filter scaled by pi/n_angles (linear convolution)."""
    p = _f64(p).reshape(g.na, g.nd)
    out = np.empty_like(p)
    _load().orc_ramp(g.na, g.nd, _p(p), _p(out))
    return out


def fbp(g: Geometry, p) -> np.ndarray:
    """Global FBP W^T C_h p on the N x N grid."""
    p = _f64(p).reshape(g.na, g.nd)
    out = np.empty((g.N, g.N), np.float64)
    _load().orc_fbp(*g._g(), _p(p), _p(out))
    return out


def fov(g: Geometry, x) -> np.ndarray:
    """x (N x N) with the pixels outside the field of view -- centre farther than
    min(N, N_d)/2 from the rotation axis -- set to 0 (a copy)."""
    x = _f64(x).reshape(g.N, g.N).copy()
    _load().orc_fov(g.N, g.nd, _p(x))
    return x


def exterior(g: Geometry, box, p, xfbp) -> np.ndarray:
    """p' = p - W M_F M_V x_fbp over the whole sinogram (M_V: the field of view, see fov)."""
    p = _f64(p).reshape(g.na, g.nd)
    xfbp = _f64(xfbp).reshape(g.N, g.N)
    out = np.empty_like(p)
    _load().orc_exterior(*g._g(), *_rect(box), _p(p), _p(xfbp), _p(out))
    return out


def rowcol_sums(g: Geometry, box):
    """(W_L 1 as [n_angles][n_det], W_L^T 1 as [h][w])."""
    b = _rect(box)
    rows = np.empty((g.na, g.nd), np.float64)
    cols = np.empty((b[3], b[2]), np.float64)
    _load().orc_rowcol_sums(*g._g(), *b, _p(rows), _p(cols))
    return rows, cols


def sirt(g: Geometry, box, pprime, iters: int, alpha=None, weighting: int = 0, nonneg: int = 1) -> np.ndarray:
    """Local SIRT on the box from x^0 = 0; alpha defaults to 1/(n_angles n_det)."""
    b = _rect(box)
    if alpha is None:
        alpha = 1.0 / (g.na * g.nd)
    pp = _f64(pprime).reshape(g.na, g.nd)
    x = np.empty((b[3], b[2]), np.float64)
    _load().orc_sirt(*g._g(), *b, _p(pp), int(iters), float(alpha), int(weighting), int(nonneg), _p(x))
    return x


def power_norm(g: Geometry, box, iters: int = 100) -> float:
    """||[W_L; grad]||_2 by power iteration from the all-ones image."""
    return float(_load().orc_power_norm(*g._g(), *_rect(box), int(iters)))


def cp_tv(g: Geometry, box, pprime, iters: int, lam: float, precond: int = 1, L=None) -> np.ndarray:
    """Chambolle-Pock TV on the box (preconditioned, or scalar steps 0.99/L)."""
    b = _rect(box)
    pp = _f64(pprime).reshape(g.na, g.nd)
    if not precond and L is None:
        L = power_norm(g, box)
    x = np.empty((b[3], b[2]), np.float64)
    _load().orc_cp(*g._g(), *b, _p(pp), int(iters), float(lam), int(precond), float(L or 0.0), _p(x))
    return x


def objective(g: Geometry, box, pprime, x, lam: float) -> float:
    """||W_L x - p'||^2 (rays reaching the box) + lam * isotropic TV(x)."""
    b = _rect(box)
    pp = _f64(pprime).reshape(g.na, g.nd)
    xx = _f64(x).reshape(b[3], b[2])
    return float(_load().orc_objective(*g._g(), *b, _p(pp), _p(xx), float(lam)))


def grad(x):
    """Forward differences (gx, gy) with a zero last difference."""
    x = _f64(x)
    h, w = x.shape
    gx = np.empty_like(x)
    gy = np.empty_like(x)
    _load().orc_grad(w, h, _p(x), _p(gx), _p(gy))
    return gx, gy


def div(vx, vy):
    """Divergence, the negative adjoint of ``grad``."""
    vx = _f64(vx)
    vy = _f64(vy)
    h, w = vx.shape
    out = np.empty_like(vx)
    _load().orc_div(w, h, _p(vx), _p(vy), _p(out))
    return out


def roi_box(N: int, cx: float, cy: float, radius: float, margin: float):
    """Extended ROI box (x0, y0, w, h): the 2R x 2R pixels, R = ceil(radius + margin),
    whose centre indices lie nearest to [c - R, c + R), clipped to the grid
    (Sec. 3.3 pads the local part by a margin; the box is the local part L)."""
    import math

    R = math.ceil(radius + margin)
    x0 = math.floor(cx - R + 0.5)
    y0 = math.floor(cy - R + 0.5)
    x1, y1 = x0 + 2 * R, y0 + 2 * R
    x0, y0 = max(x0, 0), max(y0, 0)
    x1, y1 = min(x1, N), min(y1, N)
    return (x0, y0, max(x1 - x0, 0), max(y1 - y0, 0))


def solve_local(g: Geometry, p, region, reg: str = "sirt", iters: int = 200, lam: float = 0.0,
                weighting: int = 0, precond: int = 1, xfbp=None):
    """The whole local pipeline: FBP -> exterior subtraction -> local solve.

    ``region`` = (cx, cy, radius, margin) in pixel-index units.  Returns
    ``(x_box, box, pprime, xfbp)``.
    """
    box = roi_box(g.N, *region)
    if xfbp is None:
        xfbp = fbp(g, p)
    pp = exterior(g, box, p, xfbp)
    if reg == "sirt":
        x = sirt(g, box, pp, iters, weighting=weighting)
    else:
        x = cp_tv(g, box, pp, iters, lam, precond=precond)
    return x, box, pp, xfbp


# ---- the paper's own local method (Sec. 3) ------------------------------------------

def filtcalc(g: Geometry, n: int, alpha=None) -> np.ndarray:
    """Alg. filtcalc: filters u_k = alpha W' q_k, k = 1..n, [n][n_angles][2 n_det - 1]
    (tap m at index m + n_det - 1)."""
    alpha = 1.0 / (g.na * g.nd) if alpha is None else float(alpha)
    out = np.empty((int(n), g.na, 2 * g.nd - 1), np.float64)
    _load().orc_filtcalc(*g._g(), int(n), alpha, _p(out))
    return out


def filter_conv(g: Geometry, uk, p) -> np.ndarray:
    """C_{u_k} p: per-angle linear convolution of the sinogram with filter uk [n_angles][2 n_det - 1]."""
    uk = _f64(uk).reshape(g.na, 2 * g.nd - 1)
    p = _f64(p).reshape(g.na, g.nd)
    out = np.empty_like(p)
    _load().orc_filter_conv(g.na, g.nd, _p(uk), _p(p), _p(out))
    return out


def disc(g: Geometry, p):
    """Disc subtraction (Sec. 3.3): (grey value, p - g W D, D)."""
    p = _f64(p).reshape(g.na, g.nd)
    pd = np.empty_like(p)
    D = np.empty((g.N, g.N), np.float64)
    gv = _load().orc_disc(*g._g(), _p(p), _p(pd), _p(D))
    return gv, pd, D


def filter_method(g: Geometry, box, p, u, n=None, alpha=None, shift=None, lo=0.0, hi=np.inf) -> np.ndarray:
    """Alg. method with the box constraint [lo, hi] on the local part ``box``; ``p`` is the
    (disc-subtracted) sinogram, ``u`` the filters of ``filtcalc``, ``shift`` the image added
    back after reconstruction (box-shaped, or None)."""
    alpha = 1.0 / (g.na * g.nd) if alpha is None else float(alpha)
    n = u.shape[0] if n is None else int(n)
    box = _rect(box)
    p = _f64(p).reshape(g.na, g.nd)
    u = _f64(u)
    x = np.empty((box[3], box[2]), np.float64)
    sh = None if shift is None else _f64(shift).reshape(box[3], box[2])
    _load().orc_filter_method(*g._g(), *box, _p(p), n, alpha, _p(u), _p(sh) if sh is not None else None,
                              float(lo), float(hi), _p(x))
    return x


def filter_solve(g: Geometry, p, region, iters: int, u=None, nonneg: bool = True):
    """The paper's local method end to end: disc subtraction, filters, Alg. method with
    x >= 0 (or no constraint), the disc added back on the box.  Returns (x_box, box)."""
    box = roi_box(g.N, *region)
    gv, pd, D = disc(g, p)
    if u is None:
        u = filtcalc(g, iters)
    x0, y0, w, h = box
    shift = gv * D[y0:y0 + h, x0:x0 + w]
    x = filter_method(g, box, pd, u, n=iters, shift=shift, lo=0.0 if nonneg else -np.inf)
    return x, box


def fgp(z, lam: float, iters: int) -> np.ndarray:
    """FGP for min ||x - z||^2 + 2 lam TV(x) (isotropic, forward differences)."""
    z = _f64(z)
    h, w = z.shape
    x = np.empty_like(z)
    _load().orc_fgp(w, h, _p(z), float(lam), int(iters), _p(x))
    return x


def filter_fista(g: Geometry, box, p, u, lam: float, n_fgp: int = 100, n=None, alpha=None, shift=None):
    """Alg. methodfista on the local part ``box``: FISTA for ||p - Wx||^2 + lam TV(x) with the
    SIRT step approximated by the filters ``u`` and the TV prox by FGP."""
    alpha = 1.0 / (g.na * g.nd) if alpha is None else float(alpha)
    n = u.shape[0] if n is None else int(n)
    box = _rect(box)
    p = _f64(p).reshape(g.na, g.nd)
    u = _f64(u)
    x = np.empty((box[3], box[2]), np.float64)
    sh = None if shift is None else _f64(shift).reshape(box[3], box[2])
    _load().orc_filter_fista(*g._g(), *box, _p(p), n, alpha, _p(u), _p(sh) if sh is not None else None,
                             float(lam), int(n_fgp), _p(x))
    return x


def filter_fista_solve(g: Geometry, p, region, iters: int, lam: float, n_fgp: int = 100, u=None):
    """Alg. methodfista end to end: disc subtraction, filters, FISTA-TV on the box, disc added
    back.  Returns (x_box, box)."""
    box = roi_box(g.N, *region)
    gv, pd, D = disc(g, p)
    if u is None:
        u = filtcalc(g, iters)
    x0, y0, w, h = box
    shift = gv * D[y0:y0 + h, x0:x0 + w]
    return filter_fista(g, box, pd, u, lam, n_fgp=n_fgp, n=iters, shift=shift), box


def haar(x, levels: int = 32) -> np.ndarray:
    """Orthonormal 2D Haar decomposition (see orc_haar)."""
    x = _f64(x)
    h, w = x.shape
    out = np.empty_like(x)
    _load().orc_haar(w, h, int(levels), _p(x), _p(out))
    return out


def haar_inv(c, levels: int = 32) -> np.ndarray:
    c = _f64(c)
    h, w = c.shape
    out = np.empty_like(c)
    _load().orc_haar_inv(w, h, int(levels), _p(c), _p(out))
    return out


def filter_ista(g: Geometry, box, p, u, lam: float, levels: int = 32, n=None, alpha=None, shift=None):
    """Alg. method with the Haar-ISTA prior (Eq. sirtista) on the local part ``box``."""
    alpha = 1.0 / (g.na * g.nd) if alpha is None else float(alpha)
    n = u.shape[0] if n is None else int(n)
    box = _rect(box)
    p = _f64(p).reshape(g.na, g.nd)
    u = _f64(u)
    x = np.empty((box[3], box[2]), np.float64)
    sh = None if shift is None else _f64(shift).reshape(box[3], box[2])
    _load().orc_filter_ista(*g._g(), *box, _p(p), n, alpha, _p(u), _p(sh) if sh is not None else None,
                            float(lam), int(levels), _p(x))
    return x


def filter_ista_solve(g: Geometry, p, region, iters: int, lam: float, levels: int = 32, u=None):
    """Haar-ISTA in the paper's method end to end (disc subtraction and add-back)."""
    box = roi_box(g.N, *region)
    gv, pd, D = disc(g, p)
    if u is None:
        u = filtcalc(g, iters)
    x0, y0, w, h = box
    shift = gv * D[y0:y0 + h, x0:x0 + w]
    return filter_ista(g, box, pd, u, lam, levels=levels, n=iters, shift=shift), box
