"""GB300-native local region-of-interest tomographic reconstruction.

Python binding of the C ABI declared in ``include/roi_recon.h`` (Pelt & Batenburg,
arXiv 1604.02292: global FBP, exterior reprojection and subtraction, then a local
nonnegative-SIRT or Chambolle-Pock TV solve on the extended ROI).  Every step of
the pipeline runs in the CUDA library ``_lib/libroi_recon.so``; this module only
marshals arguments.  There is no CPU fallback: importing the library raises if
it cannot be built or loaded.

Functions ``roi_recon_*`` mirror the C entry points one to one and take raw
pointers (ints).  ``RoiRecon`` is a convenience wrapper taking torch tensors,
which supply device memory and the CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

from . import build as _build

__all__ = [
    "ROI_OK", "ROI_EINVAL", "ROI_ENOMEM", "ROI_ESTATE", "ROI_ECUDA", "ROI_ETIMEOUT", "ROI_EBUSY", "ROI_ECANCELED",
    "ROI_F32", "ROI_BF16", "ROI_F16", "ROI_SIRT_NONNEG", "ROI_TV_CP", "ROI_FILTER_SIRT", "ROI_FILTER_TV", "ROI_FILTER_ISTA",
    "roi_recon_filter_prepare", "roi_recon_filter_get", "roi_recon_set_sinogram_truncated",
    "roi_recon_solve_tiled", "roi_recon_state_size", "roi_recon_state_export", "roi_recon_solve_local_resume",
    "roi_recon_check_report",
    "Geometry", "Region", "SolveParams", "SolveInfo", "RoiError", "lib", "EXPORTS",
    "roi_recon_create", "roi_recon_destroy", "roi_recon_last_error", "roi_recon_set_sinogram",
    "roi_recon_fbp", "roi_recon_reproject_exterior", "roi_recon_solve_local", "roi_recon_plan",
    "roi_recon_forward_local", "roi_recon_back_local", "roi_recon_ramp_filter", "roi_recon_set_timing",
    "roi_recon_kernel_times", "roi_recon_launch_count", "roi_recon_forward_local_noalloc",
    "roi_recon_set_option", "roi_recon_sync", "ROI_OPT_SINGLE_LAUNCH", "ROI_OPT_WAIT_LIMIT_US",
    "ROI_OPT_TEST_ABSENT_BLOCKS", "RoiRecon", "plan",
    "ServerConfig", "ServerCompletion", "ServerStats", "Server", "server_footprint",
    "roi_server_create", "roi_server_destroy", "roi_server_add_sinogram", "roi_server_submit",
    "roi_server_start", "roi_server_stop", "roi_server_progress", "roi_server_poll", "roi_server_take",
    "roi_server_drain", "roi_server_stats_get", "roi_server_last_error", "roi_server_footprint",
    "roi_server_cancel", "roi_server_set_option", "roi_recon_test_fail_alloc",
    "ROI_OPT_TILE_SHAPE", "TILE_SHAPES", "roi_recon_autotune", "roi_recon_set_tile_shapes",
    "roi_recon_get_tile_shapes", "ROI_OPT_FILTER_CONV", "roi_recon_filter_conv", "roi_recon_set_team_caps",
    "roi_recon_get_team_caps", "TEAM_CAPS", "roi_recon_batch_plan_create", "roi_recon_batch_plan_launch",
    "roi_recon_batch_plan_destroy", "BatchPlan",
]

ROI_OK, ROI_EINVAL, ROI_ENOMEM, ROI_ESTATE, ROI_ECUDA, ROI_ETIMEOUT, ROI_EBUSY, ROI_ECANCELED = range(8)
ROI_F32, ROI_BF16, ROI_F16 = range(3)
ROI_SIRT_NONNEG, ROI_TV_CP, ROI_FILTER_SIRT, ROI_FILTER_TV, ROI_FILTER_ISTA = range(5)
ROI_OPT_SINGLE_LAUNCH, ROI_OPT_WAIT_LIMIT_US, ROI_OPT_TEST_ABSENT_BLOCKS, ROI_OPT_TILE_SHAPE, ROI_OPT_FILTER_CONV = range(5)
TILE_SHAPES = {0: (16, 16), 1: (8, 8), 2: (16, 8)}   # phase B tile shape: (x, y) pixels per warp
TEAM_CAPS = (4, 8, 16, 32)                             # team sizes the autotuner tries

_STATUS = {0: "ROI_OK", 1: "ROI_EINVAL", 2: "ROI_ENOMEM", 3: "ROI_ESTATE", 4: "ROI_ECUDA",
           5: "ROI_ETIMEOUT", 6: "ROI_EBUSY", 7: "ROI_ECANCELED"}


class Geometry(ctypes.Structure):
    _fields_ = [("n_pix", ctypes.c_int), ("n_angles", ctypes.c_int), ("n_det", ctypes.c_int),
                ("angles", ctypes.POINTER(ctypes.c_double)), ("storage", ctypes.c_int),
                ("image_storage", ctypes.c_int)]


class Region(ctypes.Structure):
    _fields_ = [("cx", ctypes.c_double), ("cy", ctypes.c_double), ("radius", ctypes.c_double),
                ("margin", ctypes.c_double)]


class SolveParams(ctypes.Structure):
    _fields_ = [("reg", ctypes.c_int), ("lam", ctypes.c_double), ("iters", ctypes.c_int),
                ("weighting", ctypes.c_int), ("precond", ctypes.c_int), ("crop_disk", ctypes.c_int),
                ("eval_objective", ctypes.c_int), ("inner_iters", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("box_x0", ctypes.c_int), ("box_y0", ctypes.c_int), ("box_w", ctypes.c_int),
                ("box_h", ctypes.c_int), ("window_max", ctypes.c_int), ("window_stride", ctypes.c_int),
                ("iters_done", ctypes.c_int), ("step_L", ctypes.c_double), ("objective", ctypes.c_double)]



class BatchPlan:
    """A batch of SIRT / CP-TV regions planned once on a handle and launched as one captured
    CUDA graph; launch() after set_sinogram + fbp solves the same regions on the new data
    (bit-identical to RoiRecon.solve_batch there).  close() (or the handle's close) frees it."""

    def __init__(self, rr, regions, params, outs=None):
        torch = rr._torch
        n = len(regions)
        if isinstance(params, dict):
            params = [params] * n
        regs = (Region * n)(*[Region(*map(float, r)) for r in regions])
        prms = (SolveParams * n)()
        for i, p in enumerate(params):
            prms[i] = _params(p)
        if outs is None:
            outs = [torch.empty((rr.plan(r).box[3], rr.plan(r).box[2]), dtype=torch.float32, device="cuda")
                    for r in regions]
        ptrs = (ctypes.c_void_p * n)()
        for i, o in enumerate(outs):
            ptrs[i] = rr._dev(o)
        self.infos = (SolveInfo * n)()
        self.rr, self.outs, self.h = rr, outs, None
        s, h = roi_recon_batch_plan_create(rr.h, regs, prms, ptrs, self.infos)
        rr._check(s)
        self.h = h

    def launch(self):
        self.rr._check(roi_recon_batch_plan_launch(self.rr.h, self.h))
        return self.outs

    def close(self):
        if self.h is not None and self.rr.h:
            roi_recon_batch_plan_destroy(self.rr.h, self.h)
        self.h = None


class ServerConfig(ctypes.Structure):
    _fields_ = [("device_bytes", ctypes.c_size_t), ("host_bytes", ctypes.c_size_t), ("ring_slots", ctypes.c_int),
                ("team_blocks", ctypes.c_int), ("teams", ctypes.c_int), ("large_side", ctypes.c_int),
                ("idle_us", ctypes.c_int), ("no_spill", ctypes.c_int), ("solo_queue_ms", ctypes.c_int)]


class ServerCompletion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("status", ctypes.c_int), ("sino", ctypes.c_int),
                ("box_x0", ctypes.c_int), ("box_y0", ctypes.c_int), ("box_w", ctypes.c_int),
                ("box_h", ctypes.c_int), ("pool", ctypes.c_int), ("t_submit_ms", ctypes.c_double),
                ("t_publish_ms", ctypes.c_double), ("t_done_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong),
                ("pending", ctypes.c_longlong), ("in_flight", ctypes.c_longlong),
                ("kernel_launches", ctypes.c_longlong), ("device_in_use", ctypes.c_size_t),
                ("device_peak", ctypes.c_size_t), ("host_in_use", ctypes.c_size_t), ("host_peak", ctypes.c_size_t),
                ("blocks", ctypes.c_int), ("single_units", ctypes.c_int), ("teams", ctypes.c_int),
                ("team_blocks", ctypes.c_int), ("cancelled", ctypes.c_longlong)]


# every symbol declared in include/roi_recon.h
EXPORTS = [
    "roi_recon_create", "roi_recon_destroy", "roi_recon_last_error", "roi_recon_set_sinogram",
    "roi_recon_fbp", "roi_recon_reproject_exterior", "roi_recon_solve_local", "roi_recon_plan",
    "roi_recon_forward_local", "roi_recon_back_local", "roi_recon_ramp_filter",
    "roi_recon_set_timing", "roi_recon_kernel_times", "roi_recon_launch_count",
    "roi_recon_forward_local_noalloc", "roi_recon_set_option", "roi_recon_sync", "roi_recon_solve_batch",
    "roi_server_create", "roi_server_add_sinogram", "roi_server_submit", "roi_server_start", "roi_server_stop",
    "roi_server_progress", "roi_server_poll", "roi_server_take", "roi_server_drain", "roi_server_stats_get",
    "roi_server_last_error", "roi_server_destroy", "roi_server_footprint",
    "roi_recon_filter_prepare", "roi_recon_filter_get", "roi_recon_set_sinogram_truncated",
    "roi_recon_solve_tiled", "roi_recon_state_size", "roi_recon_state_export", "roi_recon_solve_local_resume",
    "roi_recon_check_report", "roi_server_cancel", "roi_server_set_option", "roi_recon_test_fail_alloc",
    "roi_recon_autotune", "roi_recon_set_tile_shapes", "roi_recon_get_tile_shapes", "roi_recon_filter_conv",
    "roi_recon_set_team_caps", "roi_recon_get_team_caps", "roi_recon_batch_plan_create",
    "roi_recon_batch_plan_launch", "roi_recon_batch_plan_destroy",
]

_lib = None
_lock = threading.Lock()
_P = ctypes.c_void_p
_H = ctypes.c_void_p


def lib() -> ctypes.CDLL:
    """Build (if needed) and load the CUDA library; raises on failure (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build(check=os.environ.get("ROI_RECON_CHECK") == "1")
            L = ctypes.CDLL(path)
            st = ctypes.c_int
            L.roi_recon_create.argtypes = [ctypes.POINTER(Geometry), _P, ctypes.POINTER(_H)]
            L.roi_recon_create.restype = st
            L.roi_recon_destroy.argtypes = [_H]
            L.roi_recon_destroy.restype = None
            L.roi_recon_last_error.argtypes = [_H]
            L.roi_recon_last_error.restype = ctypes.c_char_p
            L.roi_recon_set_sinogram.argtypes = [_H, _P, ctypes.c_int, ctypes.c_int]
            L.roi_recon_set_sinogram.restype = st
            L.roi_recon_fbp.argtypes = [_H, _P]
            L.roi_recon_fbp.restype = st
            L.roi_recon_reproject_exterior.argtypes = [_H, ctypes.POINTER(Region), _P, _P]
            L.roi_recon_reproject_exterior.restype = st
            L.roi_recon_solve_local.argtypes = [_H, ctypes.POINTER(Region), ctypes.POINTER(SolveParams), _P,
                                                ctypes.c_int, ctypes.POINTER(SolveInfo)]
            L.roi_recon_solve_local.restype = st
            L.roi_recon_check_report.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
            L.roi_recon_check_report.restype = ctypes.c_int
            L.roi_recon_state_size.argtypes = [_H, ctypes.POINTER(ctypes.c_size_t)]
            L.roi_recon_state_size.restype = st
            L.roi_recon_state_export.argtypes = [_H, _P, ctypes.c_size_t, ctypes.c_int]
            L.roi_recon_state_export.restype = st
            L.roi_recon_solve_local_resume.argtypes = [_H, ctypes.POINTER(Region), ctypes.POINTER(SolveParams), _P,
                                                       ctypes.c_size_t, ctypes.c_int, _P, ctypes.c_int,
                                                       ctypes.POINTER(SolveInfo)]
            L.roi_recon_solve_local_resume.restype = st
            L.roi_recon_plan.argtypes = [ctypes.POINTER(Geometry), ctypes.POINTER(Region),
                                         ctypes.POINTER(SolveInfo), _P, _P]
            L.roi_recon_plan.restype = st
            L.roi_recon_forward_local.argtypes = [_H, ctypes.POINTER(Region), _P, _P]
            L.roi_recon_forward_local.restype = st
            L.roi_recon_back_local.argtypes = [_H, ctypes.POINTER(Region), _P, _P]
            L.roi_recon_back_local.restype = st
            L.roi_recon_ramp_filter.argtypes = [_H, _P]
            L.roi_recon_ramp_filter.restype = st
            L.roi_recon_set_timing.argtypes = [_H, ctypes.c_int]
            L.roi_recon_set_timing.restype = st
            L.roi_recon_kernel_times.argtypes = [_H, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                                 ctypes.POINTER(ctypes.c_double)]
            L.roi_recon_kernel_times.restype = st
            L.roi_recon_launch_count.argtypes = []
            L.roi_recon_launch_count.restype = ctypes.c_ulonglong
            L.roi_recon_forward_local_noalloc.argtypes = [ctypes.POINTER(Geometry), ctypes.POINTER(Region), _P, _P,
                                                          _P, ctypes.c_char_p, ctypes.c_int]
            L.roi_recon_forward_local_noalloc.restype = st
            L.roi_recon_set_option.argtypes = [_H, ctypes.c_int, ctypes.c_longlong]
            L.roi_recon_set_option.restype = st
            L.roi_recon_sync.argtypes = [_H]
            L.roi_recon_sync.restype = st
            L.roi_recon_solve_batch.argtypes = [_H, ctypes.c_int, ctypes.POINTER(Region), ctypes.POINTER(SolveParams),
                                                ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                                ctypes.POINTER(SolveInfo)]
            L.roi_recon_solve_batch.restype = st
            L.roi_recon_set_sinogram_truncated.argtypes = [_H, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.roi_recon_set_sinogram_truncated.restype = st
            L.roi_recon_solve_tiled.argtypes = [_H, ctypes.c_int, ctypes.c_int, ctypes.POINTER(SolveParams), _P]
            L.roi_recon_solve_tiled.restype = st
            L.roi_recon_filter_prepare.argtypes = [_H, ctypes.c_int]
            L.roi_recon_filter_prepare.restype = st
            L.roi_recon_filter_get.argtypes = [_H, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_double)]
            L.roi_recon_filter_get.restype = st
            L.roi_recon_filter_conv.argtypes = [_H, ctypes.c_int, _P, _P, _P]
            L.roi_recon_filter_conv.restype = st
            L.roi_recon_batch_plan_create.argtypes = [_H, ctypes.c_int, ctypes.POINTER(Region),
                                                      ctypes.POINTER(SolveParams), ctypes.POINTER(ctypes.c_void_p),
                                                      ctypes.POINTER(SolveInfo), ctypes.POINTER(_H)]
            L.roi_recon_batch_plan_create.restype = st
            L.roi_recon_batch_plan_launch.argtypes = [_H, _H]
            L.roi_recon_batch_plan_launch.restype = st
            L.roi_recon_batch_plan_destroy.argtypes = [_H, _H]
            L.roi_recon_batch_plan_destroy.restype = st
            L.roi_recon_set_team_caps.argtypes = [_H, ctypes.POINTER(ctypes.c_int)]
            L.roi_recon_set_team_caps.restype = st
            L.roi_recon_get_team_caps.argtypes = [_H, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
            L.roi_recon_get_team_caps.restype = st
            L.roi_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(_H)]
            L.roi_server_create.restype = st
            L.roi_server_add_sinogram.argtypes = [_H, _H, ctypes.POINTER(ctypes.c_int)]
            L.roi_server_add_sinogram.restype = st
            L.roi_server_submit.argtypes = [_H, ctypes.c_int, ctypes.POINTER(Region), ctypes.POINTER(SolveParams),
                                            ctypes.POINTER(ctypes.c_longlong)]
            L.roi_server_submit.restype = st
            for name in ("roi_server_start", "roi_server_stop", "roi_server_progress"):
                getattr(L, name).argtypes = [_H]
                getattr(L, name).restype = st
            L.roi_server_poll.argtypes = [_H, ctypes.POINTER(ServerCompletion), ctypes.c_int]
            L.roi_server_poll.restype = ctypes.c_int
            L.roi_server_take.argtypes = [_H, ctypes.c_longlong, _P]
            L.roi_server_take.restype = st
            L.roi_server_drain.argtypes = [_H, ctypes.c_double]
            L.roi_server_drain.restype = st
            L.roi_server_stats_get.argtypes = [_H, ctypes.POINTER(ServerStats)]
            L.roi_server_stats_get.restype = st
            L.roi_server_last_error.argtypes = [_H]
            L.roi_server_last_error.restype = ctypes.c_char_p
            L.roi_server_destroy.argtypes = [_H]
            L.roi_server_destroy.restype = None
            L.roi_server_footprint.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.POINTER(Region),
                                               ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                                               ctypes.POINTER(ctypes.c_int)]
            L.roi_server_footprint.restype = st
            L.roi_server_cancel.argtypes = [_H, ctypes.c_longlong]
            L.roi_server_cancel.restype = st
            L.roi_server_set_option.argtypes = [_H, ctypes.c_int, ctypes.c_longlong]
            L.roi_server_set_option.restype = st
            L.roi_recon_test_fail_alloc.argtypes = [ctypes.c_int]
            L.roi_recon_test_fail_alloc.restype = st
            L.roi_recon_autotune.argtypes = [_H, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_double)]
            L.roi_recon_autotune.restype = st
            L.roi_recon_set_tile_shapes.argtypes = [_H, ctypes.POINTER(ctypes.c_int)]
            L.roi_recon_set_tile_shapes.restype = st
            L.roi_recon_get_tile_shapes.argtypes = [_H, ctypes.POINTER(ctypes.c_int)]
            L.roi_recon_get_tile_shapes.restype = st
            _lib = L
    return _lib


# ---- one-to-one wrappers of the C entry points (raw pointers as ints) ----------------

def roi_recon_create(geom: Geometry, stream: int):
    h = _H()
    s = lib().roi_recon_create(ctypes.byref(geom), stream or None, ctypes.byref(h))
    return s, h.value


def roi_recon_destroy(h) -> None:
    lib().roi_recon_destroy(h)


def roi_recon_last_error(h) -> str:
    return lib().roi_recon_last_error(h).decode()


def roi_recon_set_sinogram(h, p: int, dtype: int, on_device: int) -> int:
    return lib().roi_recon_set_sinogram(h, p, dtype, on_device)


def roi_recon_fbp(h, out: int | None) -> int:
    return lib().roi_recon_fbp(h, out or None)


def roi_recon_reproject_exterior(h, region: Region, window_out: int | None, d0_out: int | None) -> int:
    return lib().roi_recon_reproject_exterior(h, ctypes.byref(region), window_out or None, d0_out or None)


def roi_recon_solve_local(h, region: Region, params: SolveParams, out: int, out_on_device: int,
                          info: SolveInfo | None) -> int:
    return lib().roi_recon_solve_local(h, ctypes.byref(region), ctypes.byref(params), out, out_on_device,
                                       ctypes.byref(info) if info is not None else None)


def roi_recon_check_report() -> tuple[int, int, int]:
    """(count, site, index) of the check build's out-of-range indices since the last call."""
    site, index = ctypes.c_int(0), ctypes.c_int(0)
    n = lib().roi_recon_check_report(ctypes.byref(site), ctypes.byref(index))
    return n, site.value, index.value


def roi_recon_state_size(h) -> tuple[int, int]:
    n = ctypes.c_size_t(0)
    st = lib().roi_recon_state_size(h, ctypes.byref(n))
    return st, n.value


def roi_recon_state_export(h, dst: int, nbytes: int, on_device: int) -> int:
    return lib().roi_recon_state_export(h, dst, nbytes, on_device)


def roi_recon_solve_local_resume(h, region: Region, params: SolveParams, state: int, nbytes: int,
                                 state_on_device: int, out: int, out_on_device: int, info: SolveInfo | None) -> int:
    return lib().roi_recon_solve_local_resume(h, ctypes.byref(region), ctypes.byref(params), state, nbytes,
                                              state_on_device, out, out_on_device,
                                              ctypes.byref(info) if info is not None else None)


def roi_recon_plan(geom: Geometry, region: Region, info: SolveInfo, d0: int | None, width: int | None) -> int:
    return lib().roi_recon_plan(ctypes.byref(geom), ctypes.byref(region), ctypes.byref(info), d0 or None,
                                width or None)


def roi_recon_forward_local(h, region: Region, x: int, y: int) -> int:
    return lib().roi_recon_forward_local(h, ctypes.byref(region), x, y)


def roi_recon_back_local(h, region: Region, y: int, x: int) -> int:
    return lib().roi_recon_back_local(h, ctypes.byref(region), y, x)


def roi_recon_ramp_filter(h, q: int) -> int:
    return lib().roi_recon_ramp_filter(h, q)


def roi_recon_set_timing(h, enable: int) -> int:
    return lib().roi_recon_set_timing(h, int(enable))


def roi_recon_kernel_times(h, kernel: int):
    n = ctypes.c_int()
    ms = ctypes.c_double()
    s = lib().roi_recon_kernel_times(h, int(kernel), ctypes.byref(n), ctypes.byref(ms))
    return s, n.value, ms.value


def roi_recon_launch_count() -> int:
    return int(lib().roi_recon_launch_count())


def roi_recon_forward_local_noalloc(geom: Geometry, region: Region, x: int, y: int, stream: int):
    """Allocation-free W_L x (see the header); returns (status, message)."""
    buf = ctypes.create_string_buffer(256)
    s = lib().roi_recon_forward_local_noalloc(ctypes.byref(geom), ctypes.byref(region), x, y, stream or None,
                                              buf, len(buf))
    return s, buf.value.decode()


def roi_recon_set_option(h, opt: int, value: int) -> int:
    return lib().roi_recon_set_option(h, int(opt), int(value))


def roi_recon_sync(h) -> int:
    return lib().roi_recon_sync(h)


def roi_recon_solve_batch(h, regions, params, outs, out_on_device: int, infos=None) -> int:
    """regions, params: ctypes arrays (Region * n, SolveParams * n); outs: (c_void_p * n) pointers."""
    n = len(regions)
    return lib().roi_recon_solve_batch(h, n, regions, params, outs, int(out_on_device), infos)


def roi_recon_batch_plan_create(h, regions, params, outs, infos=None):
    """regions, params: ctypes arrays; outs: (c_void_p * n) device pointers.  Returns (status, plan)."""
    plan = _H()
    s = lib().roi_recon_batch_plan_create(h, len(regions), regions, params, outs, infos, ctypes.byref(plan))
    return s, plan.value


def roi_recon_batch_plan_launch(h, plan) -> int:
    return lib().roi_recon_batch_plan_launch(h, plan)


def roi_recon_batch_plan_destroy(h, plan) -> int:
    return lib().roi_recon_batch_plan_destroy(h, plan)


def roi_recon_set_sinogram_truncated(h, p: int, dtype: int, on_device: int, n_measured: int) -> int:
    return lib().roi_recon_set_sinogram_truncated(h, p, int(dtype), int(on_device), int(n_measured))


def roi_recon_solve_tiled(h, tile: int, margin: int, params: SolveParams, out: int) -> int:
    return lib().roi_recon_solve_tiled(h, int(tile), int(margin), ctypes.byref(params), out)


def roi_recon_filter_prepare(h, n_iters: int) -> int:
    return lib().roi_recon_filter_prepare(h, int(n_iters))


def roi_recon_filter_get(h, n_filters: int, u_out: int | None):
    g = ctypes.c_double(0.0)
    s = lib().roi_recon_filter_get(h, int(n_filters), u_out or None, ctypes.byref(g))
    return s, g.value


def roi_recon_set_team_caps(h, caps) -> int:
    arr = (ctypes.c_int * 3)(*[int(c) for c in caps])
    return lib().roi_recon_set_team_caps(h, arr)


def roi_recon_get_team_caps(h):
    caps = (ctypes.c_int * 3)()
    ms = (ctypes.c_double * 12)()
    s = lib().roi_recon_get_team_caps(h, caps, ms)
    return s, list(caps), [list(ms[4 * c:4 * c + 4]) for c in range(3)]


def roi_recon_filter_conv(h, n: int, u: int, p: int, out: int) -> int:
    return lib().roi_recon_filter_conv(h, int(n), u, p, out)


def roi_server_create(cfg: ServerConfig | None):
    h = _H()
    s = lib().roi_server_create(ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(h))
    return s, h.value


def roi_server_destroy(s) -> None:
    lib().roi_server_destroy(s)


def roi_server_add_sinogram(s, h):
    i = ctypes.c_int(-1)
    st = lib().roi_server_add_sinogram(s, h, ctypes.byref(i))
    return st, i.value


def roi_server_submit(s, sino: int, region: Region, params: SolveParams):
    i = ctypes.c_longlong(0)
    st = lib().roi_server_submit(s, int(sino), ctypes.byref(region), ctypes.byref(params), ctypes.byref(i))
    return st, i.value


def roi_server_start(s) -> int:
    return lib().roi_server_start(s)


def roi_server_stop(s) -> int:
    return lib().roi_server_stop(s)


def roi_server_progress(s) -> int:
    return lib().roi_server_progress(s)


def roi_server_poll(s, out, max_n: int) -> int:
    """out: (ServerCompletion * k) array, k >= max_n."""
    return lib().roi_server_poll(s, out, int(max_n))


def roi_server_take(s, rid: int, dst: int | None) -> int:
    return lib().roi_server_take(s, int(rid), dst or None)


def roi_server_drain(s, timeout_ms: float) -> int:
    return lib().roi_server_drain(s, float(timeout_ms))


def roi_server_stats_get(s, out: ServerStats) -> int:
    return lib().roi_server_stats_get(s, ctypes.byref(out))


def roi_server_last_error(s) -> str:
    return (lib().roi_server_last_error(s) or b"").decode()


def roi_server_cancel(s, rid: int) -> int:
    return lib().roi_server_cancel(s, int(rid))


def roi_server_set_option(s, opt: int, value: int) -> int:
    return lib().roi_server_set_option(s, int(opt), int(value))


def roi_recon_test_fail_alloc(nth: int) -> int:
    return lib().roi_recon_test_fail_alloc(int(nth))


def roi_recon_autotune(h, regions_per_class: int, iters: int):
    """(status, shapes [3], ms [3][3])."""
    shapes = (ctypes.c_int * 3)()
    ms = (ctypes.c_double * 9)()
    st = lib().roi_recon_autotune(h, int(regions_per_class), int(iters), shapes, ms)
    return st, list(shapes), [list(ms[3 * c:3 * c + 3]) for c in range(3)]


def roi_recon_set_tile_shapes(h, shapes) -> int:
    arr = (ctypes.c_int * 3)(*[int(v) for v in shapes])
    return lib().roi_recon_set_tile_shapes(h, arr)


def roi_recon_get_tile_shapes(h):
    arr = (ctypes.c_int * 3)()
    st = lib().roi_recon_get_tile_shapes(h, arr)
    return st, list(arr)


def roi_server_footprint(n_pix: int, n_angles: int, n_det: int, storage: int, region: Region):
    dev, host, side = ctypes.c_size_t(0), ctypes.c_size_t(0), ctypes.c_int(0)
    st = lib().roi_server_footprint(int(n_pix), int(n_angles), int(n_det), int(storage), ctypes.byref(region),
                                    ctypes.byref(dev), ctypes.byref(host), ctypes.byref(side))
    return st, dev.value, host.value, side.value


# ---- convenience layer -----------------------------------------------------------------

class RoiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


def _geometry(N, n_angles, n_det, angles=None, storage=ROI_F32, image_storage=ROI_F32):
    g = Geometry(int(N), int(n_angles), int(n_det), None, int(storage), int(image_storage))
    keep = None
    if angles is not None:
        import numpy as np
        keep = np.ascontiguousarray(angles, dtype=np.float64)
        assert keep.shape == (int(n_angles),)
        g.angles = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return g, keep


@dataclass
class Plan:
    box: tuple          # (x0, y0, w, h)
    window_max: int
    window_stride: int
    d0: list
    width: list


def plan(N, n_angles, n_det, region, angles=None) -> Plan:
    """Host-only ROI plan (box and per-angle detector windows); needs no GPU."""
    import numpy as np
    g, _keep = _geometry(N, n_angles, n_det, angles)
    info = SolveInfo()
    d0 = np.zeros(int(n_angles), np.int32)
    wd = np.zeros(int(n_angles), np.int32)
    s = roi_recon_plan(g, Region(*map(float, region)), info, d0.ctypes.data, wd.ctypes.data)
    if s != ROI_OK:
        raise RoiError(s, "roi_recon_plan failed")
    return Plan((info.box_x0, info.box_y0, info.box_w, info.box_h), info.window_max, info.window_stride,
                d0.tolist(), wd.tolist())


class RoiRecon:
    """Handle over one geometry, with device memory and the stream taken from torch.

    ``region`` arguments are ``(cx, cy, radius, margin)`` in pixel-index units.
    Tensors must be contiguous float32 CUDA tensors on the current device.
    """

    def __init__(self, N, n_angles, n_det, angles=None, stream=None, storage=ROI_F32, image_storage=None):
        """storage: ROI_F32, ROI_BF16 or ROI_F16 -- the type the resident sinogram is stored
        in; image_storage: the type of the cached FBP image and of the projector images of
        batched / served solves (None: the same as storage)."""
        import torch
        self._torch = torch
        self.N, self.n_angles, self.n_det = int(N), int(n_angles), int(n_det)
        self.storage = int(storage)
        self.image_storage = int(storage if image_storage is None else image_storage)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        g, self._angles_keep = _geometry(N, n_angles, n_det, angles, storage, self.image_storage)
        s, h = roi_recon_create(g, self.stream.cuda_stream)
        if s != ROI_OK:
            raise RoiError(s, "roi_recon_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            roi_recon_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, s):
        if s != ROI_OK:
            raise RoiError(s, roi_recon_last_error(self.h))

    def _dev(self, t, shape=None):
        torch = self._torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise TypeError("expected a contiguous float32 CUDA tensor")
        if shape is not None and tuple(t.shape) != tuple(shape):
            raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
        return t.data_ptr()

    def plan(self, region) -> Plan:
        return plan(self.N, self.n_angles, self.n_det, region,
                    None if self._angles_keep is None else self._angles_keep)

    def set_sinogram(self, p):
        """p: [n_angles][n_det], a CUDA tensor (float32, bfloat16 or float16) or a host
        float32 array (numpy / CPU tensor); converted to the handle's storage type."""
        torch = self._torch
        shape = (self.n_angles, self.n_det)
        if isinstance(p, torch.Tensor) and p.is_cuda:
            dts = {torch.float32: ROI_F32, torch.bfloat16: ROI_BF16, torch.float16: ROI_F16}
            if p.dtype not in dts or not p.is_contiguous() or tuple(p.shape) != shape:
                raise TypeError(f"device sinogram must be a contiguous float32/bfloat16/float16 tensor {shape}")
            self._check(roi_recon_set_sinogram(self.h, p.data_ptr(), dts[p.dtype], 1))
            self._sino_keep = p
        else:
            import numpy as np
            arr = p.numpy() if isinstance(p, torch.Tensor) else np.asarray(p)
            if arr.dtype != np.float32 or not arr.flags["C_CONTIGUOUS"] or arr.shape != shape:
                raise TypeError(f"host sinogram must be C-contiguous float32 of shape {shape}")
            self._check(roi_recon_set_sinogram(self.h, arr.ctypes.data, ROI_F32, 0))
            self._sino_keep = arr

    def set_sinogram_truncated(self, p):
        """p: [n_angles][n_measured] float32 CUDA tensor, the central bins of the detector;
        the rest of each row is padded with its edge values (Sec. 5.6)."""
        torch = self._torch
        if not (isinstance(p, torch.Tensor) and p.is_cuda and p.dtype == torch.float32 and p.is_contiguous()
                and p.dim() == 2 and p.shape[0] == self.n_angles):
            raise TypeError("expected a contiguous float32 CUDA tensor [n_angles][n_measured]")
        self._check(roi_recon_set_sinogram_truncated(self.h, p.data_ptr(), ROI_F32, 1, p.shape[1]))
        self._sino_keep = p

    def fbp(self, out=None):
        self._check(roi_recon_fbp(self.h, self._dev(out, (self.N, self.N)) if out is not None else None))
        return out

    def reproject_exterior(self, region, window_out=None):
        pl = self.plan(region)
        d0 = None
        import numpy as np
        d0 = np.zeros(self.n_angles, np.int32)
        ptr = self._dev(window_out, (self.n_angles, pl.window_stride)) if window_out is not None else None
        self._check(roi_recon_reproject_exterior(self.h, Region(*map(float, region)), ptr, d0.ctypes.data))
        return d0

    def solve_local(self, region, reg=ROI_SIRT_NONNEG, iters=200, lam=0.0, weighting=0, precond=1,
                    crop_disk=0, eval_objective=0, out=None, inner_iters=0, resume=None):
        """Returns (out, info); out is a CUDA tensor [box_h][box_w] or a host numpy array.
        resume: a state from state() (host numpy uint8 array or CUDA uint8 tensor); the solve
        then runs `iters` further iterations from it."""
        torch = self._torch
        pl = self.plan(region)
        shape = (pl.box[3], pl.box[2])
        prm = SolveParams(int(reg), float(lam), int(iters), int(weighting), int(precond), int(crop_disk),
                          int(eval_objective), int(inner_iters))
        info = SolveInfo()
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device="cuda")
        if isinstance(out, torch.Tensor) and out.is_cuda:
            optr, odev = self._dev(out, shape), 1
        else:
            import numpy as np
            if out.dtype != np.float32 or out.shape != shape or not out.flags["C_CONTIGUOUS"]:
                raise TypeError(f"host output must be C-contiguous float32 of shape {shape}")
            optr, odev = out.ctypes.data, 0
        if resume is None:
            s = roi_recon_solve_local(self.h, Region(*map(float, region)), prm, optr, odev, info)
        else:
            if isinstance(resume, torch.Tensor):
                if not (resume.is_cuda and resume.dtype == torch.uint8 and resume.is_contiguous()):
                    raise TypeError("a device state must be a contiguous uint8 CUDA tensor")
                sptr, sn, sdev = resume.data_ptr(), resume.numel(), 1
            else:
                import numpy as np
                if resume.dtype != np.uint8 or not resume.flags["C_CONTIGUOUS"]:
                    raise TypeError("a host state must be a C-contiguous uint8 numpy array")
                sptr, sn, sdev = resume.ctypes.data, resume.nbytes, 0
            s = roi_recon_solve_local_resume(self.h, Region(*map(float, region)), prm, sptr, sn, sdev, optr, odev,
                                             info)
        self._check(s)
        return out, info

    def state(self, on_device=False):
        """The iterate state of the last solve_local (checkpoint): a host numpy uint8 array, or a
        CUDA uint8 tensor when on_device."""
        st, n = roi_recon_state_size(self.h)
        self._check(st)
        if on_device:
            buf = self._torch.empty(n, dtype=self._torch.uint8, device="cuda")
            self._check(roi_recon_state_export(self.h, buf.data_ptr(), n, 1))
        else:
            import numpy as np
            buf = np.empty(n, np.uint8)
            self._check(roi_recon_state_export(self.h, buf.ctypes.data, n, 0))
        return buf

    def solve_batch(self, regions, params, outs=None):
        """Solve many regions in one call.  regions: list of (cx, cy, r, m); params: list of dicts
        (reg, iters, lam, weighting, crop_disk) or one dict for all.  Returns (outs, infos);
        outs are CUDA tensors unless host numpy arrays are passed."""
        torch = self._torch
        n = len(regions)
        if isinstance(params, dict):
            params = [params] * n
        regs = (Region * n)(*[Region(*map(float, r)) for r in regions])
        prms = (SolveParams * n)()
        for i, p in enumerate(params):
            prms[i] = _params(p)
        infos = (SolveInfo * n)()
        on_device = 1
        if outs is None:
            outs = []
            for i, r in enumerate(regions):
                try:
                    pl = self.plan(r)
                except RoiError as e:
                    raise RoiError(e.status, f"solve_batch: region {i}: extended box misses the grid or is invalid")
                outs.append(torch.empty((pl.box[3], pl.box[2]), dtype=torch.float32, device="cuda"))
        ptrs = (ctypes.c_void_p * n)()
        for i, o in enumerate(outs):
            if isinstance(o, torch.Tensor) and o.is_cuda:
                ptrs[i] = o.data_ptr()
            else:
                on_device = 0
                ptrs[i] = o.ctypes.data
        if on_device == 0 and any(isinstance(o, torch.Tensor) and o.is_cuda for o in outs):
            raise TypeError("outs must be all CUDA tensors or all host arrays")
        self._check(roi_recon_solve_batch(self.h, regs, prms, ptrs, on_device, infos))
        return outs, list(infos)

    def batch_plan(self, regions, params, outs=None):
        """A batch planned once and replayed as a captured CUDA graph (roi_recon_batch_plan_*):
        returns a BatchPlan whose launch() solves the regions on the handle's current sinogram
        into its outs (CUDA tensors, allocated here unless given)."""
        return BatchPlan(self, regions, params, outs)

    def forward_local(self, region, x, y=None):
        pl = self.plan(region)
        if y is None:
            y = self._torch.zeros((self.n_angles, pl.window_stride), dtype=self._torch.float32, device="cuda")
        self._check(roi_recon_forward_local(self.h, Region(*map(float, region)),
                                            self._dev(x, (pl.box[3], pl.box[2])),
                                            self._dev(y, (self.n_angles, pl.window_stride))))
        return y

    def back_local(self, region, y, x=None):
        pl = self.plan(region)
        if x is None:
            x = self._torch.zeros((pl.box[3], pl.box[2]), dtype=self._torch.float32, device="cuda")
        self._check(roi_recon_back_local(self.h, Region(*map(float, region)),
                                         self._dev(y, (self.n_angles, pl.window_stride)),
                                         self._dev(x, (pl.box[3], pl.box[2]))))
        return x

    def solve_tiled(self, tile: int, margin: int, params: dict, out=None):
        """The whole image as non-overlapping tile x tile local solves (Sec. 5.5); returns a CUDA
        tensor [N][N].  params: dict as for solve_batch."""
        if out is None:
            out = self._torch.empty((self.N, self.N), dtype=self._torch.float32, device="cuda")
        self._check(roi_recon_solve_tiled(self.h, tile, margin, _params(params), self._dev(out, (self.N, self.N))))
        return out

    def filter_prepare(self, n_iters: int):
        """The paper's own method (Sec. 3): filters of Alg. filtcalc for n_iters iterations, disc
        subtraction and filtered sinograms of the resident sinogram (then solve_local with
        reg=ROI_FILTER_SIRT and iters <= n_iters)."""
        self._check(roi_recon_filter_prepare(self.h, n_iters))

    def filters(self, n_filters: int):
        """(u [n][n_angles][2 n_det - 1] CUDA tensor, disc grey value) after filter_prepare."""
        u = self._torch.empty((n_filters, self.n_angles, 2 * self.n_det - 1), dtype=self._torch.float32,
                              device="cuda")
        s, g = roi_recon_filter_get(self.h, n_filters, u.data_ptr())
        self._check(s)
        return u, g

    def filter_conv(self, u, p, out=None):
        """out[k][a][d] = sum_e u[k][a][d - e + n_det - 1] p[a][e] (roi_recon_filter_conv):
        u CUDA float32 [n][n_angles][2 n_det - 1], p [n_angles][n_det]; returns out [n][n_angles][n_det]."""
        n = int(u.shape[0])
        # u and p stay referenced here until the call returns (their memory must not be reused for out)
        u_ptr = self._dev(u, (n, self.n_angles, 2 * self.n_det - 1))
        p_ptr = self._dev(p, (self.n_angles, self.n_det))
        if out is None:
            out = self._torch.empty((n, self.n_angles, self.n_det), dtype=self._torch.float32, device="cuda")
        self._check(roi_recon_filter_conv(self.h, n, u_ptr, p_ptr, self._dev(out, (n, self.n_angles, self.n_det))))
        return out

    def set_option(self, opt: int, value: int):
        self._check(roi_recon_set_option(self.h, opt, value))

    def autotune(self, regions_per_class: int = 0, iters: int = 0):
        """Pick the phase B tile shape per box-size class by timing (roi_recon_autotune);
        returns (shapes, ms) -- ms[class][shape] in milliseconds."""
        st, shapes, ms = roi_recon_autotune(self.h, regions_per_class, iters)
        self._check(st)
        return shapes, ms

    @property
    def tile_shapes(self):
        st, shapes = roi_recon_get_tile_shapes(self.h)
        self._check(st)
        return shapes

    @tile_shapes.setter
    def tile_shapes(self, shapes):
        self._check(roi_recon_set_tile_shapes(self.h, shapes))

    @property
    def team_caps(self):
        """Largest team per region of a few-region batch, per box-size class (roi_recon_get_team_caps)."""
        st, caps, _ = roi_recon_get_team_caps(self.h)
        self._check(st)
        return caps

    @team_caps.setter
    def team_caps(self, caps):
        self._check(roi_recon_set_team_caps(self.h, caps))

    def team_caps_ms(self):
        """The autotuner's milliseconds per class for team caps TEAM_CAPS (zeros before it ran)."""
        st, _, ms = roi_recon_get_team_caps(self.h)
        self._check(st)
        return ms

    def sync(self):
        """Wait for the handle's stream; raises RoiError(ROI_ETIMEOUT) if a device wait gave up."""
        self._check(roi_recon_sync(self.h))

    def set_timing(self, enable: bool):
        self._check(roi_recon_set_timing(self.h, int(enable)))

    def kernel_times(self, kernel: int):
        """(launches, total device ms) of kernel class 0 (forward), 1 (back), 2 (single-launch or
        batched solve) or 3 (filtered sinograms)."""
        s, n, ms = roi_recon_kernel_times(self.h, kernel)
        self._check(s)
        return n, ms

    def ramp_filter(self, q=None):
        if q is None:
            q = self._torch.empty((self.n_angles, self.n_det), dtype=self._torch.float32, device="cuda")
        self._check(roi_recon_ramp_filter(self.h, self._dev(q, (self.n_angles, self.n_det))))
        return q


def _params(p: dict) -> SolveParams:
    return SolveParams(int(p.get("reg", ROI_SIRT_NONNEG)), float(p.get("lam", 0.0)), int(p.get("iters", 200)),
                       int(p.get("weighting", 0)), 1, int(p.get("crop_disk", 0)), 0, int(p.get("inner_iters", 0)))


def server_footprint(N, n_angles, n_det, region, storage=ROI_F32):
    """(device_bytes, host_bytes, box_side) the server budgets for a request; host only."""
    st, dev, host, side = roi_server_footprint(N, n_angles, n_det, storage, Region(*map(float, region)))
    if st != ROI_OK:
        raise RoiError(st, "roi_server_footprint failed")
    return dev, host, side


class Server:
    """ROI server over resident sinograms (continuous batching; see roi_server_* in the C header).

    ``add(recon)`` registers a RoiRecon whose FBP is done; ``submit(sino, region, params)``
    queues a request and returns its id; ``poll()`` returns completion records (dicts);
    ``take(id)`` returns the result as a float32 numpy array [box_h][box_w].
    """

    def __init__(self, device_bytes=0, host_bytes=0, ring_slots=0, team_blocks=0, teams=-1, large_side=0,
                 idle_us=0, no_spill=0, start=True, solo_queue_ms=0):
        cfg = ServerConfig(int(device_bytes), int(host_bytes), int(ring_slots), int(team_blocks), int(teams),
                           int(large_side), int(idle_us), int(no_spill), int(solo_queue_ms))
        st, s = roi_server_create(cfg)
        if st != ROI_OK:
            raise RoiError(st, "roi_server_create failed")
        self.s = s
        self._recons = []
        self._buf = (ServerCompletion * 256)()
        self._start = bool(start)
        self._started = False

    def _check(self, st):
        if st != ROI_OK:
            raise RoiError(st, roi_server_last_error(self.s))

    def add(self, recon) -> int:
        st, i = roi_server_add_sinogram(self.s, recon.h)
        self._check(st)
        self._recons.append(recon)
        return i

    def start(self):
        self._check(roi_server_start(self.s))
        self._started = True

    def stop(self):
        self._check(roi_server_stop(self.s))
        self._started = False

    def progress(self):
        self._check(roi_server_progress(self.s))

    def submit(self, sino: int, region, params: dict | None = None) -> int:
        st, rid = roi_server_submit(self.s, sino, Region(*map(float, region)), _params(params or {}))
        self._check(st)
        if self._start and not self._started:
            self.start()
        return rid

    def poll(self):
        out = []
        while True:
            n = roi_server_poll(self.s, self._buf, len(self._buf))
            if n < 0:
                raise RoiError(ROI_EINVAL, "roi_server_poll failed")
            for c in self._buf[:n]:
                out.append(dict(id=c.id, status=c.status, sino=c.sino, box=(c.box_x0, c.box_y0, c.box_w, c.box_h),
                                pool=c.pool, t_submit_ms=c.t_submit_ms, t_publish_ms=c.t_publish_ms,
                                t_done_ms=c.t_done_ms))
            if n < len(self._buf):
                return out

    def take(self, rid: int, shape=None):
        import numpy as np
        if shape is None:
            raise ValueError("take: pass the (box_h, box_w) shape from the completion record")
        out = np.empty(shape, np.float32)
        self._check(roi_server_take(self.s, rid, out.ctypes.data))
        return out

    def drain(self, timeout_ms: float = 600000.0):
        self._check(roi_server_drain(self.s, timeout_ms))

    def cancel(self, rid: int):
        """Removes a queued request (its completion then reports ROI_ECANCELED); RoiError with
        ROI_EBUSY once it is on the device."""
        self._check(roi_server_cancel(self.s, rid))

    def set_option(self, opt: int, value: int):
        self._check(roi_server_set_option(self.s, opt, value))

    def stats(self) -> dict:
        st = ServerStats()
        self._check(roi_server_stats_get(self.s, st))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "s", None):
            roi_server_destroy(self.s)
            self.s = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
