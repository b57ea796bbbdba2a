#!/usr/bin/env python3
"""Benchmark: local ROI reconstructions per second on one GB300 (or N, one rank each).

One step = one pass of the whole local pipeline on one region of the 1024 x 1024
workload (256 angles, 1024 bins, 50 ellipses + fine texture, I0 = 5e3, ROI radius
64 px + margin 32 px, Chambolle-Pock TV lambda = 0.01, 500 iterations, FP32):
copy the resident sinogram into the handle, Ram-Lak FBP, ROI plan, exterior
reprojection and subtraction, 500 CP iterations on the 192 x 192 box, crop.
Steps cycle over 8 seeded regions so each plans a new box.

Timing: W warm-up steps; then K steps between a barrier + synchronize on both
sides; each step is bracketed by CUDA events on the library's stream and a
256 MB write flushes L2 between steps (outside the events).  ``value`` is
(steps x ranks) / max over ranks of the summed step time.  ``e2e`` repeats the
step through the C ABI with host buffers: pinned host sinogram in, host image out.

The default line also carries ``serving``: the 2048 x 2048 serving workload (8
resident sinograms, Poisson arrivals at 2000 requests/s, radii log-uniform in
[16, 256] px, SIRT/TV 50/50, 200 iterations; ``--requests`` of them) served with
continuous batching, against the same requests solved one at a time ("plain"):
solves/s and p50/p99 latency from arrival to the result in host memory.

``--workload roi_batch_2048`` and ``--workload roi_serve_2048`` print the batched and
served workloads' own lines instead.

``--impl reference`` times the FP64 CPU oracle on the host cores instead (rank 0
only): each step is FBP + exterior + a bounded number of CP iterations, scaled to
a whole solve.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1604_02292_gb300 import shard  # noqa: E402
from paper_1604_02292_gb300 import workloads as WL  # noqa: E402

WORKLOAD = "roi_cptv_1024"
N_REGIONS = 8
FLUSH_BYTES = 256 << 20
# lerps one SM can retire per clock: a Joseph interpolation needs two shared/L1 loads
# (32 lanes per clock per SM) and ~8 FP32-pipe instructions (128 lanes per clock per SM),
# both giving 16 lerps per clock per SM
LERPS_PER_CLK_SM = 16
N_SM = 152
PERSIST_SRCS = ("paper_1604_02292_gb300/csrc/persist.cu", "paper_1604_02292_gb300/csrc/dev_common.cuh")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=sorted(WL.WORKLOADS) + sorted(WL.BATCHES) + sorted(WL.SERVING) + sorted(WL.PRECISION)
                    + ["roi_large_2048"])
    ap.add_argument("--storage", default="bf16", choices=["f32", "bf16", "f16"],
                    help="precision workloads: storage type measured against float32 storage")
    ap.add_argument("--batch-count", type=int, default=None,
                    help="batch workloads: solve this many of the regions per step (default: all)")
    ap.add_argument("--requests", type=int, default=256, help="serving workloads: requests in the run")
    ap.add_argument("--iters", type=int, default=0,
                    help="batch and large-box workloads: iterations per region (0: the workload's)")
    ap.add_argument("--radius", type=float, default=128.0, help="large-box workload: ROI radius (margin r/2)")
    ap.add_argument("--rate", type=float, default=None, help="serving workloads: arrival rate (default: workload's)")
    ap.add_argument("--team-blocks", type=int, default=0, help="serving: blocks per team (0: library default)")
    ap.add_argument("--teams", type=int, default=-1, help="serving: teams (-1: library default)")
    ap.add_argument("--large-side", type=int, default=0, help="serving: box side served by teams (0: default)")
    ap.add_argument("--solo-queue-ms", type=int, default=0,
                    help="serving: queued work (ms) that ends a solo launch (0: library default)")
    ap.add_argument("--no-plain", action="store_true", help="serving: skip the one-at-a-time comparison")
    ap.add_argument("--no-serving", action="store_true", help="default workload: skip the serving comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-global", action="store_true", help="default workload: skip the local-vs-global report")
    ap.add_argument("--no-batch", action="store_true", help="default workload: skip the batching figure")
    ap.add_argument("--no-precision", action="store_true", help="default workload: skip the precision figure")
    ap.add_argument("--autotune", action="store_true", help="batch workloads: autotune the tile shapes first")
    ap.add_argument("--rates", default="50,100,150",
                    help="default workload: arrival rates (requests/s) of the sustainable-rate serving points")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def profile_traffic(kernel_srcs, profile_md):
    """DRAM bytes per launch from a committed ncu summary, only while the kernel's sources
    (concatenated) still hash to the value recorded with the counters (else None: the kernel
    has changed)."""
    import hashlib
    try:
        text = open(os.path.join(ROOT, profile_md)).read()
        src = b"".join(open(os.path.join(ROOT, f), "rb").read() for f in kernel_srcs)
    except OSError:
        return None
    fields = dict(line.split(":", 1) for line in text.splitlines() if line.startswith(("source_sha256:", "dram_bytes_per_launch:")))
    if fields.get("source_sha256", "").strip() != hashlib.sha256(src).hexdigest():
        return None
    try:
        return int(fields["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        smi = shutil.which("nvidia-smi")
        if smi and self.gpu is not None:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen([smi, f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def lerps_per_launch(pl, w):
    """Algorithmic work of the two projector kernels for one box: forward = window rays x
    samples (the box side along the stepping axis); back = pixels x angles."""
    nx, ny = pl.box[2], pl.box[3]
    th = np.arange(w.n_angles) * math.pi / w.n_angles
    row = np.abs(np.cos(th)) >= np.abs(np.sin(th)) - 1e-12
    steps = np.where(row, ny, nx)
    fwd = int(np.sum(np.asarray(pl.width) * steps))
    back = int(nx * ny * w.n_angles)
    return fwd, back


def bytes_per_launch(pl, w):
    """Algorithmic DRAM-level bytes (each operand once) of the CP projector kernels."""
    n = pl.box[2] * pl.box[3]
    win = int(np.sum(pl.width))
    fwd = 4 * (n + 4 * win)          # read xbar; read p', sigma, u; write u
    back = 4 * (win + 4 * n + 3 * n)  # read u; read x, tau, vx, vy; write x, xbar, xbar^T
    return fwd, back


# --------------------------------------------------------------------------- oracle arm

def oracle_solve(w, p, region):
    """Time one whole FP64 oracle solve: FBP + exterior + all w.iters iterations; returns
    (seconds, (fbp, exterior, iterations))."""
    import oracle
    g = oracle.Geometry(*w.geometry())
    box = oracle.roi_box(w.N, *region)
    t0 = time.perf_counter()
    xf = oracle.fbp(g, p.astype(np.float64))
    t1 = time.perf_counter()
    pp = oracle.exterior(g, box, p.astype(np.float64), xf)
    t2 = time.perf_counter()
    if w.reg == "sirt":
        oracle.sirt(g, box, pp, w.iters)
    else:
        oracle.cp_tv(g, box, pp, w.iters, w.lam, precond=1)
    t3 = time.perf_counter()
    return t3 - t0, (t1 - t0, t2 - t1, t3 - t2)


def oracle_warm(w, p, region):
    """Untimed warm-up of the oracle: FBP and exterior step (threads started, pages touched)."""
    import oracle
    g = oracle.Geometry(*w.geometry())
    xf = oracle.fbp(g, p.astype(np.float64))
    oracle.exterior(g, oracle.roi_box(w.N, *region), p.astype(np.float64), xf)


def omp_threads():
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else (os.cpu_count() or 1)


def run_reference(args):
    """The FP64 oracle on the host cores, on our arm's workload: every timed step is one
    whole local solve (FBP + exterior + all iterations) of one region, measured, nothing
    scaled; warm-up steps run the oracle's FBP and exterior step only."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = WL.WORKLOADS[args.workload]
    p = WL.sinogram(w, 0)
    regions = [WL.region(w, seed=s) for s in range(N_REGIONS)]
    for k in range(args.warmup):
        oracle_warm(w, p, regions[k % N_REGIONS])
    times, parts = [], []
    for k in range(args.steps):
        t, pt = oracle_solve(w, p, regions[k % N_REGIONS])
        times.append(t)
        parts.append(pt)
    total = sum(times)
    value = args.steps / total
    mean = [statistics.mean(x[i] for x in parts) for i in range(3)]
    sample = (f"each step: one whole oracle solve of one region (FBP {mean[0]:.2f} s + exterior {mean[1]:.2f} s + "
              f"{w.iters} {'CP' if w.reg == 'tv' else 'SIRT'} iterations {mean[2]:.2f} s, means), measured; "
              f"warm-up steps: FBP + exterior only")
    line = {
        "impl": "reference", "metric": "roi_solves_per_s", "value": value, "unit": "solves/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "N": w.N, "n_angles": w.n_angles, "n_det": w.n_det,
                   "roi_radius": w.radius, "roi_margin": w.margin, "solver": w.reg, "iters": w.iters,
                   "lambda": w.lam},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": omp_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "timed_s": total,
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------ our arm

def large_box_measure(reps=3):
    """Lone large regions through roi_recon_solve_local on the 2048 x 2048 / 180-angle serving
    geometry: radius 128 and 256 px (boxes 384 and 768), SIRT and CP-TV, 200 iterations,
    solved by the whole-region solver as one team of every block (the default) and by one
    launch per operator (ROI_OPT_SINGLE_LAUNCH = 0); CUDA-event time per solve and the
    projector lerps/s (forward window rays x box side + gather pixels x angles, per iteration)."""
    import torch

    import paper_1604_02292_gb300 as R

    w = WL.SERVING["roi_serve_2048"]
    stream = torch.cuda.Stream()
    rr = R.RoiRecon(*w.geometry(), stream=stream)
    c = (w.N - 1) / 2.0
    out = []
    with torch.cuda.stream(stream):
        rr.set_sinogram(torch.from_numpy(WL.sinogram(w, 0)).cuda())
        rr.fbp()
        for r in (128.0, 256.0):
            region = (c + 100.0, c - 150.0, r, r / 2.0)
            pl = rr.plan(region)
            nx, ny = pl.box[2], pl.box[3]
            lerps = w.iters * (sum(pl.width) * max(nx, ny) + nx * ny * w.n_angles)
            for reg, lam in ((R.ROI_SIRT_NONNEG, 0.0), (R.ROI_TV_CP, w.lam)):
                row = {"radius": r, "box": nx, "solver": "sirt" if reg == R.ROI_SIRT_NONNEG else "tv",
                       "iters": w.iters}
                for key, single in (("team", 1), ("per_operator", 0)):
                    rr.set_option(R.ROI_OPT_SINGLE_LAUNCH, single)
                    rr.solve_local(region, reg, iters=w.iters, lam=lam)  # warm-up (allocations)
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    for _ in range(reps):
                        rr.solve_local(region, reg, iters=w.iters, lam=lam)
                    b.record(stream)
                    torch.cuda.synchronize()
                    ms = a.elapsed_time(b) / reps
                    row[key] = {"ms": ms, "solves_per_s": 1e3 / ms, "Glerp_s": lerps / (ms * 1e-3) / 1e9}
                rr.set_option(R.ROI_OPT_SINGLE_LAUNCH, 1)
                row["speedup"] = row["per_operator"]["ms"] / row["team"]["ms"]
                out.append(row)
    rr.close()
    return out


def small_measure(steps=20, warmup=3):
    """The 128 x 128 workload (64 angles, 128 bins, ROI radius 16 + margin 8: box 48 x 48,
    200 nonnegative SIRT iterations): one step = set sinogram + FBP + exterior + solve, like
    the default line's step; CUDA events around each step; steps cycle over 8 regions."""
    import torch

    import paper_1604_02292_gb300 as R

    w = WL.WORKLOADS["roi_sirt_128"]
    p_dev = torch.from_numpy(WL.sinogram(w, 0)).cuda()
    regions = [WL.region(w, seed=s) for s in range(N_REGIONS)]
    stream = torch.cuda.Stream()
    rr = R.RoiRecon(*w.geometry(), stream=stream)
    plans = [rr.plan(r) for r in regions]
    outs = [torch.empty((pl.box[3], pl.box[2]), dtype=torch.float32, device="cuda") for pl in plans]

    def step(k):
        rr.set_sinogram(p_dev)
        rr.fbp()
        rr.solve_local(regions[k % N_REGIONS], R.ROI_SIRT_NONNEG, iters=w.iters, out=outs[k % N_REGIONS])

    with torch.cuda.stream(stream):
        for k in range(warmup):
            step(k)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for k in range(steps):
            ev[k][0].record(stream)
            step(k)
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    rr.close()
    return {"workload": w.name, "value": steps / (sum(ms) / 1e3), "unit": "solves/s",
            "ms_per_step": statistics.mean(ms), "box": plans[0].box[2], "iters": w.iters, "solver": w.reg,
            "path": "single cooperative launch per solve (k_persist)"}


FCONV_SRCS = ["paper_1604_02292_gb300/csrc/filterconv_tc.cu", "paper_1604_02292_gb300/csrc/dev_common.cuh"]


def tc_issued_flops(n, na, nd):
    """Tensor-pipe FLOPs of one launch of the tensor-core filtered-sinogram kernel: per work
    item (angle, 256 output bins), each 128-bin tile runs 3 tf32 MMAs (hi*hi, hi*lo, lo*hi)
    of 128 x nb x 8 per tap group it meets (nb = filters rounded up to 16)."""
    kb = -(-n // 256)
    nb = -(-(-(-n // kb)) // 16) * 16
    t1n = (2 * nd - 1 + 7) // 8
    steps = 0
    for d0 in range(0, nd, 128):
        steps += min(t1n - 1, (d0 + 127 + nd - 1) // 8) - d0 // 8 + 1
    return na * kb * steps * 3 * 2 * 128 * nb * 8


def filter_conv_measure(reps=3):
    """The filtered sinograms of the paper's own method (Sec. 3.1) at the 1024 filter workload
    (256 angles, 1024 bins, 200 filters from Alg. filtcalc): the tensor-core kernel against
    the FMA-pipe kernel, CUDA events around each launch (the filter packing excluded)."""
    import torch

    import paper_1604_02292_gb300 as R

    w = WL.WORKLOADS["roi_filter_1024"]
    n = w.iters
    rr = R.RoiRecon(*w.geometry())
    p = torch.from_numpy(WL.sinogram(w, 0)).cuda()
    rr.set_sinogram(p)
    rr.filter_prepare(n)
    u, _ = rr.filters(n)
    out = {}
    res = {}
    for path, name in ((0, "tensor_cores"), (1, "fma")):
        rr.set_option(R.ROI_OPT_FILTER_CONV, path)
        res[name] = rr.filter_conv(u, p)  # warm-up
        rr.set_timing(True)
        for _ in range(reps):
            rr.filter_conv(u, p, res[name])
        k, ms = rr.kernel_times(3)
        rr.set_timing(False)
        out[name + "_ms"] = ms / max(k, 1)
    rr.set_option(R.ROI_OPT_FILTER_CONV, 0)
    d = (res["tensor_cores"] - res["fma"]).double()
    out["rel_l2_tensor_vs_fma"] = float(d.norm() / res["fma"].double().norm())
    alg = 2.0 * n * w.n_angles * w.n_det * w.n_det
    issued = tc_issued_flops(n, w.n_angles, w.n_det)
    pk, src = peaks()
    tf32_peak = float(pk.get("bf16_tflops", 1900.0)) * 1.1 / 2.25
    t = out["tensor_cores_ms"] * 1e-3
    out.update({"workload": w.name, "filters": n, "n_angles": w.n_angles, "n_det": w.n_det,
                "algorithmic_gflop": alg / 1e9, "tensor_pipe_gflop": issued / 1e9,
                "speedup_vs_fma": out["fma_ms"] / out["tensor_cores_ms"],
                "roofline": {"bound": "tensor", "kernel": "k_filter_conv_tc", "unit": "TFLOP/s",
                             "achieved": issued / t / 1e12, "peak": tf32_peak, "frac": issued / t / 1e12 / tf32_peak,
                             "algorithmic_TFLOP_s": alg / t / 1e12,
                             "peak_source": f"tf32 dense = {src} bf16 burst x 1.1/2.25 (nominal ratio)",
                             "achieved_counts": "tf32 MMA FLOPs issued (3 split products, padded tiles)",
                             "traffic": profile_traffic(FCONV_SRCS, "profiles/k_filter_conv_tc_filter_1024.md"),
                             "traffic_unit": "DRAM bytes per launch (ncu, profiles/)"}})
    rr.close()
    return out


def local_vs_global(rr, w, p_dev, region, reg, stream):
    """The regularized local solve of `region` against the same solver, lambda and
    iterations on a box covering the whole grid, inside the ROI disk (report only)."""
    import torch

    N = w.N
    glob_region = (0.5 * (N - 1), 0.5 * (N - 1), 0.7072 * N + 1.0, 0.0)
    with torch.cuda.stream(stream):
        rr.set_sinogram(p_dev)
        rr.fbp()
        t0 = time.perf_counter()
        xg, ginfo = rr.solve_local(glob_region, reg, iters=w.iters, lam=w.lam)
        torch.cuda.synchronize()
        t_glob = time.perf_counter() - t0
        xl, linfo = rr.solve_local(region, reg, iters=w.iters, lam=w.lam)
    torch.cuda.synchronize()
    xg, xl = xg.cpu().numpy(), xl.cpu().numpy()
    cx, cy, r, _ = region
    ii, jj = np.meshgrid(np.arange(linfo.box_h) + linfo.box_y0, np.arange(linfo.box_w) + linfo.box_x0,
                         indexing="ij")
    inside = (jj - cx) ** 2 + (ii - cy) ** 2 <= r * r
    a = xl[inside].astype(np.float64)
    b = xg[ii[inside] - ginfo.box_y0, jj[inside] - ginfo.box_x0].astype(np.float64)
    return {"rel_l2_in_roi": float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)),
            "mean_in_roi": [float(a.mean()), float(b.mean())],
            "max_abs_in_roi": [float(np.abs(a).max()), float(np.abs(b).max())],
            "global_box": [ginfo.box_x0, ginfo.box_y0, ginfo.box_w, ginfo.box_h],
            "global_solve_s": t_glob, "solver": w.reg, "iters": w.iters, "lambda": w.lam}


def run_ours(args):
    import torch

    import paper_1604_02292_gb300 as R

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = WL.WORKLOADS[args.workload]
    p_host = WL.sinogram(w, seed=rank)
    regions = [WL.region(w, seed=rank * 1000 + s) for s in range(N_REGIONS)]
    reg = R.ROI_TV_CP if w.reg == "tv" else R.ROI_SIRT_NONNEG
    stream = torch.cuda.Stream()
    rr = R.RoiRecon(*w.geometry(), stream=stream)
    plans = [rr.plan(r) for r in regions]
    p_dev = torch.from_numpy(p_host).cuda()
    outs = [torch.empty((pl.box[3], pl.box[2]), dtype=torch.float32, device="cuda") for pl in plans]
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()

    def step(k):
        j = k % N_REGIONS
        rr.set_sinogram(p_dev)
        rr.fbp()
        rr.solve_local(regions[j], reg, iters=w.iters, lam=w.lam, out=outs[j])

    with torch.cuda.stream(stream):
        for k in range(args.warmup):
            step(k)
    torch.cuda.synchronize()

    # ---- timed region
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    n0 = R.roi_recon_launch_count()
    t_wall0 = time.perf_counter()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.fill_(float(k))          # evict L2 between steps (outside the events)
                ev[k][0].record(stream)
                step(k)
                ev[k][1].record(stream)
        torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    if dist:
        dist.barrier()
    launches = R.roi_recon_launch_count() - n0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    tmax = shard.max_over_ranks(total_s, dist, device="cuda")
    value = shard.throughput(args.steps, ws, tmax)

    # ---- kernels: per-launch device time from CUDA events recorded inside the solve
    pk, pk_src = peaks()
    clocks = clk.summary()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    peak_glerps = N_SM * LERPS_PER_CLK_SM * sm_max * 1e6 / 1e9
    lf, lb = lerps_per_launch(plans[0], w)
    bf, bb = bytes_per_launch(plans[0], w)
    rr.set_timing(True)
    with torch.cuda.stream(stream):
        step(0)
    n_single, ms_single = rr.kernel_times(2)
    rr.set_timing(False)
    # the same solve with one launch per operator, for per-projector figures
    rr.set_option(R.ROI_OPT_SINGLE_LAUNCH, 0)
    rr.set_timing(True)
    with torch.cuda.stream(stream):
        step(0)
    nf, msf = rr.kernel_times(0)
    nb, msb = rr.kernel_times(1)
    rr.set_timing(False)
    rr.set_option(R.ROI_OPT_SINGLE_LAUNCH, 1)
    avg_f, avg_b = msf / max(nf, 1), msb / max(nb, 1)
    if n_single:
        kernel = "k_persist (single-launch CP solve)"
        lerps = w.iters * (lf + lb)
        avg_ms = ms_single / n_single
        alg_bytes = w.iters * (bf + bb)
    else:
        kernel = "k_back (CP)" if msb >= msf else "k_forward (CP)"
        lerps, avg_ms, alg_bytes = (lb, avg_b, bb) if msb >= msf else (lf, avg_f, bf)
    achieved = lerps / (avg_ms * 1e-3) / 1e9
    traffic = profile_traffic(PERSIST_SRCS, "profiles/k_persist_cptv_1024.md") if n_single else None

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        p_pin = torch.from_numpy(p_host).pin_memory()
        outs_h = [torch.empty((pl.box[3], pl.box[2]), dtype=torch.float32).pin_memory().numpy() for pl in plans]
        with torch.cuda.stream(stream):
            for k in range(2):
                rr.set_sinogram(p_pin.numpy())
                rr.fbp()
                rr.solve_local(regions[k % N_REGIONS], reg, iters=w.iters, lam=w.lam, out=outs_h[k % N_REGIONS])
            torch.cuda.synchronize()
            ke = max(3, args.steps // 2)
            t0 = time.perf_counter()
            for k in range(ke):
                j = k % N_REGIONS
                rr.set_sinogram(p_pin.numpy())
                rr.fbp()
                rr.solve_local(regions[j], reg, iters=w.iters, lam=w.lam, out=outs_h[j])  # synchronizes
            te = time.perf_counter() - t0
        te = shard.max_over_ranks(te, dist, device="cuda")
        e2e = {"value": shard.throughput(ke, ws, te), "unit": "solves/s", "h2d_bytes_per_step": int(p_host.nbytes),
               "d2h_bytes_per_step": int(outs_h[0].nbytes), "steps": ke}

    # ---- local vs global regularized solve inside the ROI disk (reported, not a parity claim):
    # the same solver, lambda and iterations on a box covering the whole grid; on the noisy
    # workload sinogram and on the noise-free analytic sinogram of the same phantom
    local_global = None
    if rank == 0 and not args.no_global:
        local_global = local_vs_global(rr, w, p_dev, regions[0], reg, stream)
        local_global["note"] = ("report only (local, global): at this lambda the data term dominates and "
                                "both iterates amplify noise, the local one more")
        p_clean = torch.from_numpy(WL.sinogram(w, seed=rank, noise=False)).cuda()
        local_global["noise_free"] = local_vs_global(rr, w, p_clean, regions[0], reg, stream)

    # ---- serving on the 2048 x 2048 serving workload: continuous batching vs one at a time,
    # in overload (the workload's 2000 requests/s) and at sustainable rates
    serving = None
    if not args.no_serving:
        serving = serve_measure(args, args.requests, dist, ws, rank, local, clock=False)
        serving.pop("w")
        serving.pop("clocks")
        pts = []
        for r in [float(v) for v in args.rates.split(",") if v.strip()]:
            m = serve_measure(args, args.requests, dist, ws, rank, local, clock=False, rate=r)
            pts.append({"rate_per_s": r, "value": m["value"], "latency_ms": m["latency_ms"],
                        "plain": m["plain"], "kernel_launches": m["server"]["kernel_launches"]})
        serving["rates"] = pts

    # ---- the 128 x 128 workload (box 48, 200 SIRT iterations)
    small = None
    if rank == 0 and not args.no_batch:
        small = small_measure()

    # ---- the paper's own method: the filtered sinograms on the tensor cores vs the FMA pipe
    fconv = None
    if rank == 0 and not args.no_batch:
        fconv = filter_conv_measure()

    # ---- lone large boxes (beyond the single-launch solver): team of all blocks vs per operator
    large = None
    if rank == 0 and not args.no_batch:
        large = large_box_measure()

    # ---- batching on the 2048 x 2048 batch workload: all 4096 regions in one persistent launch
    batch = None
    if not args.no_batch:
        wb = WL.BATCHES["roi_batch_2048"]
        batch = batch_measure(wb, None, 1, 1, dist, ws, rank, local, clock=False, tune=True, graph=True)
        batch.pop("clocks")
        batch.update({"workload": wb.name, "N": wb.N, "n_angles": wb.n_angles, "n_det": wb.n_det,
                      "radius": [wb.r_lo, wb.r_hi], "iters": wb.iters, "solvers": "SIRT/TV 50/50",
                      "timing": "CUDA events around one solve_batch call (one persistent launch)"})

    # ---- precision on the 4096 x 4096 precision workload: one wave of regions (one per team
    # of 8 blocks), bfloat16 sinogram with float32 images and with bfloat16 images
    precision = None
    if rank == 0 and not args.no_precision:
        wp = WL.PRECISION["roi_precision_4096"]
        teams = N_SM // 8
        precision = precision_measure(wp, teams, "bf16", 8, teams, local, clock=False)
        precision.pop("clocks")
        precision.update({"workload": wp.name, "N": wp.N, "n_angles": wp.n_angles, "n_det": wp.n_det,
                          "iters": wp.iters, "solver": "CP-TV", "lambda": wp.lam, "I0": wp.I0})

    # ---- CPU baseline: whole oracle solves, measured (rank 0, one GPU only), until about
    # ten seconds of work
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        ts, pts = [], []
        while not ts or (sum(ts) < 10.0 and len(ts) < N_REGIONS):
            t, pt = oracle_solve(w, p_host, regions[len(ts)])
            ts.append(t)
            pts.append(pt)
        mean = [statistics.mean(x[i] for x in pts) for i in range(3)]
        cpu = {"value": len(ts) / sum(ts), "unit": "solves/s", "cores": omp_threads(), "kind": "oracle",
               "sample": (f"{len(ts)} whole FP64 oracle solve(s) of the workload's regions, measured: FBP "
                          f"{mean[0]:.2f} s + exterior {mean[1]:.2f} s + {w.iters} iterations {mean[2]:.2f} s "
                          f"(means)")}

    if rank == 0:
        sm = sorted(step_ms)
        line = {
            "metric": "roi_solves_per_s", "value": value, "unit": "solves/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": w.name, "N": w.N, "n_angles": w.n_angles, "n_det": w.n_det,
                       "roi_radius": w.radius, "roi_margin": w.margin, "box": plans[0].box[2],
                       "solver": w.reg, "iters": w.iters, "lambda": w.lam, "regions": N_REGIONS,
                       "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{ws}"},
            "latency_ms": {"p50": sm[len(sm) // 2], "p99": sm[min(len(sm) - 1, int(math.ceil(0.99 * len(sm))) - 1)],
                           "min": sm[0], "max": sm[-1]},
            "wall_s_timed_region": t_wall,
            "gpu_launches": int(launches),
            "roofline": {"bound": "alu", "kernel": kernel, "achieved": achieved,
                         "peak": peak_glerps, "unit": "Glerp/s", "frac": achieved / peak_glerps,
                         "traffic": traffic, "traffic_unit": "DRAM bytes per launch (ncu, profiles/)", "peak_source": f"derived: {N_SM} SMs x {LERPS_PER_CLK_SM} lerp/clk x "
                                                         f"{sm_max:.0f} MHz ({pk_src} sm_max_mhz)",
                         "launch_ms": avg_ms, "lerps_per_launch": lerps,
                         "algorithmic_GBps": alg_bytes / (avg_ms * 1e-3) / 1e9,
                         "hbm_peak_GBps": pk.get("hbm_gbs")},
            "projectors": {"path": "one launch per operator", "forward_ms": avg_f, "back_ms": avg_b,
                           "forward_lerps": lf, "back_lerps": lb, "launches": [nf, nb],
                           "forward_Glerp_s": lf / max(avg_f, 1e-9) / 1e6, "back_Glerp_s": lb / max(avg_b, 1e-9) / 1e6},
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "local_vs_global": local_global,
            "serving": serving,
            "batch": batch,
            "precision": precision,
            "large_box": large,
            "small_box": small,
            "filter_conv": fconv,
        }
        print(json.dumps(line), flush=True)
    rr.close()
    if dist:
        dist.destroy_process_group()
    return 0


def batch_measure(w, count, steps, warmup, dist, ws, rank, local, clock=True, tune=False, iters=0, graph=False):
    """Batched solves: one step = roi_recon_solve_batch over the regions (one persistent
    launch); the warm-up steps run every region for one iteration (same boxes, so the same
    device slots).  Returns regions/s over all ranks, the per-step times and the lerps/s of
    rank 0 against the derived ceiling.  tune: the phase B tile shapes are first chosen by
    roi_recon_autotune on this sinogram (timed apart), and the default table (16 x 16 for
    every box size) is measured as well.  graph: the same batch is then planned once
    (roi_recon_batch_plan_create) and one step replayed as its captured CUDA graph."""
    import torch

    import paper_1604_02292_gb300 as R

    p = WL.sinogram(w, seed=0)
    all_items = WL.batch_regions(w, seed=0, count=count)
    if iters:
        all_items = [(r, dict(prm, iters=iters)) for r, prm in all_items]
    share = shard.assign([shard.region_cost(r, prm["iters"], w.n_angles) for r, prm in all_items], ws)[rank]
    items = [all_items[i] for i in share]
    regions = [r for r, _ in items]
    params = [prm for _, prm in items]
    warm = [dict(prm, iters=1) for prm in params]
    stream = torch.cuda.Stream()
    rr = R.RoiRecon(*w.geometry(), stream=stream)
    outs = None
    with torch.cuda.stream(stream):
        rr.set_sinogram(torch.from_numpy(p).cuda())
        rr.fbp()
        for _ in range(warmup):
            outs, _ = rr.solve_batch(regions, warm, outs)
    torch.cuda.synchronize()

    def timed_steps():
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        with torch.cuda.stream(stream):
            for k in range(steps):
                ev[k][0].record(stream)
                rr.solve_batch(regions, params, outs)
                ev[k][1].record(stream)
        torch.cuda.synchronize()
        rr.sync()
        return [a.elapsed_time(b) for a, b in ev]

    tuning = None
    if tune:
        default_ms = timed_steps()  # the default table: 16 x 16 tiles for every box size
        t0 = time.perf_counter()
        shapes, tms = rr.autotune()
        tuning = {"shapes_per_class": [list(R.TILE_SHAPES[sh]) for sh in shapes],
                  "classes": ["box side <= 96", "97..216", "217..384"], "trial_ms": tms,
                  "autotune_s": time.perf_counter() - t0,
                  "default_solves_per_s": len(all_items) * steps / (sum(default_ms) / 1e3),
                  "team_caps_per_class": rr.team_caps, "team_cap_candidates": list(R.TEAM_CAPS),
                  "team_trial_ms": rr.team_caps_ms(),
                  "team_note": "team size of few-region batches (8 regions of the class); the 4096-region "
                               "batch itself runs one block per region"}
    if dist:
        dist.barrier()
    n0 = R.roi_recon_launch_count()
    with ClockSampler(local if clock else None) as clk:
        ms = timed_steps()
    launches = int(R.roi_recon_launch_count() - n0)
    graph_out = None
    if graph:
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            plan = rr.batch_plan(regions, params, outs)
        t_plan = time.perf_counter() - t0
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            plan.launch()
            b.record(stream)
        torch.cuda.synchronize()
        g_ms = a.elapsed_time(b)
        plan.close()
        graph_out = {"value": len(items) / (g_ms / 1e3), "unit": "solves/s", "ms": g_ms,
                     "plan_create_s": t_plan,
                     "note": "the batch planned once (tables, descriptors and order uploaded) and replayed "
                             "as one captured CUDA graph: the queue reset and the persistent kernel"}
    n_lerps = 0
    for reg, prm in items:
        pl = rr.plan(reg)
        nx, ny = pl.box[2], pl.box[3]
        n_lerps += prm["iters"] * (sum(pl.width) * max(nx, ny) + nx * ny * w.n_angles)
    rr.close()
    t_mine = sum(ms) / 1e3
    t = shard.max_over_ranks(t_mine, dist, device="cuda")
    pk, pk_src = peaks()
    peak = N_SM * LERPS_PER_CLK_SM * float(pk.get("sm_max_mhz", 2070.0)) * 1e6 / 1e9
    achieved = n_lerps * steps / t_mine / 1e9
    return {"value": len(all_items) * steps / t, "unit": "solves/s", "regions": len(all_items), "steps": steps,
            "ms_per_step": statistics.mean(ms), "gpu_launches": launches,
            "projector_Glerp_s_rank0": achieved, "lerp_ceiling_Glerp_s": peak, "frac_of_ceiling": achieved / peak,
            "autotune": tuning, "graph": graph_out, "clocks": clk.summary()}


def run_batch(args):
    """Batch workload line (see batch_measure); value = regions solved per second."""
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = WL.BATCHES[args.workload]
    m = batch_measure(w, args.batch_count, args.steps, args.warmup, dist, ws, rank, local, tune=args.autotune,
                      iters=args.iters)
    line = {
        "metric": "roi_solves_per_s", "value": m["value"], "unit": "solves/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True,
        "dtype": "f32", "data": "synthetic",
        "scaling": "strong",
        "config": {"workload": w.name, "N": w.N, "n_angles": w.n_angles, "n_det": w.n_det, "regions": m["regions"],
                   "radius": [w.r_lo, w.r_hi], "iters": args.iters or w.iters, "solvers": "SIRT/TV 50/50"},
        "gpu_launches": m["gpu_launches"],
        "projector_Glerp_s_rank0": m["projector_Glerp_s_rank0"],
        "frac_of_lerp_ceiling": m["frac_of_ceiling"],
        "autotune": m["autotune"],
        "clocks": m["clocks"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def _pct(v, q):
    v = sorted(v)
    if not v:
        return None
    k = min(len(v) - 1, max(0, int(math.ceil(q / 100.0 * len(v))) - 1))
    return v[k]


def serve_measure(args, count, dist, ws, rank, local, clock=True, rate=None):
    """Serving run on the serving workload: the requests arrive by a seeded Poisson process
    and are submitted to the server (continuous batching over resident sinograms) at their
    arrival times; latency = completion seen on the host - arrival.  The same requests are
    then solved one at a time with roi_recon_solve_local (FP32, whole GPU per request, host
    output) in arrival order ("plain"), each starting at max(arrival, previous completion).
    Times are host monotonic clocks; results land in host memory in both arms."""
    import torch

    import paper_1604_02292_gb300 as R

    w = WL.SERVING["roi_serve_2048"] if args.workload not in WL.SERVING else WL.SERVING[args.workload]
    rate = args.rate if rate is None else rate
    reqs = WL.serve_requests(w, seed=0, count=count)
    arr = WL.arrivals(w, seed=0, count=count, rate=rate)
    mine = [i for i in range(count) if i % ws == rank]
    recons = []
    for k in range(w.n_sinos):
        rr = R.RoiRecon(*w.geometry())
        rr.set_sinogram(torch.from_numpy(WL.sinogram(w, k)).cuda())
        rr.fbp()
        recons.append(rr)
    torch.cuda.synchronize()
    srv = R.Server(team_blocks=args.team_blocks, teams=args.teams, large_side=args.large_side,
                   solo_queue_ms=args.solo_queue_ms)
    for rr in recons:
        srv.add(rr)
    # warm-up: a few short requests through both paths (first launch, ring allocation)
    for sino, reg, prm in WL.serve_requests(w, seed=99, count=max(args.warmup, 1)):
        srv.submit(sino, reg, dict(prm, iters=5))
        recons[sino].solve_local(reg, reg=prm["reg"], iters=5, lam=prm["lam"])
    srv.drain()
    for c in srv.poll():
        srv.take(c["id"], (c["box"][3], c["box"][2]))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    # ---- served
    n0 = R.roi_recon_launch_count()
    lat, done, who = [], {}, {}
    nbytes = 0
    with ClockSampler(local if clock else None) as clk:
        t0 = time.monotonic()
        i = 0
        while len(done) < len(mine):
            now = time.monotonic()
            while i < len(mine) and t0 + arr[mine[i]] <= now:
                k = mine[i]
                sino, reg, prm = reqs[k]
                who[srv.submit(sino, reg, prm)] = k
                i += 1
            got = srv.poll()
            for c in got:
                if c["status"] != R.ROI_OK:
                    raise R.RoiError(c["status"], "served request failed")
                k = who[c["id"]]
                x = srv.take(c["id"], (c["box"][3], c["box"][2]))
                nbytes += x.nbytes
                done[k] = c
                lat.append(c["t_done_ms"] - (t0 + arr[k]) * 1e3)
            if not got:
                time.sleep(50e-6)
        t_served = max(c["t_done_ms"] for c in done.values()) / 1e3 - t0
    st = srv.stats()
    srv.close()
    launches = int(R.roi_recon_launch_count() - n0)
    # ---- plain: one request at a time, whole GPU, in arrival order
    plain = None
    if not args.no_plain:
        plat = []
        t0 = time.monotonic()
        for k in mine:
            a = t0 + arr[k]
            while time.monotonic() < a:
                time.sleep(20e-6)
            sino, reg, prm = reqs[k]
            pl = recons[sino].plan(reg)
            out = np.empty((pl.box[3], pl.box[2]), np.float32)
            recons[sino].solve_local(reg, reg=prm["reg"], iters=prm["iters"], lam=prm["lam"], out=out)
            plat.append((time.monotonic() - a) * 1e3)
        t_plain = time.monotonic() - t0
        t_plain = shard.max_over_ranks(t_plain, dist, device="cuda")
        plain = {"value": count / t_plain, "unit": "solves/s", "p50_ms": _pct(plat, 50), "p99_ms": _pct(plat, 99),
                 "mean_ms": statistics.mean(plat)}
    t_served = shard.max_over_ranks(t_served, dist, device="cuda")
    n_lerps = 0
    for k in mine:
        sino, reg, prm = reqs[k]
        pl = recons[sino].plan(reg)
        nx, ny = pl.box[2], pl.box[3]
        n_lerps += prm["iters"] * (sum(pl.width) * max(nx, ny) + nx * ny * w.n_angles)
    for rr in recons:
        rr.close()
    return {
        "workload": w.name, "requests": count, "rate_per_s": rate or w.rate, "value": count / t_served,
        "unit": "solves/s", "wall_s": t_served,
        "latency_ms": {"p50": _pct(lat, 50), "p99": _pct(lat, 99), "mean": statistics.mean(lat)},
        "plain": plain,
        "server": {k: st[k] for k in ("blocks", "single_units", "teams", "team_blocks", "kernel_launches",
                                      "device_peak", "host_peak")},
        "d2h_bytes": nbytes, "gpu_launches": launches, "Glerp_s_rank0": n_lerps / t_served / 1e9,
        "clocks": clk.summary(), "w": w,
    }


def run_serve(args):
    """Serving workload line (see serve_measure)."""
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    m = serve_measure(args, args.requests, dist, ws, rank, local)
    w = m.pop("w")
    line = {
        "metric": "roi_solves_per_s_served", "value": m["value"], "unit": "solves/s", "n_gpus": ws,
        "steps": 1, "warmup": args.warmup, "ms_per_step": m["wall_s"] * 1e3, "higher_is_better": True,
        "dtype": "f32", "data": "synthetic", "scaling": "strong",
        "config": {"workload": w.name, "N": w.N, "n_angles": w.n_angles, "n_det": w.n_det, "sinograms": w.n_sinos,
                   "requests": m["requests"], "rate_per_s": m["rate_per_s"], "radius": [w.r_lo, w.r_hi],
                   "iters": w.iters, "solvers": "SIRT/TV 50/50", "timing": "host monotonic clock, arrival to result"},
        "latency_ms": m["latency_ms"],
        "plain": m["plain"],
        "server": m["server"],
        "e2e": {"value": m["value"], "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": m["d2h_bytes"]},
        "gpu_launches": m["gpu_launches"],
        "projector_Glerp_s_rank0": m["Glerp_s_rank0"],
        "clocks": m["clocks"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def precision_measure(w, count, storage, team_blocks, teams, local, clock=True):
    """Precision workload: `count` regions solved through the server (all by teams of
    team_blocks blocks, submitted at once) with the sinogram stored in `storage` ("bf16" or
    "f16"), once with float32 images and once with the FBP and projector images stored in
    `storage` too; then with float32 storage on the same quantized data and on the
    unrounded data.  Errors per result, relative L2: each 16-bit run against the float32
    run fed the same quantized sinogram (the error the storage adds), and against the
    float32 run on the unrounded data (with the rounding of the data themselves)."""
    import torch

    import paper_1604_02292_gb300 as R
    from paper_1604_02292_gb300 import synth

    items = WL.precision_regions(w, seed=0, count=count)
    phantom = synth.random_phantom(w.N, w.n_ellipses, texture=w.texture, seed=0)
    p = synth.poisson_noise(synth.analytic_sinogram(phantom, w.n_angles, w.n_det), w.I0, seed=1000).astype(np.float32)
    st_code = {"f32": R.ROI_F32, "bf16": R.ROI_BF16, "f16": R.ROI_F16}[storage]
    tdt = {R.ROI_F32: torch.float32, R.ROI_BF16: torch.bfloat16, R.ROI_F16: torch.float16}[st_code]
    p_dev = torch.from_numpy(p).cuda()
    p_q = p_dev.to(tdt)  # the quantized data, as the 16-bit handle stores it

    def serve(sino_st, img_st, sino):
        rr = R.RoiRecon(*w.geometry(), storage=sino_st, image_storage=img_st)
        rr.set_sinogram(sino)
        rr.fbp()
        torch.cuda.synchronize()
        srv = R.Server(team_blocks=team_blocks, teams=teams, large_side=1, idle_us=1000)
        srv.add(rr)
        srv.submit(0, items[0][0], dict(items[0][1], iters=2))  # warm-up
        srv.drain()
        for c in srv.poll():
            srv.take(c["id"], (c["box"][3], c["box"][2]))
        time.sleep(0.05)  # the serving kernel leaves after 1 ms idle: the timed run launches it
        n0 = R.roi_recon_launch_count()
        with ClockSampler(local if clock else None) as clk:
            t0 = time.monotonic()
            ids = {srv.submit(0, reg, prm): k for k, (reg, prm) in enumerate(items)}
            srv.drain(3600e3)
            t = time.monotonic() - t0
        res = {}
        for c in srv.poll():
            if c["status"] != R.ROI_OK:
                raise R.RoiError(c["status"], "served request failed")
            res[ids[c["id"]]] = srv.take(c["id"], (c["box"][3], c["box"][2]))
        st = srv.stats()
        srv.close()
        launches = int(R.roi_recon_launch_count() - n0)
        rr.close()
        return t, res, st, launches, clk.summary()

    def rel(a, b):
        return float(np.linalg.norm(a.astype(np.float64) - b) / max(np.linalg.norm(b), 1e-30))

    t_all, r_all, st16, launches, clocks = serve(st_code, st_code, p_dev)
    t_sino, r_sino, _, launches_s, _ = serve(st_code, R.ROI_F32, p_dev)
    t32, r32q, _, _, _ = serve(R.ROI_F32, R.ROI_F32, p_q)    # float32 storage, same quantized data
    _, r32, _, _, _ = serve(R.ROI_F32, R.ROI_F32, p_dev)      # float32 storage, unrounded data

    def errs(r):
        e_store = [rel(r[k], r32q[k]) for k in range(count)]
        e_total = [rel(r[k], r32[k]) for k in range(count)]
        return ({"max": max(e_store), "median": statistics.median(e_store), "per_result": e_store},
                {"max": max(e_total), "median": statistics.median(e_total)})

    pl = R.plan(*w.geometry(), items[0][0])
    nx, ny = pl.box[2], pl.box[3]
    lerps_one = w.iters * (sum(pl.width) * max(nx, ny) + nx * ny * w.n_angles)
    e_all = errs(r_all)
    e_sino = errs(r_sino)
    return {"value": count / t_all, "unit": "solves/s", "regions": count, "box": nx, "wall_s": t_all,
            "storage": storage, "image_storage": storage,
            "error_vs_float32_same_data": e_all[0], "error_vs_float32_unrounded_data": e_all[1],
            "sinogram_only": {"value": count / t_sino, "unit": "solves/s", "image_storage": "f32",
                              "error_vs_float32_same_data": e_sino[0],
                              "error_vs_float32_unrounded_data": e_sino[1]},
            "float32_storage": {"value": count / t32, "unit": "solves/s"},
            "server": {k: st16[k] for k in ("teams", "team_blocks", "device_peak")},
            "gpu_launches": launches + launches_s, "projector_Glerp_s": lerps_one * count / t_all / 1e9,
            "clocks": clocks, "path": "server, teams of blocks, all submitted at once"}


def run_precision(args):
    """Precision workload line (see precision_measure); value = regions/s with 16-bit
    sinogram and images."""
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    w = WL.PRECISION[args.workload]
    count = args.batch_count or 32
    m = precision_measure(w, count, args.storage, args.team_blocks or 8, args.teams, local)
    line = {
        "metric": "roi_solves_per_s", "value": m["value"], "unit": "solves/s", "n_gpus": ws, "steps": 1,
        "warmup": 1, "ms_per_step": m["wall_s"] * 1e3, "higher_is_better": True,
        "dtype": args.storage + " storage, f32 math", "data": "synthetic", "scaling": "strong",
        "config": {"workload": w.name, "N": w.N, "n_angles": w.n_angles, "n_det": w.n_det, "regions": count,
                   "radius": w.radius, "margin": w.margin, "box": m["box"], "iters": w.iters, "solver": "CP-TV",
                   "lambda": w.lam, "I0": w.I0, "path": m["path"]},
    }
    line.update({k: m[k] for k in ("error_vs_float32_same_data", "error_vs_float32_unrounded_data", "sinogram_only",
                                   "float32_storage", "server", "gpu_launches", "projector_Glerp_s", "clocks")})
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_filter(args):
    """The paper's own method (Sec. 3) on the 1024 geometry: preparation (Alg. filtcalc
    filters on the whole grid, disc subtraction, filtered sinograms for every iteration)
    timed once; then the regions solved one at a time (one launch per operator and
    iteration) and as one batch (whole-region solver), against the exterior-subtraction
    nonnegative SIRT of the same regions and iterations.  Quality: relative L2 inside each
    ROI disk against global nonnegative SIRT (the same iterations on the whole grid)."""
    import torch

    import paper_1604_02292_gb300 as R

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    w = WL.WORKLOADS[args.workload]
    p = WL.sinogram(w, seed=0)
    regions = [WL.region(w, seed=s) for s in range(N_REGIONS)]
    rr = R.RoiRecon(*w.geometry())
    rr.set_sinogram(torch.from_numpy(p).cuda())
    rr.fbp()
    torch.cuda.synchronize()
    n0 = R.roi_recon_launch_count()
    t0 = time.perf_counter()
    rr.filter_prepare(w.iters)
    torch.cuda.synchronize()
    t_prep = time.perf_counter() - t0
    # the sinogram-level part alone: a new sinogram with the same geometry
    rr.set_sinogram(torch.from_numpy(WL.sinogram(w, seed=1)).cuda())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rr.filter_prepare(w.iters)
    torch.cuda.synchronize()
    t_sino = time.perf_counter() - t0
    rr.set_sinogram(torch.from_numpy(p).cuda())
    rr.fbp()
    rr.filter_prepare(w.iters)
    torch.cuda.synchronize()

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(reps):
            fn()
        ev[1].record()
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / 1e3 / reps

    # batches of one region per SM (the whole-region solver gives each region one block)
    many = [WL.region(w, seed=s) for s in range(152)]
    with ClockSampler(local) as clk:
        outs_single = {}

        def single():
            for k, reg in enumerate(regions):
                outs_single[k], _ = rr.solve_local(reg, R.ROI_FILTER_SIRT, iters=w.iters)

        t_single = timed(single, max(1, args.steps // 4)) / len(regions)
        prm_f = dict(reg=R.ROI_FILTER_SIRT, iters=w.iters)
        prm_s = dict(reg=R.ROI_SIRT_NONNEG, iters=w.iters)
        res = {}

        def batch_f():
            res["f"], _ = rr.solve_batch(many, [prm_f] * len(many))

        def batch_s():
            res["s"], _ = rr.solve_batch(many, [prm_s] * len(many))

        t_batch_f = timed(batch_f, args.steps) / len(many)
        t_batch_s = timed(batch_s, args.steps) / len(many)
    launches = int(R.roi_recon_launch_count() - n0)
    # quality against global nonnegative SIRT
    c = (w.N - 1) / 2.0
    xg, _ = rr.solve_local((c, c, w.N / 2.0, 0.0), R.ROI_SIRT_NONNEG, iters=w.iters)
    xg = xg.cpu().numpy()
    q_f, q_s = [], []
    for k, reg in enumerate(regions):
        pl = rr.plan(reg)
        x0, y0, bw, bh = pl.box
        jj, ii = np.meshgrid(np.arange(bw) + x0, np.arange(bh) + y0)
        m = (jj - reg[0]) ** 2 + (ii - reg[1]) ** 2 <= reg[2] ** 2
        gref = xg[y0:y0 + bh, x0:x0 + bw][m]
        for out, q in ((res["f"][k], q_f), (res["s"][k], q_s)):
            v = out.cpu().numpy()[m]
            q.append(float(np.linalg.norm(v - gref) / max(np.linalg.norm(gref), 1e-30)))
    pl = rr.plan(regions[0])
    nx, ny = pl.box[2], pl.box[3]
    line = {
        "metric": "roi_solves_per_s", "value": 1.0 / t_batch_f, "unit": "solves/s", "n_gpus": ws,
        "steps": args.steps, "warmup": 1, "ms_per_step": t_batch_f * len(many) * 1e3, "higher_is_better": True,
        "dtype": "f32", "data": "synthetic", "scaling": "weak",
        "config": {"workload": w.name, "N": w.N, "n_angles": w.n_angles, "n_det": w.n_det, "regions": len(many),
                   "roi_radius": w.radius, "roi_margin": w.margin, "box": nx, "iters": w.iters,
                   "method": "Sec. 3 (Alg. filtcalc + Alg. method, x >= 0, disc subtraction)"},
        "prepare_s": {"filters_and_sinogram": t_prep, "sinogram_only": t_sino},
        "single_region_path_solves_per_s": 1.0 / t_single,
        "exterior_sirt_batch_solves_per_s": 1.0 / t_batch_s,
        "quality_regions": len(regions),
        "rel_l2_vs_global_sirt_in_roi": {"paper_method": q_f, "exterior_sirt": q_s},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    rr.close()
    return 0


def run_tile(args):
    """Tiling (Sec. 5.5): the whole 1024 x 1024 image as 64 non-overlapping 128 x 128 local
    reconstructions by the paper's method (x >= 0, 200 iterations) in one batched launch,
    against 200 nonnegative SIRT iterations on the whole grid -- the method the local
    approximation approximates.  Times with CUDA events (the filters and filtered sinograms
    are prepared once, outside the timing); relative L2 difference of the two images inside
    the disk of radius N/2."""
    import torch

    import paper_1604_02292_gb300 as R

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    w = WL.WORKLOADS[args.workload]
    tile = int(2 * w.radius)
    rr = R.RoiRecon(*w.geometry())
    rr.set_sinogram(torch.from_numpy(WL.sinogram(w, seed=0)).cuda())
    rr.fbp()
    t0 = time.perf_counter()
    rr.filter_prepare(w.iters)
    torch.cuda.synchronize()
    t_prep = time.perf_counter() - t0
    prm = dict(reg=R.ROI_FILTER_SIRT, iters=w.iters)
    out = torch.empty((w.N, w.N), device="cuda")
    c = (w.N - 1) / 2.0

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3 / reps

    glob = {}

    def global_solve():
        glob["x"], _ = rr.solve_local((c, c, w.N / 2.0, 0.0), R.ROI_SIRT_NONNEG, iters=w.iters)

    n0 = R.roi_recon_launch_count()
    with ClockSampler(local) as clk:
        t_tiled = timed(lambda: rr.solve_tiled(tile, int(w.margin), prm, out), args.steps)
        t_global = timed(global_solve, max(1, args.steps // 2))
    launches = int(R.roi_recon_launch_count() - n0)
    xt, xg = out.cpu().numpy(), glob["x"].cpu().numpy()
    jj, ii = np.meshgrid(np.arange(w.N) - c, c - np.arange(w.N))
    m = jj ** 2 + ii ** 2 <= (w.N / 2.0) ** 2
    diff = float(np.linalg.norm((xt - xg)[m]) / max(np.linalg.norm(xg[m]), 1e-30))
    line = {
        "metric": "image_reconstructions_per_s", "value": 1.0 / t_tiled, "unit": "images/s", "n_gpus": ws,
        "steps": args.steps, "warmup": 1, "ms_per_step": t_tiled * 1e3, "higher_is_better": True, "dtype": "f32",
        "data": "synthetic", "scaling": "weak",
        "config": {"workload": w.name, "N": w.N, "n_angles": w.n_angles, "n_det": w.n_det, "tiles": (w.N // tile) ** 2,
                   "tile": tile, "margin": w.margin, "method": "Sec. 3, x >= 0", "iters": w.iters},
        "prepare_s": t_prep,
        "global_sirt_ms": t_global * 1e3,
        "rel_l2_tiled_vs_global_sirt_in_disk": diff,
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    rr.close()
    return 0

def run_large(args):
    """Lone large regions through roi_recon_solve_local on the 2048 x 2048 / 180-angle serving
    geometry (one region of radius --radius, margin r/2, CP-TV, --iters iterations): the
    whole-region solver as one team of every block; one step = one solve, CUDA events."""
    import torch

    import paper_1604_02292_gb300 as R

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    w = WL.SERVING["roi_serve_2048"]
    iters = args.iters or w.iters
    c = (w.N - 1) / 2.0
    region = (c + 100.0, c - 150.0, args.radius, args.radius / 2.0)
    stream = torch.cuda.Stream()
    rr = R.RoiRecon(*w.geometry(), stream=stream)
    with torch.cuda.stream(stream):
        rr.set_sinogram(torch.from_numpy(WL.sinogram(w, 0)).cuda())
        rr.fbp()
        for _ in range(args.warmup):
            rr.solve_local(region, R.ROI_TV_CP, iters=iters, lam=w.lam)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    n0 = R.roi_recon_launch_count()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                ev[k][0].record(stream)
                rr.solve_local(region, R.ROI_TV_CP, iters=iters, lam=w.lam)
                ev[k][1].record(stream)
        torch.cuda.synchronize()
    rr.sync()
    ms = [a.elapsed_time(b) for a, b in ev]
    pl = rr.plan(region)
    nx, ny = pl.box[2], pl.box[3]
    lerps = iters * (sum(pl.width) * max(nx, ny) + nx * ny * w.n_angles)
    pk, _ = peaks()
    peak = N_SM * LERPS_PER_CLK_SM * float(pk.get("sm_max_mhz", 2070.0)) * 1e6 / 1e9
    glerps = lerps / (statistics.mean(ms) * 1e-3) / 1e9
    line = {
        "metric": "roi_solves_per_s", "value": args.steps / (sum(ms) / 1e3), "unit": "solves/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(ms), "higher_is_better": True,
        "dtype": "f32", "data": "synthetic", "scaling": "weak",
        "config": {"workload": "roi_large_2048", "N": w.N, "n_angles": w.n_angles, "n_det": w.n_det,
                   "radius": args.radius, "box": nx, "iters": iters, "solver": "CP-TV",
                   "path": "solve_local, whole-region solver, one team of every block"},
        "gpu_launches": int(R.roi_recon_launch_count() - n0),
        "projector_Glerp_s": glerps, "frac_of_lerp_ceiling": glerps / peak,
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    rr.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in WL.WORKLOADS and WL.WORKLOADS[args.workload].reg == "filter":
        return run_filter(args)
    if args.workload in WL.WORKLOADS and WL.WORKLOADS[args.workload].reg == "tile":
        return run_tile(args)
    if args.workload in WL.BATCHES:
        return run_batch(args)
    if args.workload in WL.SERVING:
        return run_serve(args)
    if args.workload in WL.PRECISION:
        return run_precision(args)
    if args.workload == "roi_large_2048":
        return run_large(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
