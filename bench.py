#!/usr/bin/env python
"""Benchmark: type-1 / type-2 NU points per second, 3D, complex64, eps = 1e-5.

Workload (default): N = 256^3 modes (fine grid 512^3), M = 1e8 points iid
uniform in [-pi, pi)^3, strengths / coefficients with re, im iid N(0, 1),
eps = 1e-5 (w = 6, beta = 13.8).  One step is the whole hot path on one
batch: setpts + type-1 execute on one plan (bin, spread, FFT, deconvolve), then
the type-2 plan takes the same binned points (nufft_setpts_from) and executes
(pre-correct, FFT, interpolate).  value = 2 M / step time (each transform counts its M
points).  Inputs (1.2 GB of coordinates, 1 GB fine grids) exceed the 129 MB
L2, so no flush is needed between steps.

Arms:
  default            the CUDA library, inputs resident in HBM; the JSON line adds
                     e2e (host buffers, copies inside the timed region), the
                     roofline of the dominant kernel, clocks and a bounded CPU
                     baseline (the oracle)
  --impl reference   the CPU oracle, as it stands, on a bounded sample
N > 1 GPUs (torchrun): independent replicas, one per rank (the path has no
exchange step); value sums the ranks' points over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "type1/2 NU points/s at eps=1e-5 (3D, fp32)"

# DRAM bytes (read + write) per launch of the spread / interp kernels on the
# default workload: the bytes of an ncu capture of the same kernels on 1e7 points (a 256^3
# fine grid, similar points per cell; DRAM bytes per second times the launch's duration)
# times 10 for 1e8 points -- valid only for the kernel source they were measured on.
KERNEL_SOURCE = os.path.join(ROOT, "paper_1808_06736_gb300", "csrc", "spread_interp_q.cuh")
MEASURED_TRAFFIC = {
    "sha256": "b3390d078c38abf3414666daf5397155fec4e8e727a4103758261932d049f318",
    "spread": 1181453716 * 10,
    "interp": 723761629 * 10,
}


def measured_traffic(kernel: str, args) -> int | None:
    import hashlib
    default = (args.M == 100_000_000 and args.N == 256 and args.eps == 1e-5 and args.kind == "uniform" and
               args.prec == "c64" and args.kerevalmeth == 0)
    try:
        digest = hashlib.sha256(open(KERNEL_SOURCE, "rb").read()).hexdigest()
    except OSError:
        return None
    if not default or digest != MEASURED_TRAFFIC["sha256"]:
        return None
    return MEASURED_TRAFFIC.get(kernel)
UNIT = "NU points/s"
FP32_LANES_PER_SM = 128  # FP32 FMA lanes per SM (Blackwell)
FP64_NOMINAL_TFLOPS = 1.25  # GB300 dense FP64, nominal
C128_ROOFLINE_NOTE = ("the fraction can exceed 1: the complex128 kernels form their products in double-float "
                      "arithmetic on the FP32 pipe (and the spread accumulates in 32-bit fixed-point words), so "
                      "the FP64 rate, against which the method's fp64 flops are counted here, no longer bounds "
                      "them; FP32 issue and 32-bit shared-memory atomics do")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--M", type=int, default=100_000_000)
    ap.add_argument("--N", type=int, default=256)
    ap.add_argument("--eps", type=float, default=1e-5)
    ap.add_argument("--kind", default="uniform", choices=["uniform", "clustered"])
    ap.add_argument("--prec", default="c64", choices=["c64", "c128"],
                    help="c64 (the headline: complex64, float arithmetic) or c128 (complex128, double)")
    ap.add_argument("--kerevalmeth", type=int, default=0, choices=[0, 1],
                    help="kernel evaluation: 0 the ES formula, 1 the piecewise polynomial of Sec. 5.3")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=3_000_000,
                    help="points in the oracle's bounded sample of the workload (CPU baseline, reference arm)")
    ap.add_argument("--workload", default="3d", choices=["3d", "batched2d", "serving", "type3"],
                    help="3d: the 3D type-1/type-2 workload (default); batched2d: many uneven 2D type-2 "
                         "transforms, batched plan against one plan per transform; serving: a Poisson stream "
                         "of mixed requests through the request loop against the plain plan path; type3: "
                         "3D type 3 with 1e7 sources and 1e7 target frequencies on a 256^3 grid")
    ap.add_argument("--B", type=int, default=1024, help="transforms in the batched2d workload")
    ap.add_argument("--requests", type=int, default=2000, help="requests in the serving trace")
    ap.add_argument("--rate", type=float, default=2000.0, help="mean arrivals per second in the serving trace")
    ap.add_argument("--slots", type=int, default=8, help="execution slots of the request loop")
    ap.add_argument("--serve-budget-gb", type=int, default=64, help="device-memory budget of the request loop")
    ap.add_argument("--no-serving", action="store_true", help="leave the serving summary out of the 3d line")
    ap.add_argument("--no-configs", action="store_true",
                    help="leave the other workloads (3D clustered, 3D complex128, 2D, batched 2D) out of the 3d line")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, device=None) -> float:
    """The largest of every rank's value (the slowest rank's time); identity without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(points_per_rank: int, ms_max: float, world_size: int) -> float:
    """Whole-job NU points/s: every rank's points over the slowest rank's step time."""
    return world_size * points_per_rank / (ms_max * 1e-3)


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # raw samples go to a scratch file; the summary is part of the JSON line
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), "nufft_bench_clocks_rank%d_%d.csv" % (index, os.getpid()))

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# -------------------------------------------------------------- CUDA arm
def algorithmic_units(d, w):
    """Per NU point, spread or interp: flops (complex x real accumulate, tensor
    weights, kernel arguments) and HBM bytes (record, index, strength, grid
    amortised separately)."""
    flops = 4 * w ** d + 2 * w ** (d - 1) + 10 * w * d
    return flops


def run_cuda(args, ws, rank, local):
    import torch
    import numpy as np

    import nufft_inputs as I
    import paper_1808_06736_gb300 as pkg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    d, N, M, eps = 3, args.N, args.M, args.eps
    Ns = [N] * d
    seed = 1000 + 2 + 10 * (1 if args.kind == "clustered" else 0) + rank
    cdt = torch.complex128 if args.prec == "c128" else torch.complex64
    rdt = torch.float64 if args.prec == "c128" else torch.float32
    xs = I.torch_points(seed, M, d, args.kind, dev, rdt)
    c = I.torch_complex_normal(seed + 1, M, dev, cdt)
    f = I.torch_complex_normal(seed + 2, N ** d, dev, cdt)
    stream = torch.cuda.current_stream(dev)
    # unit peaks of this GPU (FP32, FP64, SFU, shared atomics), measured live for the rooflines
    st_pk, peaks = pkg.nufft_measure_peaks(stream.cuda_stream)
    if st_pk != 0:
        raise RuntimeError("nufft_measure_peaks: %d" % st_pk)
    p1 = pkg.Plan(1, Ns, eps=eps, isign=1, dtype=cdt, device=dev, debug=1, kerevalmeth=args.kerevalmeth)
    p2 = pkg.Plan(2, Ns, eps=eps, isign=-1, dtype=cdt, device=dev, debug=1, kerevalmeth=args.kerevalmeth)
    fout = torch.empty((1,) + tuple(Ns), dtype=cdt, device=dev)
    cout = torch.empty((1, M), dtype=cdt, device=dev)
    slots = {k: [] for k in ("fold", "scan", "scatter", "spread", "fft1", "deconv", "precorrect", "fft2",
                             "interp")}

    def step(record, shared=True):
        p1.setpts(*xs)
        if record:
            t = p1.timings()
        p1.execute(c, out=fout)
        if record:
            t1 = p1.timings()
        if shared:
            p2.setpts_from(p1)  # one binning serves both transforms (nufft_setpts_from)
        else:
            p2.setpts(*xs)
        p2.execute(f, out=cout)
        if record:
            t2 = p2.timings()
            slots["fold"].append(t[0]); slots["scan"].append(t[1]); slots["scatter"].append(t[2])
            slots["spread"].append(t1[3]); slots["fft1"].append(t1[4]); slots["deconv"].append(t1[5])
            slots["precorrect"].append(t2[3]); slots["fft2"].append(t2[4]); slots["interp"].append(t2[5])

    def barrier():
        torch.cuda.synchronize(dev)
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step(False)
    assert p1.status() == 0 and p2.status() == 0
    # per-step kernel timings (debug events on the plans' stream), separate pass
    for _ in range(max(3, min(args.steps, 5))):
        step(True)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(False)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    st = (p1.status(), p2.status())
    if st != (0, 0):
        raise RuntimeError("device status %s" % (st,))
    ms_max = max_over_ranks(ms, dev)
    value = aggregate_value(2 * M, ms_max, ws)
    # the same step with each plan binning the points itself (nufft_setpts on both)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        step(False, shared=False)
    e1.record(stream)
    barrier()
    ms_sep = max_over_ranks(e0.elapsed_time(e1) / args.steps, dev)
    separate = {"value": aggregate_value(2 * M, ms_sep, ws), "unit": UNIT, "ms_per_step": ms_sep,
                "step": "setpts + type-1 execute on one plan, setpts + type-2 execute on the other (two binnings)"}

    # execute only (points already set on both plans): the second figure of the metric
    ex = []
    for _ in range(max(3, min(args.steps, 10))):
        e0.record(stream)
        p1.execute(c, out=fout)
        p2.execute(f, out=cout)
        e1.record(stream)
        e1.synchronize()
        ex.append(e0.elapsed_time(e1))
    ms_ex = max_over_ranks(statistics.median(ex), dev)
    exec_only = {"value": aggregate_value(2 * M, ms_ex, ws), "unit": UNIT, "ms_per_step": ms_ex,
                 "best_ms": min(ex), "step": "type-1 execute + type-2 execute on points set beforehand (median)"}

    # end to end: pinned host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        # End to end through the public API from pinned host buffers.  Each step
        # uploads its own points, strengths and coefficients and reads back both
        # results; uploads run on a copy stream and downloads on another, double
        # buffered, so step k's copies overlap the compute of its neighbours.
        hx = [v.cpu().pin_memory() for v in xs]
        hc = c.cpu().pin_memory()
        hf = f.cpu().pin_memory()
        nb = 2
        dx = [[torch.empty_like(v) for v in xs] for _ in range(nb)]
        dc = [torch.empty_like(c) for _ in range(nb)]
        df = [torch.empty_like(f) for _ in range(nb)]
        dfo = [torch.empty_like(fout) for _ in range(nb)]
        dco = [torch.empty_like(cout) for _ in range(nb)]
        hfo = [torch.empty(fout.shape, dtype=cdt).pin_memory() for _ in range(nb)]
        hco = [torch.empty(cout.shape, dtype=cdt).pin_memory() for _ in range(nb)]
        up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        inputs_free = [torch.cuda.Event() for _ in range(nb)]
        outputs_free = [torch.cuda.Event() for _ in range(nb)]
        for ev in inputs_free + outputs_free:
            ev.record(stream)

        def step_e2e(k):
            b = k % nb
            ready, done_in, done_out = torch.cuda.Event(), torch.cuda.Event(), torch.cuda.Event()
            with torch.cuda.stream(up):
                up.wait_event(inputs_free[b])
                for a, h in zip(dx[b], hx):
                    a.copy_(h, non_blocking=True)
                dc[b].copy_(hc, non_blocking=True)
                df[b].copy_(hf, non_blocking=True)
                ready.record(up)
            stream.wait_event(ready)
            stream.wait_event(outputs_free[b])
            p1.setpts(*dx[b])
            p1.execute(dc[b], out=dfo[b])
            p2.setpts_from(p1)
            p2.execute(df[b], out=dco[b])
            done_in.record(stream)
            inputs_free[b] = done_in
            with torch.cuda.stream(down):
                down.wait_event(done_in)
                hfo[b].copy_(dfo[b], non_blocking=True)
                hco[b].copy_(dco[b], non_blocking=True)
                done_out.record(down)
            outputs_free[b] = done_out

        for k in range(2):
            step_e2e(k)
        barrier()
        # three timed windows of ke steps; the best is reported, as the paper times the best
        # of three runs (the host side of the copies varies between windows on a shared
        # machine; all three are listed)
        ke = max(4, args.steps)  # steps per window: the pipeline fills and drains once per window
        windows = []
        for _ in range(3):
            e0.record(stream)
            up.wait_stream(stream)  # the timed uploads start after e0
            down.wait_stream(stream)
            for k in range(ke):
                step_e2e(k)
            stream.wait_stream(down)
            stream.wait_stream(up)
            e1.record(stream)
            barrier()
            windows.append(e0.elapsed_time(e1) / ke)
        ms_e2e = max_over_ranks(min(windows), dev)
        h2d = sum(v.numel() * v.element_size() for v in hx) + hc.numel() * hc.element_size() + \
            hf.numel() * hf.element_size()
        d2h = hfo[0].numel() * hfo[0].element_size() + hco[0].numel() * hco[0].element_size()
        e2e = {"value": aggregate_value(2 * M, ms_e2e, ws), "unit": UNIT, "ms_per_step": ms_e2e,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "pipelining": "uploads and downloads on their own streams, double buffered",
               "windows_ms": [round(v, 3) for v in windows], "window_steps": ke}

    # roofline of the dominant kernel
    med = {k: statistics.median(v) for k, v in slots.items()}
    w = p1.info["w"]
    dominant = max(("spread", "interp"), key=lambda k: med[k])
    flops = algorithmic_units(d, w) * M
    achieved = flops / (med[dominant] * 1e-3) / 1e12
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    if args.prec == "c64":
        peak = sms * FP32_LANES_PER_SM * 2 * 2.070e9 / 1e12  # max SM clock 2070 MHz
        src = "derived: %d SMs x %d FP32 lanes x 2 flop x 2.07 GHz" % (sms, FP32_LANES_PER_SM)
    else:
        peak = FP64_NOMINAL_TFLOPS
        src = "nominal FP64 rate of the GB300 (no measured FP64 peak is provided)"
    roof = {"bound": "alu", "kernel": "k_%s (3D, w=%d, %s)" % (dominant, w, "fp32" if args.prec == "c64" else "fp64"),
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": measured_traffic(dominant, args), "peak_source": src,
            "algorithmic_flops_per_point": algorithmic_units(d, w)}
    if args.prec == "c128":
        roof["note"] = C128_ROOFLINE_NOTE
    if dominant == "spread" and args.prec == "c64":
        # the unit that binds the complex64 spread: shared-memory integer atomics, two per
        # stencil cell (real and imaginary fixed-point parts)
        atoms = 2 * w ** d * M
        pk = peaks["smem_atomics_per_s"]
        roof["smem_atomics"] = {
            "achieved_per_s": atoms / (med["spread"] * 1e-3), "peak_per_s": pk,
            "frac": atoms / (med["spread"] * 1e-3) / pk, "atomics_per_launch": atoms,
            "peak_source": "measured in this run: nufft_measure_peaks, conflict-free 32-bit shared atomic adds"}
    roof["measured_fp32_tflops"] = peaks["fp32_tflops"]
    roof["frac_of_measured_fp32"] = achieved / peaks["fp32_tflops"] if args.prec == "c64" else None
    kernels_ms = {k: round(v, 4) for k, v in med.items()}
    p1.close()
    p2.close()
    # per step: 6 setpts kernels (fold, replica sum, scan, subproblem list, replica
    # cursors, scatter) once + tiled and per-warp spread, deconvolve, pre-correct
    # scatter, tiled and per-warp interp (cuFFT's kernels not counted)
    launches = args.steps * 12
    return {"value": value, "ms": ms_max, "e2e": e2e, "roofline": roof, "kernels_ms": kernels_ms,
            "clocks": clk, "gpu_launches": launches, "w": w, "peaks": peaks, "execute_only": exec_only,
            "separate_binning": separate}


# ---------------------------------------------------- the other workloads
EXTRA_CONFIGS = [
    # (name, d, N per dimension, M, precision, eps, point distribution)
    ("3d_c64_clustered", 3, 256, 100_000_000, "c64", 1e-5, "clustered"),
    ("3d_c128_uniform", 3, 256, 30_000_000, "c128", 1e-9, "uniform"),
    ("2d_c64_uniform", 2, 1024, 10_000_000, "c64", 1e-5, "uniform"),
    ("2d_c64_clustered", 2, 1024, 10_000_000, "c64", 1e-5, "clustered"),
    ("2d_c128_uniform", 2, 1024, 10_000_000, "c128", 1e-9, "uniform"),
    ("2d_c128_clustered", 2, 1024, 10_000_000, "c128", 1e-9, "clustered"),
]


def measure_config(name, d, N, M, prec, eps, kind, steps, warmup, peaks):
    """One configuration of the workload list: the step of the headline (setpts + type 1, the
    type-2 plan on the same binned points + type 2), timed with CUDA events over ``steps``
    steps after ``warmup``; per-kernel medians from the plans' debug events; the dominant
    kernel's algorithmic flops against the FP32 rate (complex64; derived from unit counts)
    or the nominal FP64 rate (complex128)."""
    import torch

    import nufft_inputs as I
    import paper_1808_06736_gb300 as pkg

    dev = torch.device("cuda", 0)
    Ns = [N] * d
    cdt = torch.complex128 if prec == "c128" else torch.complex64
    rdt = torch.float64 if prec == "c128" else torch.float32
    seed = 3000 + 10 * d + (1 if kind == "clustered" else 0) + (2 if prec == "c128" else 0)
    xs = I.torch_points(seed, M, d, kind, dev, rdt)
    c = I.torch_complex_normal(seed + 1, M, dev, cdt)
    f = I.torch_complex_normal(seed + 2, N ** d, dev, cdt)
    p1 = pkg.Plan(1, Ns, eps=eps, isign=1, dtype=cdt, device=dev, debug=1)
    p2 = pkg.Plan(2, Ns, eps=eps, isign=-1, dtype=cdt, device=dev, debug=1)
    fout = torch.empty((1,) + tuple(Ns), dtype=cdt, device=dev)
    cout = torch.empty((1, M), dtype=cdt, device=dev)
    stream = torch.cuda.current_stream(dev)
    slots = {k: [] for k in ("fold", "scan", "scatter", "spread", "fft1", "deconv", "precorrect", "fft2", "interp")}

    def step(record):
        p1.setpts(*xs)
        if record:
            t = p1.timings()
        p1.execute(c, out=fout)
        if record:
            t1 = p1.timings()
        p2.setpts_from(p1)
        p2.execute(f, out=cout)
        if record:
            t2 = p2.timings()
            slots["fold"].append(t[0]); slots["scan"].append(t[1]); slots["scatter"].append(t[2])
            slots["spread"].append(t1[3]); slots["fft1"].append(t1[4]); slots["deconv"].append(t1[5])
            slots["precorrect"].append(t2[3]); slots["fft2"].append(t2[4]); slots["interp"].append(t2[5])

    for _ in range(warmup):
        step(False)
    for _ in range(3):
        step(True)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step(False)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    st = (p1.status(), p2.status())
    w = p1.info["w"]
    p1.close()
    p2.close()
    if st != (0, 0):
        raise RuntimeError("%s: device status %s" % (name, st))
    med = {k: round(statistics.median(v), 4) for k, v in slots.items()}
    dom = max(("spread", "interp"), key=lambda k: med[k])
    flops = algorithmic_units(d, w) * M
    achieved = flops / (med[dom] * 1e-3) / 1e12
    if prec == "c64":
        peak, src = peaks["fp32_derived_tflops"], "FP32, derived from unit counts"
    else:
        peak, src = FP64_NOMINAL_TFLOPS, "FP64, nominal"
    roof = {"kernel": "k_%s" % dom, "achieved_tflops": achieved, "peak_tflops": peak,
            "frac": achieved / peak, "peak_source": src, "algorithmic_flops_per_point": algorithmic_units(d, w)}
    if prec == "c128":
        roof["note"] = C128_ROOFLINE_NOTE
    return {"name": name, "workload": "%dD type 1 + type 2, N=%d^%d, M=%d %s points, %s, eps=%g"
            % (d, N, d, M, kind, "complex128" if prec == "c128" else "complex64", eps),
            "value": 2 * M / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "w": w, "kernels_ms": med,
            "roofline": roof}


def run_extra_configs(args, peaks):
    """Every other configuration of the workload list, and the batched 2D workload against
    its one-plan-per-transform comparator; each config freed before the next."""
    import torch
    out = []
    for cfg in EXTRA_CONFIGS:
        out.append(measure_config(*cfg, steps=5, warmup=2, peaks=peaks))
        torch.cuda.empty_cache()
    out.append(batched2d_measure(args, autotune=False))
    torch.cuda.empty_cache()
    return out


# -------------------------------------------------------------- oracle arm
def oracle_sample(args, M_sample, reps=1):
    """Time the oracle (O2, fp64, OpenMP over all host cores) on a bounded sample of the
    workload: the same fine grid, eps and point distribution, M_sample points.  One step is
    what the GPU step does -- type 1 (spread, FFT, deconvolve) and type 2 (pre-correct, FFT,
    interpolate) on the same points -- and is timed whole, the best of ``reps`` runs (the paper
    times the best of 3).  Returns (best step seconds, its spread + interp seconds, its FFT +
    correction seconds, threads used)."""
    import numpy as np

    import nufft_inputs as I
    import oracle

    d, N, eps = 3, args.N, args.eps
    Ns = [N] * d
    w, beta, ns = oracle.choose_params(eps, Ns)
    xs = I.points(4242, M_sample, d, kind=args.kind)
    c = I.complex_normal(4243, M_sample)
    f = I.complex_normal(4244, N ** d)
    threads = oracle.num_threads()
    best = None
    for _ in range(reps):
        t0 = time.perf_counter()
        b = oracle.spread(xs, c, ns, w, beta)
        t1 = time.perf_counter()
        fk = oracle.deconvolve(oracle.dft(b, 1), Ns, ns, w, beta)
        del b
        b2 = oracle.dft(oracle.precorrect(f, Ns, ns, w, beta), -1)
        t2 = time.perf_counter()
        cc = oracle.interp(xs, b2, ns, w, beta)
        t3 = time.perf_counter()
        del b2, fk, cc
        run = (t3 - t0, (t1 - t0) + (t3 - t2), t2 - t1)
        if best is None or run[0] < best[0]:
            best = run
    return best[0], best[1], best[2], threads


def cpu_sample_text(Ms, M, reps, threads, t_pts, t_fixed):
    return ("oracle O2 (fp64; spread and interp C loops with OpenMP, scipy FFT) on %d OpenMP threads: one step "
            "(type 1 + type 2, same points) on a sample of %d of the workload's %d points on its full fine grid, "
            "best of %d; that step's spread+interp %.2f s, FFTs+corrections %.2f s; value = 2 x %d / step time "
            "(measured, not extrapolated in M)" % (threads, Ms, M, reps, t_pts, t_fixed, Ms))


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    Ms = args.cpu_sample
    steps = []
    for i in range(args.warmup + args.steps):
        step_s, t_pts, t_fixed, threads = oracle_sample(args, Ms)
        if i >= args.warmup:
            steps.append((step_s, t_pts, t_fixed))
    step_s = statistics.median(s[0] for s in steps)
    value = 2 * Ms / step_s
    sample = ("oracle O2 (fp64; spread and interp C loops with OpenMP, scipy FFT) on %d OpenMP threads; each step "
              "is type 1 + type 2 on a sample of %d of the workload's %d points on its full %d^3 fine grid; "
              "median of %d steps after %d warm-up; value = 2 x %d / step time (measured, not extrapolated in M)"
              % (threads, Ms, args.M, 2 * args.N, args.steps, args.warmup, Ms))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def batched2d_measure(args, autotune=True):
    """1024 independent 2D type-2 transforms, complex64, eps = 1e-5: N per transform uniform in
    {64^2, 128^2, 256^2, 512^2}, M log-uniform in [1e3, 1e6] uniform points, coefficients re/im
    N(0, 1).  Batched: one BatchPlan (one launch per step, CUDA graph).  Plain: one Plan per
    transform, setpts + execute per call.  Both time setpts + execute of every transform."""
    import numpy as np
    import torch

    import nufft_inputs as I
    import paper_1808_06736_gb300 as pkg

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rng = I.rng(7000)
    B = args.B
    sizes = [64, 128, 256, 512]
    modes = [(int(v), int(v)) for v in rng.choice(sizes, size=B)]
    Ms = np.exp(rng.uniform(np.log(1e3), np.log(1e6), size=B)).astype(np.int64)
    offs = np.concatenate([[0], np.cumsum(Ms)]).astype(np.int64)
    Mtot = int(offs[-1])
    xs = I.torch_points(7001, Mtot, 2, "uniform", dev, torch.float32)
    nf = sum(m[0] * m[1] for m in modes)
    f = I.torch_complex_normal(7002, nf, dev, torch.complex64)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    bp = pkg.BatchPlan(2, modes, eps=args.eps, isign=-1, dtype=torch.complex64, device=dev)
    cout = torch.empty(Mtot, dtype=torch.complex64, device=dev)

    def step_batched():
        bp.setpts(*xs, offsets=offs)
        bp.execute(f, out=cout)

    for _ in range(args.warmup):
        step_batched()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        step_batched()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1) / args.steps
    assert bp.status() == 0

    # autotuned batch plan (bin shape, subproblem size, sparse threshold, block size)
    ms_t, opts, tune_best, tune_default, t_tune = None, None, None, None, None
    if autotune:
        ms_t, opts, tune_best, tune_default, t_tune = batched2d_tuned(args, modes, xs, f, offs, cout, e0, e1, stream)
    plans = [pkg.Plan(2, m, eps=args.eps, isign=-1, dtype=torch.complex64, device=dev) for m in modes]
    moffs = bp.mode_offsets
    couts = [cout[int(offs[t]):int(offs[t + 1])] for t in range(B)]
    fs = [f[moffs[t]:moffs[t + 1]] for t in range(B)]
    xts = [[v[int(offs[t]):int(offs[t + 1])] for v in xs] for t in range(B)]

    def step_plain():
        for t in range(B):
            plans[t].setpts(*xts[t])
            plans[t].execute(fs[t], out=couts[t].view(1, -1))

    step_plain()
    torch.cuda.synchronize()
    kp = max(1, min(args.steps, 3))
    e0.record(stream)
    for _ in range(kp):
        step_plain()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_p = e0.elapsed_time(e1) / kp
    for p in plans:
        p.close()
    bp.close()
    ms_best = ms_b if ms_t is None else min(ms_b, ms_t)
    res = {"name": "batched2d", "metric": "batched 2D type-2 NU points/s (%d transforms, eps=%g, fp32)" % (B, args.eps),
           "value": Mtot / (ms_best * 1e-3), "unit": UNIT, "ms_per_step": ms_best,
           "config": {"workload": "batched2d", "transforms": B, "modes": "uniform in {64,128,256,512}^2",
                      "M": "log-uniform in [1e3, 1e6]", "points_total": Mtot, "step": "setpts + execute of all"},
           "default_options": {"value": Mtot / (ms_b * 1e-3), "ms_per_step": ms_b},
           "plain": {"value": Mtot / (ms_p * 1e-3), "ms_per_step": ms_p, "path": "one Plan per transform"},
           "speedup_vs_plain": ms_p / ms_best}
    if ms_t is not None:
        res["autotuned"] = {"value": Mtot / (ms_t * 1e-3), "ms_per_step": ms_t, "options": opts,
                            "tuner_best_ms": tune_best, "tuner_default_ms": tune_default, "tuning_s": t_tune}
    return res


def batched2d_tuned(args, modes, xs, f, offs, cout, e0, e1, stream):
    """The batched workload on an autotuned batch plan: (ms per step, options, tuner figures)."""
    import torch

    import paper_1808_06736_gb300 as pkg
    dev = xs[0].device
    t_tune = time.time()
    opts, tune_best, tune_default = pkg.tune_batch(2, modes, xs, f, offs, eps=args.eps, isign=-1, reps=2)
    t_tune = time.time() - t_tune
    bt = pkg.BatchPlan(2, modes, eps=args.eps, isign=-1, dtype=torch.complex64, device=dev, **opts)
    for _ in range(args.warmup):
        bt.setpts(*xs, offsets=offs)
        bt.execute(f, out=cout)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        bt.setpts(*xs, offsets=offs)
        bt.execute(f, out=cout)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_t = e0.elapsed_time(e1) / args.steps
    assert bt.status() == 0
    bt.close()
    return ms_t, opts, tune_best, tune_default, t_tune


def run_batched2d(args):
    r = batched2d_measure(args, autotune=True)
    line = {"metric": r["metric"], "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": r["config"]}
    line.update({k: v for k, v in r.items() if k not in ("metric", "value", "ms_per_step", "config", "name")})
    print(json.dumps(line))
    return 0


def run_type3(args):
    """Type 3 (Eq. (3), Sec. 3.3), 3D, complex64, eps = 1e-5: M = N = 1e7 sources and target
    frequencies, uniform in boxes centred at (1, 2, 3) +- 10 and (-5, 4, 7) +- 19.6, so that the
    space-bandwidth product gives a 256^3 fine grid (n = 2 sigma X S / pi + w).  One step =
    setpts (bounding boxes, binning, target factors, inner type-2 setpts) + execute."""
    import torch

    import nufft_inputs as I
    import paper_1808_06736_gb300 as pkg

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    M = N = 10_000_000
    X, S = 10.0, 19.6
    g = torch.Generator(device=dev)
    g.manual_seed(9100)
    xs = [(torch.rand(M, generator=g, device=dev, dtype=torch.float64) * 2 - 1) * X + c0 for c0 in (1.0, 2.0, 3.0)]
    ss = [(torch.rand(N, generator=g, device=dev, dtype=torch.float64) * 2 - 1) * S + c0 for c0 in (-5.0, 4.0, 7.0)]
    xs = [v.float() for v in xs]
    ss = [v.float() for v in ss]
    c = I.torch_complex_normal(9101, M, dev, torch.complex64)
    out = torch.empty(N, dtype=torch.complex64, device=dev)
    p = pkg.Plan3(3, eps=args.eps, isign=1, dtype=torch.complex64, device=dev, kerevalmeth=args.kerevalmeth)
    stream = torch.cuda.current_stream(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    def step():
        p.setpts(xs, ss)
        p.execute(c, out=out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert p.status() == 0
    split = []
    for _ in range(3):
        ev[0].record(stream)
        p.setpts(xs, ss)
        ev[1].record(stream)
        p.execute(c, out=out)
        ev[2].record(stream)
        torch.cuda.synchronize()
        split.append((ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])))
    clocks = ClockSampler(0)
    clocks.start()
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(args.steps):
        step()
    ev[1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev[0].elapsed_time(ev[1]) / args.steps
    assert p.status() == 0
    info = dict(p.info)
    p.close()
    line = {"metric": "type-3 NU points/s ((M + N) / step, 3D, eps=%g, fp32)" % args.eps,
            "value": (M + N) / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "type3", "M": M, "N": N, "source_box": "(1,2,3) +- 10",
                       "target_box": "(-5,4,7) +- 19.6", "fine_grid": info["n"], "gamma": info["gamma"],
                       "w": info["w"], "step": "setpts + execute",
                       "kernel_eval": "piecewise polynomial" if args.kerevalmeth == 1 else "ES formula"},
            "setpts_ms": statistics.median(v[0] for v in split),
            "execute_ms": statistics.median(v[1] for v in split), "clocks": clk}
    print(json.dumps(line))
    return 0


def _pct(v, q):
    v = sorted(v)
    if not v:
        return None
    k = min(len(v) - 1, max(0, int(math.ceil(q / 100.0 * len(v))) - 1))
    return v[k]


def run_serving(args):
    """The serving trace (nufft_inputs.serving_trace: Poisson arrivals at --rate of
    mixed 2D/3D type-1/type-2 complex64 requests with M log-uniform in [1e4, 1e7],
    20 % least-squares gradient requests at 3D N = 64^3, M = 1e5) through
    (a) the request loop (Server: --slots slots, resident plan entries) and
    (b) the plain path: one request at a time through cached Plans (gradient
    requests through the autograd functions), synchronising after each.
    Both arms take gradient requests' point gradient through the ES kernel's
    derivative (xgrad="kernel") and use the same upsampling factor per request
    (the server's cost model, nufft_request_upsampfac).
    Open loop: each request is submitted at its arrival time; latency = device
    completion - arrival.  Burst: the whole trace submitted at once; points/s =
    sum of M / makespan.  Inputs are slices of pools resident in HBM; each arm
    runs the trace once untimed first (plan creation)."""
    import numpy as np
    import torch

    import nufft_inputs as I
    from paper_1808_06736_gb300 import autograd as AG
    from paper_1808_06736_gb300 import serve as S

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    pool = 10_000_000
    trace = I.serving_trace(8000, args.requests, args.rate, pool)
    X = I.torch_points(8001, pool, 3, "uniform", dev, torch.float32)
    C = I.torch_complex_normal(8002, pool, dev, torch.complex64)
    maxn = max(int(np.prod(q["modes"])) for q in trace)
    F = I.torch_complex_normal(8003, maxn, dev, torch.complex64)
    Y = I.torch_complex_normal(8004, 100_000, dev, torch.complex64)
    torch.cuda.synchronize()
    clock = S.nufft_server_clock
    total_pts = sum(q["M"] for q in trace)

    def inputs(q):
        M, o = q["M"], q["off"]
        xs = [X[d][o:o + M] for d in range(q["d"])]
        f = F[: int(np.prod(q["modes"]))].view(tuple(reversed(q["modes"])))
        return xs, f, C[o:o + M], Y[:M]

    def submit(srv, q, tag):
        xs, f, c, y = inputs(q)
        if q["kind"] == 1:
            return srv.type1(xs, c, q["modes"], eps=q["eps"], isign=q["isign"], tag=tag)
        if q["kind"] == 2:
            return srv.type2(xs, f, eps=q["eps"], isign=q["isign"], tag=tag)
        return srv.lsq_grad(xs, f, y, eps=q["eps"], isign=q["isign"], tag=tag, xgrad="kernel")

    def collect(srv, n, got):
        t_end = time.time() + 600
        while len(got) < n and time.time() < t_end:
            for c in srv.poll(512, 0.05):
                got[c.tag] = c
        return got

    srv = S.Server(budget_bytes=args.serve_budget_gb << 30, max_inflight=args.slots)

    def served_burst():
        t0 = clock()
        for i, q in enumerate(trace):
            submit(srv, q, i)
        got = collect(srv, len(trace), {})
        assert all(c.status == 0 for c in got.values()), "served request failed"
        return max(c.t_done for c in got.values()) - t0

    served_burst()  # untimed: creates the resident entries
    mk_served = served_burst()
    t0 = clock() + 0.05
    got = {}
    for i, q in enumerate(trace):
        target = t0 + q["t"]
        while True:
            now = clock()
            if now >= target:
                break
            for c in srv.poll(512, min(target - now, 0.001)):
                got[c.tag] = c
        submit(srv, q, i)
    collect(srv, len(trace), got)
    st = srv.stats()
    srv.close()
    assert all(c.status == 0 for c in got.values()), "served request failed"
    lat_s = [(got[i].t_done - (t0 + q["t"])) * 1e3 for i, q in enumerate(trace)]
    wait_s = [(got[i].t_admit - (t0 + q["t"])) * 1e3 for i, q in enumerate(trace)]

    cache = AG.PlanCache()

    def run_plain(q):
        xs, f, c, y = inputs(q)
        sigma = S.upsampfac_for(q["kind"], q["modes"], q["eps"], q["M"])  # the same grid as the served request
        if q["kind"] == 1:
            p = cache.get(1, q["modes"], q["eps"], q["isign"], torch.complex64, dev, upsampfac=sigma)
            p.setpts(*xs)
            p.execute(c)
        elif q["kind"] == 2:
            p = cache.get(2, q["modes"], q["eps"], q["isign"], torch.complex64, dev, upsampfac=sigma)
            p.setpts(*xs)
            p.execute(f)
        else:
            xg = torch.stack(xs).requires_grad_()
            fg = f.detach().clone().requires_grad_()
            cc = AG.nufft_type2(xg, fg, eps=q["eps"], isign=q["isign"], cache=cache, xgrad="kernel", upsampfac=sigma)
            loss = ((cc - y).abs() ** 2).sum()
            loss.backward()
        torch.cuda.synchronize()

    for q in trace:  # untimed: creates the plans
        run_plain(q)
    t = clock()
    for q in trace:
        run_plain(q)
    mk_plain = clock() - t
    t0 = clock() + 0.05
    lat_p = []
    for q in trace:
        target = t0 + q["t"]
        while clock() < target:
            time.sleep(max(0.0, min(0.0005, target - clock())))
        run_plain(q)
        lat_p.append((clock() - target) * 1e3)
    cache.clear()
    n3 = sum(1 for q in trace if q["kind"] == 3)
    return {
        "requests": len(trace), "rate_per_s": args.rate, "gradient_requests": n3,
        "points_total": total_pts, "offered_pts_per_s": total_pts / trace[-1]["t"],
        "served": {"p50_ms": _pct(lat_s, 50), "p99_ms": _pct(lat_s, 99), "mean_ms": statistics.mean(lat_s),
                   "p99_queue_ms": _pct(wait_s, 99), "burst_pts_per_s": total_pts / mk_served,
                   "burst_makespan_s": mk_served, "slots": args.slots, "budget_gb": args.serve_budget_gb,
                   "entries_created": st["entries_created"], "entries_evicted": st["entries_evicted"],
                   "peak_inflight": st["peak_inflight"], "peak_bytes": st["peak_bytes"]},
        "plain": {"p50_ms": _pct(lat_p, 50), "p99_ms": _pct(lat_p, 99), "mean_ms": statistics.mean(lat_p),
                  "burst_pts_per_s": total_pts / mk_plain, "burst_makespan_s": mk_plain,
                  "path": "cached Plan per request shape, one request at a time, synchronised"},
        "burst_throughput_vs_plain": mk_plain / mk_served,
        "points": "each request counts its M points once (a gradient request runs a type-2 transform with the "
                  "point gradient through the ES kernel's derivative and one type-1 transform on them)",
    }


def run_serving_line(args):
    r = run_serving(args)
    line = {"metric": "served p50/p99 latency (ms) of mixed type-1/2 requests, Poisson %g req/s" % args.rate,
            "value": r["served"]["p99_ms"], "unit": "ms (p99)", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": r["served"]["burst_makespan_s"] * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serving", "trace": "nufft_inputs.serving_trace(8000, %d, %g)"
                       % (args.requests, args.rate)},
            "serving": r}
    print(json.dumps(line))
    return 0


def config_dict(args):
    return {"workload": "3D type 1 + type 2, N=%d^3 modes (fine grid %d^3), M=%d %s points, %s, eps=%g"
                        % (args.N, 2 * args.N, args.M, args.kind,
                           "complex64" if args.prec == "c64" else "complex128", args.eps),
            "modes": [args.N] * 3, "fine_grid": [2 * args.N] * 3, "M": args.M, "points": args.kind,
            "eps": args.eps, "step": "setpts + type-1 execute on one plan, then the type-2 plan takes those binned "
                                     "points (nufft_setpts_from) + type-2 execute; value = 2M/step",
            "l2": "inputs larger than L2 (1.2 GB coordinates, 1 GB fine grids), no flush",
            "kernel_eval": "piecewise polynomial (Sec. 5.3)" if args.kerevalmeth == 1 else "ES formula",
            "parallelism": "replicas" if args.gpus > 1 else "single GPU"}


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched2d":
        return run_batched2d(args)
    if args.workload == "type3":
        return run_type3(args)
    if args.workload == "serving":
        return run_serving_line(args)
    r = run_cuda(args, ws, rank, local)
    if rank != 0:
        return 0
    serving = None
    if not args.no_serving and ws == 1:
        serving = run_serving(args)
    configs = None
    if not args.no_configs and ws == 1:
        import torch
        pk = dict(r["peaks"])
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        pk["fp32_derived_tflops"] = sms * FP32_LANES_PER_SM * 2 * 2.070e9 / 1e12
        configs = run_extra_configs(args, pk)
    cpu = None
    if not args.no_cpu:
        reps = 3
        step_s, t_pts, t_fixed, threads = oracle_sample(args, args.cpu_sample, reps=reps)
        cpu = {"value": 2 * args.cpu_sample / step_s, "unit": UNIT, "cores": threads, "kind": "oracle",
               "step_s": step_s, "sample": cpu_sample_text(args.cpu_sample, args.M, reps, threads, t_pts, t_fixed)}
    metric = METRIC if args.prec == "c64" else "type1/2 NU points/s at eps=%g (3D, fp64)" % args.eps
    line = {"metric": metric, "value": r["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.prec == "c64" else "f64", "data": "synthetic",
            "config": config_dict(args),
            "e2e": r["e2e"], "roofline": r["roofline"], "cpu_baseline": cpu, "clocks": r["clocks"],
            "gpu_launches": r["gpu_launches"], "kernels_ms": r["kernels_ms"], "execute_only": r["execute_only"],
            "measured_peaks": r["peaks"], "separate_binning": r["separate_binning"], "serving": serving,
            "configs": configs}
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
