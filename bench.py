#!/usr/bin/env python3
"""Throughput benchmark of the split Godunov sweep on GB300.

A bench step is one full time step of the scheme (dt, x sweep, y sweep, the
order alternating; §1, Fig. 5) of the workload.  Metric: cell-updates/s
(cells x steps / time), whole job, with HBM GB/s of the sweep kernels against
the measured copy bandwidth.

Default workload (`modes8192`): the 8192x8192 periodic random-mode field,
a smooth non-uniform flow with a genuine Riemann problem at every
interface.  The line's value is the FP32 path; the FP64 path on the same
initial state is timed beside it (`fp64`), and `precision_report` gives the
FP32 density error against FP64 after 200 steps on the FP64 dt sequence.
Other workloads (`--workload`): the Sedov blast (copy-dominated at early
steps: most cells are ambient gas), the Sod tube, the 512-grid batch, the
Kelvin-Helmholtz layer and the paper's 10000^2 point explosion.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   # the FP64 CPU oracle, bounded sample

Under torchrun (N > 1) every rank advances its own replica (the grids are
independent: weak scaling, no collective on the data path); rank 0 prints
one JSON line.  Timing: CUDA events on the library's stream bracketed by a
barrier and a device synchronize, max over ranks.  The default state
(2 x 1.07 GB in FP32) is far larger than the 129 MB L2, so no flush is
needed between steps.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2106_13465_gb300 import problems as pr  # noqa: E402

METRIC = "cell-updates/s"
UNIT = "cell-updates/s"
L2_BYTES = 129 * 1024 * 1024

# name -> (builder, precision, description)
WORKLOADS = {
    "sedov2048_fp64": (lambda: [pr.sedov(2048)], 64,
                       "2048x2048 Sedov blast, FP64, reflective, CFL 0.8, minmod, Newton Riemann (<=10 it); "
                       "early steps are ~99.97 % ambient cells copied by the exact uniform-state shortcuts"),
    "sedov128_fp64": (lambda: [pr.sedov(128)], 64, "128x128 Sedov blast, FP64"),
    "sodx4096_fp64": (lambda: [pr.sod(4096, 16, 0)], 64, "4096x16 Sod tube along x, FP64"),
    "modes4096_fp32": (lambda: [pr.random_modes(4096)], 32,
                       "4096x4096 periodic random-mode field, FP32 (profiling size)"),
    "modes8192_fp32": (lambda: [pr.random_modes(8192)], 32,
                       "8192x8192 periodic random-mode field (8 density and 8 velocity modes, |k| <= 8), FP32 "
                       "storage and arithmetic, FP64 near vacuum, dt and sums; CFL 0.8, minmod, Newton Riemann"),
    "modes2048_fp64": (lambda: [pr.random_modes(2048)], 64,
                       "2048x2048 periodic random-mode field, FP64 (profiling size)"),
    "modes8192_fp64": (lambda: [pr.random_modes(8192)], 64,
                       "8192x8192 periodic random-mode field (8 density and 8 velocity modes, |k| <= 8), FP64"),
    "batch512_fp32": (lambda: pr.batch(512), 32, "512 ragged grids, sides in [32,512], FP32"),
    "batch512_fp64": (lambda: pr.batch(512), 64, "512 ragged grids, sides in [32,512], FP64"),
    "kh16384_fp32": (lambda: [pr.kelvin_helmholtz(16384)], 32,
                     "16384x16384 periodic Kelvin-Helmholtz, FP32"),
    "explosion10000_fp64": (lambda: [pr.sedov(10000)], 64,
                            "10000x10000 point explosion (Sedov blast in the corner), FP64: the "
                            "grid of the paper's own runs (10 steps there)"),
}
# Workloads run in both precisions: the line's value is the first (FP32),
# the second (FP64, same initial state) is reported beside it in `fp64`,
# and `precision_report` holds the FP32 density error after the given number
# of steps against the FP64 run, on the FP64 run's dt sequence.
PAIRS = {
    "modes8192": ("modes8192_fp32", "modes8192_fp64", 200),
}
DEFAULT_WORKLOAD = "modes8192"


def load_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


SWEEP_SOURCES = ("godunov.cuh", "kernels.h", "sweep_tma.cuh", "fused_tma.cuh", "sweep_f64.cu", "sweep_f32.cu")

# FP64 pipe of a GB300: 152 SMs x 2 DFMA per clock x 2 flops x 2070 MHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def strip_comments(src: str) -> str:
    """C/C++ source without its comments and with whitespace runs collapsed
    (string and character literals kept as written), so that an edit of the
    comments alone does not change kernel_source_hash."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        elif c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_source_hash() -> str:
    """Hash of the sweep kernels' sources, comments and layout aside."""
    h = hashlib.sha256()
    for f in SWEEP_SOURCES:
        with open(os.path.join(ROOT, "paper_2106_13465_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(f.encode() + strip_comments(fh.read()).encode())
    return h.hexdigest()[:16]


def recorded_profile(workload: str) -> dict:
    """Figures of the committed ncu summary for this workload's sweep kernel,
    if they were taken on the current kernel sources; else {}."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return {}
    ent = rec.get(workload)
    if not ent or ent.get("source_hash") != kernel_source_hash():
        return {}
    return ent


# ---------------------------------------------------------------- clocks --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "100"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict | None:
        if not self.proc:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if "Active" in r[5 + k] and "Not" not in r[5 + k]:
                    reasons.add(nm)
        busy = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(busy) if busy else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def gpu_uuid(torch, dev: int) -> str | None:
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


# -------------------------------------------------------------- oracle ----
def sample_problem(workload: str, win: int = 512):
    """A bounded sample of the workload for the CPU oracle: its first grid (the
    largest, for a batch) cut to a win x win corner window with the same h
    and boundary conditions.  Field workloads generate only the band of rows
    the window needs (same values as inside the full field)."""
    builder, _prec, _desc = WORKLOADS[workload]
    big = {"modes8192": lambda r: pr.random_modes(8192, rows=r),
           "kh16384": lambda r: pr.kelvin_helmholtz(16384, rows=r)}
    key = workload.rsplit("_", 1)[0]
    if key in big:
        pb = big[key](slice(0, win))
        full = (pb.nx, pb.nx)
    else:
        pbs = builder()
        pb = max(pbs, key=lambda p: p.nx * p.ny)
        full = (pb.nx, pb.ny)
    U = np.ascontiguousarray(pb.U[:, :win, :win])
    if U.shape[1:] == (full[1], full[0]):
        desc = f"the full {full[0]}x{full[1]} {pb.name} grid"
    else:
        desc = (f"{U.shape[2]}x{U.shape[1]} corner window of the {full[0]}x{full[1]} {pb.name} "
                f"state (same h and boundary conditions)")
    return U, pb.h, pb.bc, desc


def oracle_cores() -> int:
    return os.cpu_count() or 1


def oracle_rate(workload: str, budget_s: float, threads: int | None):
    """The FP64 oracle as it stands on a bounded sample of the workload,
    single-threaded (threads None) or its OpenMP build on `threads` threads.
    Returns (cell-updates/s, sample description, steps, seconds)."""
    import oracle as O
    U, h, bc, desc = sample_problem(workload)
    ny, nx = U.shape[1:]
    steps, t0 = 0, time.perf_counter()
    while True:
        U, _, _ = O.run(U, h, bc, 1, step0=steps, threads=threads)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return nx * ny * steps / el, desc, steps, el


def openmp_threads() -> int | None:
    """Threads of the OpenMP oracle build on this host, or None if it cannot
    be built or loaded here."""
    import oracle as O
    try:
        return O.set_threads(oracle_cores())
    except (OSError, subprocess.CalledProcessError):
        return None


def run_reference(args, rank: int):
    if rank != 0:
        return
    import oracle as O
    primary = PAIRS.get(args.workload, (args.workload,))[0]
    U, h, bc, desc = sample_problem(primary)
    ny, nx = U.shape[1:]
    threads = openmp_threads()
    cores = threads or 1
    for k in range(args.warmup):
        U, _, _ = O.run(U, h, bc, 1, step0=k, threads=threads)
    t0 = time.perf_counter()
    for k in range(args.steps):
        U, _, _ = O.run(U, h, bc, 1, step0=args.warmup + k, threads=threads)
    el = time.perf_counter() - t0
    value = nx * ny * args.steps / el
    build = f"OpenMP build on {cores} threads" if threads else "single-threaded build"
    sample = f"each step: one FP64 oracle step ({build}) of the {desc}"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "description": WORKLOADS[primary][2]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------- ours ------
def timed_steps(ctx, steps: int, warmup: int, stream, dist, torch, sampler=None) -> dict:
    """Warm up, then time exactly `steps` steps with CUDA events on the
    library's stream, bracketed by a barrier and a device synchronize; the
    max over ranks.  Then the per-launch durations of a few more steps."""
    ctx.step(warmup)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = ctx.stats()["kernel_launches"]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.step(steps)
    e1.record(stream)
    launches = ctx.stats()["kernel_launches"] - launches0
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    # per-kernel durations (same stream, CUDA events around each launch)
    kp = max(2, min(steps, 20))
    kstep0 = ctx.get_step()
    kern = ctx.step_profiled(kp)
    par = (kstep0 + np.arange(kp)) % 2  # even steps sweep x first, odd steps y first
    return {"ms": ms, "launches": launches, "clocks": clocks,
            "sweep_ms": float(np.mean(kern[:, 1:])), "prologue_ms": float(np.mean(kern[:, 0])),
            "step_kernels_ms": float(np.mean(kern[:, 1] + kern[:, 2])),
            "x_ms": float(np.mean(np.where(par == 0, kern[:, 1], kern[:, 2]))),
            "y_ms": float(np.mean(np.where(par == 0, kern[:, 2], kern[:, 1])))}


def roofline_for(workload: str, prec: int, cells: int, m: dict, fused: bool = False) -> dict:
    """Roofline of the dominant kernel: the sweep kernel (mean of the x and y
    launches), or with fused steps the step kernel.  HBM view: algorithmic
    bytes, a read and a write of the 4 planes of every cell per launch (a
    sweep, or a whole fused step); FP64 with a recorded flop count also the
    FP64-pipe view; `bound` is the one with the larger fraction.  `traffic`:
    ncu DRAM bytes per launch recorded on the current kernel sources, else
    null."""
    peaks = load_peaks()
    key = workload + ("_fused" if fused else "")
    prof = recorded_profile(key)
    esz = 8 if prec == 64 else 4
    sweep_ms = m["step_kernels_ms"] if fused else m["sweep_ms"]
    alg_bytes = 2.0 * 4 * esz * cells
    hbm_peak = peaks.get("hbm_gbs") or 6800.0
    hbm_achieved = alg_bytes / (sweep_ms * 1e-3) / 1e9
    hbm = {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
           "frac": hbm_achieved / hbm_peak,
           "peak_source": "measured" if peaks.get("hbm_gbs") else "fallback"}
    flops_cell = prof.get("fp64_flops_per_cell_sweep")
    alu = None
    if prec == 64 and flops_cell:
        # a fused launch does both sweeps of every cell
        achieved = flops_cell * (2 if fused else 1) * cells / (sweep_ms * 1e-3) / 1e12
        alu = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
               "frac": achieved / FP64_PEAK_TFLOPS,
               "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (FP64 pipe)",
               "flops_per_cell_sweep": flops_cell}
    if alu and alu["frac"] >= hbm["frac"]:
        roof = dict(alu, hbm_view=hbm)
    else:
        roof = dict(hbm)
        if alu:
            roof["alu_view"] = alu
    roof["traffic"] = prof.get("dram_bytes_per_sweep")
    if fused:
        kname = "fused_step_kernel (with its second pass)"
    elif prec == 64:
        kname = "sweep_walk_kernel, x and y walks (mean of both)"
    else:
        kname = "sweep_x_kernel (x segments) / sweep_walk_kernel (y walk), mean of both"
    roof.update({"kernel": kname,
                 "launch_ms": sweep_ms, "algorithmic_bytes_per_launch": alg_bytes})
    return roof


def run_ours(args, rank: int, world: int, local_rank: int):
    import torch
    from paper_2106_13465_gb300 import hydro as H

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    wl = args.workload
    primary, companion, l1_default = PAIRS.get(wl, (wl, None, 0))
    l1_steps = l1_default if args.l1_steps is None else args.l1_steps
    builder, prec, desc = WORKLOADS[primary]
    pbs = builder()
    grids = [(p.nx, p.ny, p.h, p.bc) for p in pbs]
    cells = sum(p.nx * p.ny for p in pbs)
    esz = 8 if prec == 64 else 4
    state_bytes = sum(4 * p.ny * ((p.nx + 31) // 32 * 32) * esz for p in pbs)

    tuning = None
    if args.autotune:
        from paper_2106_13465_gb300.autotune import autotune
        tuning = autotune(pbs, precision=prec, steps=3, warmup=1).tuning()

    stream = torch.cuda.Stream()
    ctx = H.Context(grids, precision=prec, stream=stream.cuda_stream)
    if args.fused is not None:
        tuning = dict(tuning or {}, fused=args.fused)
    if tuning:
        ctx.set_tuning(graph_steps=20, **tuning)
    for g, p in enumerate(pbs):
        ctx.set_state(g, p.U)

    # ---- timed region: K steps, state resident in HBM --------------------
    sampler = ClockSampler(gpu_uuid(torch, local_rank)) if rank == 0 else None
    m = timed_steps(ctx, args.steps, args.warmup, stream, dist, torch, sampler)
    value = world * cells * args.steps / (m["ms"] * 1e-3)

    # ---- end to end through the C ABI with host buffers -------------------
    ke = max(1, min(args.steps, 10))
    host = [torch.empty((4, p.ny, p.nx), dtype=torch.float64).pin_memory() for p in pbs]
    for g, p in enumerate(pbs):
        host[g].numpy()[:] = ctx.get_state(g)
    step0 = ctx.get_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for k in range(ke):
        for g, p in enumerate(pbs):
            H.hydro_set_state(ctx.ctx, g, host[g].data_ptr(), 0)
        ctx.set_step(step0 + k)
        ctx.step(1)
        for g, p in enumerate(pbs):
            ctx._check(H.hydro_get_state(ctx.ctx, g, host[g].data_ptr(), 0))
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    if dist:
        t = torch.tensor([el], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        el = float(t.item())
    del host
    bytes_io = 4 * cells * 8
    e2e = {"value": world * cells * ke / el, "unit": UNIT, "h2d_bytes_per_step": bytes_io,
           "d2h_bytes_per_step": bytes_io, "steps": ke,
           "path": "hydro_set_state from pinned FP64 host arrays, hydro_step(1), hydro_get_state"}
    stats = ctx.stats()
    ctx.close()

    # ---- FP64 on the same problem: the L1 reference run, then its timing ----
    fp64 = None
    precision_report = None
    if companion or (prec == 32 and l1_steps > 0):
        c64 = H.Context(grids, precision=64, stream=stream.cuda_stream)
        if args.fused is not None:
            c64.set_tuning(graph_steps=20, fused=args.fused)
        for g, p in enumerate(pbs):
            c64.set_state(g, p.U)
        dts = ref = None
        if l1_steps > 0 and rank == 0:
            dts = c64.step(l1_steps, record_dt=True)
            ref = [c64.get_state(g)[0] for g in range(len(pbs))]
        if companion:
            m64 = timed_steps(c64, args.steps, args.warmup, stream, dist, torch)
            v64 = world * cells * args.steps / (m64["ms"] * 1e-3)
            fp64 = {"workload": companion, "description": WORKLOADS[companion][2],
                    "value": v64, "unit": UNIT, "ms_per_step": m64["ms"] / args.steps,
                    "steps": args.steps, "warmup": args.warmup, "gpu_launches": m64["launches"],
                    "start_step": (l1_steps if rank == 0 else 0),
                    "kernels_ms": {"prologue": m64["prologue_ms"], "sweep": m64["sweep_ms"],
                                   "step_kernels": m64["step_kernels_ms"],
                                   "x_sweep": m64["x_ms"], "y_sweep": m64["y_ms"]},
                    "roofline": roofline_for(companion, 64, cells, m64, bool(args.fused))}
        c64.close()
        if ref is not None:
            with H.Context(grids, precision=32, stream=stream.cuda_stream) as c32:
                for g, p in enumerate(pbs):
                    c32.set_state(g, p.U)
                c32.step(l1_steps, dt_override=dts)
                got = [c32.get_state(g)[0] for g in range(len(pbs))]
                fb = c32.stats()["riemann_fp64"]
            num = sum(float(np.abs(a - b).sum()) for a, b in zip(got, ref))
            den = sum(float(np.abs(b).sum()) for b in ref)
            precision_report = {"l1_rho_rel_fp32_vs_fp64": num / den, "steps": l1_steps,
                                "definition": "sum |rho32 - rho64| / sum |rho64| over all cells",
                                "dt": "the FP64 run's dt sequence replayed in FP32",
                                "riemann_fp64_solves": fb}

    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    roofline = roofline_for(primary, prec, cells, m, bool(args.fused))

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        half = args.cpu_seconds / 2
        r1, sample, s1, t1 = oracle_rate(primary, half, None)
        threads = openmp_threads()
        if threads:
            rn, _, sn, tn = oracle_rate(primary, half, threads)
            cpu = {"value": rn, "unit": UNIT, "cores": threads, "kind": "oracle",
                   "sample": f"{sample}; OpenMP build (lines of a sweep shared among threads, "
                             f"bit-identical results): {sn} steps in {tn:.1f} s",
                   "single_thread": {"value": r1, "cores": 1, "steps": s1, "seconds": round(t1, 2)}}
        else:
            cpu = {"value": r1, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"{sample}; single-threaded build: {s1} steps in {t1:.1f} s"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == 64 else "f32",
        "data": "synthetic",
        "config": {"workload": wl, "description": desc, "grids": len(pbs), "cells": cells,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": f"state {2 * state_bytes / 1e6:.0f} MB > L2 {L2_BYTES / 1e6:.0f} MB, no flush",
                   "tuning": tuning or "model default"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": m["launches"],
        "clocks": m["clocks"],
        "kernels_ms": {"prologue": m["prologue_ms"], "sweep": m["sweep_ms"],
                       "step_kernels": m["step_kernels_ms"], "x_sweep": m["x_ms"],
                       "y_sweep": m["y_ms"]},
        "riemann_fp64_fallbacks": stats["riemann_fp64"],
        "fp64": fp64,
        "precision_report": precision_report,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS) + sorted(PAIRS))
    ap.add_argument("--cpu-seconds", type=float, default=16.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--l1-steps", type=int, default=None,
                    help="FP32 workloads: report the L1 density error against FP64 after this many "
                         "steps (default: 200 for the paired workloads, else 0)")
    ap.add_argument("--autotune", action="store_true",
                    help="time candidate launch shapes first and use the fastest")
    ap.add_argument("--fused", type=int, default=None, choices=[0, 1],
                    help="1: one fused step kernel per step (both sweeps of a tile in shared memory); "
                         "0: two sweep kernels; default: the library default (0)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
