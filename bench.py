#!/usr/bin/env python3
"""Throughput benchmark of the split Godunov sweep on GB300.

A bench step is one full time step of the scheme (dt, x sweep, y sweep, the
order alternating; §1, Fig. 5) of the workload.  Default workload: the
2048x2048 FP64 Sedov blast (reflective box, total energy 1 in the corner
cell).  Metric: cell-updates/s (cells x steps / time), whole job.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   # the FP64 CPU oracle, bounded sample

Under torchrun (N > 1) every rank advances its own replica (the grids are
independent: weak scaling, no collective on the data path); rank 0 prints
one JSON line.  Timing: CUDA events on the library's stream bracketed by a
barrier and a device synchronize, max over ranks.  The state (2 x 134 MB for
the default workload) is larger than the 129 MB L2, so no flush is needed
between steps.
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
                       "2048x2048 Sedov blast, FP64, reflective, CFL 0.8, minmod, Newton Riemann (<=10 it)"),
    "sedov128_fp64": (lambda: [pr.sedov(128)], 64, "128x128 Sedov blast, FP64"),
    "sodx4096_fp64": (lambda: [pr.sod(4096, 16, 0)], 64, "4096x16 Sod tube along x, FP64"),
    "modes4096_fp32": (lambda: [pr.random_modes(4096)], 32,
                       "4096x4096 periodic random-mode field, FP32 (profiling size)"),
    "modes8192_fp32": (lambda: [pr.random_modes(8192)], 32,
                       "8192x8192 periodic random-mode field, FP32"),
    "modes2048_fp64": (lambda: [pr.random_modes(2048)], 64,
                       "2048x2048 periodic random-mode field, FP64 (profiling size)"),
    "modes8192_fp64": (lambda: [pr.random_modes(8192)], 64,
                       "8192x8192 periodic random-mode field, FP64"),
    "batch512_fp32": (lambda: pr.batch(512), 32, "512 ragged grids, sides in [32,512], FP32"),
    "batch512_fp64": (lambda: pr.batch(512), 64, "512 ragged grids, sides in [32,512], FP64"),
    "kh16384_fp32": (lambda: [pr.kelvin_helmholtz(16384)], 32,
                     "16384x16384 periodic Kelvin-Helmholtz, FP32"),
    "explosion10000_fp64": (lambda: [pr.sedov(10000)], 64,
                            "10000x10000 point explosion (Sedov blast in the corner), FP64: the "
                            "grid of the paper's own runs (10 steps there)"),
}
DEFAULT_WORKLOAD = "sedov2048_fp64"


def load_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


SWEEP_SOURCES = ("godunov.cuh", "kernels.h", "sweep_tma.cuh", "sweep_f64.cu", "sweep_f32.cu")

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
def oracle_rate(workload: str, budget_s: float, max_steps: int | None = None):
    """The FP64 oracle as it stands, single-threaded, on a bounded sample of the
    workload.  Returns (cell-updates/s, sample description, steps, seconds)."""
    import oracle as O
    O.build()
    pbs = WORKLOADS[workload][0]()
    pb = max(pbs, key=lambda p: p.nx * p.ny)
    win = 512
    if pb.nx > win or pb.ny > win:
        U = pb.U[:, :win, :win].copy()
        sample = (f"{win}x{win} corner window of the {pb.nx}x{pb.ny} {pb.name} state "
                  f"(same h and boundary conditions), oracle steps run back to back")
    else:
        U = pb.U.copy()
        sample = f"the full {pb.nx}x{pb.ny} {pb.name} grid"
    ny, nx = U.shape[1:]
    steps, t0 = 0, time.perf_counter()
    while True:
        U, _, _ = O.run(U, pb.h, pb.bc, 1, step0=steps)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (max_steps and steps >= max_steps):
            break
    return nx * ny * steps / el, sample, steps, el


def run_reference(args, rank: int):
    if rank != 0:
        return
    wl = args.workload
    import oracle as O
    O.build()
    pbs = WORKLOADS[wl][0]()
    pb = max(pbs, key=lambda p: p.nx * p.ny)
    win = min(512, pb.nx), min(512, pb.ny)
    U = pb.U[:, :win[1], :win[0]].copy()
    for k in range(args.warmup):
        U, _, _ = O.run(U, pb.h, pb.bc, 1, step0=k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        U, _, _ = O.run(U, pb.h, pb.bc, 1, step0=args.warmup + k)
    el = time.perf_counter() - t0
    value = win[0] * win[1] * args.steps / el
    sample = (f"each step: one oracle step of the {win[0]}x{win[1]} corner window of "
              f"{pb.name} (same h and boundary conditions)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wl, "description": WORKLOADS[wl][2]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------- ours ------
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
    builder, prec, desc = WORKLOADS[wl]
    pbs = builder()
    cells = sum(p.nx * p.ny for p in pbs)
    esz = 8 if prec == 64 else 4
    state_bytes = sum(4 * p.ny * ((p.nx + 31) // 32 * 32) * esz for p in pbs)

    tuning = None
    if args.autotune:
        from paper_2106_13465_gb300.autotune import autotune
        tuning = autotune(pbs, precision=prec, steps=3, warmup=1).tuning()

    stream = torch.cuda.Stream()
    ctx = H.Context([(p.nx, p.ny, p.h, p.bc) for p in pbs], precision=prec,
                    stream=stream.cuda_stream)
    if tuning:
        ctx.set_tuning(graph_steps=20, **tuning)
    for g, p in enumerate(pbs):
        ctx.set_state(g, p.U)
    ctx.step(args.warmup)
    torch.cuda.synchronize()

    # ---- timed region: K steps, state resident in HBM --------------------
    sampler = ClockSampler(gpu_uuid(torch, local_rank)) if rank == 0 else None
    if sampler:
        sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = ctx.stats()["kernel_launches"]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.step(args.steps)
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
    value = world * cells * args.steps / (ms * 1e-3)

    # ---- per-kernel durations (same stream, CUDA events per launch) -------
    kp = max(2, min(args.steps, 20))
    kstep0 = ctx.get_step()
    kern = ctx.step_profiled(kp)
    sweep_ms = float(np.mean(kern[:, 1:]))
    prologue_ms = float(np.mean(kern[:, 0]))
    # even steps sweep x first, odd steps y first
    par = (kstep0 + np.arange(kp)) % 2
    x_ms = float(np.mean(np.where(par == 0, kern[:, 1], kern[:, 2])))
    y_ms = float(np.mean(np.where(par == 0, kern[:, 2], kern[:, 1])))

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
    bytes_io = 4 * cells * 8
    e2e = {"value": world * cells * ke / el, "unit": UNIT, "h2d_bytes_per_step": bytes_io,
           "d2h_bytes_per_step": bytes_io, "steps": ke}

    stats = ctx.stats()
    ctx.close()

    # ---- FP32 against FP64 on the same dt sequence (outside the timing) ----
    precision_report = None
    if prec == 32 and args.l1_steps > 0 and world == 1:
        grids = [(p.nx, p.ny, p.h, p.bc) for p in pbs]
        with H.Context(grids, precision=64) as c64:
            for g, p in enumerate(pbs):
                c64.set_state(g, p.U)
            dts = c64.step(args.l1_steps, record_dt=True)
            ref = [c64.get_state(g)[0] for g in range(len(pbs))]
        with H.Context(grids, precision=32) as c32:
            for g, p in enumerate(pbs):
                c32.set_state(g, p.U)
            c32.step(args.l1_steps, dt_override=dts)
            got = [c32.get_state(g)[0] for g in range(len(pbs))]
            fb = c32.stats()["riemann_fp64"]
        num = sum(float(np.abs(a - b).sum()) for a, b in zip(got, ref))
        den = sum(float(np.abs(b).sum()) for b in ref)
        precision_report = {"l1_rho_rel_fp32_vs_fp64": num / den, "steps": args.l1_steps,
                            "dt": "FP64 run's dt sequence replayed in FP32",
                            "riemann_fp64_solves": fb}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (the sweep) ----------------------
    peaks = load_peaks()
    prof = recorded_profile(wl)
    alg_bytes = 2.0 * 4 * esz * cells  # one read + one write of the 4 planes of every cell per sweep
    hbm_peak = peaks.get("hbm_gbs") or 6800.0
    hbm_achieved = alg_bytes / (sweep_ms * 1e-3) / 1e9
    hbm = {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
           "frac": hbm_achieved / hbm_peak,
           "peak_source": "measured" if peaks.get("hbm_gbs") else "fallback"}
    flops_cell = prof.get("fp64_flops_per_cell_sweep")
    alu = None
    if prec == 64 and flops_cell:
        # FP64 pipe: flops per cell-sweep counted by ncu on this kernel and workload
        achieved = flops_cell * cells / (sweep_ms * 1e-3) / 1e12
        alu = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
               "frac": achieved / FP64_PEAK_TFLOPS,
               "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (FP64 pipe)",
               "flops_per_cell_sweep": flops_cell}
    # the bound reported is the resource the kernel uses the larger fraction of
    # (an FP64 workload whose cells are mostly uniform copies is closer to HBM)
    if alu and alu["frac"] >= hbm["frac"]:
        roofline = dict(alu, hbm_view=hbm)
    else:
        roofline = dict(hbm)
        if alu:
            roofline["alu_view"] = alu
    roofline["traffic"] = prof.get("dram_bytes_per_sweep")
    roofline.update({"kernel": "sweep_kernel", "launch_ms": sweep_ms,
                     "algorithmic_bytes_per_launch": alg_bytes})

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        rate, sample, osteps, osec = oracle_rate(wl, budget_s=args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{sample}; {osteps} steps in {osec:.1f} s"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == 64 else "f32",
        "data": "synthetic",
        "config": {"workload": wl, "description": desc, "grids": len(pbs), "cells": cells,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": f"state {2 * state_bytes / 1e6:.0f} MB > L2 {L2_BYTES / 1e6:.0f} MB, no flush",
                   "tuning": tuning or "model default"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "kernels_ms": {"prologue": prologue_ms, "sweep": sweep_ms, "x_sweep": x_ms, "y_sweep": y_ms},
        "riemann_fp64_fallbacks": stats["riemann_fp64"],
        "precision_report": precision_report,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--l1-steps", type=int, default=0,
                    help="FP32 workloads: also report the L1 density error against FP64 after this many steps")
    ap.add_argument("--autotune", action="store_true",
                    help="time candidate launch shapes first and use the fastest")
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
