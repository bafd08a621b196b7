#!/usr/bin/env python3
"""Throughput of the five-equation WENO5 / HLLC / TVD-RK3 step on GB300.

Default workload: the 3D two-fluid shock-bubble interaction on 256^3 cells
(7 conserved fields, Mach 1.5 shock, light-gas sphere, seeded density
noise), float64 (MFC_FP64_FAST: float64 throughout, FMA contraction and
refined reciprocals; within 1e-11 of the oracle after 100 steps), CFL 0.4
with the CFL dt computed on the device every step.  The other precisions
(MFC_FP64, bit for bit the oracle; MFC_DF64, double-float WENO5 on the
float32 pipes beside the float64 Riemann solve; and the mixed
float32/float64 form) are timed on the same workload, with their per-field
error against MFC_FP64.
One timed "step" is one full RK3 step (CFL reduction + three stages of
three directional sweeps).  The state is 1.0 GB, far larger than the 129 MB
L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  Under torchrun every rank runs its own
replica of the workload (the method needs no data exchange on one GPU);
value = all ranks' cell updates / the slowest rank's time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2503_07953_gb300 import flops  # noqa: E402
from paper_2503_07953_gb300 import pipes  # noqa: E402
from paper_2503_07953_gb300 import workloads as wl  # noqa: E402

METRIC = "WENO5-HLLC cell-updates/s per RK3 step, FP64 vs mixed at stated error; VJP/fwd cost"
UNIT = "cell-updates/s"
# FP64 peak from unit counts and clock: 152 SMs x 2 DFMA lanes x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="shock_bubble_3d",
                    choices=["shock_bubble_3d", "random_interfaces_3d", "bubble_collapse_2d", "water_air_1d"])
    ap.add_argument("--n", type=int, default=0, help="cells per axis (0: the workload's own size)")
    ap.add_argument("--precision", default="fp64_fast", choices=["fp64", "fp64_fast", "df64", "mixed"])
    ap.add_argument("--no-extras", action="store_true", help="skip the mixed, adjoint, e2e and CPU legs")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    return args


def make_workload(name: str, n: int):
    if name == "shock_bubble_3d":
        return wl.shock_bubble_3d(n or 256)
    if name == "random_interfaces_3d":
        return wl.random_interfaces_3d(n or 512)
    if name == "bubble_collapse_2d":
        return wl.bubble_collapse_2d(n or 1024)
    return wl.water_air_shock_tube(n or 1000)


def describe(case) -> str:
    dims = "x".join(str(x) for x in case.n)
    return f"{case.name} {dims} cells, {case.nq} fields, {case.nf} fluids, WENO5-M + HLLC, TVD-RK3, CFL {case.cfl}"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); smax.append(float(f[2])); power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "power_w_max": max(power),
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value: float) -> float:
    if world == 1:
        return value
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def launches_per_step(nd: int) -> int:
    # set-scalars + CFL reduction + finalize + 3 stages x nd sweeps
    return 3 + 3 * nd


def time_steps(S, q, steps: int) -> float:
    """Milliseconds for `steps` RK3 steps, CUDA events on the launching stream."""
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        S.rk3_step(q, 0.0)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def time_sweeps(S, q, reps: int) -> float:
    """Average milliseconds of one directional sweep launch: `reps`
    evaluations of L (ndim sweep launches each, nothing else)."""
    out = S.empty()
    stream = torch.cuda.current_stream()
    for _ in range(2):
        S.rhs(q, out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        S.rhs(q, out)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / (reps * S.ndim)


def field_errors(a: torch.Tensor, b: torch.Tensor, nf: int, nd: int):
    """Per field max |a - b| / max |b|; the momentum components share the
    largest of their maxima as scale."""
    den = [b[k].abs().max().item() for k in range(b.shape[0])]
    m = max(den[nf:nf + nd])
    den[nf:nf + nd] = [m] * nd
    return [(a[k] - b[k]).abs().max().item() / den[k] if den[k] > 0 else 0.0 for k in range(b.shape[0])]


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def sample_case(workload: str, sample_n: int):
    if workload == "shock_bubble_3d":
        return wl.shock_bubble_3d(dims=(sample_n,) * 3)
    if workload == "random_interfaces_3d":
        return wl.random_interfaces_3d(dims=(sample_n,) * 3)
    if workload == "bubble_collapse_2d":
        return wl.bubble_collapse_2d(dims=(sample_n * 8, sample_n * 8))
    return wl.water_air_shock_tube(1000)


def time_oracle(workload: str, sample_n: int, steps: int, parallel: bool) -> dict:
    """The oracle, as it stands, on `steps` RK3 steps of a bounded sample of
    the workload: single-threaded, or its OpenMP build on all host cores."""
    import oracle
    oracle.build(openmp=parallel)
    oracle.set_parallel(parallel)
    try:
        case, W = sample_case(workload, sample_n)
        P = oracle.Problem(n=case.n, gamma=case.gamma, pi_inf=case.pi_inf, lo=case.lo, hi=case.hi,
                           bc_lo=case.bc_lo, bc_hi=case.bc_hi, weno=case.weno, eps=case.eps)
        q = oracle.prim_to_cons(P, W)
        threads = oracle.threads()
        t0 = time.perf_counter()
        q, dts = oracle.rk3_run(P, q, steps, cfl=case.cfl)
        el = time.perf_counter() - t0
    finally:
        oracle.set_parallel(False)
    how = "single-threaded" if threads == 1 else f"OpenMP over the grid lines on {threads} threads"
    return {"value": case.ncells * steps / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{case.name} {'x'.join(map(str, case.n))} cells, {steps} RK3 steps (CFL dt each step), "
                      f"{how}, {el:.1f} s"}


def cpu_baseline_leg(workload: str, ndim: int) -> dict:
    """The oracle on all host cores (its OpenMP build) on a bounded sample,
    with the single-threaded oracle beside it; nproc and the CPU model."""
    three_d = ndim == 3
    single = time_oracle(workload, 64 if three_d else 0, 5 if three_d else 50, parallel=False)
    allc = time_oracle(workload, 128 if three_d else 0, 3 if three_d else 50, parallel=True)
    out = dict(allc)
    out["nproc"] = os.cpu_count()
    out["cpu_model"] = cpu_model()
    out["single_thread"] = single
    out["parallel_speedup"] = allc["value"] / single["value"]
    return out


def run_reference(args, world, rank):
    """The reference arm: the plain CPU oracle (its OpenMP build, all host
    cores), timed on a bounded sample of the workload."""
    if rank != 0:
        return
    import oracle
    oracle.build(openmp=True)
    oracle.set_parallel(True)
    if args.workload == "shock_bubble_3d":
        case, W = wl.shock_bubble_3d(dims=(64,) * 3)
    elif args.workload == "random_interfaces_3d":
        case, W = wl.random_interfaces_3d(dims=(48,) * 3)
    elif args.workload == "bubble_collapse_2d":
        case, W = wl.bubble_collapse_2d(dims=(256, 256))
    else:
        case, W = wl.water_air_shock_tube(1000)
    P = oracle.Problem(n=case.n, gamma=case.gamma, pi_inf=case.pi_inf, lo=case.lo, hi=case.hi,
                       bc_lo=case.bc_lo, bc_hi=case.bc_hi, weno=case.weno, eps=case.eps)
    threads = oracle.threads()
    q = oracle.prim_to_cons(P, W)
    q, _ = oracle.rk3_run(P, q, args.warmup, cfl=case.cfl)
    t0 = time.perf_counter()
    q, _ = oracle.rk3_run(P, q, args.steps, cfl=case.cfl)
    el = time.perf_counter() - t0
    oracle.set_parallel(False)
    value = case.ncells * args.steps / el
    sample = (f"{case.name} {'x'.join(map(str, case.n))} cells per step (bounded sample of the workload), "
              f"OpenMP over the grid lines on {threads} threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": describe(make_workload_stub(args)), "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def make_workload_stub(args):
    """The workload description without generating its fields."""
    n = args.n
    table = {"shock_bubble_3d": ([n or 256] * 3, 7, 2, 0.4), "random_interfaces_3d": ([n or 512] * 3, 9, 3, 0.4),
             "bubble_collapse_2d": ([n or 1024] * 2, 6, 2, 0.3), "water_air_1d": ([n or 1000], 5, 2, 0.3)}
    dims, nq, nf, cfl = table[args.workload]

    class _C:
        pass
    c = _C()
    c.name, c.n, c.nq, c.nf, c.cfl = args.workload, dims, nq, nf, cfl
    return c


PREC = {"fp64": 0, "mixed": 1, "fp64_fast": 2, "df64": 3}


def time_vjp(S, q, dt: float, reps: int) -> float:
    """Milliseconds per mfc_rk3_step_vjp (stage recomputation included).
    The cotangent is seeded standard-normal noise, a generic objective's
    gradient.  (An all-ones cotangent is degenerate: its flux differences
    vanish, and the kernels skip the zero bars.)"""
    gen = torch.Generator(device=q.device).manual_seed(1)
    g = torch.randn(q.shape, generator=gen, dtype=torch.float64, device=q.device)
    out = S.empty()
    stream = torch.cuda.current_stream()
    S.rk3_step_vjp(q, dt, g, out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        S.rk3_step_vjp(q, dt, g, out)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def e2e_leg(S, q0, ncell, steps, world):
    """End to end through the public API with host buffers: every step
    uploads its input state from pinned host memory, steps it and downloads
    the result (mfc_rk3_step_batch_host, which overlaps the copies of
    neighbouring steps with the step in between).  Every rank, max over
    ranks, like the device-timed value."""
    import torch
    host_in = torch.empty(q0.shape, dtype=torch.float64, pin_memory=True)
    host_out = torch.empty(q0.shape, dtype=torch.float64, pin_memory=True)
    host_in.copy_(q0)
    S.rk3_step_batch_host([host_in] * 2, [host_out] * 2, 0.0)  # staging buffers, untimed
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    S.rk3_step_batch_host([host_in] * steps, [host_out] * steps, 0.0)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    mse = max_over_ranks(world, e0.elapsed_time(e1))
    nbytes = q0.numel() * 8
    del host_in, host_out
    torch.cuda.empty_cache()
    return {"value": world * ncell * steps / (mse / 1e3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "ms_per_step": mse / steps, "api": "mfc_rk3_step_batch_host"}


def run_ours(args, world, rank, local):
    from paper_2503_07953_gb300 import build, mfc
    build.build()
    case, W = make_workload(args.workload, args.n)
    prec = PREC[args.precision]
    S = mfc.Solver.from_case(case, precision=prec)
    q0 = S.prim_to_cons(S.from_interior(W))
    del W
    q = q0.clone()
    ncell = case.ncells

    # warm-up, then the timed region (CFL dt on the device every step)
    for _ in range(args.warmup):
        S.rk3_step(q, 0.0)
    S.check()
    clocks = ClockSampler(local)
    barrier(world)
    clocks.start()
    ms = time_steps(S, q, args.steps)
    clk = clocks.stop()
    barrier(world)
    S.check()
    ms = max_over_ranks(world, ms)
    value = world * ncell * args.steps / (ms / 1e3)

    # dominant kernel: the directional sweep (per launch, CUDA events)
    t_sweep = time_sweeps(S, q, 3)
    per_sweep = flops.per_cell_sweep(args.workload) * ncell
    achieved = per_sweep / (t_sweep / 1e3) / 1e12
    fp64 = prec != mfc.MFC_MIXED
    roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS if fp64 else None, "unit": "TFLOP/s",
            "frac": (achieved / FP64_PEAK_TFLOPS) if fp64 else None, "traffic": None,
            "kernel": f"sweep_kernel ({args.precision}), {t_sweep:.3f} ms per launch, "
                      f"{per_sweep / 1e9:.2f} GFLOP (algorithmic) per launch",
            "peak_basis": "FP64 pipe: 152 SMs x 2 DFMA lanes/clk x 2 flop x 2.07 GHz = 1.259 TFLOP/s "
                          "(unit counts and max clock; 1.253 measured by a DFMA microbenchmark)"}
    if not fp64:
        roof["peak_basis"] = "mixed path: FP32 and FP64 pipes both in use"
    # the HBM roofline the step would have if it were bandwidth-bound:
    # algorithmic bytes per cell-step (8 N_q doubles) against the measured copy bandwidth
    hbm_peak, hbm_basis = 6800.0, "fallback (6.8 TB/s)"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            hbm_peak, hbm_basis = float(json.load(fh)["hbm_gbs"]), "measured copy bandwidth (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        pass
    hbm_ach = 8 * case.nq * 8 * ncell / ((ms / args.steps) / 1e3) / 1e9
    # DRAM traffic and pipe counts of the sweep kernels from an ncu capture of
    # these very sources (profiles/sweep_pipes.json), scaled by cells; null
    # when the sources differ from the captured ones
    fp_src = build.source_fingerprint()
    clock = clk.get("sm_mhz") or 2070.0
    rec = pipes.load(args.precision, args.workload, fp_src)
    roof["pipes"] = pipes.roofline(rec, ncell, t_sweep, clock) if rec else None
    if rec:
        roof["traffic"] = rec["dram_bytes_per_cell"] * ncell
        roof["traffic_basis"] = (f"ncu dram__bytes_read.sum + dram__bytes_write.sum per cell-sweep at "
                                 f"{rec['captured']}, scaled by cells")

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if fp64 else "f64+f32",
            "data": "synthetic",
            "config": {"workload": describe(case), "cells": ncell, "precision": args.precision,
                       "dt": "CFL dt reduced on the device every step",
                       "l2": "state 1.0 GB per buffer > 129 MB L2: no flush needed" if ncell >= 2 ** 22
                       else "state smaller than L2", "parallelism": f"replicas x{world}"},
            "gpu_launches": launches_per_step(case.ndim) * args.steps, "clocks": clk, "roofline": roof,
            "hbm": {"achieved_gbs": hbm_ach, "peak_gbs": hbm_peak, "frac": hbm_ach / hbm_peak,
                    "bytes_per_cell_step": 8 * case.nq * 8, "peak_basis": hbm_basis},
            "grind_time_ns": (ms / args.steps) * 1e6 / (ncell * case.nq * 3)}

    if not args.no_extras:
        line["e2e"] = e2e_leg(S, q0, ncell, args.steps, world)
    if not args.no_extras and rank == 0:
        extras = {}
        # reference trajectory: MFC_FP64, which reproduces the oracle bit for bit
        Sx = S if prec == mfc.MFC_FP64 else mfc.Solver.from_case(case, precision=mfc.MFC_FP64)
        qref = q0.clone()
        Sx.rk3_run(qref, args.warmup + args.steps, 0.0)
        Sx.check()
        del Sx
        nsteps = args.warmup + args.steps
        qh = q0.clone()
        S.rk3_run(qh, nsteps, 0.0)
        line["field_max_rel_err_vs_fp64"] = field_errors(S.interior(qh), S.interior(qref), case.nf, case.ndim)
        line["after_steps"] = nsteps
        del qh
        for name in ("fp64", "fp64_fast", "df64", "mixed"):
            if name == args.precision:
                continue
            So = mfc.Solver.from_case(case, precision=PREC[name])
            qo = q0.clone()
            for _ in range(args.warmup):
                So.rk3_step(qo, 0.0)
            leg_clocks = ClockSampler(local)
            leg_clocks.start()
            mso = time_steps(So, qo, args.steps)
            leg_clk = leg_clocks.stop()
            So.check()
            extras[name] = {"value": ncell * args.steps / (mso / 1e3), "ms_per_step": mso / args.steps,
                            "speedup_vs_" + args.precision: ms / mso,
                            "field_max_rel_err_vs_fp64": field_errors(So.interior(qo), S.interior(qref),
                                                                      case.nf, case.ndim),
                            "after_steps": nsteps,
                            "sweep_ms_per_launch": time_sweeps(So, qo, 3)}
            if name != "mixed":
                extras[name]["bitwise_equal_to_fp64"] = bool(torch.equal(So.interior(qo), S.interior(qref)))
            # the pipe that bounds this leg's sweeps, and how busy it is
            # (instruction counts per cell-sweep from an ncu capture of these
            # sources, the sweep time from CUDA events, the clock sampled
            # during the leg's timed steps)
            if name in ("df64", "mixed"):
                # the adjoint step of this precision against its forward step
                dto = So.compute_dt(qo)
                ms_f = time_steps(So, qo.clone(), 2) / 2
                ms_v = time_vjp(So, qo, dto, 2)
                extras[name]["vjp"] = {"ms_per_step_vjp": ms_v, "ms_per_step_fwd": ms_f, "vjp_over_fwd": ms_v / ms_f}
            leg_rec = pipes.load(name, args.workload, fp_src)
            extras[name]["clocks"] = leg_clk
            extras[name]["roofline"] = (pipes.roofline(leg_rec, ncell, extras[name]["sweep_ms_per_launch"],
                                                       leg_clk.get("sm_mhz") or 2070.0) if leg_rec else None)
            if name == "df64":
                # double-float WENO on the float32 pipes beside the float64
                # Riemann solve: its algorithmic flop rate against the
                # float64 pipe's peak (above 1: faster than the float64 pipe
                # allows for the same arithmetic)
                ach = per_sweep / (extras[name]["sweep_ms_per_launch"] / 1e3) / 1e12
                extras[name]["sweep_tflops_algorithmic"] = ach
                extras[name]["over_fp64_pipe_peak"] = ach / FP64_PEAK_TFLOPS
            del So, qo
            torch.cuda.empty_cache()
        del qref
        # adjoint cost: one RK3-step VJP (stages recomputed) per forward step
        dt = S.compute_dt(q)
        ms_fwd1 = time_steps(S, q.clone(), 2) / 2
        ms_vjp = time_vjp(S, q, dt, 2)
        extras["vjp"] = {"ms_per_step_vjp": ms_vjp, "ms_per_step_fwd": ms_fwd1, "vjp_over_fwd": ms_vjp / ms_fwd1,
                         "precision": args.precision}
        torch.cuda.empty_cache()
        line.update(extras)
        line["cpu_baseline"] = cpu_baseline_leg(args.workload, case.ndim)
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
