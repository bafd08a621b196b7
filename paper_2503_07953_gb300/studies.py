"""Measurements of the paper-shaped workloads beyond the headline benchmark.

    python -m paper_2503_07953_gb300.studies sizes   [--sizes 128 256 384 512 640] [--precisions ...]
    python -m paper_2503_07953_gb300.studies mixed-error [--n 512] [--steps 50]
    python -m paper_2503_07953_gb300.studies adjoint [--n 1024] [--steps 500] [--directions 16]
    python -m paper_2503_07953_gb300.studies tube    [--n 1000] [--steps 200]

Each prints JSON lines (one per measured configuration).  Every number is
taken through the library's public API on synthetic inputs from
`workloads.py`, timed with CUDA events on the launching stream after
warm-up steps; the states are larger than L2 except in `tube`.

- sizes: the 3D shock-bubble at N^3 cells; cell-updates/s per RK3 step,
  sweep time per launch, algorithmic FP64 TFLOP/s of the sweep (flops.py),
  algorithmic HBM GB/s of the step (8 N_q 8 bytes per cell-step), and the
  cost of one RK3-step VJP against one forward step, with the bytes one
  checkpoint snapshot holds.
- mixed-error: the three-fluid random-interface field, the mixed
  float32/float64 mode against a float64 mode after the same steps, per
  field (max |a - b| / max |b|, momenta sharing one scale), with both runs'
  throughput.
- adjoint: the 2D bubble collapse; J = time-integrated pressure impulse on
  the x = 1 wall, gradient with respect to the initial volume fraction by
  the checkpointed VJP, against central differences along seeded
  directions, per precision.
- tube: the 1D water/air shock tube; steps/s with a launch per kernel and
  with the whole run captured once in a CUDA graph and replayed.
"""
from __future__ import annotations

import argparse
import json
import sys

import torch

from . import adjoint as adj
from . import checkpoint, flops, mfc
from . import workloads as wl

PREC = {"fp64": mfc.MFC_FP64, "fp64_fast": mfc.MFC_FP64_FAST, "df64": mfc.MFC_DF64, "mixed": mfc.MFC_MIXED}


def _emit(rec: dict) -> None:
    print(json.dumps(rec), flush=True)


def _timed(fn, reps: int) -> float:
    """Milliseconds per call of fn(), CUDA events on the current stream."""
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _field_errors(a: torch.Tensor, b: torch.Tensor, nf: int, nd: int):
    den = [b[k].abs().max().item() for k in range(b.shape[0])]
    m = max(den[nf:nf + nd])
    den[nf:nf + nd] = [m] * nd
    return [(a[k] - b[k]).abs().max().item() / den[k] if den[k] > 0 else 0.0 for k in range(b.shape[0])]


def sizes(args) -> None:
    for n in args.sizes:
        case, W = wl.shock_bubble_3d(n)
        ncell = case.ncells
        for pname in args.precisions:
            S = mfc.Solver.from_case(case, precision=PREC[pname])
            q = S.prim_to_cons(S.from_interior(W))
            for _ in range(args.warmup):
                S.rk3_step(q, 0.0)
            S.check()
            ms = _timed(lambda: S.rk3_step(q, 0.0), args.steps)
            out = S.empty()
            ms_sweep = _timed(lambda: S.rhs(q, out), 2) / case.ndim
            S.check()
            rec = {"study": "sizes", "workload": f"shock_bubble_3d {n}^3", "precision": pname, "cells": ncell,
                   "steps": args.steps, "ms_per_step": ms, "cell_updates_per_s": ncell / (ms / 1e3),
                   "sweep_ms_per_launch": ms_sweep,
                   "sweep_alg_tflops": flops.per_cell_sweep("shock_bubble_3d") * ncell / (ms_sweep / 1e3) / 1e12,
                   "step_alg_hbm_gbs": 8 * case.nq * 8 * ncell / (ms / 1e3) / 1e9,
                   "grind_time_ns": ms * 1e6 / (ncell * case.nq * 3)}
            if args.vjp:
                dt = S.compute_dt(q)
                # seeded noise: an all-ones cotangent would make the flux
                # differences vanish, and the kernels skip zero bars
                gen = torch.Generator(device=q.device).manual_seed(1)
                bar = torch.randn(q.shape, generator=gen, dtype=torch.float64, device=q.device)
                S.rk3_step_vjp(q, dt, bar)
                ms_vjp = _timed(lambda: S.rk3_step_vjp(q, dt, bar), 2)
                rec.update({"ms_per_step_vjp": ms_vjp, "vjp_over_fwd": ms_vjp / ms,
                            "snapshot_bytes": q.numel() * 8,
                            "adjoint_scratch_bytes": 6 * q.numel() * 8})
                del bar
            _emit(rec)
            del S, q, out
            torch.cuda.empty_cache()


def mixed_error(args) -> None:
    case, W = wl.random_interfaces_3d(args.n)
    runs = {}
    for pname in [args.reference, "mixed"]:
        S = mfc.Solver.from_case(case, precision=PREC[pname])
        q = S.prim_to_cons(S.from_interior(W))
        dts = torch.zeros(args.steps, dtype=torch.float64, device=q.device)
        ms = _timed(lambda: S.rk3_run(q, args.steps, 0.0, dts), 1) / args.steps
        S.check()
        runs[pname] = (S.interior(q).clone(), ms, dts.cpu())
        del S, q
        torch.cuda.empty_cache()
    ref, ms_ref, dts_ref = runs[args.reference]
    mix, ms_mix, dts_mix = runs["mixed"]
    _emit({"study": "mixed-error", "workload": f"random_interfaces_3d {args.n}^3, 3 fluids, periodic",
           "steps": args.steps, "reference": args.reference,
           "field_max_rel_err_mixed_vs_reference": _field_errors(mix, ref, case.nf, case.ndim),
           "fields": ["a1r1", "a2r2", "a3r3", "ru", "rv", "rw", "rE", "a1", "a2"],
           "dt_max_rel_diff": float(((dts_mix - dts_ref).abs() / dts_ref).max()),
           "ms_per_step": {args.reference: ms_ref, "mixed": ms_mix},
           "cell_updates_per_s": {args.reference: case.ncells / (ms_ref / 1e3), "mixed": case.ncells / (ms_mix / 1e3)},
           "speedup_mixed": ms_ref / ms_mix})


def _stored_derivatives(path: str) -> dict:
    """J, dt figures and dJ_direction_k of a wall_impulse_jvp_<N>.txt file."""
    out = {}
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()
            out[k] = float(v)
    return out


def adjoint_study(args) -> None:
    case, W = wl.bubble_collapse_2d(args.n)
    a1 = torch.as_tensor(W[case.nf + case.ndim + 1].copy(), dtype=torch.float64, device="cuda")
    band = ((a1 > 1e-3) & (a1 < 1 - 1e-3)).double()
    stored = _stored_derivatives(args.compare) if args.compare else None
    fixed_dts = None
    if args.dt_from_fp64:
        # the CFL dt sequence of the bit-exact float64 mode (the oracle's, bit
        # for bit), held by every precision below
        S0 = mfc.Solver.from_case(case, precision=mfc.MFC_FP64)
        q = adj.alpha_to_state(S0, case, W, a1).detach()
        log = torch.zeros(args.steps, dtype=torch.float64, device="cuda")
        S0.rk3_run(q, args.steps, 0.0, log)
        S0.check()
        fixed_dts = [float(x) for x in log.cpu()]
        del S0, q
        torch.cuda.empty_cache()
    for pname, h in zip(args.precisions, args.h):
        S = mfc.Solver.from_case(case, precision=PREC[pname])
        q0 = adj.alpha_to_state(S, case, W, a1).detach()
        t0 = torch.cuda.Event(enable_timing=True); t1 = torch.cuda.Event(enable_timing=True)
        if fixed_dts is not None:
            dts = fixed_dts
        else:
            _, _, dts, _ = adj.rollout_gradient(S, q0, args.steps, lambda n, q: q.sum() * 0.0, 1)
        loss = adj.wall_pressure_objective(S, case, dts)
        torch.cuda.synchronize(); t0.record()
        J, gq, _, st = adj.rollout_gradient(S, q0, args.steps, loss, args.snapshots, dts)
        t1.record(); torch.cuda.synchronize()
        ms_grad = t0.elapsed_time(t1)
        a = a1.clone().requires_grad_(True)
        (adj.alpha_to_state(S, case, W, a) * gq).sum().backward()
        ga = a.grad

        def J_of(alpha):
            q = adj.alpha_to_state(S, case, W, alpha).detach()
            tot = torch.zeros((), dtype=torch.float64, device=q.device)
            for k in range(args.steps):
                S.rk3_step(q, dts[k])
                tot += loss(k, q)
            return float(tot)

        t0.record()
        J_check = J_of(a1)
        t1.record(); torch.cuda.synchronize()
        ms_fwd = t0.elapsed_time(t1)
        gen = torch.Generator(device="cpu").manual_seed(0)
        rel, ads, fds = [], [], []
        ndir = max(args.directions, 2 if stored else 0)
        for k in range(ndir):
            d = torch.randn(a1.shape, generator=gen, dtype=torch.float64).to(a1.device) * band
            d = d / float(d.abs().max())
            ad = float((ga * d).sum())
            ads.append(ad)
            if k < args.directions:
                fd = (J_of(a1 + h * d) - J_of(a1 - h * d)) / (2 * h)
                rel.append(abs(ad - fd) / abs(fd))
                fds.append(fd)
        S.check()
        vs_oracle = None
        if stored:
            # the oracle's forward-mode derivatives along the same seeded directions
            vs_oracle = {"J_oracle": stored.get("J"), "J_rel_diff": abs(J - stored["J"]) / abs(stored["J"]),
                         "dJ_oracle": [stored[f"dJ_direction_{k}"] for k in range(2)],
                         "dJ_adjoint": ads[:2],
                         "dJ_rel_diff": [abs(ads[k] - stored[f"dJ_direction_{k}"]) / abs(stored[f"dJ_direction_{k}"])
                                         for k in range(2)],
                         "dt_sum_rel_diff": (abs(sum(dts) - stored["dt_sum"]) / stored["dt_sum"]
                                             if "dt_sum" in stored else None)}
        _emit({"study": "adjoint", "workload": f"bubble_collapse_2d {args.n}x{args.n}, {args.steps} steps",
               "precision": pname, "J": J, "J_forward_only": J_check, "snapshots": args.snapshots,
               "max_live_snapshots": st.max_live_snapshots, "recomputed_steps": st.advances, "vjp_steps": st.vjps,
               "snapshot_bytes": q0.numel() * 8, "ms_gradient": ms_grad, "ms_forward_with_objective": ms_fwd,
               "gradient_over_forward": ms_grad / ms_fwd, "fd_step": h, "fd_directions": args.directions,
               "grad_abs_sum": float(ga.abs().sum()), "directional_adjoint": ads, "directional_fd": fds,
               "fd_rel_diff": rel, "fd_rel_diff_max": max(rel) if rel else None,
               "fd_rel_diff_median": sorted(rel)[len(rel) // 2] if rel else None,
               "dts": "bit-exact float64 mode's CFL sequence" if fixed_dts is not None else "own CFL sequence",
               "vs_oracle_forward_mode": vs_oracle})
        del S, q0, gq, ga
        torch.cuda.empty_cache()


def tube(args) -> None:
    case, W = wl.water_air_shock_tube(args.n, args.steps)
    for pname in args.precisions:
        S = mfc.Solver.from_case(case, precision=PREC[pname])
        q0 = S.prim_to_cons(S.from_interior(W))
        q = q0.clone()
        for _ in range(3):
            S.rk3_step(q, 0.0)
        q.copy_(q0)
        ms = _timed(lambda: S.rk3_run(q, args.steps, 0.0), 1)
        S.check()
        # the whole run as one CUDA graph (the library launches on the
        # capturing stream and neither allocates nor synchronises in a step)
        qg = q0.clone()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            S.rk3_run(qg, 3, 0.0)
        torch.cuda.current_stream().wait_stream(s)
        qg.copy_(q0)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            S.rk3_run(qg, args.steps, 0.0)
        qg.copy_(q0)
        ms_graph = _timed(g.replay, 1)
        same = bool(torch.equal(S.interior(qg), S.interior(q)))
        S.check()
        _emit({"study": "tube", "workload": f"water_air_1d {args.n} cells, {args.steps} steps", "precision": pname,
               "steps_per_s": args.steps / (ms / 1e3), "steps_per_s_graph": args.steps / (ms_graph / 1e3),
               "us_per_step": ms * 1e3 / args.steps, "us_per_step_graph": ms_graph * 1e3 / args.steps,
               "graph_result_bitwise_equal": same})
        del S, q, qg, g
        torch.cuda.empty_cache()


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(prog="python -m paper_2503_07953_gb300.studies")
    sub = ap.add_subparsers(dest="study", required=True)
    p = sub.add_parser("sizes")
    p.add_argument("--sizes", type=int, nargs="+", default=[128, 256, 384, 512, 640])
    p.add_argument("--precisions", nargs="+", default=["fp64_fast", "df64", "mixed"], choices=sorted(PREC))
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--no-vjp", dest="vjp", action="store_false")
    p = sub.add_parser("mixed-error")
    p.add_argument("--n", type=int, default=512)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--reference", default="fp64_fast", choices=["fp64", "fp64_fast"])
    p = sub.add_parser("adjoint")
    p.add_argument("--n", type=int, default=1024)
    p.add_argument("--steps", type=int, default=500)
    p.add_argument("--snapshots", type=int, default=20)
    p.add_argument("--directions", type=int, default=16)
    p.add_argument("--precisions", nargs="+", default=["fp64_fast", "mixed"], choices=sorted(PREC))
    p.add_argument("--h", type=float, nargs="+", default=[1e-6, 1e-3],
                   help="central-difference step per precision (directions are max-normalised)")
    p.add_argument("--dt-from-fp64", action="store_true",
                   help="hold the bit-exact float64 mode's CFL dt sequence in every precision")
    p.add_argument("--compare", default=None,
                   help="a wall_impulse_jvp_<N>.txt file of oracle forward-mode derivatives to compare with")
    p = sub.add_parser("tube")
    p.add_argument("--n", type=int, default=1000)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--precisions", nargs="+", default=["fp64", "fp64_fast", "mixed"], choices=sorted(PREC))
    args = ap.parse_args(argv)
    if not torch.cuda.is_available():
        sys.exit("studies need a CUDA device")
    mfc.lib()
    {"sizes": sizes, "mixed-error": mixed_error, "adjoint": adjoint_study, "tube": tube}[args.study](args)


if __name__ == "__main__":
    main()
