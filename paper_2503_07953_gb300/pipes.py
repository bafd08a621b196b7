"""Per-pipe roofline of the directional sweeps.

The sweeps are bound by plain ALU pipes, not by HBM: the float64 pipe (2
operations per SM per clock on GB300), the float32 FMA pipes (128 per SM per
clock) or instruction issue (4 warp instructions per SM per clock).  An ncu
capture of one RK3 stage's sweep kernels gives, per cell and sweep, the
float64 and float32 arithmetic instructions the kernels execute and the warp
instructions they issue; ``roofline`` turns those counts and a measured
sweep time into the time each pipe needs at the measured clock, names the
pipe that needs the most (the bound) and the fraction of the measured time
that pipe is busy.

The counts are kept in ``profiles/sweep_pipes.json`` with the fingerprint of
the sweep sources they were captured on (``build.source_fingerprint``); a
record whose fingerprint differs from the current sources is not used.

  python -m paper_2503_07953_gb300.pipes CSV --precision P --workload W --n N --sweeps S --command CMD

reads an ``ncu --csv --metrics ...`` log of S directional sweeps on an N^3
grid (the launches of every kernel of those sweeps) and adds or replaces the
record of (P, W) in profiles/sweep_pipes.json.
"""
from __future__ import annotations

import argparse
import csv
import json
import os

SMS = 152
FP64_PER_SM_CLK = 2.0      # float64 add / mul / fma thread operations
FP32_PER_SM_CLK = 128.0    # float32 add / mul / fma thread operations
ISSUE_PER_SM_CLK = 4.0     # warp instructions

METRICS = [
    "gpu__time_duration.sum",
    "sm__inst_executed.sum",
    "sm__inst_executed_pipe_fp64.sum",
    "sm__sass_thread_inst_executed_op_dadd_pred_on.sum",
    "sm__sass_thread_inst_executed_op_dmul_pred_on.sum",
    "sm__sass_thread_inst_executed_op_dfma_pred_on.sum",
    "sm__sass_thread_inst_executed_op_fadd_pred_on.sum",
    "sm__sass_thread_inst_executed_op_fmul_pred_on.sum",
    "sm__sass_thread_inst_executed_op_ffma_pred_on.sum",
    "sm__sass_thread_inst_executed_op_fadd2_pred_on.sum",
    "sm__sass_thread_inst_executed_op_fmul2_pred_on.sum",
    "sm__sass_thread_inst_executed_op_ffma2_pred_on.sum",
    "sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_elapsed",
    "sm__inst_executed.avg.per_cycle_elapsed",
    "dram__bytes_read.sum",
    "dram__bytes_write.sum",
]

HERE = os.path.dirname(os.path.abspath(__file__))
RECORDS = os.path.join(os.path.dirname(HERE), "profiles", "sweep_pipes.json")


def _num(s: str) -> float:
    return float(s.replace(",", "")) if s not in ("", "n/a") else 0.0


def parse_ncu_csv(path: str) -> list:
    """Rows of an ncu --csv metrics log: one dict per (launch, metric)."""
    with open(path, newline="") as fh:
        lines = [ln for ln in fh if ln.startswith('"')]
    return list(csv.DictReader(lines))


def counts_from_rows(rows: list, cells: int, sweeps: int) -> dict:
    """Per cell and sweep: float64 and float32 arithmetic thread
    instructions, issued warp instructions, DRAM bytes; per kernel name the
    launches and time."""
    tot = {}
    kernels = {}
    launches = set()
    for r in rows:
        name, unit, val = r["Metric Name"], r.get("Metric Unit", ""), _num(r["Metric Value"])
        lid = r["ID"]
        kname = r["Kernel Name"].split("(")[0].split("<")[0].strip()
        if name == "gpu__time_duration.sum":
            scale = {"ns": 1.0, "nsecond": 1.0, "us": 1e3, "usecond": 1e3, "ms": 1e6, "msecond": 1e6,
                     "s": 1e9, "second": 1e9}[unit]
            k = kernels.setdefault(kname, {"launches": 0, "ns": 0.0})
            k["launches"] += 1
            k["ns"] += val * scale
        if name.startswith("dram__bytes"):
            scale = {"byte": 1.0, "Kbyte": 1e3, "KB": 1e3, "Mbyte": 1e6, "MB": 1e6, "Gbyte": 1e9, "GB": 1e9}[unit]
            val *= scale
        if name.endswith(".sum"):
            tot[name] = tot.get(name, 0.0) + val
        launches.add(lid)
    per = float(cells) * sweeps
    f64 = sum(tot.get(f"sm__sass_thread_inst_executed_op_{o}_pred_on.sum", 0.0) for o in ("dadd", "dmul", "dfma"))
    f32 = sum(tot.get(f"sm__sass_thread_inst_executed_op_{o}_pred_on.sum", 0.0) for o in ("fadd", "fmul", "ffma"))
    f32 += 2.0 * sum(tot.get(f"sm__sass_thread_inst_executed_op_{o}2_pred_on.sum", 0.0)
                     for o in ("fadd", "fmul", "ffma"))
    return {
        "fp64_ops_per_cell": f64 / per,
        "dfma_share": tot.get("sm__sass_thread_inst_executed_op_dfma_pred_on.sum", 0.0) / f64 if f64 else None,
        "fp64_pipe_warp_inst_per_cell": tot.get("sm__inst_executed_pipe_fp64.sum", 0.0) / per,
        "fp32_ops_per_cell": f32 / per,
        "warp_inst_per_cell": tot.get("sm__inst_executed.sum", 0.0) / per,
        "dram_bytes_per_cell": (tot.get("dram__bytes_read.sum", 0.0) + tot.get("dram__bytes_write.sum", 0.0)) / per,
        "kernels": kernels,
        "launches": len(launches),
    }


def roofline(rec: dict, cells: int, sweep_ms: float, clock_mhz: float) -> dict:
    """Time each pipe needs for one sweep of `cells` cells at `clock_mhz`
    against the measured `sweep_ms`; the bound is the pipe that needs the
    most, frac its busy fraction of the measured time."""
    f = clock_mhz * 1e6
    need = {
        "fp64": rec["fp64_ops_per_cell"] * cells / (SMS * FP64_PER_SM_CLK * f),
        "fp32": rec["fp32_ops_per_cell"] * cells / (SMS * FP32_PER_SM_CLK * f),
        "issue": rec["warp_inst_per_cell"] * cells / (SMS * ISSUE_PER_SM_CLK * f),
    }
    t = sweep_ms / 1e3
    bound = max(need, key=need.get)
    return {"bound": bound, "frac": need[bound] / t, "unit": "pipe-busy fraction",
            "pipe_fracs": {k: v / t for k, v in need.items()},
            "per_cell_sweep": {"fp64_ops": rec["fp64_ops_per_cell"], "fp32_ops": rec["fp32_ops_per_cell"],
                               "warp_inst": rec["warp_inst_per_cell"], "dfma_share": rec.get("dfma_share")},
            "peaks_per_sm_clk": {"fp64": FP64_PER_SM_CLK, "fp32": FP32_PER_SM_CLK, "issue": ISSUE_PER_SM_CLK},
            "clock_mhz": clock_mhz, "sweep_ms": sweep_ms, "captured": rec.get("captured")}


def load(precision: str, workload: str, fingerprint: str):
    """The record of (precision, workload) captured on the current sources, or None."""
    try:
        with open(RECORDS) as fh:
            recs = json.load(fh)
    except (OSError, ValueError):
        return None
    for r in recs:
        if r.get("precision") == precision and r.get("workload") == workload and \
                r.get("source_fingerprint") == fingerprint:
            return r
    return None


def main(argv=None) -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("csv")
    ap.add_argument("--precision", required=True)
    ap.add_argument("--workload", default="shock_bubble_3d")
    ap.add_argument("--n", type=int, required=True, help="cells per axis of the captured grid")
    ap.add_argument("--sweeps", type=int, default=3, help="directional sweeps covered by the captured launches")
    ap.add_argument("--command", default="")
    args = ap.parse_args(argv)
    from . import build
    rows = parse_ncu_csv(args.csv)
    cells = args.n ** 3
    rec = counts_from_rows(rows, cells, args.sweeps)
    rec.update({"source_fingerprint": build.source_fingerprint(), "precision": args.precision,
                "workload": args.workload, "captured": f"{args.n}^3 cells, {args.sweeps} sweeps "
                                                      f"({rec['launches']} launches)",
                "command": args.command})
    try:
        with open(RECORDS) as fh:
            recs = json.load(fh)
    except (OSError, ValueError):
        recs = []
    recs = [r for r in recs if not (r.get("precision") == args.precision and r.get("workload") == args.workload)]
    recs.append(rec)
    with open(RECORDS, "w") as fh:
        json.dump(recs, fh, indent=1)
    print(json.dumps(rec, indent=1))


if __name__ == "__main__":
    main()
