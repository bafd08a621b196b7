"""Host logic of the per-pipe roofline (paper_2503_07953_gb300/pipes.py): the
per-cell counts taken from an ncu --csv metrics log, the time each pipe
needs and the bound, and the lookup of a record by the sweep sources'
fingerprint.  CPU only: the log below is written here, in the layout ncu
prints."""
import json

import pytest

from paper_2503_07953_gb300 import pipes

HEADER = '"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"\n'


def row(lid, kernel, metric, unit, value):
    return f'"{lid}","{kernel}","{metric}","{unit}","{value}"\n'


def synthetic_log(tmp_path):
    """Two launches of two kernels with round numbers (thread instructions,
    warp instructions, bytes), as ncu writes them (thousands separators,
    mixed time and byte units), after ncu's own preamble lines."""
    k1 = "void sweep_kernel<2, 3, 0, 2>(mfc::Consts, mfc::SweepArgs)"
    k2 = "void sweep_x_kernel<2, 3, 1>(mfc::Consts, mfc::SweepArgs)"
    lines = ["==PROF== Connected to process 1\n", HEADER]
    for lid, k, ms in ((0, k1, "1.5"), (1, k2, "0.5")):
        lines += [
            row(lid, k, "gpu__time_duration.sum", "msecond", ms),
            row(lid, k, "sm__inst_executed.sum", "inst", "1,000"),
            row(lid, k, "sm__inst_executed_pipe_fp64.sum", "inst", "100"),
            row(lid, k, "sm__sass_thread_inst_executed_op_dadd_pred_on.sum", "inst", "2,000"),
            row(lid, k, "sm__sass_thread_inst_executed_op_dmul_pred_on.sum", "inst", "3,000"),
            row(lid, k, "sm__sass_thread_inst_executed_op_dfma_pred_on.sum", "inst", "5,000"),
            row(lid, k, "sm__sass_thread_inst_executed_op_ffma_pred_on.sum", "inst", "400"),
            row(lid, k, "sm__sass_thread_inst_executed_op_ffma2_pred_on.sum", "inst", "300"),
            row(lid, k, "dram__bytes_read.sum", "Kbyte", "2"),
            row(lid, k, "dram__bytes_write.sum", "byte", "500"),
        ]
    path = tmp_path / "log.csv"
    path.write_text("".join(lines))
    return str(path)


def test_counts_per_cell_and_sweep(tmp_path):
    rows = pipes.parse_ncu_csv(synthetic_log(tmp_path))
    rec = pipes.counts_from_rows(rows, cells=10, sweeps=2)
    per = 10 * 2
    assert rec["fp64_ops_per_cell"] == pytest.approx(2 * (2000 + 3000 + 5000) / per)
    assert rec["dfma_share"] == pytest.approx(5000 / 10000)
    # a paired float32 instruction counts two operations
    assert rec["fp32_ops_per_cell"] == pytest.approx(2 * (400 + 2 * 300) / per)
    assert rec["warp_inst_per_cell"] == pytest.approx(2 * 1000 / per)
    assert rec["fp64_pipe_warp_inst_per_cell"] == pytest.approx(2 * 100 / per)
    assert rec["dram_bytes_per_cell"] == pytest.approx(2 * (2000 + 500) / per)
    assert rec["launches"] == 2
    assert rec["kernels"]["void sweep_kernel"] == {"launches": 1, "ns": pytest.approx(1.5e6)}
    assert rec["kernels"]["void sweep_x_kernel"] == {"launches": 1, "ns": pytest.approx(0.5e6)}


def test_roofline_names_the_pipe_that_needs_the_most_time():
    cells, clock_mhz = 1_000_000, 2000.0
    f = clock_mhz * 1e6
    rec = {"fp64_ops_per_cell": 900.0, "fp32_ops_per_cell": 1000.0, "warp_inst_per_cell": 160.0,
           "dfma_share": 0.4, "captured": "test"}
    need64 = 900.0 * cells / (pipes.SMS * pipes.FP64_PER_SM_CLK * f)
    need32 = 1000.0 * cells / (pipes.SMS * pipes.FP32_PER_SM_CLK * f)
    needis = 160.0 * cells / (pipes.SMS * pipes.ISSUE_PER_SM_CLK * f)
    sweep_ms = 2.0 * need64 * 1e3  # the float64 pipe busy half the measured time
    r = pipes.roofline(rec, cells, sweep_ms, clock_mhz)
    assert r["bound"] == "fp64"
    assert r["frac"] == pytest.approx(0.5)
    assert r["pipe_fracs"]["fp32"] == pytest.approx(need32 / (sweep_ms / 1e3))
    assert r["pipe_fracs"]["issue"] == pytest.approx(needis / (sweep_ms / 1e3))
    # an issue-heavy, float64-light record is bound by issue
    rec2 = dict(rec, fp64_ops_per_cell=8.0, warp_inst_per_cell=60.0)
    assert pipes.roofline(rec2, cells, 1.0, clock_mhz)["bound"] == "issue"


def test_records_are_keyed_by_precision_workload_and_fingerprint(tmp_path, monkeypatch):
    path = tmp_path / "records.json"
    recs = [{"precision": "fp64_fast", "workload": "shock_bubble_3d", "source_fingerprint": "aa", "x": 1},
            {"precision": "mixed", "workload": "shock_bubble_3d", "source_fingerprint": "aa", "x": 2}]
    path.write_text(json.dumps(recs))
    monkeypatch.setattr(pipes, "RECORDS", str(path))
    assert pipes.load("mixed", "shock_bubble_3d", "aa")["x"] == 2
    assert pipes.load("mixed", "shock_bubble_3d", "bb") is None  # captured on other sources
    assert pipes.load("df64", "shock_bubble_3d", "aa") is None
    monkeypatch.setattr(pipes, "RECORDS", str(tmp_path / "missing.json"))
    assert pipes.load("mixed", "shock_bubble_3d", "aa") is None
