"""The measurement studies run end to end on small sizes and report
consistent numbers (the full-size runs are summarised under profiles/)."""
import json

import pytest

from paper_2503_07953_gb300 import studies

pytestmark = pytest.mark.gpu


def run(capsys, argv):
    studies.main(argv)
    return [json.loads(line) for line in capsys.readouterr().out.splitlines() if line.startswith("{")]


def test_sizes(capsys, cuda_device):
    recs = run(capsys, ["sizes", "--sizes", "24", "--steps", "1", "--precisions", "fp64_fast", "mixed"])
    assert [r["precision"] for r in recs] == ["fp64_fast", "mixed"]
    for r in recs:
        assert r["cells"] == 24 ** 3 and r["cell_updates_per_s"] > 0 and r["vjp_over_fwd"] > 0


def test_mixed_error(capsys, cuda_device):
    (r,) = run(capsys, ["mixed-error", "--n", "24", "--steps", "3"])
    assert len(r["field_max_rel_err_mixed_vs_reference"]) == 9
    assert max(r["field_max_rel_err_mixed_vs_reference"]) < 1e-3


def test_adjoint(capsys, cuda_device):
    # 100 steps: the collapse's pressure waves reach the wall (after ~20
    # steps the wall pressure hardly depends on the bubble yet and the
    # derivative is at rounding level)
    (r,) = run(capsys, ["adjoint", "--n", "32", "--steps", "100", "--snapshots", "4", "--directions", "2",
                        "--precisions", "fp64_fast", "--h", "1e-6"])
    assert r["max_live_snapshots"] <= 4 and r["vjp_steps"] == 100
    assert r["J"] == pytest.approx(r["J_forward_only"], rel=1e-12)
    assert r["fd_rel_diff_max"] < 1e-4


def test_tube_graph_replay_matches(capsys, cuda_device):
    recs = run(capsys, ["tube", "--n", "200", "--steps", "20"])
    assert len(recs) == 3 and all(r["graph_result_bitwise_equal"] for r in recs)
