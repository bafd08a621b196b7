"""The algorithmic operation counts used by the benchmark's roofline are the
oracle's operation counts of each building block."""
import pytest

from paper_2503_07953_gb300 import flops
from paper_2503_07953_gb300 import workloads as wl
from tests.helpers import oracle_problem

MAKERS = {
    "shock_bubble_3d": lambda: wl.shock_bubble_3d(dims=(8, 8, 8)),
    "random_interfaces_3d": lambda: wl.random_interfaces_3d(dims=(8, 8, 8)),
    "bubble_collapse_2d": lambda: wl.bubble_collapse_2d(dims=(8, 8)),
    "water_air_1d": lambda: wl.water_air_shock_tube(8),
}


@pytest.mark.parametrize("name", sorted(MAKERS))
def test_block_counts_match_oracle(oracle_lib, name):
    case, W = MAKERS[name]()
    P = oracle_problem(oracle_lib, case)
    q = oracle_lib.prim_to_cons(P, W).reshape(case.nq, -1)
    counts = oracle_lib.block_counts(P, q[:, 0].copy(), q[:, 1].copy())
    b = flops.BLOCKS[name]
    assert b["nq"] == case.nq and b["nd"] == case.ndim
    for blk, c in counts.items():
        assert b[blk] == c["add"] + c["mul"] + c["div"] + c["sqrt"], blk


def test_per_step_total_is_close_to_the_oracle_count(oracle_lib):
    """The oracle recomputes primitives six times per face and the smoothness
    indicators per edge; removing exactly that redundancy from its counted
    step must give the algorithmic count."""
    case, W = wl.shock_bubble_3d(dims=(6, 6, 6))
    case.bc_lo = [0, 0, 0]
    case.bc_hi = [0, 0, 0]
    P = oracle_problem(oracle_lib, case)
    q = oracle_lib.prim_to_cons(P, W)
    c = oracle_lib.rk3_step_counts(P, q, 1e-4)
    total = c["add"] + c["mul"] + c["div"] + c["sqrt"]
    b = flops.BLOCKS["shock_bubble_3d"]
    ncell = 6 ** 3
    faces = 36 * 7  # the oracle computes the n + 1 faces of each of the 36 lines
    # oracle: per face 6 c2p and 2 nq full edges; per cell one cell term per direction
    oracle_per_sweep = faces * (6 * b["c2p"] + 2 * b["nq"] * b["weno_edge"] + b["face_check"] + b["hllc"]) \
        + ncell * b["cell_term"]
    rk = ncell * (3 * b["rk_update"] - 2 * b["nq"])  # stage 1 is q + dt L: 2 ops per field instead of 5
    # accumulation into L: nq adds per cell per direction
    acc = ncell * b["nq"] * 3
    expect = 3 * (3 * oracle_per_sweep + acc) + rk
    # the HLLC branch mix of this state differs from the star-region count
    assert abs(total - expect) / expect < 0.02, (total, expect)
