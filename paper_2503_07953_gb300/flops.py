"""Algorithmic floating-point operation counts of the method, per cell.

Each building block is counted once per use the method needs (add, sub,
mul, div and sqrt each count as one operation; comparisons are not
counted).  The per-block numbers below were obtained by running the blocks
with an operation-counting scalar type on a representative face (HLLC in
its star region, the costlier branch); tests/test_flop_counts.py re-derives
them and fails if they drift.

Per cell and per directional sweep the method needs one
conservative-to-primitive conversion, the WENO5 edge values of N_q
primitives on both edges of the cell (the smoothness indicators of a cell's
three stencils are shared by its two edges), the physical-state test of the
two reconstructed states and one HLLC solve (one face per cell), and one
flux difference.  One RK3 step makes ndim sweeps per stage,
three stages, three stage updates and one CFL evaluation.
"""
from __future__ import annotations

BLOCKS = {
    # nf, nd, WENO-M: per-call counts of each block
    "shock_bubble_3d": {"nq": 7, "nd": 3, "c2p": 23, "weno_edge": 115, "weno_beta": 33, "hllc": 125,
                        "cell_term": 18, "rk_update": 35, "cfl_cell": 21, "face_check": 24},
    "random_interfaces_3d": {"nq": 9, "nd": 3, "c2p": 29, "weno_edge": 115, "weno_beta": 33, "hllc": 143,
                             "cell_term": 26, "rk_update": 45, "cfl_cell": 27, "face_check": 36},
    "bubble_collapse_2d": {"nq": 6, "nd": 2, "c2p": 20, "weno_edge": 115, "weno_beta": 33, "hllc": 113,
                           "cell_term": 16, "rk_update": 30, "cfl_cell": 19, "face_check": 24},
    "water_air_1d": {"nq": 5, "nd": 1, "c2p": 17, "weno_edge": 115, "weno_beta": 33, "hllc": 101,
                     "cell_term": 14, "rk_update": 25, "cfl_cell": 17, "face_check": 24},
}


def per_cell_sweep(workload: str) -> int:
    """Operations per cell of one directional sweep (excluding the stage update)."""
    b = BLOCKS[workload]
    weno = b["nq"] * (2 * b["weno_edge"] - b["weno_beta"])
    return b["c2p"] + weno + b["face_check"] + b["hllc"] + b["cell_term"]


def per_cell_step(workload: str) -> int:
    """Operations per cell of one RK3 step with its CFL evaluation."""
    b = BLOCKS[workload]
    return 3 * b["nd"] * per_cell_sweep(workload) + 3 * b["rk_update"] + b["cfl_cell"]
