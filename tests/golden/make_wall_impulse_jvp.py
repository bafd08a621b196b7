"""Write wall_impulse_jvp_<N>.txt: the 2D bubble-collapse wall impulse on
N x N cells over a number of CFL steps (Sec. 3.5-shaped workload, WENO5-M,
HLLC), its value J and its derivatives along two seeded directions of the
initial volume fraction, from the oracle alone: a forward run for the dt
sequence, then the forward-mode (dual-number) derivative of every RK3 step
at those dts.

    J = sum_n dt_n dy sum_j p(q^{n+1})[last x cell, j]

    python tests/golden/make_wall_impulse_jvp.py                    # 256 x 256, 500 steps
    python tests/golden/make_wall_impulse_jvp.py --n 1024 --steps 1800 --openmp

256 x 256 over 500 steps runs for about 15 minutes single-threaded.  At
1024 x 1024 the collapse's pressure waves need about 1360 steps to reach the
wall, so the 1800-step file has a wall impulse that depends on the initial
state; it runs for about 2.5 hours on 8 host threads (--openmp: the
oracle's OpenMP build, bit for bit the single-threaded one)."""
import argparse
import os
import sys

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2503_07953_gb300 import workloads as wl  # noqa: E402


def directions(a1, count=2):
    """Seeded directions supported where 1e-3 < alpha_1 < 1 - 1e-3, max-normalised."""
    band = ((a1 > 1e-3) & (a1 < 1 - 1e-3)).astype(float)
    gen = torch.Generator(device="cpu").manual_seed(0)
    for _ in range(count):
        d = torch.randn(a1.shape, generator=gen, dtype=torch.float64).numpy() * band
        yield d / np.abs(d).max()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--openmp", action="store_true")
    args = ap.parse_args()
    N, STEPS = args.n, args.steps
    if args.openmp:
        O.build(openmp=True)
        O.set_parallel(True)
    case, W = wl.bubble_collapse_2d(N)
    P = O.Problem(n=case.n, gamma=case.gamma, pi_inf=case.pi_inf, lo=case.lo, hi=case.hi,
                  bc_lo=case.bc_lo, bc_hi=case.bc_hi, weno=case.weno, eps=case.eps)
    nf, nd = case.nf, case.ndim
    a1 = W[nf + nd + 1].copy()
    r1, r2 = W[0] / a1, W[1] / (1 - a1)

    def q_of(alpha):
        Wp = W.copy()
        Wp[0], Wp[1], Wp[nf + nd + 1] = alpha * r1, (1 - alpha) * r2, alpha
        return O.prim_to_cons(P, Wp)

    q0 = q_of(a1)
    qT, dts = O.rk3_run(P, q0, STEPS, case.cfl)
    g = [1 / (x - 1) for x in case.gamma]
    h = [x * p / (x - 1) for x, p in zip(case.gamma, case.pi_inf)]
    dy = case.dx(1)

    def pressure_and_tangent(q, dq):
        rho, drho = q[0] + q[1], dq[0] + dq[1]
        ke = sum(q[nf + e] ** 2 for e in range(nd)) / (2 * rho)
        dke = sum(q[nf + e] * dq[nf + e] for e in range(nd)) / rho - ke * drho / rho
        a, da = q[nf + nd + 1], dq[nf + nd + 1]
        Gam, Pi = a * g[0] + (1 - a) * g[1], a * h[0] + (1 - a) * h[1]
        p = (q[nf + nd] - ke - Pi) / Gam
        dp = (dq[nf + nd] - dke - da * (h[0] - h[1])) / Gam - p * da * (g[0] - g[1]) / Gam
        return p, dp

    lines = [f"# bubble_collapse_2d {N}x{N}, {STEPS} CFL steps, WENO5-M + HLLC; written by make_wall_impulse_jvp.py"]
    if STEPS != 500 or N != 256:
        lines.append(f"dt_first {float(dts[0])!r}")
        lines.append(f"dt_last {float(dts[-1])!r}")
        lines.append(f"dt_sum {float(np.sum(dts))!r}")
    J = None
    for k, d in enumerate(directions(a1)):
        dq = (q_of(a1 + d) - q_of(a1 - d)) / 2  # the map alpha -> q is affine
        q = q0.copy()
        tot, dtot = 0.0, 0.0
        for s in range(STEPS):
            q, dq = O.rk3_step_jvp(P, q, dq, dts[s])
            p, dp = pressure_and_tangent(q, dq)
            tot += dts[s] * dy * p[0, :, -1].sum()
            dtot += dts[s] * dy * dp[0, :, -1].sum()
        J = tot
        lines.append(f"dJ_direction_{k} {float(dtot)!r}")
    lines.insert(1, f"J {float(J)!r}")
    with open(os.path.join(HERE, f"wall_impulse_jvp_{N}.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
