"""Oracle against exact Riemann solutions (single-fluid Sod, two-fluid
stiffened-gas water/air), and the exact solver's own self-checks."""
import os

import numpy as np
import pytest

from oracle import exact_riemann as er
from paper_2503_07953_gb300 import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))

CASES = {
    "sod": (er.Side(1.0, 0.0, 1.0, 1.4, 0.0), er.Side(0.125, 0.0, 0.1, 1.4, 0.0)),
    "water_air": (er.Side(1000.0, 0.0, 1e9, 4.4, 6e8), er.Side(50.0, 0.0, 1e5, 1.4, 0.0)),
    "double_shock": (er.Side(1.0, 2.0, 1.0, 1.4, 0.0), er.Side(1.0, -2.0, 1.0, 1.4, 0.0)),
    "double_rarefaction": (er.Side(1.0, -1.0, 1.0, 1.4, 0.0), er.Side(1.0, 1.0, 1.0, 1.4, 0.0)),
    "air_water_stiff": (er.Side(1.2, 0.0, 1e7, 1.4, 0.0), er.Side(1000.0, 0.0, 1e5, 6.1, 2e9)),
}


def test_sod_star_state_matches_toro():
    vals = {}
    with open(os.path.join(HERE, "golden", "sod_star_state.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    ps, us = er.star_state(*CASES["sod"])
    assert round(ps, 5) == vals["p_star"]
    assert round(us, 5) == vals["u_star"]


@pytest.mark.parametrize("name", sorted(CASES))
def test_exact_solver_jump_conditions(name):
    res = er.check_waves(*CASES[name])
    for k, v in res.items():
        assert v < 1e-12, (k, v)


@pytest.mark.parametrize("name", sorted(CASES))
def test_exact_solution_pressure_velocity_continuous_at_contact(name):
    L, R = CASES[name]
    ps, us = er.star_state(L, R)
    eps = 1e-9 * max(1.0, abs(us))
    rho, u, p, side = er.sample(L, R, np.array([us - eps, us + eps]))
    assert side.tolist() == [0, 1]
    assert u[0] == pytest.approx(u[1], rel=1e-12, abs=1e-12)
    assert p[0] == pytest.approx(p[1], rel=1e-12)


def _run_to(oracle_lib, case, W, t_end, cfl, riemann=0):
    P = oracle_lib.Problem(n=case.n, gamma=case.gamma, pi_inf=case.pi_inf,
                           bc_lo=case.bc_lo, bc_hi=case.bc_hi, riemann=riemann)
    q = oracle_lib.prim_to_cons(P, W)
    t, bad = 0.0, 0
    while t < t_end * (1 - 1e-14):
        dt = min(oracle_lib.cfl_dt(P, q, cfl), t_end - t)
        q, b = oracle_lib.rk3_step(P, q, dt, return_bad=True)
        bad += b
        t += dt
    return oracle_lib.cons_to_prim(P, q), bad


@pytest.mark.parametrize("riemann", [0, 1])
def test_sod_converges_to_exact_solution(oracle_lib, riemann):
    """HLLC and HLL (Sec. 3.2.2) both converge to the exact solution."""
    L, R = CASES["sod"]
    errs = []
    for n in (100, 200, 400):
        case, W = wl.riemann_1d(n, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.5, [1.4], [0.0])
        w, bad = _run_to(oracle_lib, case, W, 0.2, 0.4, riemann)
        assert bad == 0
        rho, u, p, _ = er.cell_averages(L, R, 0.5, 0.2, n)
        errs.append([np.abs(w[0, 0, 0] - rho).mean(), np.abs(w[1, 0, 0] - u).mean(),
                     np.abs(w[2, 0, 0] - p).mean()])
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert errs[-1, 0] < 1.5e-3 and errs[-1, 2] < 1e-3
    assert (rates > 0.8).all(), rates


def test_water_air_shock_tube_converges(oracle_lib):
    """The two-fluid workload's Riemann problem (water at 1e9 Pa against air
    at 1e5 Pa, different stiffened gases), run to a fixed time."""
    L, R = CASES["water_air"]
    t_end = 2.0e-5
    errs = []
    for n in (250, 500, 1000):
        case, W = wl.water_air_shock_tube(n)
        w, bad = _run_to(oracle_lib, case, W, t_end, 0.3)
        assert bad == 0
        rho, u, p, _ = er.cell_averages(L, R, 0.7, t_end, n)
        errs.append([np.abs(w[2, 0, 0] - u).mean() / 500.0, np.abs(w[3, 0, 0] - p).mean() / 1e9])
        # the pressure stays between the initial extremes (no large overshoot)
        assert w[3].min() > 0.5e5 and w[3].max() < 1.05e9
    errs = np.array(errs)
    assert (errs[1:] < errs[:-1]).all(), errs
    assert errs[-1, 0] < 5e-3 and errs[-1, 1] < 5e-3
