"""Pins of the oracle's Kapila model (Sec. 2.1.1): the K div(u) term of the
volume-fraction equation with the Wood mixture sound speed, two fluids.

A homogeneous water / air mixture carries sound at Wood's speed,
1/(rho c^2) = sum_i alpha_i / (rho_i c_i^2), far below the speed of the
K = 0 model's single mixture stiffened gas; a pressure pulse must travel at
that speed, and each phase must stay on its own isentrope.  Both follow from
the K term alone (the wave-speed estimate of the Riemann solver only sets
the dissipation), so they pin its form and sign."""
import math

import numpy as np
import pytest

from paper_2503_07953_gb300 import workloads as wl

GAMMA = [4.4, 1.4]
PI = [6e8, 0.0]
RHO = [1000.0, 1.2]
P0 = 1.0e5


def pulse_case(n, model, a1=0.5, amp=1e-3, width=0.03):
    case = wl.Case("pulse", [n], [0.0], [1.0], [wl.PERIODIC], [wl.PERIODIC], GAMMA, PI, cfl=0.4, steps=0)
    case.model = model
    X, _, _ = wl._centres(case)
    dp = amp * P0 * np.exp(-((X - 0.5) / width) ** 2)
    p = P0 + dp
    # each phase compressed along its own isentrope: rho_i ~ (p + pi_i)^(1/gamma_i)
    rho = [RHO[i] * ((p + PI[i]) / (P0 + PI[i])) ** (1.0 / GAMMA[i]) for i in range(2)]
    a = np.full_like(X, a1)
    W = wl._assemble(case, [a, 1.0 - a], rho, [np.zeros_like(X)], p)
    return case, W


def wood_speed(a1):
    z = [GAMMA[i] * (P0 + PI[i]) for i in range(2)]
    rho = a1 * RHO[0] + (1 - a1) * RHO[1]
    return 1.0 / math.sqrt(rho * (a1 / z[0] + (1 - a1) / z[1]))


def frozen_mixture_speed(a1):
    g = [1 / (x - 1) for x in GAMMA]
    h = [x * p / (x - 1) for x, p in zip(GAMMA, PI)]
    G = a1 * g[0] + (1 - a1) * g[1]
    Pm = a1 * h[0] + (1 - a1) * h[1]
    rho = a1 * RHO[0] + (1 - a1) * RHO[1]
    return math.sqrt(((G + 1) * P0 + Pm) / (G * rho))


def run(oracle_lib, case, W, t_end, nsteps):
    P = oracle_lib.Problem(n=case.n, gamma=case.gamma, pi_inf=case.pi_inf, lo=case.lo, hi=case.hi,
                           bc_lo=case.bc_lo, bc_hi=case.bc_hi, model=case.model)
    q0 = oracle_lib.prim_to_cons(P, W)
    q, _, bad = oracle_lib.rk3_run(P, q0, nsteps, dts=np.full(nsteps, t_end / nsteps), return_bad=True)
    assert bad == 0
    return P, q, oracle_lib.cons_to_prim(P, q)


def right_peak(x, v):
    """Position of the maximum of v over x > 0.5, refined by a parabola."""
    m = x > 0.5
    i = int(np.argmax(np.where(m, v, -np.inf)))
    y0, y1, y2 = v[i - 1], v[i], v[i + 1]
    h = x[1] - x[0]
    return x[i] + 0.5 * h * (y0 - y2) / (y0 - 2 * y1 + y2)


@pytest.mark.parametrize("a1", [0.5, 0.1])
def test_pressure_pulse_travels_at_wood_speed(oracle_lib, a1):
    n = 400
    c_w = wood_speed(a1)
    assert c_w < 0.2 * frozen_mixture_speed(a1)  # the two models differ a lot here
    t_end = 0.25 / c_w
    case, W = pulse_case(n, 1, a1)
    nsteps = int(math.ceil(t_end / (0.4 / n / c_w)))
    P, q, w = run(oracle_lib, case, W, t_end, nsteps)
    x = (np.arange(n) + 0.5) / n
    speed = (right_peak(x, w[3, 0, 0]) - 0.5) / t_end
    assert speed == pytest.approx(c_w, rel=0.02), (speed, c_w)


def test_phases_stay_on_their_isentropes(oracle_lib):
    """Under the pulse's compression alpha_1 = (alpha_1 rho_1) / rho_1(p) with
    rho_1(p) on the water isentrope through the initial state: the Kapila
    model keeps it (to the scheme's error); the K = 0 model leaves alpha
    unchanged under uniform compression and misses it by the full amount."""
    n, a1 = 400, 0.5
    c_w = wood_speed(a1)
    t_end = 0.2 / c_w
    errs = {}
    for model in (0, 1):
        # (a larger pulse steepens into a shock within 0.06 m in this very
        # nonlinear mixture, where the non-conservative K term is unstable,
        # as Sec. 2.1.1 warns)
        case, W = pulse_case(n, model, a1, amp=1e-3)
        c = c_w if model == 1 else frozen_mixture_speed(a1)
        nsteps = int(math.ceil(t_end / (0.4 / n / c)))
        P, q, w = run(oracle_lib, case, W, t_end, nsteps)
        p = w[3, 0, 0]
        rho1 = RHO[0] * ((p + PI[0]) / (P0 + PI[0])) ** (1 / GAMMA[0])
        rho2 = RHO[1] * ((p + PI[1]) / (P0 + PI[1])) ** (1 / GAMMA[1])
        # both phasic masses are carried by the same velocity: compare the
        # volume fraction with the one the two isentropes imply
        m1, m2 = w[0, 0, 0], w[1, 0, 0]
        a_isen = (m1 / rho1) / (m1 / rho1 + m2 / rho2)
        dev = np.abs(w[4, 0, 0] - a_isen).max()
        swing = np.abs(a_isen - a1).max()
        errs[model] = dev / swing
    assert errs[1] < 0.05, errs
    assert errs[0] > 0.5, errs


def test_identical_fluids_reduce_to_the_k0_model(oracle_lib):
    """With identical (gamma, pi_inf) K vanishes and Wood's speed is the
    mixture speed: the two models give the same trajectory to rounding."""
    case = wl.Case("same", [24, 20], [0, 0], [1.0, 0.8], [0, 1], [0, 2], [1.4, 1.4], [0.0, 0.0], 0.4, 0)
    W = wl.random_smooth_state(case, seed=6, amp=0.2)
    out = []
    for model in (0, 1):
        P = oracle_lib.Problem(n=case.n, gamma=case.gamma, pi_inf=case.pi_inf, lo=case.lo, hi=case.hi,
                               bc_lo=case.bc_lo, bc_hi=case.bc_hi, model=model)
        q0 = oracle_lib.prim_to_cons(P, W)
        q, _ = oracle_lib.rk3_run(P, q0, 20, dts=np.full(20, 2e-3))
        out.append(q)
    for k in range(case.nq):
        assert np.abs(out[1][k] - out[0][k]).max() <= 1e-12 * np.abs(out[0][k]).max()


def test_kapila_needs_two_fluids(oracle_lib):
    P = oracle_lib.Problem(n=[8], gamma=[1.4, 1.6, 4.4], pi_inf=[0, 0, 1], model=1)
    with pytest.raises(Exception):
        oracle_lib.rhs(P, np.ones(P.shape))
