"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

MFC_FP64 evaluates every formula in the oracle's operation order with IEEE
division and square root and no fused multiply-add, so it must agree with
the oracle bit for bit, for one evaluation of L and after 100+ steps.

MFC_FP64_FAST differs from the oracle by rounding only; per field,
max |gpu - oracle| / max |oracle| <= 1e-11 (the FP64 target) on workloads
whose own rounding sensitivity is far below that (the 3D shock-bubble).
Momentum components share one scale (tests.helpers.field_errors).

Some workloads amplify rounding by many orders of magnitude (measured on
the oracle itself: a 1-ulp perturbation of the 1D water/air state grows to
~1e-6 in 200 steps with WENO-M's eps = 1e-40), which is why the
reproducible mode exists and carries the long-run comparisons.
"""
import numpy as np
import pytest
import torch

from paper_2503_07953_gb300 import workloads as wl
from tests.helpers import case_errors, oracle_problem, solver_for, to_host

pytestmark = pytest.mark.gpu

TOL = 1e-11


def four_fluid_case(dims=(13, 11, 9)):
    case = wl.Case("four_fluid", list(dims), [0.0] * 3, [1.0, 0.9, 0.8], [0, 1, 2], [0, 2, 1],
                   [1.4, 1.67, 4.4, 6.1], [0.0, 0.0, 10.0, 30.0], cfl=0.4, steps=0)
    return case, wl.random_smooth_state(case, seed=11, amp=0.15)


def sod_single_fluid(n=200):
    return wl.riemann_1d(n, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.5, [1.4], [0.0])


CASES = {
    "shock_bubble_3d": lambda: wl.shock_bubble_3d(dims=(37, 29, 21)),
    "random_interfaces_3d": lambda: wl.random_interfaces_window(dims=(26, 24, 22)),
    "bubble_collapse_2d": lambda: wl.bubble_collapse_2d(dims=(41, 33)),
    "water_air_1d": lambda: wl.water_air_shock_tube(1000),
    "sod_single_fluid_1d": lambda: sod_single_fluid(),
    "four_fluid_3d": four_fluid_case,
}


def setup(oracle_lib, mfc_lib, make, **kw):
    case, W = make()
    P = oracle_problem(oracle_lib, case)
    S = solver_for(mfc_lib, case, **kw)
    q_o = oracle_lib.prim_to_cons(P, W)
    q_g = S.prim_to_cons(S.from_interior(W))
    return case, W, P, S, q_o, q_g


@pytest.mark.parametrize("name", sorted(CASES))
def test_prim_cons_maps_bitwise(oracle_lib, mfc_lib, cuda_device, name):
    case, W, P, S, q_o, q_g = setup(oracle_lib, mfc_lib, CASES[name])
    assert np.array_equal(to_host(S, q_g), q_o)
    assert np.array_equal(to_host(S, S.cons_to_prim(q_g)), oracle_lib.cons_to_prim(P, q_o))


@pytest.mark.parametrize("name", sorted(CASES))
def test_rhs_bitwise(oracle_lib, mfc_lib, cuda_device, name):
    case, W, P, S, q_o, q_g = setup(oracle_lib, mfc_lib, CASES[name])
    L_o, bad = oracle_lib.rhs(P, q_o, return_bad=True)
    assert bad == 0
    L_g = to_host(S, S.rhs(S.from_interior(q_o)))
    assert np.array_equal(L_g, L_o), case_errors(case, L_g, L_o)
    S.check()


@pytest.mark.parametrize("name", sorted(CASES))
def test_rhs_fast(oracle_lib, mfc_lib, cuda_device, name):
    """MFC_FP64_FAST: one evaluation of L to rounding."""
    case, W, P, S, q_o, q_g = setup(oracle_lib, mfc_lib, CASES[name], precision=mfc_lib.MFC_FP64_FAST)
    L_o = oracle_lib.rhs(P, q_o)
    err = case_errors(case, to_host(S, S.rhs(S.from_interior(q_o))), L_o)
    assert (err <= TOL).all(), err


@pytest.mark.parametrize("name", sorted(CASES))
def test_step_mixed(oracle_lib, mfc_lib, cuda_device, name):
    """MFC_MIXED: float32 reconstruction, Riemann solve and flux difference.
    One RK3 step at the CFL dt agrees with the oracle per field to the
    float32 rounding of fluxes much larger than their difference: <= 1e-4
    of each field's maximum (measured: up to 4e-5 on the momenta of the
    bubble collapse, which start from rest and are driven by 1e7 Pa
    pressure fluxes)."""
    case, W, P, S, q_o, q_g = setup(oracle_lib, mfc_lib, CASES[name], precision=mfc_lib.MFC_MIXED)
    dt = oracle_lib.cfl_dt(P, q_o, case.cfl)
    q = S.from_interior(q_o)
    S.rk3_step(q, dt)
    S.check()
    err = case_errors(case, to_host(S, q), oracle_lib.rk3_step(P, q_o, dt))
    assert (err <= 1e-4).all(), err


@pytest.mark.parametrize("weno", [0, 2, 3])
@pytest.mark.parametrize("prec", [0, 2])
def test_rhs_weno_variants(oracle_lib, mfc_lib, cuda_device, weno, prec):
    case, W = wl.shock_bubble_3d(dims=(19, 16, 14))
    case.weno = weno
    case.eps = 1e-6 if weno == 0 else 1e-40
    P = oracle_problem(oracle_lib, case)
    S = solver_for(mfc_lib, case, precision=prec)
    q_o = oracle_lib.prim_to_cons(P, W)
    L_g = to_host(S, S.rhs(S.from_interior(q_o)))
    L_o = oracle_lib.rhs(P, q_o)
    if prec == mfc_lib.MFC_FP64:
        assert np.array_equal(L_g, L_o)
    else:
        assert (case_errors(case, L_g, L_o) <= TOL).all()


def test_compute_dt_bitwise(oracle_lib, mfc_lib, cuda_device):
    for make in (CASES["shock_bubble_3d"], CASES["water_air_1d"], CASES["random_interfaces_3d"]):
        case, W, P, S, q_o, q_g = setup(oracle_lib, mfc_lib, make)
        assert S.compute_dt(S.from_interior(q_o)) == oracle_lib.cfl_dt(P, q_o, case.cfl)


@pytest.mark.parametrize("prec", [1, 2])
def test_compute_dt_fast_arithmetic(oracle_lib, mfc_lib, cuda_device, prec):
    """MFC_FP64_FAST and MFC_MIXED take the CFL step with refined
    reciprocals (float64): within a few ulps of the oracle's."""
    for make in (CASES["shock_bubble_3d"], CASES["water_air_1d"], CASES["random_interfaces_3d"]):
        case, W, P, S, q_o, q_g = setup(oracle_lib, mfc_lib, make, precision=prec)
        assert S.compute_dt(S.from_interior(q_o)) == pytest.approx(oracle_lib.cfl_dt(P, q_o, case.cfl), rel=1e-14)


RUNS = {
    "shock_bubble_3d": (lambda: wl.shock_bubble_3d(dims=(20, 18, 16)), 100),
    "bubble_collapse_2d": (lambda: wl.bubble_collapse_2d(dims=(64, 60)), 100),
    "water_air_1d": (lambda: wl.water_air_shock_tube(1000), 200),
    "random_interfaces_3d": (lambda: wl.random_interfaces_window(origin=(10, 300, 420), dims=(24, 22, 20)), 50),
}


@pytest.mark.parametrize("name", sorted(RUNS))
def test_rk3_run_bitwise(oracle_lib, mfc_lib, cuda_device, name):
    """The paper-shaped workloads (small grids) for their full step counts
    with the CFL dt of every step: identical dt sequences and final states."""
    make, steps = RUNS[name]
    case, W, P, S, q_o, q_g = setup(oracle_lib, mfc_lib, make)
    q_g = S.from_interior(q_o)
    dt_log = torch.zeros(steps, dtype=torch.float64, device=cuda_device)
    S.rk3_run(q_g, steps, 0.0, dt_log)
    S.check()
    q_end, dts, bad = oracle_lib.rk3_run(P, q_o, steps, cfl=case.cfl, return_bad=True)
    assert bad == 0
    assert np.array_equal(dt_log.cpu().numpy(), dts)
    got = to_host(S, q_g)
    assert np.array_equal(got, q_end), case_errors(case, got, q_end)


@pytest.mark.parametrize("name", ["shock_bubble_3d", "water_air_1d"])
def test_rk3_run_teno_bitwise(oracle_lib, mfc_lib, cuda_device, name):
    """TENO weights (Sec. 4.2.2), MFC_FP64: 50 CFL steps bit for bit."""
    make, _ = RUNS[name]
    case, W = make()
    case.weno = 3
    P = oracle_problem(oracle_lib, case)
    S = solver_for(mfc_lib, case)
    q_o = oracle_lib.prim_to_cons(P, W)
    q_g = S.from_interior(q_o)
    S.rk3_run(q_g, 50, 0.0)
    S.check()
    q_end, _ = oracle_lib.rk3_run(P, q_o, 50, cfl=case.cfl)
    got = to_host(S, q_g)
    assert np.array_equal(got, q_end), case_errors(case, got, q_end)


def kapila_pulse(n=400):
    """A small pressure pulse in a 50/50 water / air mixture at rest."""
    case = wl.Case("pulse", [n], [0.0], [1.0], [wl.PERIODIC], [wl.PERIODIC], [4.4, 1.4], [6e8, 0.0], 0.4, 0)
    case.model = 1
    X, _, _ = wl._centres(case)
    p = 1e5 * (1 + 1e-3 * np.exp(-((X - 0.5) / 0.03) ** 2))
    rho = [1000.0 * ((p + 6e8) / (1e5 + 6e8)) ** (1 / 4.4), 1.2 * (p / 1e5) ** (1 / 1.4)]
    a = np.full_like(X, 0.5)
    return case, wl._assemble(case, [a, 1 - a], rho, [np.zeros_like(X)], p)


def kapila_shock_bubble():
    case, W = wl.shock_bubble_3d(dims=(20, 18, 16))
    case.model = 1
    return case, W


@pytest.mark.parametrize("make,steps", [(kapila_pulse, 100), (kapila_shock_bubble, 50)])
def test_rk3_run_kapila_bitwise(oracle_lib, mfc_lib, cuda_device, make, steps):
    """The Kapila K div u term with the Wood sound speed (Sec. 2.1.1),
    MFC_FP64: CFL steps bit for bit, dt sequence included."""
    case, W = make()
    P = oracle_problem(oracle_lib, case)
    S = solver_for(mfc_lib, case)
    q_o = oracle_lib.prim_to_cons(P, W)
    q_g = S.from_interior(q_o)
    dt_log = torch.zeros(steps, dtype=torch.float64, device=cuda_device)
    S.rk3_run(q_g, steps, 0.0, dt_log)
    S.check()
    q_end, dts, bad = oracle_lib.rk3_run(P, q_o, steps, cfl=case.cfl, return_bad=True)
    assert bad == 0
    assert np.array_equal(dt_log.cpu().numpy(), dts)
    got = to_host(S, q_g)
    assert np.array_equal(got, q_end), case_errors(case, got, q_end)


@pytest.mark.parametrize("prec,tol", [(2, 1e-11), (1, 1e-4)])
def test_step_kapila_fast_and_mixed(oracle_lib, mfc_lib, cuda_device, prec, tol):
    case, W = kapila_shock_bubble()
    P = oracle_problem(oracle_lib, case)
    S = solver_for(mfc_lib, case, precision=prec)
    q_o = oracle_lib.prim_to_cons(P, W)
    dt = oracle_lib.cfl_dt(P, q_o, case.cfl)
    q = S.from_interior(q_o)
    S.rk3_step(q, dt)
    S.check()
    err = case_errors(case, to_host(S, q), oracle_lib.rk3_step(P, q_o, dt))
    assert (err <= tol).all(), err


SOLVERS = [(1, 0), (0, 1), (0, 2), (1, 1)]  # (riemann, low_mach): HLL, HLLC+Thornber, HLLC+APC, HLL+Thornber


@pytest.mark.parametrize("riemann,low_mach", SOLVERS)
def test_rk3_run_riemann_variants_bitwise(oracle_lib, mfc_lib, cuda_device, riemann, low_mach):
    """HLL and the low-Mach corrections (Sec. 3.2.2, Sec. 4.2.4), MFC_FP64:
    the Gresho vortex at M = 0.01 (40 steps) and the shock-bubble
    (20 steps), bit for bit with their dt sequences."""
    for make, steps in ((lambda: wl.gresho_vortex(24, 1e-2), 40), (lambda: wl.shock_bubble_3d(dims=(16, 14, 12)), 20)):
        case, W = make()
        case.riemann, case.low_mach = riemann, low_mach
        P = oracle_problem(oracle_lib, case)
        S = solver_for(mfc_lib, case)
        q_o = oracle_lib.prim_to_cons(P, W)
        q_g = S.from_interior(q_o)
        dt_log = torch.zeros(steps, dtype=torch.float64, device=cuda_device)
        S.rk3_run(q_g, steps, 0.0, dt_log)
        S.check()
        q_end, dts, bad = oracle_lib.rk3_run(P, q_o, steps, cfl=case.cfl, return_bad=True)
        assert bad == 0
        assert np.array_equal(dt_log.cpu().numpy(), dts)
        got = to_host(S, q_g)
        assert np.array_equal(got, q_end), case_errors(case, got, q_end)


@pytest.mark.parametrize("riemann,low_mach", SOLVERS)
@pytest.mark.parametrize("prec,tol", [(2, 1e-11), (1, 1e-4)])
def test_step_riemann_variants_fast_and_mixed(oracle_lib, mfc_lib, cuda_device, riemann, low_mach, prec, tol):
    case, W = wl.shock_bubble_3d(dims=(16, 14, 12))
    case.riemann, case.low_mach = riemann, low_mach
    P = oracle_problem(oracle_lib, case)
    S = solver_for(mfc_lib, case, precision=prec)
    q_o = oracle_lib.prim_to_cons(P, W)
    dt = oracle_lib.cfl_dt(P, q_o, case.cfl)
    q = S.from_interior(q_o)
    S.rk3_step(q, dt)
    S.check()
    err = case_errors(case, to_host(S, q), oracle_lib.rk3_step(P, q_o, dt))
    assert (err <= tol).all(), err


def test_rk3_run_fast_shock_bubble(oracle_lib, mfc_lib, cuda_device):
    """MFC_FP64_FAST, 100 CFL steps of the 3D shock-bubble: <= 1e-11 per field."""
    make, steps = RUNS["shock_bubble_3d"]
    case, W, P, S, q_o, q_g = setup(oracle_lib, mfc_lib, make, precision=mfc_lib.MFC_FP64_FAST)
    q_g = S.from_interior(q_o)
    S.rk3_run(q_g, steps, 0.0)
    S.check()
    q_end, dts = oracle_lib.rk3_run(P, q_o, steps, cfl=case.cfl)
    err = case_errors(case, to_host(S, q_g), q_end)
    assert (err <= TOL).all(), err


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_full_size_step_sampled(oracle_lib, mfc_lib, cuda_device, prec):
    """The 256^3 shock-bubble workload in the benchmarked configuration: one
    step on the GPU, checked at sampled cells (corners, walls, the shock and
    the bubble interface) against the oracle's domain-of-dependence
    evaluation of the same step.  Bitwise in MFC_FP64, 1e-11 in
    MFC_FP64_FAST, 1e-5 in MFC_MIXED (float32 fluxes)."""
    case, W = wl.shock_bubble_3d(256)
    P = oracle_problem(oracle_lib, case)
    S = solver_for(mfc_lib, case, precision=prec)
    q_g = S.prim_to_cons(S.from_interior(W))
    q_o = to_host(S, q_g)  # the oracle steps the GPU's own initial state
    dt = oracle_lib.cfl_dt(P, q_o, case.cfl)
    S.rk3_step(q_g, dt)
    S.check()
    out_g = to_host(S, q_g)
    rng = np.random.default_rng(0)
    cells = [(0, 0, 0), (255, 255, 255), (0, 255, 128), (255, 0, 3), (64, 128, 128), (63, 127, 200),
             (89, 128, 128), (128, 90, 128), (128, 128, 166), (167, 128, 128), (128, 1, 254)]
    cells += [tuple(int(v) for v in rng.integers(0, 256, 3)) for _ in range(9)]
    ref = oracle_lib.rk3_step_sampled(P, q_o, dt, cells)
    got = np.stack([out_g[:, k, j, i] for (i, j, k) in cells])
    if prec == mfc_lib.MFC_FP64:
        assert np.array_equal(got, ref)
    else:
        scale = np.abs(out_g).max(axis=(1, 2, 3))
        scale[case.nf:case.nf + case.ndim] = scale[case.nf:case.nf + case.ndim].max()
        err = (np.abs(got - ref) / scale).max(axis=0)
        assert (err <= (TOL if prec == mfc_lib.MFC_FP64_FAST else 1e-5)).all(), err


@pytest.mark.parametrize("ghost", [0, 5])
def test_ghost_padding_does_not_change_results(oracle_lib, mfc_lib, cuda_device, ghost):
    case, W = wl.shock_bubble_3d(dims=(17, 13, 11))
    S3 = solver_for(mfc_lib, case)
    Sg = solver_for(mfc_lib, case, ghost=ghost)
    a = S3.prim_to_cons(S3.from_interior(W))
    b = Sg.prim_to_cons(Sg.from_interior(W))
    S3.rk3_run(a, 3)
    Sg.rk3_run(b, 3)
    assert np.array_equal(to_host(S3, a), to_host(Sg, b))


@pytest.mark.parametrize("dims,bc", [
    ((3,), 0),            # smallest periodic axis
    ((5,), 1),
    ((3, 3, 3), 0),
    ((7, 1), 1),          # one cell across a transmissive axis
    ((1, 6, 4), 1),
    ((67, 3, 18), 2),     # ragged segments along x, smallest reflective axis
])
def test_degenerate_sizes(oracle_lib, mfc_lib, cuda_device, dims, bc):
    nd = len(dims)
    case = wl.Case("tiny", list(dims), [0.0] * nd, [1.0] * nd, [bc] * nd, [bc] * nd, [1.4, 1.67],
                   [0.0, 0.0], cfl=0.4, steps=0)
    W = wl.random_smooth_state(case, seed=1, amp=0.1)
    P = oracle_problem(oracle_lib, case)
    S = solver_for(mfc_lib, case)
    q_o = oracle_lib.prim_to_cons(P, W)
    q_g = S.from_interior(q_o)
    S.rk3_run(q_g, 5)
    q_end, _ = oracle_lib.rk3_run(P, q_o, 5, cfl=case.cfl)
    assert np.array_equal(to_host(S, q_g), q_end)


def test_positivity_fallback_matches_oracle(oracle_lib, mfc_lib, cuda_device):
    """Three stiff fluids at 1e5 Pa on a coarse 24x22x20 grid of the whole
    cube: WENO overshoots make thousands of reconstructed states
    non-physical (c^2 < 0 without the fallback); both sides fall back to
    first order at exactly those faces."""
    case, W = wl.random_interfaces_3d(dims=(24, 22, 20))
    P = oracle_problem(oracle_lib, case)
    q_o = oracle_lib.prim_to_cons(P, W)
    L_o, bad = oracle_lib.rhs(P, q_o, return_bad=True)
    assert bad == 0
    S = solver_for(mfc_lib, case)
    assert np.array_equal(to_host(S, S.rhs(S.from_interior(q_o))), L_o)


def test_nonphysical_state_reported(oracle_lib, mfc_lib, cuda_device):
    case, W = wl.shock_bubble_3d(dims=(8, 8, 8))
    S = solver_for(mfc_lib, case)
    q = S.prim_to_cons(S.from_interior(W))
    S.interior(q)[case.nf + case.ndim, 4, 4, 4] = -10.0  # negative energy -> p + pi < 0
    with pytest.raises(mfc_lib.MfcError) as ei:
        S.compute_dt(q)
    assert ei.value.status == mfc_lib.MFC_ERR_NONPHYSICAL
    S.check()  # the flag was cleared


def test_rejects_bad_arguments(mfc_lib, cuda_device):
    case, W = wl.shock_bubble_3d(dims=(8, 8, 8))
    S = solver_for(mfc_lib, case)
    q = S.empty()
    with pytest.raises(mfc_lib.MfcError) as ei:
        mfc_lib.mfc_rhs(S.ctx, q.data_ptr(), q.data_ptr(), None)
    assert ei.value.status == mfc_lib.MFC_ERR_ARG
    with pytest.raises(mfc_lib.MfcError):
        mfc_lib.mfc_rk3_step(S.ctx, 0, 0.0, None, None)
