"""The hand-written adjoint (mfc_rhs_vjp, mfc_rk3_step_vjp) against the
oracle's forward-mode derivatives of the same computation.

Dot-product identity <v, J w> = <J^T v, w> with J w from the oracle's dual
numbers and J^T v from the CUDA adjoint; full Jacobians on tiny grids
(every column from the oracle, every row from the GPU); central finite
differences of the GPU's own forward step.

Where to compare.  The initial states of the workloads sit on the
non-smooth set of the method: at rest (u = 0) every face has S* = 0, the
switch between the two HLLC star states, and with WENO-M's eps = 1e-40 a
flat stencil gives weights whose derivatives are ratios of indicators of
rounding size.  Each side differentiates the branch its own forward pass
takes, so ties are only comparable where the forward passes are identical
(MFC_FP64 recomputes the oracle's forward bit for bit); and derivatives
taken at rounding-size indicators are ill-conditioned in any evaluation
order (forward-mode dual numbers and the reverse sweep round differently,
and sums of terms of size 1/beta cancel).  The Jiang-Shu eps = 1e-6 is an
absolute constant: against a pressure of 1e9 Pa the rounding residue of a
"flat" indicator (the square of an ulp of 3p, ~1e-13) is no longer
negligible, and a 1-ulp change of the state moves a Jacobian entry by up to
1e-5 relative.  The checks therefore use smooth states with the mapped
weights (both float64 modes), and the workloads' own initial states with
the Jiang-Shu weights in reduced units (densities over 1000 kg/m^3,
pressures over the workload's pressure scale), where the indicators'
rounding residue is ~1e-32, in MFC_FP64.
"""
import numpy as np
import pytest
import torch

from paper_2503_07953_gb300 import workloads as wl
from tests.helpers import field_scales, oracle_problem, solver_for, to_host

pytestmark = pytest.mark.gpu


def smooth_case(dims, bc_lo, bc_hi, gamma=(1.4, 4.4), pi=(0.0, 10.0), seed=3):
    nd = len(dims)
    hi = [1.0, 0.9, 0.8][:nd]
    case = wl.Case("adj", list(dims), [0.0] * nd, hi, list(bc_lo), list(bc_hi), list(gamma), list(pi),
                   cfl=0.4, steps=0)
    return case, wl.random_smooth_state(case, seed=seed, amp=0.15)


def js(make, rho0=1.0, p0=1.0):
    """The Jiang-Shu variant (eps = 1e-6) of a workload, in reduced units."""
    def f():
        case, W = wl.reduced_units(*make(), rho0, p0)
        case.weno, case.eps = 0, 1e-6
        return case, W
    return f


def teno(cw):
    case, W = cw
    case.weno, case.eps = 3, 1e-40
    return case, W


def solver(cw, riemann, low_mach):
    case, W = cw
    case.riemann, case.low_mach = riemann, low_mach
    return case, W


def kapila(cw):
    case, W = cw
    case.model = 1
    return case, W


def stiff_smooth_case(dims=(13, 11), seed=4):
    """Smooth water-like / air-like mixture at 1e9 Pa, moving at ~100 m/s."""
    nd = len(dims)
    case = wl.Case("adj_stiff", list(dims), [0.0] * nd, [1.0, 0.9, 0.8][:nd], [0] * nd, [0] * nd,
                   [4.4, 1.4], [6e8, 0.0], cfl=0.4, steps=0)
    W = wl.random_smooth_state(case, seed=seed, amp=0.15)
    nf = case.nf
    W[0] *= 1000.0
    W[1] *= 50.0
    for d in range(nd):
        W[nf + d] *= 300.0
    W[nf + nd] *= 1e9
    return case, W


CASES = {
    "smooth_3d_mixed_bc": lambda: smooth_case((11, 9, 7), (0, 1, 2), (0, 2, 1)),
    "stiff_smooth_2d": stiff_smooth_case,
    "smooth_2d_periodic": lambda: smooth_case((19, 17), (0, 0), (0, 0)),
    "smooth_2d_teno": lambda: teno(smooth_case((19, 17), (0, 1), (0, 2))),
    "smooth_2d_kapila": lambda: kapila(smooth_case((19, 17), (1, 0), (2, 0))),
    "smooth_2d_hll_thornber": lambda: solver(smooth_case((19, 17), (0, 1), (0, 2)), 1, 1),
    "smooth_2d_apc": lambda: solver(smooth_case((19, 17), (2, 0), (1, 0)), 0, 2),
    "shock_bubble_3d_js": js(lambda: wl.shock_bubble_3d(dims=(21, 18, 17))),
    "water_air_1d_js": js(lambda: wl.water_air_shock_tube(300), 1000.0, 1e9),
    "random_interfaces_js": js(lambda: wl.random_interfaces_window(dims=(12, 11, 10)), 1000.0, 1e5),
    "bubble_collapse_2d_js": js(lambda: wl.bubble_collapse_2d(dims=(24, 22)), 1000.0, 1e7),
}
SMOOTH = ["smooth_3d_mixed_bc", "smooth_2d_periodic", "stiff_smooth_2d", "smooth_2d_teno", "smooth_2d_kapila",
          "smooth_2d_hll_thornber", "smooth_2d_apc"]
# MFC_DF64: the adjoint sweeps of a double-float context run the reverse
# WENO5 in double-float (JS and mapped weights; the other variants in float64)
PARAMS = [(name, 0) for name in sorted(CASES)] + [(name, 2) for name in SMOOTH] + [(name, 3) for name in SMOOTH]


def dot(a, b):
    return float(np.sum(a * b))


def directions(case, q, seed):
    """w in the units of each field, v in the inverse units: <v, J w> is then a
    sum of nondimensional terms."""
    rng = np.random.default_rng(seed)
    scale = field_scales(case, q).reshape(-1, 1, 1, 1)
    return rng.normal(size=q.shape) * scale, rng.normal(size=q.shape) / scale


@pytest.mark.parametrize("name,prec", PARAMS)
def test_rhs_vjp_dot_product(oracle_lib, mfc_lib, cuda_device, name, prec):
    case, W = CASES[name]()
    P = oracle_problem(oracle_lib, case)
    S = solver_for(mfc_lib, case, precision=prec)
    q = oracle_lib.prim_to_cons(P, W)
    w, v = directions(case, q, 7)
    _, Jw = oracle_lib.rhs_jvp(P, q, w)
    qb = S.rhs_vjp(S.from_interior(q), S.from_interior(v))
    lhs = dot(v, Jw)
    rhs = dot(to_host(S, qb), w)
    assert rhs == pytest.approx(lhs, rel=1e-10), (lhs, rhs)


@pytest.mark.parametrize("name,prec", PARAMS)
def test_rk3_step_vjp_dot_product(oracle_lib, mfc_lib, cuda_device, name, prec):
    case, W = CASES[name]()
    P = oracle_problem(oracle_lib, case)
    S = solver_for(mfc_lib, case, precision=prec)
    q = oracle_lib.prim_to_cons(P, W)
    dt = oracle_lib.cfl_dt(P, q, case.cfl)
    w, v = directions(case, q, 8)
    _, Jw = oracle_lib.rk3_step_jvp(P, q, w, dt)
    qb = S.rk3_step_vjp(S.from_interior(q), dt, S.from_interior(v))
    lhs = dot(v, Jw)
    rhs = dot(to_host(S, qb), w)
    assert rhs == pytest.approx(lhs, rel=1e-10), (lhs, rhs)


def full_jacobians(oracle_lib, S, P, q):
    N = q.size
    J = np.empty((N, N))
    for j in range(N):
        e = np.zeros(N); e[j] = 1.0
        J[:, j] = oracle_lib.rhs_jvp(P, q, e.reshape(q.shape))[1].ravel()
    qg = S.from_interior(q)
    JT = np.empty((N, N))
    for i in range(N):
        e = np.zeros(N); e[i] = 1.0
        JT[i] = to_host(S, S.rhs_vjp(qg, S.from_interior(e.reshape(q.shape)))).ravel()
    return J, JT


@pytest.mark.parametrize("model,riemann,low_mach", [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (0, 0, 2),
                                                    (0, 1, 1), (1, 0, 2)])
@pytest.mark.parametrize("dims,bc_lo,bc_hi", [
    ((17,), (2,), (2,)),        # two segments, the second one cell long, reflective
    ((19,), (0,), (0,)),        # periodic with two segments
    ((40,), (1,), (2,)),        # three segments, transmissive / reflective
    ((6, 5), (0, 2), (0, 1)),   # 2D, every boundary type
    ((3, 4), (0, 1), (0, 1)),   # smallest periodic axis
])
def test_rhs_full_jacobian(oracle_lib, mfc_lib, cuda_device, dims, bc_lo, bc_hi, model, riemann, low_mach):
    """Every column of dL/dq from the oracle's dual numbers equals every row
    of the GPU adjoint: the transposed Jacobian matches entry by entry
    (model 1: the Kapila K div u term and the Wood sound speed; riemann 1:
    HLL; low_mach 1, 2: Thornber, anti-dissipation pressure correction)."""
    case, W = smooth_case(dims, bc_lo, bc_hi)
    case.model, case.riemann, case.low_mach = model, riemann, low_mach
    P = oracle_problem(oracle_lib, case)
    S = solver_for(mfc_lib, case)
    q = oracle_lib.prim_to_cons(P, W)
    J, JT = full_jacobians(oracle_lib, S, P, q)
    assert np.abs(JT - J).max() <= 1e-12 * np.abs(J).max()


@pytest.mark.parametrize("weno", [0, 1])
@pytest.mark.parametrize("dims,bc_lo,bc_hi", [((17,), (2,), (2,)), ((19,), (0,), (0,)), ((6, 5), (0, 2), (0, 1))])
def test_rhs_full_jacobian_df64(oracle_lib, mfc_lib, cuda_device, dims, bc_lo, bc_hi, weno):
    """The double-float adjoint (reverse WENO5 in double-float arithmetic,
    48-bit significand) against the oracle's dual numbers, entry by entry:
    within 1e-10 of the Jacobian's largest entry."""
    case, W = smooth_case(dims, bc_lo, bc_hi)
    case.weno, case.eps = weno, (1e-6 if weno == 0 else 1e-40)
    P = oracle_problem(oracle_lib, case)
    S = solver_for(mfc_lib, case, precision=mfc_lib.MFC_DF64)
    q = oracle_lib.prim_to_cons(P, W)
    J, JT = full_jacobians(oracle_lib, S, P, q)
    assert np.abs(JT - J).max() <= 1e-10 * np.abs(J).max()


@pytest.mark.parametrize("weno", [0, 1, 2])
@pytest.mark.parametrize("dims,bc_lo,bc_hi", [((17,), (2,), (2,)), ((19,), (0,), (0,)), ((6, 5), (0, 2), (0, 1)),
                                              ((5, 4, 3), (1, 0, 2), (2, 0, 1))])
def test_rhs_full_jacobian_fast(oracle_lib, mfc_lib, cuda_device, dims, bc_lo, bc_hi, weno):
    """The MFC_FP64_FAST adjoint (the reverse WENO5 on consecutive
    differences, one reciprocal per normalisation; Jiang-Shu, mapped and Z
    weights) against the oracle's dual numbers, entry by entry: within 1e-11
    of the Jacobian's largest entry (measured on GB300: at most 3.3e-13, the
    Jiang-Shu weights in 1D)."""
    case, W = smooth_case(dims, bc_lo, bc_hi)
    case.weno, case.eps = weno, (1e-6 if weno == 0 else 1e-40)
    P = oracle_problem(oracle_lib, case)
    S = solver_for(mfc_lib, case, precision=mfc_lib.MFC_FP64_FAST)
    q = oracle_lib.prim_to_cons(P, W)
    J, JT = full_jacobians(oracle_lib, S, P, q)
    assert np.abs(JT - J).max() <= 1e-11 * np.abs(J).max()


@pytest.mark.parametrize("weno", [0, 1, 2])
@pytest.mark.parametrize("dims,bc_lo,bc_hi", [((17,), (2,), (2,)), ((19,), (0,), (0,)), ((6, 5), (0, 2), (0, 1)),
                                              ((5, 4, 3), (1, 0, 2), (2, 0, 1))])
def test_rhs_full_jacobian_mixed(oracle_lib, mfc_lib, cuda_device, dims, bc_lo, bc_hi, weno):
    """The MFC_MIXED adjoint (float32 reverse WENO5 with the edges paired,
    float32 HLLC adjoint, float64 pressure recovery) against the oracle's
    float64 dual numbers, entry by entry.  Measured on GB300: at most
    2.1e-5 of the Jacobian's largest entry over these cases (Z weights in
    2D); the bound is 1e-4."""
    case, W = smooth_case(dims, bc_lo, bc_hi)
    case.weno, case.eps = weno, (1e-6 if weno == 0 else 1e-40)
    P = oracle_problem(oracle_lib, case)
    S = solver_for(mfc_lib, case, precision=mfc_lib.MFC_MIXED)
    q = oracle_lib.prim_to_cons(P, W)
    J, JT = full_jacobians(oracle_lib, S, P, q)
    assert np.abs(JT - J).max() <= 1e-4 * np.abs(J).max()


@pytest.mark.parametrize("name,weno", [("water_air", 1), ("water_air", 0), ("bubble", 1), ("bubble", 0),
                                       ("shock_bubble", 1), ("stiff_smooth", 1), ("stiff_smooth", 0),
                                       ("water_air", 3), ("shock_bubble", 3), ("stiff_smooth", 3)])
def test_rhs_full_jacobian_workload_states(oracle_lib, mfc_lib, cuda_device, name, weno):
    """Entry by entry on tiny versions of the workloads' initial states
    (stiff interfaces, fluid at rest, sharp jumps), MFC_FP64: the same
    branches on both sides; the Jiang-Shu variants in reduced units.  Entries are compared in nondimensional form
    (each row and column scaled by its field's magnitude), against the
    largest entry: the volume-fraction rows of a fluid at rest are exactly
    zero up to rounding on both sides."""
    if name == "water_air":
        (case, W), rho0, p0 = wl.water_air_shock_tube(14), 1000.0, 1e9
    elif name == "bubble":
        (case, W), rho0, p0 = wl.bubble_collapse_2d(dims=(8, 7)), 1000.0, 1e7
    elif name == "stiff_smooth":
        (case, W), rho0, p0 = stiff_smooth_case(dims=(7, 6)), 1.0, 1.0
    else:
        (case, W), rho0, p0 = wl.shock_bubble_3d(dims=(6, 5, 4)), 1.0, 1.0
    if weno == 0:
        case, W = wl.reduced_units(case, W, rho0, p0)
    case.weno, case.eps = weno, (1e-6 if weno == 0 else 1e-40)
    P = oracle_problem(oracle_lib, case)
    S = solver_for(mfc_lib, case)
    q = oracle_lib.prim_to_cons(P, W)
    J, JT = full_jacobians(oracle_lib, S, P, q)
    # nondimensional Jacobian D^-1 J D, D = the field scales of every entry of q
    d = np.repeat(field_scales(case, q), q[0].size)
    Jn = J * d[None, :] / d[:, None]
    JTn = JT * d[None, :] / d[:, None]
    err = np.abs(JTn - Jn) / np.abs(Jn).max()
    ncell = q[0].size
    worst = np.argsort(err.ravel())[::-1][:6]
    report = [(float(err.ravel()[k]), (k // err.shape[1] // ncell, k // err.shape[1] % ncell),
               (k % err.shape[1] // ncell, k % err.shape[1] % ncell),
               float(J.ravel()[k]), float(JT.ravel()[k])) for k in worst]
    assert err.max() <= 1e-12, report


@pytest.mark.parametrize("name", ["smooth_3d_mixed_bc", "smooth_2d_periodic"])
def test_rk3_step_vjp_central_differences(mfc_lib, cuda_device, name):
    """The GPU adjoint against central differences of the GPU's own step."""
    case, W = CASES[name]()
    S = solver_for(mfc_lib, case)
    q = S.prim_to_cons(S.from_interior(W))
    dt = S.compute_dt(q)
    qi = S.interior(q).cpu().numpy()
    w, v = directions(case, qi, 3)
    w = S.from_interior(w)
    v = S.from_interior(v)
    qb = S.rk3_step_vjp(q, dt, v)
    ad = float((S.interior(qb) * S.interior(w)).sum())
    for h in (1e-5, 1e-6, 1e-7):
        qp = q + h * w
        qm = q - h * w
        S.rk3_step(qp, dt)
        S.rk3_step(qm, dt)
        fd = float((S.interior(v) * (S.interior(qp) - S.interior(qm))).sum()) / (2 * h)
        if abs(fd - ad) <= 1e-5 * abs(ad):
            return
    raise AssertionError((ad, fd))


def test_mixed_precision_adjoint_dot_product(oracle_lib, mfc_lib, cuda_device):
    """Float32 reconstruction / Riemann adjoint: same identity at float32 accuracy."""
    case, W = CASES["smooth_3d_mixed_bc"]()
    P = oracle_problem(oracle_lib, case)
    S = solver_for(mfc_lib, case, precision=mfc_lib.MFC_MIXED)
    q = oracle_lib.prim_to_cons(P, W)
    dt = oracle_lib.cfl_dt(P, q, case.cfl)
    w, v = directions(case, q, 9)
    _, Jw = oracle_lib.rk3_step_jvp(P, q, w, dt)
    qb = S.rk3_step_vjp(S.from_interior(q), dt, S.from_interior(v))
    assert dot(to_host(S, qb), w) == pytest.approx(dot(v, Jw), rel=1e-4)


def test_vjp_aliasing_and_arguments(mfc_lib, cuda_device):
    case, W = wl.shock_bubble_3d(dims=(12, 10, 9))
    S = solver_for(mfc_lib, case)
    q = S.prim_to_cons(S.from_interior(W))
    dt = S.compute_dt(q)
    g = S.from_interior(torch.ones(S.interior_shape, dtype=torch.float64))
    ref = S.rk3_step_vjp(q, dt, g)
    g2 = g.clone()
    S.rk3_step_vjp(q, dt, g2, g2)  # qn_bar may alias qnp1_bar
    assert torch.equal(S.interior(ref), S.interior(g2))
    with pytest.raises(mfc_lib.MfcError):
        S.rk3_step_vjp(q, 0.0, g)  # the adjoint needs the step's dt
    with pytest.raises(mfc_lib.MfcError):
        S.rhs_vjp(q, g, q)
