"""Pins of the oracle's viscous stress (Sec. 2.1.1): T = 2 eta (D - tr(D) I/3),
D = (grad u + (grad u)^T)/2, entering the momentum flux as -T and the energy
flux as -T.u, with the mixture viscosity eta = sum_i alpha_i eta_i and
second-order central differences on the faces (readings; the paper prints
neither).

- The face differences are exact on velocity fields of degree two, so the
  viscous right-hand side of such fields has a closed form: 2 eta for
  u = y^2, (8/3) eta for u = x^2 (the bulk -2/3 term), eta/3 for the cross
  terms of u = xy, eta a^2 of viscous heating for Couette flow u = a y.
- A shear wave v = A sin(2 pi x) is an exact solution of the semi-discrete
  scheme that decays at the rate of the discrete Laplacian's eigenvalue,
  eta 2 (1 - cos(2 pi h)) / h^2 (and at second order in h at eta (2 pi)^2).
- The 2D Taylor-Green vortex loses kinetic energy as exp(-4 nu t) over an
  inviscid run's numerical dissipation.
"""
import math

import numpy as np
import pytest

from paper_2503_07953_gb300 import workloads as wl
from tests.helpers import oracle_problem

ETA = 0.3


def poly_case(dims, nf=1, eta=(ETA,), bc=wl.TRANSMISSIVE):
    nd = len(dims)
    return wl.Case("poly", list(dims), [0.0] * nd, [1.0] * nd, [bc] * nd, [bc] * nd,
                   [1.4, 1.67][:nf], [0.0, 0.0][:nf], 0.4, 0, eta=list(eta))


def state(case, vel, rho=2.0, p=1e5, alpha=None):
    one = np.ones(case.shape[1:])
    vel = [v * one for v in vel]
    if case.nf == 1:
        return wl._assemble(case, [one], [rho * one], vel, p * one)
    a = alpha * one
    return wl._assemble(case, [a, 1.0 - a], [rho * one, rho * one], vel, p * one)


def viscous_interior(oracle_lib, case, W, margin=2):
    P = oracle_problem(oracle_lib, case)
    V = oracle_lib.viscous_rhs(P, oracle_lib.prim_to_cons(P, W))
    # array axes (field, z, y, x): trim the active axes (x is axis 0)
    sl = [slice(None)] + [slice(margin, -margin) if a < case.ndim else slice(None) for a in (2, 1, 0)]
    return V[tuple(sl)]


@pytest.mark.parametrize("field,row,want", [
    ("y2", "u", 2.0 * ETA),               # d/dy (eta du/dy)
    ("x2", "u", 8.0 / 3.0 * ETA),         # d/dx (4/3 eta du/dx)
    ("xy_u", "u", 0.0),
    ("xy_v", "v", ETA / 3.0),             # eta d2u/dxdy - 2/3 eta d(div u)/dy
])
def test_quadratic_fields_2d(oracle_lib, field, row, want):
    case = poly_case([12, 12])
    X, Y, _ = wl._centres(case)
    u = {"y2": Y ** 2, "x2": X ** 2, "xy_u": X * Y, "xy_v": X * Y}[field]
    V = viscous_interior(oracle_lib, case, state(case, [u, 0.0 * X]))
    k = case.nf + (0 if row == "u" else 1)
    np.testing.assert_allclose(V[k], want, rtol=0, atol=1e-13)
    other = case.nf + (1 if row == "u" else 0)
    if field in ("y2", "x2"):
        assert np.abs(V[other]).max() < 1e-13


def test_cross_terms_3d(oracle_lib):
    """w = x z: V_u = -2/3 eta d(div u)/dx + eta d2w/dxdz = eta/3, V_v = V_w = 0."""
    case = poly_case([8, 8, 8])
    X, Y, Z = wl._centres(case)
    V = viscous_interior(oracle_lib, case, state(case, [0.0 * X, 0.0 * X, X * Z]))
    np.testing.assert_allclose(V[1], ETA / 3.0, rtol=0, atol=1e-13)
    assert np.abs(V[2]).max() < 1e-13
    assert np.abs(V[3]).max() < 1e-13


def test_couette_heating_and_mixture_viscosity(oracle_lib):
    """u = a y with alpha_1 = c0 + c1 y and eta = alpha_1 eta_1 + alpha_2 eta_2:
    V_u = a c1 (eta_1 - eta_2) and V_E = a^2 d(eta y)/dy (heating), both
    exact; with one fluid V_u = 0 and V_E = eta a^2."""
    a = 3.0
    case = poly_case([12, 12])
    X, Y, _ = wl._centres(case)
    V = viscous_interior(oracle_lib, case, state(case, [a * Y, 0.0 * X]))
    assert np.abs(V[1]).max() < 1e-13
    np.testing.assert_allclose(V[3], ETA * a * a, rtol=1e-13)
    eta1, eta2, c0, c1 = 0.5, 0.1, 0.2, 0.5
    case = poly_case([12, 12], nf=2, eta=(eta1, eta2))
    X, Y, _ = wl._centres(case)
    V = viscous_interior(oracle_lib, case, state(case, [a * Y, 0.0 * X], alpha=c0 + c1 * Y))
    np.testing.assert_allclose(V[2], a * c1 * (eta1 - eta2), rtol=1e-12)
    Yi = Y[:, 2:-2, :]
    want = a * a * (eta2 + (eta1 - eta2) * (c0 + 2.0 * c1 * Yi))
    np.testing.assert_allclose(V[4], np.broadcast_to(want, V[4].shape), rtol=1e-12)
    assert np.abs(V[0]).max() == 0 and np.abs(V[1]).max() == 0 and np.abs(V[5]).max() == 0


def smooth_periodic(nd, n, nf=1, seed=0):
    dims = [n] * nd
    case = wl.Case("smooth", dims, [0.0] * nd, [1.0] * nd, [wl.PERIODIC] * nd, [wl.PERIODIC] * nd,
                   [1.4, 1.67][:nf], [0.0, 0.0][:nf], 0.4, 0, eta=[0.05, 0.01][:nf])
    X, Y, Z = wl._centres(case)
    tp = 2.0 * math.pi
    r = np.random.default_rng(seed).uniform(0.5, 1.0, size=8)
    vel = [r[d] * np.sin(tp * (X + r[3] * Y + r[4] * Z) + d) for d in range(nd)]
    rho = 1.0 + 0.2 * np.cos(tp * (X - Y + Z))
    p = 1.0 + 0.1 * np.sin(tp * (Y + 2 * Z + X))
    one = np.ones(case.shape[1:])
    if nf == 1:
        W = wl._assemble(case, [one], [rho * one], vel, p * one)
    else:
        al = 0.5 + 0.3 * np.sin(tp * (X + Z)) * one
        W = wl._assemble(case, [al, 1.0 - al], [rho * one, rho * one], vel, p * one)
    return case, W


@pytest.mark.parametrize("nd,nf", [(2, 1), (3, 2)])
def test_conservation_periodic(oracle_lib, nd, nf):
    """The viscous flux is in conservation form: on a periodic grid the
    cell sums of the momentum and energy right-hand sides vanish."""
    case, W = smooth_periodic(nd, 10, nf)
    P = oracle_problem(oracle_lib, case)
    V = oracle_lib.viscous_rhs(P, oracle_lib.prim_to_cons(P, W))
    for k in range(nf, nf + nd + 1):
        assert abs(V[k].sum()) <= 1e-12 * np.abs(V[k]).sum(), k


def test_galilean_invariance(oracle_lib):
    """A uniform velocity U leaves the momentum rows unchanged and adds
    U . V_momentum to the energy row (T depends on gradients only)."""
    case, W = smooth_periodic(3, 8, 1)
    P = oracle_problem(oracle_lib, case)
    V0 = oracle_lib.viscous_rhs(P, oracle_lib.prim_to_cons(P, W))
    U = np.array([0.3, -0.2, 0.7])
    W2 = W.copy()
    for d in range(3):
        W2[1 + d] += U[d]
    V1 = oracle_lib.viscous_rhs(P, oracle_lib.prim_to_cons(P, W2))
    scale = np.abs(V0[1:4]).max()
    assert np.abs(V1[1:4] - V0[1:4]).max() < 1e-12 * scale
    want = V0[4] + sum(U[d] * V0[1 + d] for d in range(3))
    assert np.abs(V1[4] - want).max() < 1e-12 * np.abs(V0[4]).max()


def test_reflective_wall_mirror_symmetry(oracle_lib):
    """Mirroring the state about the x extent of a domain with reflective
    walls (normal velocity negated) mirrors the viscous right-hand side, its
    x-momentum row negated."""
    case = poly_case([10, 9], nf=2, eta=(0.2, 0.05), bc=wl.REFLECTIVE)
    X, Y, _ = wl._centres(case)
    W = state(case, [np.sin(3 * X) * Y, np.cos(2 * Y) + X * X], alpha=0.3 + 0.4 * X * Y)
    W[case.nf + case.ndim] = 1e5 + 10 * X
    P = oracle_problem(oracle_lib, case)
    V = oracle_lib.viscous_rhs(P, oracle_lib.prim_to_cons(P, W))
    Wm = W[..., ::-1].copy()
    Wm[case.nf] = -Wm[case.nf]
    Vm = oracle_lib.viscous_rhs(P, oracle_lib.prim_to_cons(P, Wm))[..., ::-1]
    Vm[case.nf] = -Vm[case.nf]
    assert np.abs(Vm - V).max() <= 1e-12 * np.abs(V).max()


def test_inviscid_is_unchanged(oracle_lib):
    """eta = 0 for every fluid is the inviscid method, bit for bit."""
    case, W = smooth_periodic(2, 10, 2)
    P = oracle_problem(oracle_lib, case)
    q = oracle_lib.prim_to_cons(P, W)
    case.eta = [0.0, 0.0]
    L0 = oracle_lib.rhs(oracle_problem(oracle_lib, case), q)
    case.eta = None
    L1 = oracle_lib.rhs(oracle_problem(oracle_lib, case), q)
    assert np.array_equal(L0, L1)
    assert not np.any(oracle_lib.viscous_rhs(oracle_problem(oracle_lib, case), q))


def test_rhs_is_viscous_plus_inviscid(oracle_lib):
    case, W = smooth_periodic(3, 8, 2)
    P = oracle_problem(oracle_lib, case)
    q = oracle_lib.prim_to_cons(P, W)
    L = oracle_lib.rhs(P, q)
    V = oracle_lib.viscous_rhs(P, q)
    eta = case.eta
    case.eta = None
    L0 = oracle_lib.rhs(oracle_problem(oracle_lib, case), q)
    case.eta = eta
    np.testing.assert_allclose(L, V + L0, rtol=0, atol=1e-12 * np.abs(L).max())


@pytest.mark.parametrize("n", [16, 32])
def test_shear_wave_decays_at_the_discrete_laplacian_rate(oracle_lib, n):
    case, W = wl.shear_wave_2d(n)
    P = oracle_problem(oracle_lib, case)
    q = oracle_lib.prim_to_cons(P, W)
    X, Y, _ = wl._centres(case)
    mode = np.sin(2.0 * math.pi * X) + 0.0 * Y

    def amplitude(q):
        return 2.0 * ((q[2] / q[0]) * mode).mean()

    a0 = amplitude(q)
    dt = oracle_lib.cfl_dt(P, q, case.cfl)
    steps = int(round(0.4 / dt))
    q1, dts = oracle_lib.rk3_run(P, q, steps, cfl=case.cfl)
    rate = -math.log(amplitude(q1) / a0) / float(np.sum(dts))
    eta, h = case.eta[0], 1.0 / n
    discrete = eta * 2.0 * (1.0 - math.cos(2.0 * math.pi * h)) / h ** 2
    assert rate == pytest.approx(discrete, rel=1e-8)
    # second order towards the continuous rate eta (2 pi)^2
    err = abs(rate / (eta * (2.0 * math.pi) ** 2) - 1.0)
    assert err < 1.4 * (2.0 * math.pi * h) ** 2 / 12.0
    # the wave neither moves mass nor changes the pressure at first order
    assert np.abs(q1[0] - q[0]).max() < 1e-9


def test_taylor_green_2d_viscous_dissipation(oracle_lib):
    """Kinetic energy of the viscous run over that of the inviscid run
    (which carries the scheme's own dissipation) is exp(-4 nu t), Re 100,
    Ma 0.1, t = 1 (within 1e-3: compressibility and O(h^2))."""
    out = {}
    for viscous in (True, False):
        case, W = wl.taylor_green(32, ndim=2, re=100.0, mach=0.1)
        if not viscous:
            case.eta = None
        P = oracle_problem(oracle_lib, case)
        q = oracle_lib.prim_to_cons(P, W)
        ke = lambda s: 0.5 * ((s[1] ** 2 + s[2] ** 2) / s[0]).sum()
        dt = 1.0 / 140
        q1, _ = oracle_lib.rk3_run(P, q, 140, dts=np.full(140, dt))
        out[viscous] = ke(q1) / ke(q)
    nu = 1.0 / 100.0
    assert out[True] / out[False] == pytest.approx(math.exp(-4.0 * nu * 1.0), rel=1e-3)


def test_sampled_step_matches_full_step(oracle_lib):
    """The sampled RK3 step reaches the viscous stencil's edge neighbours."""
    case, W = smooth_periodic(3, 8, 2)
    P = oracle_problem(oracle_lib, case)
    q = oracle_lib.prim_to_cons(P, W)
    dt = oracle_lib.cfl_dt(P, q, 0.4)
    full = oracle_lib.rk3_step(P, q, dt)
    cells = np.array([[0, 0, 0], [7, 3, 5], [4, 7, 0]], dtype=np.int64)
    got = oracle_lib.rk3_step_sampled(P, q, dt, cells)
    for s, (i, j, k) in enumerate(cells):
        assert np.array_equal(got[s], full[:, k, j, i]), s


def test_jvp_through_the_viscous_term(oracle_lib):
    """Forward-mode derivatives of L with viscosity against central
    differences of the oracle itself.  Jiang-Shu weights (eps 1e-6): with
    WENO-M's eps = 1e-40 the weights of a smooth 8-cell field have
    derivatives of order 1/beta that no finite step resolves, viscous or
    not."""
    case, W = smooth_periodic(2, 8, 2)
    case.weno, case.eps = wl.WENO_JS, 1e-6
    P = oracle_problem(oracle_lib, case)
    q = oracle_lib.prim_to_cons(P, W)
    dq = np.random.default_rng(3).standard_normal(q.shape) * np.abs(q).max(axis=(1, 2, 3), keepdims=True) * 1e-3
    _, dL = oracle_lib.rhs_jvp(P, q, dq)
    h = 1e-4
    fd = (oracle_lib.rhs(P, q + h * dq) - oracle_lib.rhs(P, q - h * dq)) / (2 * h)
    assert np.abs(dL - fd).max() <= 1e-6 * np.abs(fd).max()
