"""Invariants, closed forms and brute-force checks that pin the oracle."""
import math

import numpy as np
import pytest

from paper_2503_07953_gb300 import workloads as wl


def problem(oracle_lib, case, **kw):
    return oracle_lib.Problem(n=case.n, gamma=case.gamma, pi_inf=case.pi_inf, lo=case.lo, hi=case.hi,
                              bc_lo=case.bc_lo, bc_hi=case.bc_hi, **kw)


def test_rk3_tableau_is_third_order_taylor(oracle_lib):
    """I5: on y' = lambda y one step equals 1 + z + z^2/2 + z^3/6 (Sec. 3.4)."""
    for lam in (-1.0, 0.5, -3.0, 2.0):
        for dt in (0.1, 0.01, 0.37):
            z = lam * dt
            assert oracle_lib.rk3_linear(lam, 1.0, dt) == pytest.approx(1 + z + z * z / 2 + z ** 3 / 6,
                                                                        rel=1e-14)


def test_prim_cons_roundtrip(oracle_lib):
    case, W = wl.random_interfaces_3d(dims=(6, 5, 4))
    P = problem(oracle_lib, case)
    q = oracle_lib.prim_to_cons(P, W)
    W2 = oracle_lib.cons_to_prim(P, q)
    nf, nd = case.nf, case.ndim
    for k in range(case.nq):
        if k == nf + nd:
            # p = (rho E - KE - Pi)/Gamma cancels Pi ~ 2e9 against p ~ 1e5:
            # the bound is a few ulps of rho E, divided by Gamma
            tol = 1e-15 * np.abs(q[k]).max() / (1.0 / (6.1 - 1.0))
        else:
            tol = 1e-14 * max(1.0, np.abs(W[k]).max())
        assert np.abs(W2[k] - W[k]).max() <= tol
    q2 = oracle_lib.prim_to_cons(P, W2)
    for k in range(case.nq):
        assert np.abs(q2[k] - q[k]).max() <= 1e-14 * np.abs(q[k]).max()


@pytest.mark.parametrize("riemann,low_mach", [(0, 0), (1, 0), (0, 1), (0, 2), (1, 1)])
def test_hllc_equal_states_give_physical_flux(oracle_lib, riemann, low_mach):
    """Brute force: one face with L = R returns the exact Euler flux, for
    HLLC and HLL, with and without the low-Mach corrections (which vanish
    for equal states: u_L = u_R, p_d = 0)."""
    case = wl.Case("f", [4, 4, 4], [0] * 3, [1] * 3, [1] * 3, [1] * 3, [1.4, 4.4], [0.0, 6e8], 0.4, 0)
    P = problem(oracle_lib, case, riemann=riemann, low_mach=low_mach)
    g = np.array([1.4, 4.4]); pi = np.array([0.0, 6e8])
    rng = np.random.default_rng(0)
    for _ in range(20):
        a1 = rng.uniform(0.1, 0.9); rho = rng.uniform(1, 1000, 2)
        u = rng.normal(size=3) * 50; p = rng.uniform(1e5, 1e7)
        w = np.array([a1 * rho[0], (1 - a1) * rho[1], *u, p, a1])
        for d in range(3):
            F, uf, bad = oracle_lib.hllc_face(P, d, w, w)
            assert bad == 0
            r = a1 * rho[0] + (1 - a1) * rho[1]
            al = np.array([a1, 1 - a1])
            E = (al / (g - 1)).sum() * p + (al * g * pi / (g - 1)).sum() + 0.5 * r * (u @ u)
            expect = np.array([a1 * rho[0] * u[d], (1 - a1) * rho[1] * u[d],
                               *(r * u[d] * u + p * np.eye(3)[d]), (E + p) * u[d], a1 * u[d]])
            # F*_K = F_K + S_K (U*_K - U_K) rounds at the level of |S_K| |U_K|
            Gm = (al / (g - 1)).sum(); Pm = (al * g * pi / (g - 1)).sum()
            c = math.sqrt(((Gm + 1) * p + Pm) / (Gm * r))
            scale = (c + np.abs(u).max()) * max(E, r * np.abs(u).max(), rho.max())
            np.testing.assert_allclose(F, expect, rtol=1e-14, atol=1e-14 * scale)
            assert uf == pytest.approx(u[d], rel=1e-14)


def test_hllc_wall_face_has_no_mass_flux(oracle_lib):
    """A mirror state (reflective wall) gives S* = 0: no mass / alpha flux."""
    case = wl.Case("f", [4, 4], [0] * 2, [1] * 2, [1] * 2, [1] * 2, [1.4, 1.67], [0.0, 0.0], 0.4, 0)
    P = problem(oracle_lib, case)
    rng = np.random.default_rng(3)
    for _ in range(20):
        wl_ = np.array([rng.uniform(0.1, 1), rng.uniform(0.1, 1), rng.normal(), rng.normal(),
                        rng.uniform(0.5, 2), rng.uniform(0, 1)])
        for d in range(2):
            wr = wl_.copy(); wr[2 + d] = -wr[2 + d]
            F, uf, bad = oracle_lib.hllc_face(P, d, wl_, wr)
            assert uf == 0.0
            # mass and alpha fluxes vanish up to the rounding of S_L (U* - U_L)
            tol = 1e-15 * 8.0 * (abs(wl_[2 + d]) + 3.0)
            assert abs(F[0]) <= tol and abs(F[1]) <= tol and F[5] == 0.0


def test_sampled_step_equals_full_step_bitwise(oracle_lib):
    """The domain-of-dependence evaluation reproduces the full step exactly,
    including cells next to periodic, reflective and transmissive edges."""
    case = wl.Case("s", [9, 8, 7], [0] * 3, [1.0, 0.8, 0.7], [0, 2, 1], [0, 2, 2], [1.4, 1.67],
                   [0.0, 0.0], 0.4, 0)
    W = wl.random_smooth_state(case, seed=5, amp=0.1)
    P = problem(oracle_lib, case)
    q = oracle_lib.prim_to_cons(P, W)
    dt = oracle_lib.cfl_dt(P, q, 0.4)
    full = oracle_lib.rk3_step(P, q, dt)
    cells = [(0, 0, 0), (8, 7, 6), (4, 0, 3), (0, 4, 6), (8, 3, 0), (2, 6, 5)]
    out = oracle_lib.rk3_step_sampled(P, q, dt, cells)
    for n, (i, j, k) in enumerate(cells):
        assert np.array_equal(out[n], full[:, k, j, i])


def test_conservation_periodic(oracle_lib):
    """I1: partial masses, momenta and energy are conserved to round-off on a
    periodic grid (the flux form telescopes, Eq. (rhs)); alpha is not."""
    case = wl.Case("c", [16, 12], [0, 0], [1.0, 0.75], [0, 0], [0, 0], [1.4, 4.4], [0.0, 1e3], 0.4, 0)
    W = wl.random_smooth_state(case, seed=1, amp=0.2)
    P = problem(oracle_lib, case)
    q0 = oracle_lib.prim_to_cons(P, W)
    q, dts = oracle_lib.rk3_run(P, q0, 40, cfl=0.4)
    for k in range(case.nq - (case.nf - 1)):
        s0, s1 = q0[k].sum(), q[k].sum()
        scale = np.abs(q0[k]).sum()
        assert abs(s1 - s0) <= 1e-13 * scale, (k, s0, s1)
    assert abs(q[-1].sum() - q0[-1].sum()) > 1e-10 * np.abs(q0[-1]).sum()


def test_volume_fraction_does_not_leak_with_identical_eos(oracle_lib):
    """I2: with identical (gamma, pi_inf) for every fluid, Gamma and Pi do not
    depend on alpha, so changing only the alpha field leaves the partial
    densities, momentum and energy trajectories bitwise unchanged."""
    # gamma = 2, pi = 0.5 make both mixture coefficients exactly 1, so
    # (1 - alpha) * 1 + alpha * 1 rounds to exactly 1 for every alpha
    case = wl.Case("i2", [14, 10], [0, 0], [1, 1], [0, 1], [0, 2], [2.0, 2.0], [0.5, 0.5], 0.4, 0)
    W = wl.random_smooth_state(case, seed=2, amp=0.2)
    P = problem(oracle_lib, case)
    qa = oracle_lib.prim_to_cons(P, W)
    qb = qa.copy()
    # a different, smooth alpha field that stays inside (0, 1) (outside it,
    # 1 - alpha rounds and the mixture coefficients stop being exactly 1)
    x = (np.arange(14) + 0.5) / 14
    qb[-1] = 0.5 + 0.2 * np.sin(2 * np.pi * x)[None, None, :]
    dts = np.full(25, 0.2 * oracle_lib.cfl_dt(P, qa, 0.4))
    ra, _ = oracle_lib.rk3_run(P, qa, 25, dts=dts)
    rb, _ = oracle_lib.rk3_run(P, qb, 25, dts=dts)
    assert np.array_equal(ra[:-1], rb[:-1])
    assert not np.array_equal(ra[-1], rb[-1])


@pytest.mark.parametrize("name,gamma,pi,rho,p,u,tol", [
    ("air_helium", [1.4, 1.67], [0.0, 0.0], [1.0, 0.138], 1.0, 3.0, 1e-12),
    ("water_air", [4.4, 1.4], [6e8, 0.0], [1000.0, 1.0], 1e5, 300.0, 1e-8),
])
@pytest.mark.parametrize("smear", [None, 1.0])
@pytest.mark.parametrize("riemann", [0, 1])
def test_interface_equilibrium(oracle_lib, name, gamma, pi, rho, p, u, tol, smear, riemann):
    """I3: a material interface advected at uniform u and p keeps u and p
    uniform (primitive reconstruction with alpha_f u_f + alpha div u), with
    HLLC and with HLL (whose alpha face velocity is the HLL average of u).
    The stiff case loses digits in p = (rho E - 1/2 rho u^2 - Pi)/Gamma
    because Pi ~ 1e9 against p = 1e5."""
    case, W = wl.interface_advection([64], gamma, pi, rho, [u], p, smear=smear)
    P = problem(oracle_lib, case, riemann=riemann)
    q0 = oracle_lib.prim_to_cons(P, W)
    q, dts, bad = oracle_lib.rk3_run(P, q0, 100, cfl=0.4, return_bad=True)
    assert bad == 0
    w = oracle_lib.cons_to_prim(P, q)
    assert np.abs(w[2] / u - 1.0).max() < tol
    assert np.abs(w[3] / p - 1.0).max() < tol
    # the interface did move
    assert np.abs(q[-1] - q0[-1]).max() > 0.1


def test_interface_equilibrium_2d_oblique(oracle_lib):
    case, W = wl.interface_advection([24, 20], [1.4, 1.67], [0.0, 0.0], [1.0, 0.138], [1.0, -0.7], 1.0,
                                     smear=1.0)
    P = problem(oracle_lib, case)
    q, _ = oracle_lib.rk3_run(P, oracle_lib.prim_to_cons(P, W), 30, cfl=0.4)
    w = oracle_lib.cons_to_prim(P, q)
    assert np.abs(w[2] - 1.0).max() < 1e-12
    assert np.abs(w[3] + 0.7).max() < 1e-12
    assert np.abs(w[4] - 1.0).max() < 1e-12


def test_mirror_symmetry_x(oracle_lib):
    """I4: reversing x and negating u_x commutes with a step."""
    case = wl.Case("m", [17, 6], [0, 0], [1, 0.5], [1, 2], [1, 2], [1.4, 4.4], [0.0, 1e2], 0.4, 0)
    W = wl.random_smooth_state(case, seed=7, amp=0.2)
    P = problem(oracle_lib, case)
    q = oracle_lib.prim_to_cons(P, W)
    dt = oracle_lib.cfl_dt(P, q, 0.4)
    a = oracle_lib.rk3_step(P, q, dt)
    qm = q[:, :, :, ::-1].copy(); qm[case.nf] *= -1
    b = oracle_lib.rk3_step(P, qm, dt)[:, :, :, ::-1]
    b = b.copy(); b[case.nf] *= -1
    for k in range(case.nq):
        assert np.abs(a[k] - b[k]).max() <= 1e-13 * np.abs(a[k]).max() + 1e-300


def test_axis_permutation_3d(oracle_lib):
    """I4: permuting the axes of a 3D state permutes the result."""
    case = wl.Case("p", [7, 8, 9], [0] * 3, [0.7, 0.8, 0.9], [0, 1, 2], [0, 1, 2], [1.4, 1.6], [0, 0], 0.4, 0)
    W = wl.random_smooth_state(case, seed=3, amp=0.2)
    P = problem(oracle_lib, case)
    q = oracle_lib.prim_to_cons(P, W)
    dt = oracle_lib.cfl_dt(P, q, 0.4)
    a = oracle_lib.rk3_step(P, q, dt)
    # (x, y, z) -> (y, z, x): new x = old y, new y = old z, new z = old x
    case2 = wl.Case("p2", [8, 9, 7], [0] * 3, [0.8, 0.9, 0.7], [1, 2, 0], [1, 2, 0], [1.4, 1.6], [0, 0], 0.4, 0)
    P2 = problem(oracle_lib, case2)
    nf = case.nf
    def perm(arr):  # arr[field, z, y, x] -> new[field, Z=x, Y=z, X=y]
        out = np.transpose(arr, (0, 3, 1, 2)).copy()
        m = out[nf:nf + 3].copy()
        out[nf], out[nf + 1], out[nf + 2] = m[1], m[2], m[0]
        return out
    b = oracle_lib.rk3_step(P2, perm(q), dt)
    pa = perm(a)
    for k in range(case.nq):
        assert np.abs(pa[k] - b[k]).max() <= 1e-13 * np.abs(pa[k]).max()


@pytest.mark.parametrize("name", ["water_air", "bubble_collapse", "stiff_smooth"])
def test_change_of_units(oracle_lib, name):
    """Dimensional homogeneity (Sec. 2.1.1 with the stiffened-gas closure):
    dividing densities by rho0, pressures and pi_inf by p0 and velocities by
    u0 = sqrt(p0 / rho0) divides each right-hand side by its field's unit
    times u0 (unit length), and the CFL step is multiplied by u0.  A term with
    the wrong power of rho, u or p (a dropped density, u where u^2 belongs,
    sqrt(rho) for rho in the sound speed) breaks it; dimensionless factors
    are pinned elsewhere.  The mapped weights with eps = 1e-40 are
    unit-free wherever beta is above rounding size; on flat stencils the
    candidates agree to rounding, so the edge values do too."""
    if name == "water_air":
        case, W = wl.water_air_shock_tube(60); rho0, p0 = 1000.0, 1e9
    elif name == "bubble_collapse":
        case, W = wl.bubble_collapse_2d(dims=(24, 22)); rho0, p0 = 1000.0, 1e7
    else:
        case = wl.Case("s", [13, 11], [0, 0], [1.0, 0.9], [0, 2], [0, 1], [4.4, 1.4], [6e8, 0.0], 0.4, 0)
        W = wl.random_smooth_state(case, seed=4, amp=0.15)
        W[0] *= 1000.0; W[1] *= 50.0; W[2:4] *= 300.0; W[4] *= 1e9
        rho0, p0 = 997.0, 3.1e8
    case2, W2 = wl.reduced_units(case, W, rho0, p0)
    P, P2 = problem(oracle_lib, case), problem(oracle_lib, case2)
    q, q2 = oracle_lib.prim_to_cons(P, W), oracle_lib.prim_to_cons(P2, W2)
    L, L2 = oracle_lib.rhs(P, q), oracle_lib.rhs(P2, q2)
    u0 = math.sqrt(p0 / rho0)
    nf, nd = case.nf, case.ndim
    unit = np.array([rho0] * nf + [rho0 * u0] * nd + [p0] + [1.0] * (nf - 1))
    for k in range(case.nq):
        scale = np.abs(L[k]).max()
        assert np.abs(L2[k] * unit[k] * u0 - L[k]).max() <= 1e-11 * scale, k
    assert oracle_lib.cfl_dt(P2, q2, 0.4) == pytest.approx(oracle_lib.cfl_dt(P, q, 0.4) * u0, rel=1e-13)


def test_cfl_dt_closed_form(oracle_lib):
    """Uniform single-fluid state: dt = CFL dx / (|u| + c), c^2 = gamma p / rho."""
    case = wl.Case("d", [10, 5], [0, 0], [2.0, 0.5], [1, 1], [1, 1], [1.4], [0.0], 0.4, 0)
    W = np.empty(case.shape)
    W[0] = 1.3; W[1] = 2.0; W[2] = -0.5; W[3] = 0.9
    P = problem(oracle_lib, case)
    q = oracle_lib.prim_to_cons(P, W)
    c = math.sqrt(1.4 * 0.9 / 1.3)
    expect = 0.4 * min(0.2 / (2.0 + c), 0.1 / (0.5 + c))
    assert oracle_lib.cfl_dt(P, q, 0.4) == pytest.approx(expect, rel=1e-14)


def test_jvp_matches_central_differences(oracle_lib):
    case = wl.Case("j", [10, 7], [0, 0], [1, 0.7], [0, 2], [0, 1], [1.4, 4.4], [0.0, 10.0], 0.4, 0)
    W = wl.random_smooth_state(case, seed=4, amp=0.15)
    P = problem(oracle_lib, case)
    q = oracle_lib.prim_to_cons(P, W)
    dt = oracle_lib.cfl_dt(P, q, 0.4)
    rng = np.random.default_rng(0)
    dq = rng.normal(size=q.shape) * np.abs(q).max(axis=(1, 2, 3), keepdims=True)
    _, jv = oracle_lib.rk3_step_jvp(P, q, dq, dt)
    h = 1e-6
    fd = (oracle_lib.rk3_step(P, q + h * dq, dt) - oracle_lib.rk3_step(P, q - h * dq, dt)) / (2 * h)
    assert np.abs(jv - fd).max() <= 1e-6 * np.abs(jv).max()


def test_nonphysical_state_is_reported(oracle_lib):
    case = wl.Case("n", [8], [0], [1], [1], [1], [1.4, 1.4], [0, 0], 0.4, 0)
    W = np.empty(case.shape)
    W[0] = 0.5; W[1] = 0.5; W[2] = 0.0; W[3] = 1.0; W[4] = 0.5
    P = problem(oracle_lib, case)
    q = oracle_lib.prim_to_cons(P, W)
    q[3, 0, 0, 4] = -5.0  # negative energy -> negative pressure
    _, bad = oracle_lib.rhs(P, q, return_bad=True)
    assert bad > 0


def test_bad_problem_rejected(oracle_lib):
    case = wl.Case("b", [2], [0], [1], [0], [0], [1.4], [0.0], 0.4, 0)  # periodic needs >= 3 cells
    P = problem(oracle_lib, case)
    with pytest.raises(ValueError):
        oracle_lib.rhs(P, np.ones(case.shape))
    P2 = oracle_lib.Problem(n=[8], gamma=[1.0], pi_inf=[0.0])  # gamma must exceed 1
    with pytest.raises(ValueError):
        oracle_lib.rhs(P2, np.ones((3, 1, 1, 8)))
