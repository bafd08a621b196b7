"""The opt-in explicit viscous time-step limit of the oracle's CFL dt
(reading: the paper states no viscous bound; the usual limit of an explicit
step of the momentum diffusion), dt = CFL min over cells of
min(min_d dx_d / (|u_d| + c), rho min_d dx_d^2 / (2 ndim eta)), pinned by
closed forms on uniform states: the viscous bound binds exactly when it is
the smaller, with the mixture viscosity of the cell's volume fractions."""
import math

import numpy as np
import pytest

from paper_2503_07953_gb300 import workloads as wl
from tests.helpers import oracle_problem


def uniform_case(eta, alpha1, ndim=2, n=(8, 6), viscous_dt=1):
    case = wl.Case("uniform", list(n[:ndim]), [0.0] * ndim, [1.0, 0.75][:ndim], [0] * ndim, [0] * ndim,
                   [1.4, 1.6], [0.0, 0.0], cfl=0.5, steps=0, eta=list(eta), viscous_dt=viscous_dt)
    rho = (2.0, 3.0)
    shp = case.shape[1:]
    W = np.zeros(case.shape)
    W[0] = alpha1 * rho[0]
    W[1] = (1.0 - alpha1) * rho[1]
    W[case.nf + ndim] = 5.0          # p; fluid at rest
    W[case.nf + ndim + 1] = alpha1
    return case, W, rho


@pytest.mark.parametrize("eta, alpha1", [((0.5, 0.5), 0.3), ((2.0, 0.0), 0.25), ((0.0, 1.0), 0.6)])
def test_viscous_bound_closed_form(oracle_lib, eta, alpha1):
    case, W, rho = uniform_case(eta, alpha1)
    P = oracle_problem(oracle_lib, case)
    q = oracle_lib.prim_to_cons(P, W)
    rho_m = alpha1 * rho[0] + (1 - alpha1) * rho[1]
    eta_m = alpha1 * eta[0] + (1 - alpha1) * eta[1]
    dxmin = min(case.dx(a) for a in range(case.ndim))
    # convective: the mixture stiffened-gas sound speed, fluid at rest
    G = alpha1 / 0.4 + (1 - alpha1) / 0.6
    c = math.sqrt((G + 1.0) * 5.0 / (G * rho_m))
    conv = dxmin / c
    visc = rho_m * dxmin ** 2 / (2 * case.ndim * eta_m)
    dt = oracle_lib.cfl_dt(P, q, case.cfl)
    assert dt == pytest.approx(case.cfl * min(conv, visc), rel=1e-14)
    assert visc < conv  # these viscosities make the viscous bound the binding one
    # without the option the convective dt alone
    case.viscous_dt = 0
    dt0 = oracle_lib.cfl_dt(oracle_problem(oracle_lib, case), q, case.cfl)
    assert dt0 == pytest.approx(case.cfl * conv, rel=1e-14)


def test_inviscid_fluid_has_no_viscous_bound(oracle_lib):
    """A cell of the inviscid fluid alone (eta = 0 there) keeps the
    convective dt even with the option."""
    case, W, rho = uniform_case((0.0, 3.0), 1.0)
    P = oracle_problem(oracle_lib, case)
    q = oracle_lib.prim_to_cons(P, W)
    case.viscous_dt = 0
    assert oracle_lib.cfl_dt(P, q, case.cfl) == oracle_lib.cfl_dt(oracle_problem(oracle_lib, case), q, case.cfl)
