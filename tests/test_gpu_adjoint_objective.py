"""The wall-impulse objective's own arithmetic against the library.

The objective of the bubble-collapse adjoint (adjoint.wall_pressure_objective)
differentiates the pressure with torch, so adjoint.py restates the pressure
recovery of the stiffened-gas mixture (mixture_pressure) and the map from the
first volume fraction to the conservative state (alpha_to_state) in torch
operations.  Both must be the library's maps up to rounding: the pressure
against mfc_cons_to_prim, the state against mfc_prim_to_cons, on the
workloads' own states (two- and three-fluid, stiff water at 1e7 Pa, where
p = (rho E - Pi - ke)/Gamma cancels Pi ~ 8e8 against rho E)."""
import numpy as np
import pytest
import torch

from paper_2503_07953_gb300 import adjoint
from paper_2503_07953_gb300 import workloads as wl
from tests.helpers import solver_for

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("make", [
    lambda: wl.bubble_collapse_2d(dims=(48, 40)),
    lambda: wl.water_air_shock_tube(300),
    lambda: wl.shock_bubble_3d(dims=(20, 16, 12)),
    lambda: wl.random_interfaces_window(dims=(12, 10, 8)),
])
def test_mixture_pressure_matches_cons_to_prim(mfc_lib, cuda_device, make):
    case, W = make()
    S = solver_for(mfc_lib, case)
    q = S.prim_to_cons(S.from_interior(W))
    p_lib = S.interior(S.cons_to_prim(q))[case.nf + case.ndim]
    p_obj = S.interior(adjoint.mixture_pressure(S, q, case.gamma, case.pi_inf).unsqueeze(0))[0]
    scale = p_lib.abs().max().item()
    err = (p_obj - p_lib).abs().max().item() / scale
    # Pi / p up to ~80 for water at 1e7 Pa: the cancellation magnifies the
    # rounding of either evaluation by as much
    assert err <= 1e-13, err
    S.check()


@pytest.mark.parametrize("make", [
    lambda: wl.bubble_collapse_2d(dims=(48, 40)),
    lambda: wl.water_air_shock_tube(300),
])
def test_alpha_to_state_matches_prim_to_cons(mfc_lib, cuda_device, make):
    case, W = make()
    S = solver_for(mfc_lib, case)
    q_lib = S.interior(S.prim_to_cons(S.from_interior(W)))
    a1 = torch.as_tensor(W[case.nf + case.ndim + 1], dtype=torch.float64, device=cuda_device)
    q_obj = S.interior(adjoint.alpha_to_state(S, case, W, a1))
    for k in range(case.nq):
        scale = max(q_lib[k].abs().max().item(), 1e-300)
        err = (q_obj[k] - q_lib[k]).abs().max().item() / scale
        assert err <= 1e-14, (k, err)
