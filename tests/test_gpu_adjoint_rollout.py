"""Gradients of multi-step objectives through the CUDA adjoint: the
autograd wrapper, binomial checkpointing, and central finite differences
of the 2D bubble-collapse wall-pressure impulse with respect to the initial
volume fraction (a small grid of the workload)."""
import numpy as np
import pytest
import torch

from paper_2503_07953_gb300 import adjoint as adj
from paper_2503_07953_gb300 import workloads as wl
from tests.helpers import oracle_problem, solver_for, to_host

pytestmark = pytest.mark.gpu


def setup(mfc_lib, dims=(40, 36), precision=0):
    case, W = wl.bubble_collapse_2d(dims=dims)
    S = solver_for(mfc_lib, case, precision=precision)
    a1 = torch.as_tensor(W[case.nf + case.ndim + 1].copy(), dtype=torch.float64, device="cuda")
    return case, W, S, a1


def test_autograd_step_matches_vjp(mfc_lib, cuda_device):
    case, W, S, a1 = setup(mfc_lib)
    q0 = adj.alpha_to_state(S, case, W, a1).detach()
    dt = S.compute_dt(q0)
    q = q0.clone().requires_grad_(True)
    out = adj.rk3_step(q, S, dt)
    g = torch.randn(S.shape, dtype=torch.float64, device=cuda_device, generator=torch.Generator("cuda").manual_seed(0))
    g = S.from_interior(S.interior(g))
    (out * g).sum().backward()
    ref = S.rk3_step_vjp(q0, dt, g)
    assert torch.equal(q.grad, ref)
    step = q0.clone()
    S.rk3_step(step, dt)
    assert torch.equal(out.detach(), step)


def test_checkpointed_gradient_equals_store_all(mfc_lib, cuda_device):
    case, W, S, a1 = setup(mfc_lib)
    q0 = adj.alpha_to_state(S, case, W, a1).detach()
    nsteps = 24
    _, _, dts, _ = adj.rollout_gradient(S, q0, nsteps, lambda n, q: q.sum() * 0.0, 1)
    loss = adj.wall_pressure_objective(S, case, dts)
    J1, g1, _, st1 = adj.rollout_gradient(S, q0, nsteps, loss, 3, dts)
    J2, g2, _, st2 = adj.rollout_gradient(S, q0, nsteps, loss, nsteps - 1, dts)
    assert J1 == J2
    assert torch.equal(g1, g2)  # recomputed states are bit-identical
    assert st1.max_live_snapshots <= 3 and st1.advances > st2.advances


def wall_impulse_setup(mfc_lib, precision):
    """32x32 bubble collapse, 100 steps (the collapse's pressure waves reach
    the x = 1 wall), the dt sequence of the forward run held fixed, and the
    adjoint gradient dJ/d alpha_1(t=0) through the initial-condition map."""
    case, W, S, a1 = setup(mfc_lib, dims=(32, 32), precision=precision)
    nsteps = 100
    q0 = adj.alpha_to_state(S, case, W, a1).detach()
    _, _, dts, _ = adj.rollout_gradient(S, q0, nsteps, lambda n, q: q.sum() * 0.0, 1)
    loss = adj.wall_pressure_objective(S, case, dts)
    J, gq, _, _ = adj.rollout_gradient(S, q0, nsteps, loss, 6, dts)
    a = a1.clone().requires_grad_(True)
    (adj.alpha_to_state(S, case, W, a) * gq).sum().backward()
    return case, W, S, a1, dts, loss, a.grad


def seeded_directions(a1, count=4):
    """Seeded directions supported where 1e-3 < alpha_1 < 1 - 1e-3, max-normalised."""
    band = ((a1 > 1e-3) & (a1 < 1 - 1e-3)).double()
    gen = torch.Generator(device="cpu").manual_seed(0)
    for _ in range(count):
        d = torch.randn(a1.shape, generator=gen, dtype=torch.float64).to(a1.device) * band
        yield d / float(d.abs().max())


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-3)])
def test_wall_impulse_gradient_matches_oracle_forward_mode(oracle_lib, mfc_lib, cuda_device, precision, tol):
    """The checkpointed reverse sweep against the oracle's forward-mode
    derivative of the same 100 steps at the same dts.  MFC_FP64: two
    evaluation orders of one derivative of one floating-point map.
    MFC_MIXED: the float32 reconstruction and Riemann solve perturb the
    gradient by ~1e-5 relative (measured)."""
    case, W, S, a1, dts, loss, ga = wall_impulse_setup(mfc_lib, precision)
    P = oracle_problem(oracle_lib, case)
    for d in seeded_directions(a1):
        q0, dq0 = torch.func.jvp(lambda x: adj.alpha_to_state(S, case, W, x), (a1,), (d,))
        q, dq = to_host(S, q0), to_host(S, dq0)
        fwd = 0.0
        for n in range(len(dts)):
            q, dq = oracle_lib.rk3_step_jvp(P, q, dq, dts[n])
            fwd += float(torch.func.jvp(lambda x: loss(n, x), (S.from_interior(q),), (S.from_interior(dq),))[1])
        ad = float((ga * d).sum())
        assert ad == pytest.approx(fwd, rel=tol), (ad, fwd)


@pytest.mark.parametrize("precision,tol,h", [(0, 1e-5, 1e-6), (1, 5e-2, 1e-3)])
def test_wall_impulse_gradient_central_differences(mfc_lib, cuda_device, precision, tol, h):
    """Central differences of J along four seeded directions.  The map is
    only piecewise smooth (weight and HLLC switches), so the float64
    difference needs a small step: on this problem the oracle's own
    differences reach its forward-mode derivative to ~5e-4 at h = 1e-5 and
    ~2e-6 at h = 1e-6.  The float32 path needs a step large enough for the
    difference to rise above its rounding, where the truncation error of
    this non-smooth map is itself ~1e-2 (the oracle's float64 differences
    at h = 1e-3 miss by up to 2.4e-2), so it is a coarse check; the mixed
    gradient is held to 1e-3 against the oracle's forward mode above."""
    case, W, S, a1, dts, loss, ga = wall_impulse_setup(mfc_lib, precision)

    def J_of(alpha):
        q = adj.alpha_to_state(S, case, W, alpha).detach()
        tot = 0.0
        for n in range(len(dts)):
            S.rk3_step(q, dts[n])
            tot += float(loss(n, q))
        return tot

    for k, d in enumerate(seeded_directions(a1)):
        fd = (J_of(a1 + h * d) - J_of(a1 - h * d)) / (2 * h)
        ad = float((ga * d).sum())
        assert ad == pytest.approx(fd, rel=tol), (k, ad, fd)
