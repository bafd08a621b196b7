"""Adjoints through the CUDA library for torch users.

`RK3Step` is a torch.autograd.Function: forward = mfc_rk3_step at a fixed
dt, backward = mfc_rk3_step_vjp.  `rollout_gradient` differentiates a
scalar objective J = sum_n l_n(q^{n+1}) of an N-step rollout with binomial
checkpointing (`checkpoint.py`): the forward sweep keeps one state, the
reverse sweep holds at most `snapshots` states and recomputes the rest.
The dt of every step is taken from the forward sweep (CFL) and held fixed
in the reverse sweep.

Objectives and initial-condition maps are user code evaluated with torch
operations on small slices of the state (not part of the solver's path);
`wall_pressure_objective` and `alpha_to_state` are the ones the 2D
bubble-collapse workload uses.
"""
from __future__ import annotations

from typing import Callable, Optional, Sequence

import torch

from . import checkpoint
from .mfc import Solver


class RK3Step(torch.autograd.Function):
    """q^{n+1} = RK3(q^n) at a fixed dt, differentiable in q^n."""

    @staticmethod
    def forward(ctx, q: torch.Tensor, solver: Solver, dt: float):
        out = q.detach().clone()
        solver.rk3_step(out, dt)
        ctx.save_for_backward(q.detach())
        ctx.solver = solver
        ctx.dt = dt
        return out

    @staticmethod
    def backward(ctx, grad: torch.Tensor):
        (q,) = ctx.saved_tensors
        g = ctx.solver.rk3_step_vjp(q, ctx.dt, grad.contiguous())
        return g, None, None


def rk3_step(q: torch.Tensor, solver: Solver, dt: float) -> torch.Tensor:
    return RK3Step.apply(q, solver, dt)


def rollout_gradient(solver: Solver, q0: torch.Tensor, nsteps: int, loss: Callable[[int, torch.Tensor], torch.Tensor],
                     snapshots: int, dts: Optional[Sequence[float]] = None):
    """(J, dJ/dq^0, dts, stats) for J = sum_n loss(n, q^{n+1}); loss must be a
    torch function of the state (differentiated with torch.autograd)."""
    if dts is None:
        log = torch.zeros(max(nsteps, 1), dtype=torch.float64, device=q0.device)
        q = q0.clone()
        for n in range(nsteps):
            solver.rk3_step(q, 0.0, log[n:n + 1])
        solver.check()
        dts = [float(x) for x in log[:nsteps].cpu()]
    dts = list(dts)

    def advance(q, n):
        out = q.clone()
        solver.rk3_step(out, dts[n])
        return out

    def vjp(q, n, bar):
        return solver.rk3_step_vjp(q, dts[n], bar.contiguous())

    def loss_value(n, q):
        with torch.no_grad():
            return float(loss(n, q))

    def loss_grad(n, q):
        qq = q.detach().requires_grad_(True)
        (g,) = torch.autograd.grad(loss(n, qq), qq)
        return g.contiguous()

    J, g, stats = checkpoint.rollout_gradient(q0, nsteps, advance, vjp, loss_value, loss_grad,
                                              lambda t: t.clone(), snapshots)
    solver.check()
    return J, g, dts, stats


def mixture_pressure(solver: Solver, q: torch.Tensor, gamma, pi_inf) -> torch.Tensor:
    """p = (rho E - |rho u|^2 / (2 rho) - Pi) / Gamma on the whole padded array
    (torch operations; used only for objectives)."""
    nf, nd = solver.nf, solver.ndim
    g = [1.0 / (x - 1.0) for x in gamma]
    h = [gam * pi / (gam - 1.0) for gam, pi in zip(gamma, pi_inf)]
    rho = sum(q[i] for i in range(nf))
    ke = sum(q[nf + d] * q[nf + d] for d in range(nd)) / (2.0 * rho)
    alphas = [q[nf + nd + 1 + j] for j in range(nf - 1)]
    aN = 1.0 - sum(alphas) if alphas else torch.ones_like(rho)
    Gam = aN * g[nf - 1] + sum(a * g[j] for j, a in enumerate(alphas))
    Pi = aN * h[nf - 1] + sum(a * h[j] for j, a in enumerate(alphas))
    return (q[nf + nd] - ke - Pi) / Gam


def wall_pressure_objective(solver: Solver, case, dts: Sequence[float]) -> Callable[[int, torch.Tensor], torch.Tensor]:
    """l_n(q) = dt_n * sum_j p(q)[last x cell, j] * dy: the time-integrated
    pressure impulse on the x = 1 wall (the last interior column)."""
    g = solver.ghost
    nx = case.n[0]
    dy = case.dx(1) if case.ndim > 1 else 1.0

    def loss(n, q):
        col = q[:, :, g:g + case.n[1], g + nx - 1:g + nx] if case.ndim > 1 else q[:, :, :, g + nx - 1:g + nx]
        p = mixture_pressure(solver, col, case.gamma, case.pi_inf)
        return dts[n] * dy * p.sum()
    return loss


def alpha_to_state(solver: Solver, case, W, alpha1: torch.Tensor) -> torch.Tensor:
    """Conservative state (padded) from the first volume fraction, holding the
    phasic densities, velocity and pressure of the primitive field W (two
    fluids): alpha_i rho_i = alpha_i rho_i^0, rho E = Gamma(alpha) p + Pi(alpha)
    + 1/2 rho |u|^2.  Differentiable in alpha1 (interior-shaped)."""
    nf, nd = case.nf, case.ndim
    assert nf == 2
    W = torch.as_tensor(W, dtype=torch.float64, device=alpha1.device)
    a0 = W[nf + nd + 1]
    rho1 = W[0] / a0
    rho2 = W[1] / (1.0 - a0)
    u = [W[nf + d] for d in range(nd)]
    p = W[nf + nd]
    g = [1.0 / (x - 1.0) for x in case.gamma]
    h = [gam * pi / (gam - 1.0) for gam, pi in zip(case.gamma, case.pi_inf)]
    a1 = alpha1.reshape(a0.shape)
    ar1, ar2 = a1 * rho1, (1.0 - a1) * rho2
    rho = ar1 + ar2
    Gam = (1.0 - a1) * g[1] + a1 * g[0]
    Pi = (1.0 - a1) * h[1] + a1 * h[0]
    E = Gam * p + Pi + 0.5 * rho * sum(ud * ud for ud in u)
    fields = [ar1, ar2] + [rho * ud for ud in u] + [E, a1]
    q = torch.zeros(solver.shape, dtype=torch.float64, device=alpha1.device)
    sl = solver._slices()
    q[sl] = torch.stack(fields)
    return q
