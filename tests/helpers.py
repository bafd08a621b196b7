"""Shared test helpers: build the oracle problem and the GPU solver for the
same workload, move states between layouts, compare per field."""
import numpy as np
import torch


def oracle_problem(oracle, case):
    return oracle.Problem(n=case.n, gamma=case.gamma, pi_inf=case.pi_inf, lo=case.lo, hi=case.hi,
                          bc_lo=case.bc_lo, bc_hi=case.bc_hi, weno=case.weno, eps=case.eps,
                          teno_ct=case.teno_ct, model=case.model, riemann=case.riemann,
                          low_mach=case.low_mach, eta=case.eta, viscous_dt=int(getattr(case, "viscous_dt", 0)))


def solver_for(mfc, case, **kw):
    return mfc.Solver.from_case(case, **kw)


def field_errors(a, b, nf=None, nd=None):
    """Per-field max |a - b| / max |b| (b = reference).  With nf and nd the
    momentum components share one scale, the largest of their maxima: a
    component that is analytically zero (say rho v in a flow along x) holds
    only rounding noise, and its own maximum is no scale for it."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.array([np.abs(b[k]).max() for k in range(b.shape[0])])
    if nf is not None and nd is not None:
        den[nf:nf + nd] = den[nf:nf + nd].max()
    out = []
    for k in range(b.shape[0]):
        num = np.abs(a[k] - b[k]).max()
        out.append(num / den[k] if den[k] > 0 else num)
    return np.array(out)


def field_scales(case, q):
    """Characteristic magnitude of each conserved field: the maximum for the
    partial densities and the energy, sqrt(max rho * max rho E) (~ rho c)
    for the momenta, 1 for the volume fractions."""
    q = np.asarray(q)
    nf, nd = case.nf, case.ndim
    rho = np.sum(q[:nf], axis=0)
    sc = np.array([max(np.abs(q[k]).max(), 1e-300) for k in range(q.shape[0])])
    mom = np.sqrt(np.abs(rho).max() * np.abs(q[nf + nd]).max())
    sc[nf:nf + nd] = mom
    sc[nf + nd + 1:] = 1.0
    return sc


def case_errors(case, a, b):
    return field_errors(a, b, case.nf, case.ndim)


def to_host(solver, t):
    torch.cuda.synchronize()
    return solver.interior(t).double().cpu().numpy()
