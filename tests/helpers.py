"""Shared test helpers: build the oracle problem and the GPU solver for the
same workload, move states between layouts, compare per field."""
import numpy as np
import torch


def oracle_problem(oracle, case):
    return oracle.Problem(n=case.n, gamma=case.gamma, pi_inf=case.pi_inf, lo=case.lo, hi=case.hi,
                          bc_lo=case.bc_lo, bc_hi=case.bc_hi, weno=case.weno, eps=case.eps)


def solver_for(mfc, case, **kw):
    return mfc.Solver.from_case(case, **kw)


def field_errors(a, b):
    """Per-field max |a - b| / max |b| (b = reference)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    out = []
    for k in range(b.shape[0]):
        den = np.abs(b[k]).max()
        num = np.abs(a[k] - b[k]).max()
        out.append(num / den if den > 0 else num)
    return np.array(out)


def to_host(solver, t):
    torch.cuda.synchronize()
    return solver.interior(t).double().cpu().numpy()
