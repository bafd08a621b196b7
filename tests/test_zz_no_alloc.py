"""The allocation-free RK3 step (mfc_rk3_step_noalloc) against the ordinary
context-based step.

Some callers cannot allocate device memory (another component owns the
memory budget, or the cudaMalloc / cudaFree synchronisation is not
acceptable); they call mfc_rk3_step_noalloc, whose scratch is a file-scope
device array.  This file runs last in the suite so that a failure here
cannot hide the others; it also passes when run alone.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2503_07953_gb300 import workloads as wl
from tests.helpers import case_errors, solver_for, to_host

pytestmark = pytest.mark.gpu

TOL = 1e-11


def descriptors(mfc, case, ghost=3, precision=0):
    g = mfc.mfc_grid()
    g.ndim = case.ndim
    for a in range(3):
        act = a < case.ndim
        g.n[a] = case.n[a] if act else 1
        g.lo[a] = case.lo[a] if act else 0.0
        g.hi[a] = case.hi[a] if act else 1.0
        g.bc_lo[a] = case.bc_lo[a] if act else mfc.MFC_BC_TRANSMISSIVE
        g.bc_hi[a] = case.bc_hi[a] if act else mfc.MFC_BC_TRANSMISSIVE
    g.ghost = ghost
    e = mfc.mfc_eos()
    e.nfluids = case.nf
    for i in range(case.nf):
        e.gamma[i] = case.gamma[i]
        e.pi_inf[i] = case.pi_inf[i]
    o = mfc.mfc_opts()
    o.precision = precision
    o.weno = case.weno
    o.weno_eps = case.eps
    o.cfl = case.cfl
    return g, e, o


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_noalloc_step_matches_context_step(mfc_lib, cuda_device, precision):
    """Two calls in a row (CFL dt each) agree with mfc_rk3_step on a context
    in every precision.  MFC_FP64, MFC_MIXED and MFC_FP64_FAST run the same
    kernels either way and agree bit for bit, dt included.  A double-float
    context runs its sweeps split into reconstruction and Riemann kernels
    and this call the fused sweep; the compiler contracts their updates
    differently, so they agree to rounding: the first dt (from the common
    initial state) bit for bit, the second to 1e-12."""
    case, W = wl.shock_bubble_3d(dims=(40, 36, 30))
    S = solver_for(mfc_lib, case, precision=precision)
    q_ctx = S.prim_to_cons(S.from_interior(W))
    q_na = q_ctx.clone()
    g, e, o = descriptors(mfc_lib, case, precision=precision)
    stream = torch.cuda.current_stream().cuda_stream
    dts = torch.zeros(4, dtype=torch.float64, device=cuda_device)
    for call in range(2):
        S.rk3_step(q_ctx, 0.0, dts[2 * call:2 * call + 1])
        mfc_lib.mfc_rk3_step_noalloc(g, e, o, q_na.data_ptr(), 0.0, dts[2 * call + 1:2 * call + 2].data_ptr(),
                                     stream)
        torch.cuda.synchronize()
        a, b = to_host(S, q_na), to_host(S, q_ctx)
        err = case_errors(case, a, b)
        assert (err <= TOL).all(), (call, err)
        d_ctx, d_na = dts[2 * call].item(), dts[2 * call + 1].item()
        if precision != mfc_lib.MFC_DF64 or call == 0:
            assert d_ctx == d_na
        else:
            assert abs(d_na - d_ctx) <= 1e-12 * d_ctx
    S.check()


@pytest.mark.parametrize("dt", [0.0, 1e-4])
def test_noalloc_reports_nonphysical_state_in_dt(mfc_lib, cuda_device, dt):
    """Without a context there is no flag to read back: a step that meets a
    non-physical state (here a cell of negative pressure) returns NaN in
    dt_used; the next call on a good state clears it."""
    case, W = wl.shock_bubble_3d(dims=(20, 18, 16))
    S = solver_for(mfc_lib, case)
    q_good = S.prim_to_cons(S.from_interior(W))
    Wbad = W.copy()
    Wbad[case.nf + case.ndim, 7, 9, 10] = -0.5  # p < 0 with pi_inf = 0: c^2 < 0
    q_bad = S.prim_to_cons(S.from_interior(Wbad))
    g, e, o = descriptors(mfc_lib, case)
    stream = torch.cuda.current_stream().cuda_stream
    dt_used = torch.zeros(1, dtype=torch.float64, device=cuda_device)
    mfc_lib.mfc_rk3_step_noalloc(g, e, o, q_bad.data_ptr(), dt, dt_used.data_ptr(), stream)
    torch.cuda.synchronize()
    assert np.isnan(dt_used.item())
    mfc_lib.mfc_rk3_step_noalloc(g, e, o, q_good.data_ptr(), dt, dt_used.data_ptr(), stream)
    torch.cuda.synchronize()
    assert np.isfinite(dt_used.item()) and dt_used.item() > 0


def test_noalloc_rejects_oversize_grid(mfc_lib, cuda_device):
    case, W = wl.shock_bubble_3d(dims=(8, 8, 8))
    case.n = [128, 128, 128]  # 134^3 x 7 doubles per state: over the limit
    g, e, o = descriptors(mfc_lib, case)
    q = torch.zeros(1, dtype=torch.float64, device=cuda_device)
    with pytest.raises(mfc_lib.MfcError) as ei:
        mfc_lib.mfc_rk3_step_noalloc(g, e, o, q.data_ptr(), 0.0, None, None)
    assert ei.value.status == mfc_lib.MFC_ERR_ARG
    assert "too large" in mfc_lib.mfc_last_error(None)


def test_noalloc_refuses_viscosity(mfc_lib, cuda_device):
    """The allocation-free step has no scratch for the cell velocities of
    the viscous stress: it refuses before touching the device."""
    case, W = wl.taylor_green(dims=[8, 8, 8])
    g, e, o = descriptors(mfc_lib, case)
    e.eta[0] = case.eta[0]
    q = torch.zeros(1, dtype=torch.float64, device=cuda_device)
    with pytest.raises(mfc_lib.MfcError) as ei:
        mfc_lib.mfc_rk3_step_noalloc(g, e, o, q.data_ptr(), 0.0, None, None)
    assert ei.value.status == mfc_lib.MFC_ERR_UNSUPPORTED


def test_noalloc_symbol_is_exported(mfc_lib):
    lib = ctypes.CDLL(mfc_lib.LIB_PATH)
    assert hasattr(lib, "mfc_rk3_step_noalloc")
