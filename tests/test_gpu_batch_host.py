"""mfc_rk3_step_batch_host: independent states held in host memory, each
uploaded, stepped once (Sec. 3.4) and downloaded, with the copies on the
context's own streams overlapping the neighbouring states' steps.  The same
kernels run as for mfc_rk3_step, so every result must equal, bit for bit,
the in-place device step of the same state in the same precision, and in
MFC_FP64 the oracle's step."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2503_07953_gb300 import workloads as wl
from tests.helpers import case_errors, oracle_problem, solver_for

pytestmark = pytest.mark.gpu


def host_states(S, case, W, count, pinned):
    """count distinct conservative states on the host: the workload with its
    pressure scaled by 1 + 0.02 b."""
    out = []
    ip = case.nf + case.ndim
    for b in range(count):
        Wb = np.array(W, copy=True)
        Wb[ip] *= 1.0 + 0.02 * b
        q = S.prim_to_cons(S.from_interior(Wb)).cpu()
        out.append(q.pin_memory() if pinned else q)
    return out


def device_reference(S, qs, dt):
    """The in-place device step of each state, and the dt it took."""
    res, dts = [], []
    dt_used = torch.zeros(1, dtype=torch.float64, device=S.device)
    for q in qs:
        qd = q.to(S.device)
        S.rk3_step(qd, dt, dt_used)
        S.check()
        res.append(qd.cpu())
        dts.append(float(dt_used.item()))
    return res, dts


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_batch_equals_device_steps(mfc_lib, cuda_device, prec, pinned):
    case, W = wl.shock_bubble_3d(dims=(19, 16, 14))
    S = solver_for(mfc_lib, case, precision=prec)
    qs = host_states(S, case, W, 5, pinned)
    want, want_dt = device_reference(S, qs, 0.0)
    outs = [torch.empty_like(q) for q in qs]
    if pinned:
        outs = [o.pin_memory() for o in outs]
    dts = S.rk3_step_batch_host(qs, outs, 0.0)
    for b in range(len(qs)):
        assert torch.equal(outs[b], want[b]), b
    assert dts.tolist() == want_dt
    assert len(set(want_dt)) == len(want_dt)  # the states are distinct


def test_batch_matches_oracle_bitwise(oracle_lib, mfc_lib, cuda_device):
    """MFC_FP64 through host buffers: the oracle's CFL dt and RK3 step."""
    case, W = wl.shock_bubble_3d(dims=(21, 18, 13))
    P = oracle_problem(oracle_lib, case)
    S = solver_for(mfc_lib, case)
    qs = host_states(S, case, W, 3, True)
    outs = [torch.empty_like(q).pin_memory() for q in qs]
    dts = S.rk3_step_batch_host(qs, outs, 0.0)
    for b in range(3):
        q_o = S.interior(qs[b]).numpy()
        dt = oracle_lib.cfl_dt(P, q_o, case.cfl)
        assert dts[b].item() == dt
        want = oracle_lib.rk3_step(P, q_o, dt)
        got = S.interior(outs[b]).numpy()
        assert np.array_equal(got, want), case_errors(case, got, want)


def test_batch_aliasing_rules(mfc_lib, cuda_device):
    """One input read by every state, one output written by every state (it
    ends with the last), and q_out[b] = q_in[b] in place."""
    case, W = wl.water_air_shock_tube(300)
    S = solver_for(mfc_lib, case, precision=2)
    qs = host_states(S, case, W, 4, True)
    want, _ = device_reference(S, qs, 1e-7)
    shared_out = torch.empty_like(qs[0]).pin_memory()
    dts = S.rk3_step_batch_host([qs[0]] * 4, [shared_out] * 4, 1e-7)
    assert dts.tolist() == [1e-7] * 4
    assert torch.equal(shared_out, want[0])
    shared_out.zero_()
    S.rk3_step_batch_host(qs, [shared_out] * 4, 1e-7)
    assert torch.equal(shared_out, want[3])
    inplace = [q.clone().pin_memory() for q in qs]
    S.rk3_step_batch_host(inplace, inplace, 1e-7)
    for b in range(4):
        assert torch.equal(inplace[b], want[b]), b


def test_batch_longer_than_staging(mfc_lib, cuda_device):
    """More states than staging buffers and than the first dt array (64):
    the buffers are reused in turn and the dt array grows."""
    case, W = wl.water_air_shock_tube(200)
    S = solver_for(mfc_lib, case, precision=2)
    base = host_states(S, case, W, 1, True)[0]
    qs = []
    for b in range(70):
        q = base.clone()
        S.interior(q)[case.nf + case.ndim] *= 1.0 + 1e-3 * b
        qs.append(q.pin_memory())
    want, want_dt = device_reference(S, qs, 0.0)
    outs = [torch.empty_like(q).pin_memory() for q in qs]
    dts = S.rk3_step_batch_host(qs, outs, 0.0)
    assert dts.tolist() == want_dt
    for b in range(70):
        assert torch.equal(outs[b], want[b]), b


def test_batch_empty_and_bad_arguments(mfc_lib, cuda_device):
    case, W = wl.water_air_shock_tube(64)
    S = solver_for(mfc_lib, case)
    assert S.rk3_step_batch_host([], [], 0.0).numel() == 0
    q = host_states(S, case, W, 1, True)[0]
    with pytest.raises(ValueError):
        S.rk3_step_batch_host([q], [], 0.0)
    with pytest.raises(ValueError):
        S.rk3_step_batch_host([q.to(cuda_device)], [q], 0.0)
    L = mfc_lib.lib()
    VP2 = ctypes.c_void_p * 2
    good = VP2(q.data_ptr(), q.data_ptr())
    holed = VP2(q.data_ptr(), None)
    stream = torch.cuda.current_stream().cuda_stream
    assert L.mfc_rk3_step_batch_host(S.ctx, -1, good, good, 0.0, None, stream) == mfc_lib.MFC_ERR_ARG
    assert L.mfc_rk3_step_batch_host(S.ctx, 2, None, good, 0.0, None, stream) == mfc_lib.MFC_ERR_ARG
    assert L.mfc_rk3_step_batch_host(S.ctx, 2, good, holed, 0.0, None, stream) == mfc_lib.MFC_ERR_ARG
    assert b"null host buffer" in L.mfc_last_error(S.ctx)
    assert L.mfc_rk3_step_batch_host(S.ctx, 1, good, good, float("nan"), None, stream) == mfc_lib.MFC_ERR_ARG
    assert L.mfc_rk3_step_batch_host(S.ctx, 0, None, None, 0.0, None, stream) == mfc_lib.MFC_OK


def test_batch_reports_nonphysical_state(mfc_lib, cuda_device):
    case, W = wl.shock_bubble_3d(dims=(8, 8, 8))
    S = solver_for(mfc_lib, case)
    qs = host_states(S, case, W, 3, True)
    S.interior(qs[1])[case.nf + case.ndim, 4, 4, 4] = -10.0  # negative energy -> p + pi < 0
    outs = [torch.empty_like(q).pin_memory() for q in qs]
    with pytest.raises(mfc_lib.MfcError) as ei:
        S.rk3_step_batch_host(qs, outs, 1e-9)
    assert ei.value.status == mfc_lib.MFC_ERR_NONPHYSICAL
    S.check()  # the flag was cleared
    want, _ = device_reference(S, [qs[2]], 1e-9)
    assert torch.equal(outs[2], want[0])
