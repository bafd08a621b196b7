"""MFC_DF64 (double-float WENO5 on the float32 pipes, float64 elsewhere)
against the CPU oracle, through the C ABI.

The double-float reconstruction carries a 48-bit significand instead of
float64's 53 in the corrections to the centre value, so it agrees with the
oracle to rounding, not bit for bit.  The bar on states is the float64
target, max |gpu - oracle| / max |oracle| <= 1e-11 per field (momenta
sharing one scale): after 100 CFL steps of the 3D shock-bubble, after one
step of every Riemann-solver option and model, and at sampled cells of the
256^3 benchmarked configuration.

One evaluation of L is a difference of fluxes divided by dx, which
amplifies their rounding by |F| / (|L| dx): MFC_FP64_FAST itself reaches
1e-11 of max |L| on some workloads (the minority partial density of the
shock-bubble).  There the bar is 1e-11 or 16 times MFC_FP64_FAST's own
error on the same input (the ratio of the two significands' rounding,
2^-49 / 2^-53), whichever is larger."""
import numpy as np
import pytest
import torch

from paper_2503_07953_gb300 import workloads as wl
from tests.helpers import case_errors, oracle_problem, solver_for, to_host
from tests.test_gpu_parity import CASES, RUNS, SOLVERS, kapila_shock_bubble, setup

pytestmark = pytest.mark.gpu

TOL = 1e-11


def rhs_errors(oracle_lib, mfc_lib, case, W):
    """Per-field errors of one evaluation of L in MFC_DF64 and MFC_FP64_FAST."""
    P = oracle_problem(oracle_lib, case)
    q_o = oracle_lib.prim_to_cons(P, W)
    L_o = oracle_lib.rhs(P, q_o)
    errs = []
    for prec in (mfc_lib.MFC_DF64, mfc_lib.MFC_FP64_FAST):
        S = solver_for(mfc_lib, case, precision=prec)
        L_g = to_host(S, S.rhs(S.from_interior(q_o)))
        S.check()
        errs.append(case_errors(case, L_g, L_o))
    return errs


@pytest.mark.parametrize("name", sorted(CASES))
def test_rhs_df64(oracle_lib, mfc_lib, cuda_device, name):
    case, W = CASES[name]()
    err, err_fast = rhs_errors(oracle_lib, mfc_lib, case, W)
    assert (err <= np.maximum(TOL, 16 * err_fast)).all(), (err, err_fast)


@pytest.mark.parametrize("weno", [0, 2, 3])
def test_rhs_df64_weno_variants(oracle_lib, mfc_lib, cuda_device, weno):
    """Jiang-Shu (eps = 1e-6), Z and TENO weights in double-float."""
    for make in (lambda: wl.shock_bubble_3d(dims=(19, 16, 14)), lambda: wl.water_air_shock_tube(400)):
        case, W = make()
        case.weno = weno
        case.eps = 1e-6 if weno == 0 else 1e-40
        err, err_fast = rhs_errors(oracle_lib, mfc_lib, case, W)
        assert (err <= np.maximum(TOL, 16 * err_fast)).all(), (case.name, err, err_fast)


def test_rk3_run_df64_shock_bubble(oracle_lib, mfc_lib, cuda_device):
    """100 CFL steps of the 3D shock-bubble, dt computed on the device."""
    make, steps = RUNS["shock_bubble_3d"]
    case, W, P, S, q_o, q_g = setup(oracle_lib, mfc_lib, make, precision=mfc_lib.MFC_DF64)
    q_g = S.from_interior(q_o)
    S.rk3_run(q_g, steps, 0.0)
    S.check()
    q_end, _ = oracle_lib.rk3_run(P, q_o, steps, cfl=case.cfl)
    err = case_errors(case, to_host(S, q_g), q_end)
    assert (err <= TOL).all(), err


@pytest.mark.parametrize("name", ["random_interfaces_3d", "bubble_collapse_2d"])
def test_rk3_run_df64_matches_fast(oracle_lib, mfc_lib, cuda_device, name):
    """Stiff workloads over their full step counts: MFC_DF64 stays as close
    to the oracle as MFC_FP64_FAST does (both differ from it by rounding
    that these workloads amplify), within a factor of 100 or 1e-11."""
    make, steps = RUNS[name]
    errs = {}
    for prec in (mfc_lib.MFC_FP64_FAST, mfc_lib.MFC_DF64):
        case, W, P, S, q_o, q_g = setup(oracle_lib, mfc_lib, make, precision=prec)
        q_g = S.from_interior(q_o)
        S.rk3_run(q_g, steps, 0.0)
        S.check()
        if prec == mfc_lib.MFC_FP64_FAST:
            q_end, _ = oracle_lib.rk3_run(P, q_o, steps, cfl=case.cfl)
        errs[prec] = case_errors(case, to_host(S, q_g), q_end)
    bound = np.maximum(100.0 * errs[mfc_lib.MFC_FP64_FAST], TOL)
    assert (errs[mfc_lib.MFC_DF64] <= bound).all(), errs


def test_step_df64_kapila(oracle_lib, mfc_lib, cuda_device):
    case, W = kapila_shock_bubble()
    P = oracle_problem(oracle_lib, case)
    S = solver_for(mfc_lib, case, precision=mfc_lib.MFC_DF64)
    q_o = oracle_lib.prim_to_cons(P, W)
    dt = oracle_lib.cfl_dt(P, q_o, case.cfl)
    q = S.from_interior(q_o)
    S.rk3_step(q, dt)
    S.check()
    err = case_errors(case, to_host(S, q), oracle_lib.rk3_step(P, q_o, dt))
    assert (err <= TOL).all(), err


@pytest.mark.parametrize("riemann,low_mach", SOLVERS)
def test_step_df64_riemann_variants(oracle_lib, mfc_lib, cuda_device, riemann, low_mach):
    for make in (lambda: wl.gresho_vortex(24, 1e-2), lambda: wl.shock_bubble_3d(dims=(16, 14, 12))):
        case, W = make()
        case.riemann, case.low_mach = riemann, low_mach
        P = oracle_problem(oracle_lib, case)
        S = solver_for(mfc_lib, case, precision=mfc_lib.MFC_DF64)
        q_o = oracle_lib.prim_to_cons(P, W)
        dt = oracle_lib.cfl_dt(P, q_o, case.cfl)
        q = S.from_interior(q_o)
        S.rk3_step(q, dt)
        S.check()
        err = case_errors(case, to_host(S, q), oracle_lib.rk3_step(P, q_o, dt))
        assert (err <= TOL).all(), (case.name, err)


@pytest.mark.parametrize("dims,bc", [((3,), 0), ((5,), 1), ((3, 3, 3), 0), ((7, 1), 1), ((1, 6, 4), 1),
                                     ((67, 3, 18), 2)])
def test_df64_degenerate_sizes(oracle_lib, mfc_lib, cuda_device, dims, bc):
    nd = len(dims)
    case = wl.Case("tiny", list(dims), [0.0] * nd, [1.0] * nd, [bc] * nd, [bc] * nd, [1.4, 1.67],
                   [0.0, 0.0], cfl=0.4, steps=0)
    W = wl.random_smooth_state(case, seed=1, amp=0.1)
    P = oracle_problem(oracle_lib, case)
    S = solver_for(mfc_lib, case, precision=mfc_lib.MFC_DF64)
    q_o = oracle_lib.prim_to_cons(P, W)
    q_g = S.from_interior(q_o)
    S.rk3_run(q_g, 5)
    S.check()
    q_end, _ = oracle_lib.rk3_run(P, q_o, 5, cfl=case.cfl)
    err = case_errors(case, to_host(S, q_g), q_end)
    assert (err <= TOL).all(), err


def test_df64_full_size_step_sampled(oracle_lib, mfc_lib, cuda_device):
    """The 256^3 shock-bubble in the benchmarked configuration: one step,
    checked at sampled cells (corners, walls, the shock, the bubble
    interface) against the oracle's domain-of-dependence evaluation."""
    case, W = wl.shock_bubble_3d(256)
    P = oracle_problem(oracle_lib, case)
    S = solver_for(mfc_lib, case, precision=mfc_lib.MFC_DF64)
    q_g = S.prim_to_cons(S.from_interior(W))
    q_o = to_host(S, q_g)
    dt = oracle_lib.cfl_dt(P, q_o, case.cfl)
    S.rk3_step(q_g, dt)
    S.check()
    out_g = to_host(S, q_g)
    rng = np.random.default_rng(1)
    cells = [(0, 0, 0), (255, 255, 255), (0, 255, 128), (255, 0, 3), (64, 128, 128), (63, 127, 200),
             (89, 128, 128), (128, 90, 128), (128, 128, 166), (167, 128, 128), (128, 1, 254)]
    cells += [tuple(int(v) for v in rng.integers(0, 256, 3)) for _ in range(9)]
    ref = oracle_lib.rk3_step_sampled(P, q_o, dt, cells)
    got = np.stack([out_g[:, k, j, i] for (i, j, k) in cells])
    scale = np.abs(out_g).max(axis=(1, 2, 3))
    scale[case.nf:case.nf + case.ndim] = scale[case.nf:case.nf + case.ndim].max()
    err = (np.abs(got - ref) / scale).max(axis=0)
    assert (err <= TOL).all(), err


def test_df64_indicator_overflow_reported(mfc_lib, cuda_device):
    """A pressure jump of 1e20 overflows the float32 range of the
    smoothness indicators: the step reports a non-physical state instead of
    returning a silently different result."""
    case, W = wl.shock_bubble_3d(dims=(12, 10, 8))
    W = np.array(W, copy=True)
    W[case.nf + case.ndim, :, :, 6:] = 1e20
    S = solver_for(mfc_lib, case, precision=mfc_lib.MFC_DF64)
    q = S.prim_to_cons(S.from_interior(W))
    S.rhs(q)
    with pytest.raises(mfc_lib.MfcError) as ei:
        S.check()
    assert ei.value.status == mfc_lib.MFC_ERR_NONPHYSICAL
    S.check()  # the flag was cleared


@pytest.mark.parametrize("make", [lambda: wl.shock_bubble_3d(dims=(40, 36, 30)),
                                  lambda: wl.bubble_collapse_2d(dims=(64, 48)),
                                  lambda: wl.water_air_shock_tube(300)])
def test_df64_split_sweeps_equal_fused(mfc_lib, cuda_device, make):
    """A context runs the MFC_DF64 sweeps split into reconstruction and
    Riemann kernels on two streams, in chunks of lines; the allocation-free
    step runs the fused sweep.  The same operations on the same values, up to
    the compiler's fused multiply-add contraction of the update, which
    differs between the kernels: after two CFL steps the states agree to
    1e-13 per field and the first step's dt bit for bit."""
    from tests.test_zz_no_alloc import descriptors
    case, W = make()
    S = solver_for(mfc_lib, case, precision=mfc_lib.MFC_DF64)
    q_split = S.prim_to_cons(S.from_interior(W))
    q_fused = q_split.clone()
    g, e, o = descriptors(mfc_lib, case, precision=mfc_lib.MFC_DF64)
    stream = torch.cuda.current_stream().cuda_stream
    dts = torch.zeros(4, dtype=torch.float64, device=cuda_device)
    for call in range(2):
        S.rk3_step(q_split, 0.0, dts[2 * call:2 * call + 1])
        mfc_lib.mfc_rk3_step_noalloc(g, e, o, q_fused.data_ptr(), 0.0, dts[2 * call + 1:2 * call + 2].data_ptr(),
                                     stream)
    S.check()
    d = dts.cpu().numpy()
    assert d[0] == d[1] and d[2] == pytest.approx(d[3], rel=1e-14)
    err = case_errors(case, to_host(S, q_split), to_host(S, q_fused))
    assert (err <= 1e-13).all(), err


@pytest.mark.parametrize("name", ["taylor_green_3d", "walled_2d_nf2", "walled_3d_nf3"])
def test_df64_viscous(oracle_lib, mfc_lib, cuda_device, name):
    """With viscous stress the split sweeps accumulate onto the viscous
    right-hand side (float64, MODE_FAST arithmetic): one evaluation of L
    against the oracle at FAST's own rounding, and 20 steps of a walled
    three-fluid run within 1e-11."""
    from tests.test_gpu_viscous import CASES as VCASES
    case, W = VCASES[name]()
    err, err_fast = rhs_errors(oracle_lib, mfc_lib, case, W)
    assert (err <= np.maximum(TOL, 16 * err_fast)).all(), (err, err_fast)
    if name == "walled_3d_nf3":
        P = oracle_problem(oracle_lib, case)
        S = solver_for(mfc_lib, case, precision=mfc_lib.MFC_DF64)
        q_o = oracle_lib.prim_to_cons(P, W)
        q_end, dts = oracle_lib.rk3_run(P, q_o, 20, cfl=case.cfl)
        q_g = S.from_interior(q_o)
        for dt in dts:
            S.rk3_step(q_g, float(dt))
        S.check()
        err = case_errors(case, to_host(S, q_g), q_end)
        assert (err <= TOL).all(), err


def test_df64_graph_capture(mfc_lib, cuda_device):
    """A 192^3 shock-bubble (two chunks per direction, so the ring of edge
    value slots wraps within each evaluation of L): five steps captured in
    one CUDA graph, the reconstruction stream forked and joined inside the
    capture, replay equal bit for bit to the same steps run eagerly."""
    case, W = wl.shock_bubble_3d(192)
    S = solver_for(mfc_lib, case, precision=mfc_lib.MFC_DF64)
    q0 = S.prim_to_cons(S.from_interior(W))
    q = q0.clone()
    S.rk3_run(q, 5, 0.0)
    S.check()
    qg = q0.clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        S.rk3_run(qg, 1, 0.0)
    torch.cuda.current_stream().wait_stream(side)
    qg.copy_(q0)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        S.rk3_run(qg, 5, 0.0)
    qg.copy_(q0)
    g.replay()
    torch.cuda.synchronize()
    S.check()
    assert torch.equal(qg, q)


@pytest.mark.parametrize("name", ["smooth_3d_mixed_bc", "stiff_smooth_2d", "smooth_2d_kapila"])
def test_df64_rk3_step_vjp_dot_product(oracle_lib, mfc_lib, cuda_device, name):
    """The adjoint step of a double-float context recomputes the RK stages
    with the double-float sweeps and runs the adjoint sweeps in float64
    (MFC_FP64_FAST arithmetic): <v, J w> from the oracle's dual numbers
    against <J^T v, w> from the library, 1e-10 as for MFC_FP64_FAST."""
    from tests.test_gpu_adjoint import CASES as ACASES, directions, dot
    case, W = ACASES[name]()
    P = oracle_problem(oracle_lib, case)
    S = solver_for(mfc_lib, case, precision=mfc_lib.MFC_DF64)
    q = oracle_lib.prim_to_cons(P, W)
    dt = oracle_lib.cfl_dt(P, q, case.cfl)
    w, v = directions(case, q, 8)
    _, Jw = oracle_lib.rk3_step_jvp(P, q, w, dt)
    qb = S.rk3_step_vjp(S.from_interior(q), dt, S.from_interior(v))
    lhs = dot(v, Jw)
    rhs = dot(to_host(S, qb), w)
    assert rhs == pytest.approx(lhs, rel=1e-10), (lhs, rhs)
