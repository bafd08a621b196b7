"""The slab decomposition with the CUDA library (MFC_BC_HALO sides,
mfc_rk3_stage): every slab of a grid as its own context on one GPU, the
halo layers copied between their tensors before each stage and the CFL dt
reduced to the minimum over the slabs (decomp.LocalSlabs, the arithmetic of
one slab per GPU).  The gathered slabs must equal the undivided grid's run
bit for bit in every precision: the library reads the halo cells exactly
where it would read the neighbouring cells, and every face sees the same
cell width (power-of-two widths here; decomp.exact_span)."""
import numpy as np
import pytest
import torch

from paper_2503_07953_gb300 import decomp
from tests.helpers import oracle_problem, solver_for
from tests.test_decomp import make_case

pytestmark = pytest.mark.gpu

CASES = {
    "shock_bubble_x3": ("shock_bubble_3d", dict(dims=(40, 24, 20)), 0, 3, 4),
    "shock_bubble_y2": ("shock_bubble_3d", dict(dims=(24, 40, 20)), 1, 2, 4),
    "smooth_periodic_z2": ("smooth_periodic_3d", dict(dims=(20, 16, 24)), 2, 2, 3),
    "smooth_periodic_x3": ("smooth_periodic_3d", dict(dims=(24, 16, 20)), 0, 3, 3),
    "smooth_periodic_y2": ("smooth_periodic_3d", dict(dims=(16, 24, 20)), 1, 2, 3),
    "shock_bubble_z2": ("shock_bubble_3d", dict(dims=(20, 16, 24)), 2, 2, 3),
    "bubble_collapse_wall_x4": ("bubble_collapse_2d", dict(dims=(64, 48)), 0, 4, 5),
    "water_air_tube_3": ("water_air_shock_tube", dict(n=300), 0, 3, 20),
}


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("name", sorted(CASES))
def test_slabs_equal_undivided_run_bitwise(mfc_lib, cuda_device, name, prec):
    wname, kw, axis, world, steps = CASES[name]
    case, W = make_case(wname, kw)
    S = solver_for(mfc_lib, case, precision=prec)
    q0 = S.prim_to_cons(S.from_interior(W))
    ref = q0.clone()
    dts_ref = torch.zeros(steps, dtype=torch.float64, device=cuda_device)
    S.rk3_run(ref, steps, 0.0, dts_ref)
    S.check()  # the undivided run itself meets no non-physical state
    D = decomp.LocalSlabs(case, axis, world, lambda c: solver_for(mfc_lib, c, precision=prec))
    qs = D.scatter(S.interior(q0))
    scratch = [(st.empty(), st.empty()) for st in D.steppers]
    dts = [D.step(qs, scratch) for _ in range(steps)]
    for st in D.steppers:
        st.check()
    got = D.gather(qs)
    want = S.interior(ref).cpu()
    diff = (got - want).abs().amax(dim=tuple(d for d in range(4) if d != 3 - axis))
    assert dts == dts_ref.cpu().tolist(), (dts, dts_ref.cpu().tolist())
    assert torch.equal(got, want), ("largest difference per cell layer along the cut axis", diff.tolist())


def test_slabs_fp64_match_the_oracle(oracle_lib, mfc_lib, cuda_device):
    case, W = make_case("shock_bubble_3d", dict(dims=(30, 16, 12)))
    P = oracle_problem(oracle_lib, case)
    q_o = oracle_lib.prim_to_cons(P, W)
    ref, _ = oracle_lib.rk3_run(P, q_o, 3, cfl=case.cfl)
    D = decomp.LocalSlabs(case, 0, 3, lambda c: solver_for(mfc_lib, c))
    qs = D.scatter(torch.as_tensor(q_o))
    scratch = [(st.empty(), st.empty()) for st in D.steppers]
    for _ in range(3):
        D.step(qs, scratch)
    assert np.array_equal(D.gather(qs).numpy(), ref)


def test_halo_context_refuses_whole_steps(mfc_lib, cuda_device):
    case, W = make_case("shock_bubble_3d", dict(dims=(16, 8, 8)))
    st = solver_for(mfc_lib, decomp.Slab(case, 0, 2, 0).local_case())
    q = st.empty()
    for call in (lambda: st.rk3_step(q, 1e-3), lambda: st.rk3_run(q, 1, 1e-3),
                 lambda: st.rk3_step_vjp(q, 1e-3, st.empty())):
        with pytest.raises(mfc_lib.MfcError) as ei:
            call()
        assert ei.value.status == mfc_lib.MFC_ERR_UNSUPPORTED
    with pytest.raises(mfc_lib.MfcError) as ei:
        st.rk3_stage(1, q, None, q, 1e-3)  # q_out aliasing q_in
    assert ei.value.status == mfc_lib.MFC_ERR_ARG
