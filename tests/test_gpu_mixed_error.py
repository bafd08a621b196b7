"""The error of the mixed-precision mode (float32 reconstruction, Riemann
solve and directional sums; float64 pressure recovery, stage update and
CFL reduction) against the float64 oracle over many steps, per field.

Both sides take the same dt sequence (the oracle's CFL steps), so the
difference is the mixed arithmetic alone.  Per-field error: max |gpu -
oracle| / max |oracle|, the momentum components sharing one scale.  The
bounds are about three times the errors measured on GB300 (listed per
test); a change that doubles the mixed error fails them.

* 48 x 40 x 40 window of the 3D shock-bubble (the Mach 1.5 shock crosses
  the light-gas bubble in these 25 steps), measured after 25 steps:
  2.6e-6, 1.2e-5, 5.8e-6 (partial densities, rho u), 2.0e-6, 2.5e-6
  (rho v, rho w), 7.7e-6 (energy), 2.9e-6 (alpha_1).
* 32^3 window of the 512^3 three-fluid random-interface field, 50 steps:
  1.7e-6, 1.3e-6, 1.1e-6 (partial densities), 1.1e-4, 1.5e-4, 1.0e-4
  (momenta: 10 m/s flows driven by 1e5 Pa pressure fluxes rounded to
  float32), 3.4e-7 (energy), 3.0e-7, 2.3e-7 (alpha_1, alpha_2).
"""
import numpy as np
import pytest

from paper_2503_07953_gb300 import workloads as wl
from tests.helpers import case_errors, oracle_problem, solver_for, to_host

pytestmark = pytest.mark.gpu

RUNS = {
    "shock_bubble_48x40x40_25": (lambda: wl.shock_bubble_3d(dims=(48, 40, 40)), 25,
                                 [8e-6, 4e-5, 2e-5, 6e-6, 8e-6, 2.5e-5, 9e-6]),
    "random_interfaces_32_50": (lambda: wl.random_interfaces_window(dims=(32, 32, 32)), 50,
                                [5e-6, 4e-6, 3.5e-6, 3.5e-4, 4.5e-4, 3.5e-4, 1e-6, 9e-7, 7e-7]),
}


@pytest.mark.parametrize("name", sorted(RUNS))
def test_mixed_error_per_field_over_steps(oracle_lib, mfc_lib, cuda_device, name):
    make, steps, bounds = RUNS[name]
    case, W = make()
    P = oracle_problem(oracle_lib, case)
    q_o = oracle_lib.prim_to_cons(P, W)
    q_end, dts = oracle_lib.rk3_run(P, q_o, steps, cfl=case.cfl)
    S = solver_for(mfc_lib, case, precision=mfc_lib.MFC_MIXED)
    q = S.from_interior(q_o)
    for dt in dts:
        S.rk3_step(q, float(dt))
    S.check()
    err = case_errors(case, to_host(S, q), q_end)
    print(name, "per-field error", " ".join(f"{e:.2e}" for e in err))
    assert (err <= np.array(bounds)).all(), (err, bounds)
    # and the mixed error is a float32 error, not a float64 one: far above
    # the float64 modes' rounding on the same run
    assert err.max() > 1e-8
