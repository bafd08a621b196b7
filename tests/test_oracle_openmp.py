"""The OpenMP build of the oracle (used to time the CPU baseline on all host
cores) splits only the loops over grid lines and cells; every cell's
arithmetic is that of the single-threaded build, so the two agree bit for
bit: right-hand sides, CFL time steps and whole RK3 runs, inviscid and
viscous."""
import os

import numpy as np
import pytest

from paper_2503_07953_gb300 import workloads as wl
from tests.helpers import oracle_problem


@pytest.fixture()
def both(oracle_lib):
    oracle_lib.build(openmp=True)
    yield oracle_lib
    oracle_lib.set_parallel(False)


def run(oracle, parallel, case, W, steps):
    oracle.set_parallel(parallel)
    P = oracle_problem(oracle, case)
    q = oracle.prim_to_cons(P, W)
    L = oracle.rhs(P, q)
    dt = oracle.cfl_dt(P, q, case.cfl)
    qe, dts = oracle.rk3_run(P, q, steps, cfl=case.cfl)
    return L, dt, qe, dts


@pytest.mark.parametrize("make, steps", [
    (lambda: wl.shock_bubble_3d(dims=(14, 12, 10)), 3),
    (lambda: wl.random_interfaces_window(dims=(10, 9, 8)), 2),
    (lambda: wl.bubble_collapse_2d(dims=(24, 20)), 3),
    (lambda: wl.taylor_green(n=10, ndim=3), 2),
])
def test_openmp_build_is_bitwise_equal(both, make, steps):
    case, W = make()
    serial = run(both, False, case, W, steps)
    threaded = run(both, True, case, W, steps)
    assert both.threads() >= 1
    for a, b in zip(serial, threaded):
        assert np.array_equal(np.asarray(a), np.asarray(b))


def test_openmp_build_uses_the_host_cores(both):
    both.set_parallel(True)
    n = os.cpu_count() or 1
    want = int(os.environ.get("OMP_NUM_THREADS", n))
    assert both.threads() == want
    both.set_parallel(False)
    assert both.threads() == 1
