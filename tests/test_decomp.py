"""The slab decomposition (paper_2503_07953_gb300.decomp) on CPU: world size
2 and 3 over gloo, the oracle as each rank's stepper.

Each rank advances its slab with one halo exchange per RK stage and the
CFL dt reduced to the minimum over the ranks; the slabs, gathered, must
equal the undivided grid's oracle run bit for bit (every cell goes through
the same arithmetic, and a minimum does not depend on the order of its
terms).  The oracle stands in for the CUDA library here: it evaluates L on
the slab extended by its halo layers, with any boundary condition beyond
them (those cells' own right-hand sides are discarded), which is what the
library does by reading the halo cells (MFC_BC_HALO).  The same driver runs
the CUDA library in tests/test_gpu_decomp.py."""
import dataclasses
import os
import pickle
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = {
    "shock_bubble_x": ("shock_bubble_3d", dict(dims=(20, 12, 10)), 0, 3),
    "smooth_periodic_x": ("smooth_periodic_3d", dict(dims=(16, 12, 10)), 0, 2),
    "smooth_periodic_z": ("smooth_periodic_3d", dict(dims=(10, 12, 16)), 2, 2),
    "bubble_collapse_wall_x": ("bubble_collapse_2d", dict(dims=(24, 20)), 0, 3),
}


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleStepper:
    """The oracle behind the stepper interface of decomp, on CPU tensors in
    the library's padded layout [field][z][y][x] with `ghost` cells on each
    active axis."""

    def __init__(self, oracle, case, ghost=3):
        self.oracle, self.case, self.ghost = oracle, case, ghost
        self.ndim = case.ndim
        self.n = list(case.n) + [1] * (3 - case.ndim)
        pad = [self.n[a] + (2 * ghost if a < self.ndim else 0) for a in range(3)]
        self.shape = (case.nq, pad[2], pad[1], pad[0])

    def empty(self):
        return torch.zeros(self.shape, dtype=torch.float64)

    def _region(self, ext):
        """Index of the interior, extended by the ghost layers of halo sides
        when ext."""
        g, idx, nlo = self.ghost, [slice(None)], []
        for a in (2, 1, 0):
            if a >= self.ndim:
                idx.append(slice(0, 1))
                continue
            lo = g - (g if ext and self.case.bc_lo[a] == 3 else 0)
            hi = g + self.n[a] + (g if ext and self.case.bc_hi[a] == 3 else 0)
            idx.append(slice(lo, hi))
        return tuple(idx)

    def interior(self, t):
        return t[self._region(False)]

    def from_interior(self, arr):
        t = self.empty()
        t[self._region(False)] = torch.as_tensor(np.ascontiguousarray(arr))
        return t

    def _problem(self, case):
        from tests.helpers import oracle_problem
        return oracle_problem(self.oracle, case)

    def compute_dt(self, q):
        c = dataclasses.replace(self.case, bc_lo=[1 if b == 3 else b for b in self.case.bc_lo],
                                bc_hi=[1 if b == 3 else b for b in self.case.bc_hi])
        return self.oracle.cfl_dt(self._problem(c), self.interior(q).numpy(), self.case.cfl)

    def rk3_stage(self, stage, q_in, q_n, q_out, dt):
        from paper_2503_07953_gb300.decomp import exact_span
        c = self.case
        n, lo, hi, bl, bh = list(c.n), list(c.lo), list(c.hi), list(c.bc_lo), list(c.bc_hi)
        add_lo = [self.ghost if b == 3 else 0 for b in c.bc_lo]
        add_hi = [self.ghost if b == 3 else 0 for b in c.bc_hi]
        for a in range(c.ndim):
            dx = c.dx(a)
            n[a] = c.n[a] + add_lo[a] + add_hi[a]
            lo[a], hi[a] = exact_span(c.lo[a] - add_lo[a] * dx, dx, n[a])
            bl[a] = 1 if bl[a] == 3 else bl[a]
            bh[a] = 1 if bh[a] == 3 else bh[a]
        ext = dataclasses.replace(c, n=n, lo=lo, hi=hi, bc_lo=bl, bc_hi=bh)
        L = self.oracle.rhs(self._problem(ext), np.ascontiguousarray(q_in[self._region(True)].numpy()))
        sl = [slice(None)]
        for a in (2, 1, 0):
            sl.append(slice(add_lo[a], add_lo[a] + c.n[a]) if a < c.ndim else slice(0, 1))
        Li = L[tuple(sl)]
        qi = self.interior(q_in).numpy()
        if stage == 1:
            out = qi + dt * Li
        elif stage == 2:
            out = 0.75 * self.interior(q_n).numpy() + 0.25 * (qi + dt * Li)
        else:
            out = (1.0 / 3.0) * self.interior(q_n).numpy() + (2.0 / 3.0) * (qi + dt * Li)
        q_out[self._region(False)] = torch.as_tensor(out)
        return q_out


def smooth_periodic_3d(dims):
    """A smooth three-fluid state (stiffened gases) on a periodic box."""
    from paper_2503_07953_gb300 import workloads as wl
    case = wl.Case("smooth_periodic_3d", list(dims), [0.0] * 3, [1.0] * 3, [wl.PERIODIC] * 3, [wl.PERIODIC] * 3,
                   [1.4, 4.4, 6.1], [0.0, 6.0, 20.0], cfl=0.4, steps=0)
    return case, wl.random_smooth_state(case, seed=5, amp=0.1)


def make_case(name, kw):
    """The workload's state on a grid whose cell widths are powers of two
    (the largest not above the workload's own), so that every slab of any
    size has the global cell width exactly (decomp.exact_span)."""
    from paper_2503_07953_gb300 import workloads as wl
    case, W = smooth_periodic_3d(**kw) if name == "smooth_periodic_3d" else getattr(wl, name)(**kw)
    for a in range(case.ndim):
        w = 2.0 ** np.floor(np.log2(case.dx(a)))
        case.hi[a] = case.lo[a] + case.n[a] * w
    return case, W


def _rank_main(rank, world, port, name, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import oracle
    from paper_2503_07953_gb300 import decomp
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wname, kw, axis, steps = CASES[name]
    case, W = make_case(wname, kw)
    slab = decomp.Slab(case, axis, world, rank)
    st = OracleStepper(oracle, slab.local_case())
    from tests.helpers import oracle_problem
    q_glob = oracle.prim_to_cons(oracle_problem(oracle, case), W)
    q = st.from_interior(np.ascontiguousarray(slab.take(q_glob)))
    scratch = [st.empty(), st.empty()]
    ex = decomp.HaloExchange(slab, st.ghost)
    dts = [decomp.rk3_step(st, q, scratch, ex, decomp.allreduce_min) for _ in range(steps)]
    with open(os.path.join(out_dir, f"rank{rank}.pkl"), "wb") as fh:
        pickle.dump({"q": st.interior(q).numpy().copy(), "dts": dts, "offset": slab.offset}, fh)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("name", sorted(CASES))
def test_slab_decomposition_equals_undivided_run_bitwise(oracle_lib, tmp_path, name, world):
    wname, kw, axis, steps = CASES[name]
    if wname == "smooth_periodic_3d" and world == 3 and axis == 2:
        pytest.skip("one periodic case per axis is enough at world size 3")
    mp.start_processes(_rank_main, args=(world, free_port(), name, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    case, W = make_case(wname, kw)
    from tests.helpers import oracle_problem
    P = oracle_problem(oracle_lib, case)
    ref, ref_dts = oracle_lib.rk3_run(P, oracle_lib.prim_to_cons(P, W), steps, cfl=case.cfl)
    recs = [pickle.load(open(tmp_path / f"rank{r}.pkl", "rb")) for r in range(world)]
    got = np.concatenate([r["q"] for r in recs], axis=3 - axis)
    for r in recs:
        assert r["dts"] == [float(d) for d in ref_dts]
    assert np.array_equal(got, ref)


def test_slab_sides_and_sizes():
    from paper_2503_07953_gb300 import decomp
    case, _ = make_case("shock_bubble_3d", dict(dims=(10, 4, 4)))
    slabs = [decomp.Slab(case, 0, 3, r) for r in range(3)]
    assert [s.n_local for s in slabs] == [4, 3, 3] and [s.offset for s in slabs] == [0, 4, 7]
    assert (slabs[0].left, slabs[0].right, slabs[2].right) == (None, 1, None)
    lc = slabs[1].local_case()
    assert lc.bc_lo[0] == decomp.BC_HALO and lc.bc_hi[0] == decomp.BC_HALO
    assert slabs[0].local_case().bc_lo[0] == case.bc_lo[0]
    for s in slabs:
        c = s.local_case()
        assert c.dx(0) == case.dx(0)  # the global cell width, bit for bit
    per, _ = make_case("random_interfaces_3d", dict(dims=(6, 4, 4)))
    p = [decomp.Slab(per, 0, 2, r) for r in range(2)]
    assert (p[0].left, p[0].right, p[1].left, p[1].right) == (1, 1, 0, 0)
    with pytest.raises(ValueError):
        decomp.Slab(case, 0, 11, 0)
    # a width that no span of 6 float64 cells reproduces exactly is refused
    with pytest.raises(ValueError):
        decomp.exact_span(0.35, 0.05, 6)
