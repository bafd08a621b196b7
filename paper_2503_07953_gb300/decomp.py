"""Slab domain decomposition with one halo exchange per Runge-Kutta stage.

The method shards by splitting the grid into subdomains, each advanced by
its own GPU, with the cells within the stencil's reach of a neighbour
(three, for WENO5) exchanged before every evaluation of L, and the CFL time
step reduced to its minimum over the subdomains once per step (the paper's
scaling runs decompose the grid into uniformly sized chunks, one per rank,
that exchange only a small halo region around themselves; Sec. 4.3,
exascale capabilities).  Here the grid is cut along one axis into slabs:

* ``Slab`` describes rank r's slab of a case: its cells, its grid (the
  global cell width exactly, so that every face sees the same dx), and its
  sides.  A side on the cut is ``MFC_BC_HALO`` (the neighbour's cells sit in
  the ghost layer, which the library reads); the ends of the axis keep the
  case's boundary conditions, except that a periodic axis wraps: the last
  slab is the first one's left neighbour.
* ``HaloExchange`` refreshes the ghost layers of one state on the cut sides:
  each side receives the neighbour's three layers nearest to it.  Its
  transport is ``torch.distributed`` point-to-point (gloo on CPU, NCCL
  between GPUs; each rank sends into the neighbour's own memory and the
  kernels read only local memory) or, for several slabs in one process,
  direct copies between their tensors (``LocalSlabs``).
* ``rk3_step`` advances one step: dt = CFL minimum over all slabs (the
  same value as the undivided grid's, since a minimum does not depend on
  the order of its terms), then the three stages, each after the halo
  exchange of its input.  Every cell then goes through the same arithmetic
  as in the undivided grid, so the decomposed run equals it bit for bit.

A stepper is anything with the ``Solver`` methods this module calls:
``ghost``, ``shape``, ``empty()``, ``compute_dt(q)`` and
``rk3_stage(stage, q_in, q_n, q_out, dt)``.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Optional, Sequence

import torch

BC_PERIODIC, BC_TRANSMISSIVE, BC_REFLECTIVE, BC_HALO = 0, 1, 2, 3


def exact_span(lo: float, dx: float, n: int) -> tuple:
    """(lo', hi') with (hi' - lo') / n == dx in float64, so that a slab's
    cell width is the global one bit for bit (the kernels use only the cell
    width of a grid, not its position).  Tries spans starting at lo, then at
    0 (where the steps of hi' / n are finest), nudging hi' by ulps around
    lo' + n dx; raises ValueError when no span gives dx exactly (a cell
    width that is a power of two always has one)."""
    for start in (lo, 0.0):
        hi0 = torch.tensor(start + n * dx, dtype=torch.float64)
        up = torch.tensor(float("inf"), dtype=torch.float64)
        down = torch.tensor(-float("inf"), dtype=torch.float64)
        cands = [hi0]
        a, b = hi0, hi0
        for _ in range(32):
            a, b = torch.nextafter(a, up), torch.nextafter(b, down)
            cands += [a, b]
        for hi in cands:
            if (float(hi) - start) / n == dx:
                return start, float(hi)
    raise ValueError(f"no float64 span of {n} cells has the cell width {dx!r} exactly")


@dataclasses.dataclass
class Slab:
    """Rank `rank`'s slab of `case` cut along `axis` into `world` slabs (as
    equal as possible; the first n mod world slabs have one cell more)."""
    case: object
    axis: int
    world: int
    rank: int

    def __post_init__(self):
        n = self.case.n[self.axis]
        if not 0 <= self.rank < self.world or self.world > n:
            raise ValueError("need 0 <= rank < world <= cells along the axis")
        base, rem = divmod(n, self.world)
        self.sizes = [base + (1 if r < rem else 0) for r in range(self.world)]
        self.offset = sum(self.sizes[:self.rank])
        self.n_local = self.sizes[self.rank]
        periodic = self.case.bc_lo[self.axis] == BC_PERIODIC
        last = self.world - 1
        self.left = self.rank - 1 if self.rank > 0 else (last if periodic else None)
        self.right = self.rank + 1 if self.rank < last else (0 if periodic else None)

    def local_case(self):
        """The slab as a case of its own: its cells, the global cell width
        (its span along the cut axis from exact_span), halo sides on the cut
        (and on both ends of a periodic axis)."""
        c, a = self.case, self.axis
        dx = c.dx(a)
        n = list(c.n)
        lo, hi = list(c.lo), list(c.hi)
        bl, bh = list(c.bc_lo), list(c.bc_hi)
        n[a] = self.n_local
        lo[a], hi[a] = exact_span(c.lo[a] + self.offset * dx, dx, self.n_local)
        bl[a] = BC_HALO if self.left is not None else c.bc_lo[a]
        bh[a] = BC_HALO if self.right is not None else c.bc_hi[a]
        return dataclasses.replace(c, name=f"{c.name}[slab {self.rank}/{self.world} along axis {a}]", n=n, lo=lo,
                                   hi=hi, bc_lo=bl, bc_hi=bh)

    def dim(self) -> int:
        """Tensor dimension of the cut axis in a [field][z][y][x] array."""
        return 3 - self.axis

    def take(self, interior):
        """This slab's cells of a whole-grid interior array [field][z][y][x]."""
        d = self.dim()
        idx = [slice(None)] * 4
        idx[d] = slice(self.offset, self.offset + self.n_local)
        return interior[tuple(idx)]


def _layers(q: torch.Tensor, slab: Slab, ghost: int):
    """(send_left, send_right, ghost_left, ghost_right) views of a padded
    state: the slab's first and last `ghost` interior layers along the cut
    axis, and its two ghost layers there."""
    d, g, n = slab.dim(), ghost, slab.n_local
    return q.narrow(d, g, g), q.narrow(d, n, g), q.narrow(d, 0, g), q.narrow(d, g + n, g)


class HaloExchange:
    """Halo exchange of one rank's slab through torch.distributed
    (point-to-point sends and receives, posted together)."""

    def __init__(self, slab: Slab, ghost: int, group=None):
        if ghost < 3:
            raise ValueError("a halo exchange needs ghost >= 3")
        self.slab, self.ghost, self.group = slab, ghost, group

    def __call__(self, q: torch.Tensor) -> None:
        import torch.distributed as dist
        s = self.slab
        send_l, send_r, gh_l, gh_r = _layers(q, s, self.ghost)
        if s.left is not None and s.left == s.rank:  # one periodic slab: its own wrap
            gh_l.copy_(send_r)
            gh_r.copy_(send_l)
            return
        # messages travel east (a slab's last layers into its right
        # neighbour's left ghost) or west; every rank posts its sends east,
        # west, then its receives from the west and from the east, so that
        # two slabs that are each other's neighbours on both sides (a
        # periodic axis cut in two) match their messages in order, tags or no
        EAST, WEST = 0, 1
        ops, recvs = [], []
        rank_of = (lambda r: dist.get_global_rank(self.group, r)) if self.group is not None else (lambda r: r)
        if s.right is not None:
            ops.append(dist.P2POp(dist.isend, send_r.contiguous(), rank_of(s.right), self.group, tag=EAST))
        if s.left is not None:
            ops.append(dist.P2POp(dist.isend, send_l.contiguous(), rank_of(s.left), self.group, tag=WEST))
        if s.left is not None:
            buf = torch.empty_like(gh_l, memory_format=torch.contiguous_format)
            ops.append(dist.P2POp(dist.irecv, buf, rank_of(s.left), self.group, tag=EAST))
            recvs.append((gh_l, buf))
        if s.right is not None:
            buf = torch.empty_like(gh_r, memory_format=torch.contiguous_format)
            ops.append(dist.P2POp(dist.irecv, buf, rank_of(s.right), self.group, tag=WEST))
            recvs.append((gh_r, buf))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        for dst, buf in recvs:
            dst.copy_(buf)


def allreduce_min(x: float, group=None, device=None) -> float:
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
    return float(t.item())


def rk3_step(stepper, q: torch.Tensor, scratch: Sequence[torch.Tensor], exchange: Callable[[torch.Tensor], None],
             reduce_min: Callable[[float], float], dt: float = 0.0) -> float:
    """One RK3 step of one slab in place: dt (the CFL minimum over every
    slab when dt <= 0), then stage s on the halo-exchanged input of stage s.
    scratch: two states of the stepper's shape.  Returns the dt taken."""
    q1, q2 = scratch
    if dt <= 0.0:
        dt = reduce_min(stepper.compute_dt(q))
    exchange(q)
    stepper.rk3_stage(1, q, None, q1, dt)
    exchange(q1)
    stepper.rk3_stage(2, q1, q, q2, dt)
    exchange(q2)
    stepper.rk3_stage(3, q2, q, q, dt)
    return dt


class LocalSlabs:
    """All slabs of a decomposition in one process (one stepper each, run
    one after the other): the halo exchange copies between their tensors and
    the dt reduction is a plain minimum.  The same arithmetic as one slab per
    process; used to check a decomposition on one device."""

    def __init__(self, case, axis: int, world: int, make_stepper: Callable):
        self.slabs = [Slab(case, axis, world, r) for r in range(world)]
        self.steppers = [make_stepper(s.local_case()) for s in self.slabs]
        self.ghost = self.steppers[0].ghost
        if self.ghost < 3:
            raise ValueError("a halo exchange needs ghost >= 3")

    def exchange(self, qs: List[torch.Tensor]) -> None:
        views = [_layers(q, s, self.ghost) for q, s in zip(qs, self.slabs)]
        for r, s in enumerate(self.slabs):
            if s.left is not None:
                views[r][2].copy_(views[s.left][1])
            if s.right is not None:
                views[r][3].copy_(views[s.right][0])

    def scatter(self, interior) -> List[torch.Tensor]:
        """Padded per-slab states from a whole-grid interior array."""
        return [st.from_interior(s.take(interior)) for st, s in zip(self.steppers, self.slabs)]

    def gather(self, qs: List[torch.Tensor]) -> torch.Tensor:
        """The whole-grid interior array of the slabs' states."""
        parts = [st.interior(q) for st, q in zip(self.steppers, qs)]
        return torch.cat([p.cpu() for p in parts], dim=self.slabs[0].dim())

    def step(self, qs: List[torch.Tensor], scratch: List[Sequence[torch.Tensor]], dt: float = 0.0) -> float:
        """One RK3 step of every slab (the stages in lock step across slabs)."""
        if dt <= 0.0:
            dt = min(st.compute_dt(q) for st, q in zip(self.steppers, qs))
        ins = list(qs)
        for stage in (1, 2, 3):
            self.exchange(ins)
            outs = []
            for st, q, sc, x in zip(self.steppers, qs, scratch, ins):
                out = q if stage == 3 else sc[stage - 1]
                st.rk3_stage(stage, x, None if stage == 1 else q, out, dt)
                outs.append(out)
            ins = outs
        return dt
