"""Adjoints of long RK3 rollouts with binomial checkpointing.

For J = sum_{n=0}^{N-1} l_n(q^{n+1}) with q^{n+1} = step_n(q^n) (fixed dt
per step), the adjoint recursion is

    lam^N = dl_{N-1}/dq^N
    lam^n = (d step_n / d q^n)^T lam^{n+1} + dl_{n-1}/dq^n     (n >= 1)
    dJ/dq^0 = (d step_0 / d q^0)^T lam^1.

Reversing step n needs q^n.  Storing every state costs N states; with c
snapshot slots the states are recomputed from stored ones.  The schedule
here is the binomial one (Griewank): reversing s steps from a stored state
with c free slots, advance m steps, store that state, reverse the last
s - m steps with c - 1 slots, then the first m steps with c slots, with m
minimising the total number of recomputed steps
    F(s, c) = min_m [m + F(s - m, c - 1) + F(m, c)],
    F(1, c) = 0,   F(s, 0) = s (s - 1) / 2.
F and the optimal m are tabulated once per (N, c).

The functions are generic over the state type: `advance(q, n)` returns
step_n(q) as a new state, `vjp(q, n, bar)` returns (d step_n/dq)^T bar at
q = q^n, `loss_grad(n, q)` returns dl_n/dq at q = q^{n+1} (or None), and
`clone(q)` copies a state.  paper_2503_07953_gb300.adjoint binds them to
the CUDA library.
"""
from __future__ import annotations

from functools import lru_cache
from typing import Callable, List, Optional, Tuple

import numpy as np


@lru_cache(maxsize=32)
def binomial_table(nsteps: int, snaps: int) -> Tuple[np.ndarray, np.ndarray]:
    """F[c, s] (recomputed steps) and M[c, s] (optimal first advance) for
    s <= nsteps, c <= snaps."""
    S, C = nsteps, snaps
    F = np.zeros((C + 1, S + 1), dtype=np.int64)
    M = np.zeros((C + 1, S + 1), dtype=np.int64)
    s = np.arange(S + 1, dtype=np.int64)
    F[0] = s * (s - 1) // 2
    F[0, 0] = 0
    for c in range(1, C + 1):
        F[c, :2] = 0
        for n in range(2, S + 1):
            m = np.arange(1, n)
            cost = m + F[c - 1, n - m] + F[c, m]
            k = int(np.argmin(cost))
            F[c, n] = cost[k]
            M[c, n] = m[k]
    return F, M


def recompute_count(nsteps: int, snaps: int) -> int:
    """Forward steps recomputed by the binomial schedule (the forward sweep
    that evaluates J is not included)."""
    if nsteps <= 1:
        return 0
    F, _ = binomial_table(nsteps, snaps)
    return int(F[snaps, nsteps])


class Stats:
    def __init__(self):
        self.advances = 0
        self.vjps = 0
        self.max_live_snapshots = 0
        self._live = 0

    def hold(self, k: int):
        self._live += k
        self.max_live_snapshots = max(self.max_live_snapshots, self._live)


def reverse(q0, nsteps: int, lam_end, advance: Callable, vjp: Callable, loss_grad: Optional[Callable],
            clone: Callable, snaps: int, stats: Optional[Stats] = None):
    """dJ/dq^0 given q^0 and lam^N (= dl_{N-1}/dq^N), with at most `snaps`
    intermediate states held at any time."""
    stats = stats if stats is not None else Stats()
    _, M = binomial_table(max(nsteps, 1), max(snaps, 0))

    def rev(qa, a: int, b: int, c: int, lam):
        # reverse steps b-1 .. a given q^a; lam = lam^b on entry, lam^a on exit
        s = b - a
        if s == 1:
            lam = vjp(qa, a, lam)
            stats.vjps += 1
            if a >= 1 and loss_grad is not None:
                g = loss_grad(a - 1, qa)
                if g is not None:
                    lam = lam + g
            return lam
        if c == 0:
            # no free slot: recompute each state from q^a
            for k in range(b - 1, a - 1, -1):
                qk = clone(qa)
                for n in range(a, k):
                    qk = advance(qk, n)
                    stats.advances += 1
                lam = rev(qk, k, k + 1, 0, lam)
            return lam
        m = int(M[c, s])
        qm = clone(qa)
        for n in range(a, a + m):
            qm = advance(qm, n)
            stats.advances += 1
        stats.hold(1)
        lam = rev(qm, a + m, b, c - 1, lam)
        del qm
        stats.hold(-1)
        return rev(qa, a, a + m, c, lam)

    if nsteps == 0:
        return lam_end
    return rev(q0, 0, nsteps, snaps, lam_end)


def rollout_gradient(q0, nsteps: int, advance: Callable, vjp: Callable, loss: Callable, loss_grad: Callable,
                     clone: Callable, snaps: int) -> Tuple[float, object, Stats]:
    """J = sum_n loss(n, q^{n+1}) and dJ/dq^0 with binomial checkpointing.
    The forward sweep keeps only the current state."""
    stats = Stats()
    J = 0.0
    q = clone(q0)
    for n in range(nsteps):
        q = advance(q, n)
        J += float(loss(n, q))
    lam = loss_grad(nsteps - 1, q)
    g = reverse(q0, nsteps, lam, advance, vjp, loss_grad, clone, snaps, stats)
    return J, g, stats
