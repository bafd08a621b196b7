"""Binomial checkpointing (paper_2503_07953_gb300.checkpoint) on a small
nonlinear recurrence whose gradient is computed directly by storing every
state."""
import numpy as np
import pytest

from paper_2503_07953_gb300 import checkpoint as ck


def make_problem(n=8, steps=30, seed=0):
    rng = np.random.default_rng(seed)
    A = [rng.normal(size=(n, n)) / np.sqrt(n) for _ in range(steps)]
    wts = rng.normal(size=(steps, n))

    def advance(q, k):
        return np.tanh(A[k] @ q)

    def vjp(q, k, bar):
        z = A[k] @ q
        return A[k].T @ ((1 - np.tanh(z) ** 2) * bar)

    def loss(k, q):
        return 0.5 * float(wts[k] @ (q * q))

    def loss_grad(k, q):
        return wts[k] * q

    return advance, vjp, loss, loss_grad, rng.normal(size=n)


def direct_gradient(q0, steps, advance, vjp, loss, loss_grad):
    qs = [q0]
    for k in range(steps):
        qs.append(advance(qs[-1], k))
    J = sum(loss(k, qs[k + 1]) for k in range(steps))
    lam = loss_grad(steps - 1, qs[steps])
    for k in range(steps - 1, -1, -1):
        lam = vjp(qs[k], k, lam)
        if k >= 1:
            lam = lam + loss_grad(k - 1, qs[k])
    return J, lam


@pytest.mark.parametrize("steps,snaps", [(1, 0), (2, 1), (7, 0), (30, 1), (30, 3), (30, 10), (30, 40), (57, 5)])
def test_gradient_equals_store_all(steps, snaps):
    advance, vjp, loss, loss_grad, q0 = make_problem(steps=max(steps, 1))
    J, g, stats = ck.rollout_gradient(q0, steps, advance, vjp, loss, loss_grad, np.copy, snaps)
    J0, g0 = direct_gradient(q0, steps, advance, vjp, loss, loss_grad)
    assert J == pytest.approx(J0, rel=1e-13)
    np.testing.assert_allclose(g, g0, rtol=1e-12, atol=1e-14)
    assert stats.vjps == steps
    assert stats.max_live_snapshots <= snaps
    assert stats.advances == ck.recompute_count(steps, snaps)


def test_gradient_matches_finite_differences():
    steps = 25
    advance, vjp, loss, loss_grad, q0 = make_problem(steps=steps, seed=3)
    _, g, _ = ck.rollout_gradient(q0, steps, advance, vjp, loss, loss_grad, np.copy, 4)
    d = np.random.default_rng(1).normal(size=q0.shape)
    h = 1e-6

    def J(q):
        tot = 0.0
        for k in range(steps):
            q = advance(q, k)
            tot += loss(k, q)
        return tot
    fd = (J(q0 + h * d) - J(q0 - h * d)) / (2 * h)
    assert float(g @ d) == pytest.approx(fd, rel=1e-7)


def test_binomial_counts():
    """With no slot each state is recomputed from the start, s (s - 1) / 2
    steps; with s - 1 slots every state is computed once; more slots never
    cost more; and the binomial schedule beats the best single level of
    equally spaced checkpoints (a sqrt-style scheme)."""
    for s in (1, 2, 5, 17, 40):
        assert ck.recompute_count(s, 0) == s * (s - 1) // 2
        assert ck.recompute_count(s, max(s - 1, 0)) == max(s - 1, 0)
    prev = None
    for c in range(0, 12):
        r = ck.recompute_count(500, c)
        if prev is not None:
            assert r <= prev
        prev = r
    for s, c in ((500, 10), (200, 4), (64, 3)):
        # equally spaced: k segments of length L = ceil(s / k), k - 1 <= c checkpoints,
        # each segment reversed from its start with no further slot
        best = None
        for k in range(1, c + 2):
            L = -(-s // k)
            cost = (k - 1) * L + k * L * (L - 1) // 2
            best = cost if best is None else min(best, cost)
        assert ck.recompute_count(s, c) <= best
