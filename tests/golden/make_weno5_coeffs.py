"""Derive the WENO5 constants from the paper's generic construction.

Sec. 4.2.2 builds each k-cell candidate polynomial from cell averages by
Lagrange interpolation of the primitive function,

    p(x) = sum_j c_j(x) f_j,
    c_j(x) = dx_j sum_{m=j+1}^{k} [sum_{l != m} prod_{q != m, l} (x - x_{q-1/2})]
                                / prod_{l != m} (x_{m-1/2} - x_{l-1/2}),

rewrites it as p(x) = f_0 + sum_j chat_j(x) Delta f_j with Delta f_j =
f_{j+1} - f_j, evaluates the right flux of stencil r at x_{k-r-1/2}, and
writes the smoothness indicator
    beta_r = sum_{l=1}^{k-1} dx^{2l-1} int over the centre cell (p^(l))^2
as sum_{j <= m} bhat_{r,j,m} Delta f_j Delta f_m.

This script evaluates those formulas exactly (rational arithmetic) for k = 3
on a uniform grid (dx = 1, stencil boundaries x_{q-1/2} = q) and also finds
the ideal weights d_r that make sum_r d_r p_r equal the value of the
(2k-1)-cell polynomial at the same edge.  It writes weno5_coeffs.txt; the
same edge quantities are given for the left edge of the centre cell (the
mirror used for the right state of a face).  It uses no oracle code.
"""
from __future__ import annotations

import os
from fractions import Fraction as Fr

K = 3


def padd(a, b):
    n = max(len(a), len(b))
    return [(a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0) for i in range(n)]


def pscale(a, s):
    return [s * x for x in a]


def pmul(a, b):
    out = [Fr(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def pderiv(a):
    return [i * a[i] for i in range(1, len(a))] or [Fr(0)]


def peval(a, x):
    return sum(c * x ** i for i, c in enumerate(a))


def pint(a, lo, hi):
    return sum(c * (Fr(hi) ** (i + 1) - Fr(lo) ** (i + 1)) / (i + 1) for i, c in enumerate(a))


def lagrange_cell_weights(k: int):
    """c_j(x), j = 0..k-1, for k cells with boundaries 0..k (dx = 1)."""
    xb = [Fr(q) for q in range(k + 1)]
    cs = []
    for j in range(k):
        cj = [Fr(0)]
        for m in range(j + 1, k + 1):
            num = [Fr(0)]
            for l in range(k + 1):
                if l == m:
                    continue
                term = [Fr(1)]
                for q in range(k + 1):
                    if q in (m, l):
                        continue
                    term = pmul(term, [-xb[q], Fr(1)])
                num = padd(num, term)
            den = Fr(1)
            for l in range(k + 1):
                if l != m:
                    den *= xb[m] - xb[l]
            cj = padd(cj, pscale(num, 1 / den))
        cs.append(cj)
    return cs


def derive(k: int = K):
    c = lagrange_cell_weights(k)
    # chat_i(x) = sum_{j > i} c_j(x)
    chat = []
    for i in range(k - 1):
        acc = [Fr(0)]
        for j in range(i + 1, k):
            acc = padd(acc, c[j])
        chat.append(acc)
    res = {}
    for r in range(k):
        right = Fr(k - r)           # x_{k-r-1/2}
        left = Fr(k - r - 1)        # left edge of the centre cell
        res[("chat_right", r)] = [peval(chat[j], right) for j in range(k - 1)]
        res[("chat_left", r)] = [peval(chat[j], left) for j in range(k - 1)]
        b = {}
        for j in range(k - 1):
            for m in range(j, k - 1):
                s = Fr(0)
                dj, dm = chat[j], chat[m]
                for l in range(1, k):
                    dj = pderiv(dj)
                    dm = pderiv(dm)
                    s += pint(pmul(dj, dm), k - r - 1, k - r)  # dx^(2l-1) = 1
                b[(j, m)] = (2 if j != m else 1) * s
        res[("bhat", r)] = b
    # ideal weights: the (2k-1)-cell polynomial's edge value equals sum d_r p_r
    big = lagrange_cell_weights(2 * k - 1)  # cells 0..4, centre cell k-1
    for edge, x in (("right", Fr(k)), ("left", Fr(k - 1))):
        target = [peval(big[i], x) for i in range(2 * k - 1)]
        # stencil r covers big-cells (k-1-r) .. (2k-2-r) ... in the oracle's
        # ordering, stencil r = {c-2+r .. c+r}, i.e. big cells r .. r+k-1,
        # whose centre cell (big index k-1) is local cell k-1-r.
        xs = {}
        for r in range(k):
            cl = lagrange_cell_weights(k)
            xloc = x - r  # shift big coordinates to the stencil's local ones
            xs[r] = [peval(cl[j], xloc) for j in range(k)]
        # unknown d_0..d_{k-1}: sum_r d_r xs[r][i - r] = target[i]
        rows = []
        for i in range(2 * k - 1):
            rows.append([xs[r][i - r] if 0 <= i - r < k else Fr(0) for r in range(k)] + [target[i]])
        d = solve_least(rows, k)
        res[("d", edge)] = d
    return res


def solve_least(rows, n):
    """Solve the consistent overdetermined rational system by elimination."""
    A = [list(r) for r in rows]
    piv_rows = []
    col = 0
    for col in range(n):
        p = next(i for i in range(len(A)) if i not in piv_rows and A[i][col] != 0)
        piv_rows.append(p)
        for i in range(len(A)):
            if i != p and A[i][col] != 0:
                f = A[i][col] / A[p][col]
                A[i] = [a - f * b for a, b in zip(A[i], A[p])]
    for i in range(len(A)):
        if i not in piv_rows:
            assert all(x == 0 for x in A[i]), "inconsistent ideal-weight system"
    return [A[piv_rows[c]][n] / A[piv_rows[c]][c] for c in range(n)]


def write(path: str):
    res = derive()
    lines = ["# WENO5 (k = 3) constants on a uniform grid, evaluated exactly from the",
             "# generic Lagrange / Delta-f construction of Sec. 4.2.2 (p_r = f_0 + sum_j",
             "# chat_{r,j} Delta f_j over stencil r's own cells; beta_r = sum_{j<=m}",
             "# bhat_{r,j,m} Delta f_j Delta f_m; d = ideal weights).  Stencil r holds",
             "# cells c-2+r .. c+r of the five-cell stencil around centre cell c.",
             "# Written by make_weno5_coeffs.py."]
    for r in range(K):
        lines.append(f"chat_right {r} " + " ".join(str(x) for x in res[("chat_right", r)]))
        lines.append(f"chat_left {r} " + " ".join(str(x) for x in res[("chat_left", r)]))
        b = res[("bhat", r)]
        lines.append(f"bhat {r} " + " ".join(f"{j}{m}:{b[(j, m)]}" for (j, m) in sorted(b)))
    for edge in ("right", "left"):
        lines.append(f"d_{edge} " + " ".join(str(x) for x in res[("d", edge)]))
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    write(os.path.join(os.path.dirname(os.path.abspath(__file__)), "weno5_coeffs.txt"))
