"""Exact solution of the 1D Riemann problem between two stiffened gases.

Test infrastructure (part of the oracle).  Each side K has its own
(gamma_K, pi_K); with p + pi_K in place of p every stiffened-gas wave obeys
the ideal-gas relations (Menikoff & Plohr, cited for the EOS in Sec. 2.2;
Toro's exact solver, cited in Sec. 3.2.2).  Across a shock the Rankine-
Hugoniot conditions hold, across a rarefaction the isentrope and the
Riemann invariant, and across the contact the pressure and the velocity are
continuous; `check_waves` evaluates those residuals.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.optimize import brentq


@dataclass
class Side:
    rho: float
    u: float
    p: float
    gamma: float
    pi: float

    @property
    def c(self) -> float:
        return math.sqrt(self.gamma * (self.p + self.pi) / self.rho)


def _f(s: Side, pstar: float):
    """Velocity change across the left/right wave for star pressure pstar."""
    g, P, Ps = s.gamma, s.p + s.pi, pstar + s.pi
    if Ps > P:  # shock
        A = 2.0 / ((g + 1.0) * s.rho)
        B = (g - 1.0) / (g + 1.0) * P
        return (Ps - P) * math.sqrt(A / (Ps + B))
    return 2.0 * s.c / (g - 1.0) * ((Ps / P) ** ((g - 1.0) / (2.0 * g)) - 1.0)


def star_state(L: Side, R: Side):
    """(p*, u*) of the Riemann problem."""
    def F(ps):
        return _f(L, ps) + _f(R, ps) + (R.u - L.u)
    lo = -min(L.pi, R.pi) + 1e-12 * max(1.0, L.p + L.pi, R.p + R.pi)
    hi = max(L.p + L.pi, R.p + R.pi) * 10.0 + 1.0
    while F(hi) < 0:
        hi *= 10.0
    if F(lo) > 0:
        raise ValueError("vacuum generated")
    ps = brentq(F, lo, hi, xtol=1e-16 * hi, rtol=1e-15, maxiter=500)
    us = 0.5 * (L.u + R.u) + 0.5 * (_f(R, ps) - _f(L, ps))
    return ps, us


def _star_density(s: Side, ps: float) -> float:
    g, P, Ps = s.gamma, s.p + s.pi, ps + s.pi
    if Ps > P:
        r = (g - 1.0) / (g + 1.0)
        return s.rho * (Ps / P + r) / (r * Ps / P + 1.0)
    return s.rho * (Ps / P) ** (1.0 / g)


def sample(L: Side, R: Side, xi: np.ndarray):
    """(rho, u, p, side) at similarity coordinates xi = (x - x0)/t; side = 0
    where the left material is present, 1 for the right one."""
    ps, us = star_state(L, R)
    rho = np.empty_like(xi); u = np.empty_like(xi); p = np.empty_like(xi); side = np.empty(xi.shape, int)
    for n, x in enumerate(xi):
        if x <= us:
            s, sgn, side[n] = L, -1.0, 0
        else:
            s, sgn, side[n] = R, 1.0, 1
        g, P, Ps = s.gamma, s.p + s.pi, ps + s.pi
        if Ps > P:  # shock on this side
            r = (g - 1.0) / (g + 1.0)
            S = s.u + sgn * s.c * math.sqrt((g + 1.0) / (2 * g) * Ps / P + (g - 1.0) / (2 * g))
            outside = x < S if sgn < 0 else x > S
            if outside:
                rho[n], u[n], p[n] = s.rho, s.u, s.p
            else:
                rho[n], u[n], p[n] = _star_density(s, ps), us, ps
        else:  # rarefaction
            cs = s.c * (Ps / P) ** ((g - 1.0) / (2 * g))
            head = s.u + sgn * s.c
            tail = us + sgn * cs
            if (sgn < 0 and x < head) or (sgn > 0 and x > head):
                rho[n], u[n], p[n] = s.rho, s.u, s.p
            elif (sgn < 0 and x > tail) or (sgn > 0 and x < tail):
                rho[n], u[n], p[n] = _star_density(s, ps), us, ps
            else:
                uu = 2.0 / (g + 1.0) * (-sgn * s.c + (g - 1.0) / 2.0 * s.u + x)
                cc = -sgn * (uu - x)
                rho[n] = s.rho * (cc / s.c) ** (2.0 / (g - 1.0))
                u[n] = uu
                p[n] = (s.p + s.pi) * (cc / s.c) ** (2.0 * g / (g - 1.0)) - s.pi
    return rho, u, p, side


def check_waves(L: Side, R: Side) -> dict:
    """Residuals of the jump / invariant conditions the exact solution must
    satisfy (relative).  Keys: rh_mass, rh_mom, rh_energy (max over shocks),
    isentrope, invariant (max over rarefactions)."""
    ps, us = star_state(L, R)
    out = {"rh_mass": 0.0, "rh_mom": 0.0, "rh_energy": 0.0, "isentrope": 0.0, "invariant": 0.0}
    for s, sgn in ((L, -1.0), (R, 1.0)):
        g, P, Ps = s.gamma, s.p + s.pi, ps + s.pi
        rs = _star_density(s, ps)
        if Ps > P:
            S = s.u + sgn * s.c * math.sqrt((g + 1.0) / (2 * g) * Ps / P + (g - 1.0) / (2 * g))

            def e(rho, p):  # specific internal energy of the stiffened gas
                return (p + g * s.pi) / ((g - 1.0) * rho)
            m1 = s.rho * (s.u - S); m2 = rs * (us - S)
            out["rh_mass"] = max(out["rh_mass"], abs(m1 - m2) / abs(m1))
            f1 = m1 * (s.u - S) + s.p; f2 = m2 * (us - S) + ps
            out["rh_mom"] = max(out["rh_mom"], abs(f1 - f2) / max(abs(f1), abs(f2)))
            h1 = e(s.rho, s.p) + s.p / s.rho + 0.5 * (s.u - S) ** 2
            h2 = e(rs, ps) + ps / rs + 0.5 * (us - S) ** 2
            out["rh_energy"] = max(out["rh_energy"], abs(h1 - h2) / abs(h1))
        else:
            k1 = P / s.rho ** g; k2 = Ps / rs ** g
            out["isentrope"] = max(out["isentrope"], abs(k1 - k2) / k1)
            cs = math.sqrt(g * Ps / rs)
            j1 = s.u - sgn * 2 * s.c / (g - 1.0); j2 = us - sgn * 2 * cs / (g - 1.0)
            out["invariant"] = max(out["invariant"], abs(j1 - j2) / max(abs(j1), s.c))
    return out


def cell_averages(L: Side, R: Side, x0: float, t: float, n: int, sub: int = 64):
    """Cell averages of (rho, u, p, side-fraction) on n cells of [0, 1] at
    time t (midpoint sub-sampling of each cell; u and p averaged as point
    values)."""
    h = 1.0 / n
    xs = (np.arange(n * sub) + 0.5) * (h / sub)
    rho, u, p, side = sample(L, R, (xs - x0) / t)
    f = lambda a: a.reshape(n, sub).mean(axis=1)
    return f(rho), f(u), f(p), f(side.astype(float))
