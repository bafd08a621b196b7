"""Seeded synthetic inputs shaped like the paper's workloads.

This module only *defines inputs*: grids, boundary conditions, fluid
parameters and initial primitive fields.  It holds none of the method's
arithmetic (no EOS inversion, reconstruction, Riemann solve or time
stepping); converting the primitive fields to conservative variables is done
separately by each side (the oracle and the CUDA library).

Primitive fields are returned as float64 arrays shaped
``(n_fields, nz, ny, nx)`` with the slot order
``alpha_1 rho_1 .. alpha_N rho_N, u_1 .. u_ndim, p, alpha_1 .. alpha_{N-1}``.

Random numbers come from ``torch.Generator`` on the CPU with explicit seeds,
so every size and device sees the same values.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np
import torch

PERIODIC, TRANSMISSIVE, REFLECTIVE = 0, 1, 2
WENO_JS, WENO_M, WENO_Z, WENO_TENO = 0, 1, 2, 3


@dataclass
class Case:
    """A grid, its boundary conditions, the fluids and the run settings."""
    name: str
    n: List[int]
    lo: List[float]
    hi: List[float]
    bc_lo: List[int]
    bc_hi: List[int]
    gamma: List[float]
    pi_inf: List[float]
    cfl: float
    steps: int
    weno: int = WENO_M
    eps: float = 1e-40
    teno_ct: float = 1e-6     # TENO threshold C_T (weno = 3)
    model: int = 0            # 0: K = 0 (Allaire); 1: Kapila K div u (two fluids)
    riemann: int = 0          # 0: HLLC; 1: HLL
    low_mach: int = 0         # 0: none; 1: Thornber; 2: anti-dissipation pressure correction (HLLC)
    eta: Optional[List[float]] = None  # shear viscosity per fluid (Sec. 2.1.1); None: inviscid
    viscous_dt: bool = False  # the CFL dt also respects the explicit viscous limit

    @property
    def ndim(self) -> int:
        return len(self.n)

    @property
    def nf(self) -> int:
        return len(self.gamma)

    @property
    def nq(self) -> int:
        return 2 * self.nf + self.ndim

    @property
    def ncells(self) -> int:
        return int(np.prod(self.n))

    @property
    def shape(self):
        n3 = list(self.n) + [1] * (3 - self.ndim)
        return (self.nq, n3[2], n3[1], n3[0])

    def dx(self, a: int) -> float:
        return (self.hi[a] - self.lo[a]) / self.n[a]


def reduced_units(case: Case, W: np.ndarray, rho0: float, p0: float) -> tuple:
    """The same flow in reduced units: densities over rho0, pressures and
    pi_inf over p0, velocities over u0 = sqrt(p0 / rho0) (lengths unchanged,
    so times scale by u0; viscosities over rho0 u0).  The equations with the
    stiffened-gas EOS are invariant under this change of units; the WENO
    eps, an absolute constant, is not, and in reduced units it sits far
    above the rounding size of the smoothness indicators of O(1) fields.
    Returns a new (case, W)."""
    u0 = math.sqrt(p0 / rho0)
    nf, nd = case.nf, case.ndim
    W = np.array(W, dtype=np.float64, copy=True)
    W[:nf] /= rho0
    W[nf:nf + nd] /= u0
    W[nf + nd] /= p0
    out = Case(case.name, list(case.n), list(case.lo), list(case.hi), list(case.bc_lo), list(case.bc_hi),
               list(case.gamma), [x / p0 for x in case.pi_inf], case.cfl, case.steps, case.weno, case.eps,
               case.teno_ct, case.model, case.riemann, case.low_mach,
               None if case.eta is None else [x / (rho0 * u0) for x in case.eta])
    return out, W


def _centres(case: Case):
    """Cell-centre coordinate arrays broadcastable to (nz, ny, nx)."""
    n3 = list(case.n) + [1] * (3 - case.ndim)
    xs = []
    for a in range(3):
        if a < case.ndim:
            h = case.dx(a)
            xs.append(case.lo[a] + (np.arange(n3[a]) + 0.5) * h)
        else:
            xs.append(np.zeros(1))
    X = xs[0][None, None, :]
    Y = xs[1][None, :, None]
    Z = xs[2][:, None, None]
    return X, Y, Z


def _uniform(seed: int, shape, lo=-1.0, hi=1.0) -> np.ndarray:
    g = torch.Generator().manual_seed(seed)
    return (lo + (hi - lo) * torch.rand(shape, generator=g, dtype=torch.float64)).numpy()


def _assemble(case: Case, alpha: Sequence[np.ndarray], rho_phase: Sequence[np.ndarray],
              vel: Sequence[np.ndarray], p: np.ndarray) -> np.ndarray:
    """Stack alpha_i * rho_i, u_d, p, alpha_j into the primitive slot order."""
    shp = case.shape[1:]
    W = np.empty(case.shape, dtype=np.float64)
    nf, nd = case.nf, case.ndim
    for i in range(nf):
        W[i] = np.broadcast_to(alpha[i] * rho_phase[i], shp)
    for d in range(nd):
        W[nf + d] = np.broadcast_to(vel[d], shp)
    W[nf + nd] = np.broadcast_to(p, shp)
    for j in range(nf - 1):
        W[nf + nd + 1 + j] = np.broadcast_to(alpha[j], shp)
    return W


# ---------------------------------------------------------------------------
# The paper-shaped workloads
# ---------------------------------------------------------------------------

WATER = (4.4, 6.0e8)
AIR = (1.4, 0.0)


def water_air_shock_tube(n: int = 1000, steps: int = 200) -> tuple:
    """1D two-fluid shock tube: water (rho 1000, p 1e9) left of x = 0.7 with
    alpha_water = 1 - 1e-6, air (rho 50, p 1e5) right of it with
    alpha_water = 1e-6; u = 0; transmissive ends; CFL 0.3.  Both phasic
    densities are kept in both halves (water 1000, air 50)."""
    case = Case("water_air_1d", [n], [0.0], [1.0], [TRANSMISSIVE], [TRANSMISSIVE],
                [WATER[0], AIR[0]], [WATER[1], AIR[1]], cfl=0.3, steps=steps)
    X, _, _ = _centres(case)
    left = X < 0.7
    a1 = np.where(left, 1.0 - 1e-6, 1e-6)
    p = np.where(left, 1.0e9, 1.0e5)
    W = _assemble(case, [a1, 1.0 - a1], [np.full_like(a1, 1000.0), np.full_like(a1, 50.0)],
                  [np.zeros_like(a1)], p)
    return case, W


def normal_shock_state(mach: float, gamma: float, rho1: float, p1: float):
    """Post-shock (rho2, p2, u2) behind a shock moving at Mach `mach` into gas
    at rest (rho1, p1) (Rankine-Hugoniot relations for a perfect gas)."""
    m2 = mach * mach
    rho2 = rho1 * (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    p2 = p1 * (1.0 + 2.0 * gamma * (m2 - 1.0) / (gamma + 1.0))
    c1 = math.sqrt(gamma * p1 / rho1)
    u2 = mach * c1 * (1.0 - rho1 / rho2)
    return rho2, p2, u2


def shock_bubble_3d(n: int = 256, steps: int = 100, seed: int = 0, dims=None) -> tuple:
    """3D shock-bubble interaction on [0,1]^3: a Mach 1.5 planar shock in air
    (gamma 1.4, pre-shock rho = p = 1) at x = 0.25 moving +x, and a sphere of
    light gas (gamma 1.67, rho 0.138, p 1) of radius 0.15 at the centre whose
    interface is a tanh profile one cell wide; every phasic density is
    multiplied by (1 + 1e-3 U[-1, 1)) per cell (seeded); reflective y/z walls,
    transmissive x; CFL 0.4.  `dims` overrides the cell counts (nx, ny, nz)."""
    nx, ny, nz = dims if dims is not None else (n, n, n)
    case = Case("shock_bubble_3d", [nx, ny, nz], [0.0] * 3, [1.0] * 3,
                [TRANSMISSIVE, REFLECTIVE, REFLECTIVE], [TRANSMISSIVE, REFLECTIVE, REFLECTIVE],
                [1.4, 1.67], [0.0, 0.0], cfl=0.4, steps=steps)
    X, Y, Z = _centres(case)
    r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
    eps = 1e-6
    R = 0.15
    h = case.dx(0)
    a_air = eps + (1.0 - 2.0 * eps) * 0.5 * (1.0 + np.tanh((r - R) / h))
    rho2, p2, u2 = normal_shock_state(1.5, 1.4, 1.0, 1.0)
    shocked = X < 0.25
    shp = case.shape[1:]
    rho_air = np.broadcast_to(np.where(shocked, rho2, 1.0), shp)
    rho_gas = np.full(shp, 0.138)
    noise = _uniform(seed, (2,) + tuple(shp))
    rho_air = rho_air * (1.0 + 1e-3 * noise[0])
    rho_gas = rho_gas * (1.0 + 1e-3 * noise[1])
    p = np.broadcast_to(np.where(shocked, p2, 1.0), shp)
    u = np.broadcast_to(np.where(shocked, u2, 0.0), shp)
    zero = np.zeros(shp)
    W = _assemble(case, [a_air, 1.0 - a_air], [rho_air, rho_gas], [u, zero, zero], p)
    return case, W


def _fourier_field(seed: int, X, Y, Z, modes: int = 32, kmax: int = 4, amp: float = 1.0) -> np.ndarray:
    """sum_m a_m cos(2 pi kappa_m . x + theta_m), a_m ~ N(0,1)/sqrt(modes),
    theta_m ~ U[0, 2 pi), kappa_m integer vectors with |kappa|_inf <= kmax."""
    g = torch.Generator().manual_seed(seed)
    k = torch.randint(-kmax, kmax + 1, (modes, 3), generator=g).numpy()
    a = (torch.randn(modes, generator=g, dtype=torch.float64) / math.sqrt(modes)).numpy()
    th = (2.0 * math.pi * torch.rand(modes, generator=g, dtype=torch.float64)).numpy()
    out = np.zeros(np.broadcast_shapes(X.shape, Y.shape, Z.shape))
    for m in range(modes):
        ex = np.exp(2j * math.pi * k[m, 0] * X)
        ey = np.exp(2j * math.pi * k[m, 1] * Y)
        ez = np.exp(2j * math.pi * k[m, 2] * Z)
        out += amp * a[m] * np.real(np.exp(1j * th[m]) * ex * ey * ez)
    return out


def _fourier_curl(seed: int, X, Y, Z, modes: int = 32, kmax: int = 4):
    """Curl of a random periodic vector potential (three Fourier fields with
    seeds seed, seed+100, seed+200), differentiated analytically per mode."""
    comps = []
    for c in range(3):
        g = torch.Generator().manual_seed(seed + 100 * c)
        k = torch.randint(-kmax, kmax + 1, (modes, 3), generator=g).numpy()
        a = (torch.randn(modes, generator=g, dtype=torch.float64) / math.sqrt(modes)).numpy()
        th = (2.0 * math.pi * torch.rand(modes, generator=g, dtype=torch.float64)).numpy()
        comps.append((k, a, th))
    shp = np.broadcast_shapes(X.shape, Y.shape, Z.shape)
    # d psi_c / d x_e for each component c and axis e
    grad = np.zeros((3, 3) + shp)
    coords = (X, Y, Z)
    for c, (k, a, th) in enumerate(comps):
        for m in range(modes):
            phase = np.exp(1j * th[m])
            for e in range(3):
                phase = phase * np.exp(2j * math.pi * k[m, e] * coords[e])
            # d/dx_e cos(arg) = -sin(arg) * 2 pi k_e
            s = -np.imag(phase)
            for e in range(3):
                if k[m, e] != 0:
                    grad[c, e] += a[m] * s * 2.0 * math.pi * k[m, e]
    ux = grad[2, 1] - grad[1, 2]
    uy = grad[0, 2] - grad[2, 0]
    uz = grad[1, 0] - grad[0, 1]
    return ux, uy, uz


def random_interfaces_window(origin=(200, 180, 160), dims=(32, 32, 32), n: int = 512, steps: int = 50) -> tuple:
    """A dims-sized block, at cell offset `origin`, of the n^3 random
    interface field below: the same fields at the same resolution (the
    pressure noise is a function of the global cell index), with
    transmissive boundaries in place of the periodic wrap."""
    h = 1.0 / n
    lo = [origin[a] * h for a in range(3)]
    hi = [(origin[a] + dims[a]) * h for a in range(3)]
    case = Case("random_interfaces_window", list(dims), lo, hi, [TRANSMISSIVE] * 3, [TRANSMISSIVE] * 3,
                [1.4, 4.4, 6.1], [0.0, 6.0e8, 2.0e9], cfl=0.4, steps=steps)
    return case, _random_interfaces_fields(case, origin, n)


def random_interfaces_3d(n: int = 512, steps: int = 50, dims=None) -> tuple:
    """3D three-fluid random interface field on the periodic unit cube:
    fluids (gamma, pi_inf) = (1.4, 0), (4.4, 6e8), (6.1, 2e9) with phasic
    densities 1.2, 1000, 1100; alpha = softmax of three 32-mode Fourier
    fields (amplitude 4, seeds 0, 1, 2) clipped to [1e-6, 1] and renormalised;
    p = 1e5 (1 + 0.01 U[-1,1)) with U a hash of the global cell index
    (seed 4); u = curl of a random vector potential (seed 3) scaled so that
    its maximum over a 64^3 sampling of the cube is 10 m/s; CFL 0.4."""
    nx, ny, nz = dims if dims is not None else (n, n, n)
    case = Case("random_interfaces_3d", [nx, ny, nz], [0.0] * 3, [1.0] * 3,
                [PERIODIC] * 3, [PERIODIC] * 3, [1.4, 4.4, 6.1], [0.0, 6.0e8, 2.0e9],
                cfl=0.4, steps=steps)
    return case, _random_interfaces_fields(case, (0, 0, 0), nx)


def _hash_uniform(seed: int, gi, gj, gk, n: int) -> np.ndarray:
    """U[-1, 1) from the splitmix64 finaliser of the global cell index."""
    with np.errstate(over="ignore"):
        x = (gi.astype(np.uint64) + np.uint64(n) * (gj.astype(np.uint64) + np.uint64(n) * gk.astype(np.uint64))
             + np.uint64(seed) * np.uint64(0x9E3779B97F4A7C15))
        x = x + np.uint64(0x9E3779B97F4A7C15)
        x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        x = x ^ (x >> np.uint64(31))
    return (x >> np.uint64(11)).astype(np.float64) * (2.0 / 2.0 ** 53) - 1.0


_CURL_SCALE = {}


def _curl_scale() -> float:
    """10 m/s over the maximum speed of the raw curl field on a 64^3 sampling."""
    if "s" not in _CURL_SCALE:
        c = (np.arange(64) + 0.5) / 64
        ux, uy, uz = _fourier_curl(3, c[None, None, :], c[None, :, None], c[:, None, None])
        _CURL_SCALE["s"] = 10.0 / np.sqrt(ux ** 2 + uy ** 2 + uz ** 2).max()
    return _CURL_SCALE["s"]


def _random_interfaces_fields(case: Case, origin, n: int) -> np.ndarray:
    X, Y, Z = _centres(case)
    phi = np.stack([_fourier_field(s, X, Y, Z, amp=4.0) for s in (0, 1, 2)])
    phi = phi - phi.max(axis=0, keepdims=True)
    e = np.exp(phi)
    alpha = e / e.sum(axis=0, keepdims=True)
    alpha = np.clip(alpha, 1e-6, 1.0)
    alpha = alpha / alpha.sum(axis=0, keepdims=True)
    shp = case.shape[1:]
    nx, ny, nz = case.n
    gi = (origin[0] + np.arange(nx))[None, None, :]
    gj = (origin[1] + np.arange(ny))[None, :, None]
    gk = (origin[2] + np.arange(nz))[:, None, None]
    gi, gj, gk = np.broadcast_arrays(gi, gj, gk)
    p = 1.0e5 * (1.0 + 0.01 * _hash_uniform(4, gi, gj, gk, n))
    ux, uy, uz = _fourier_curl(3, X, Y, Z)
    scale = _curl_scale()
    rhos = [np.full(shp, 1.2), np.full(shp, 1000.0), np.full(shp, 1100.0)]
    return _assemble(case, [alpha[0], alpha[1], alpha[2]], rhos, [ux * scale, uy * scale, uz * scale], p)


def bubble_collapse_2d(n: int = 1024, steps: int = 500, dims=None) -> tuple:
    """2D air-in-water bubble collapse on [0,1]^2: an air bubble (rho 1,
    gamma 1.4, p 1e4) of radius 0.1 at (0.5, 0.5) in water (rho 1000,
    gamma 4.4, pi_inf 6e8, p 1e7), tanh interface one cell wide; the x = 1
    side is a reflective wall, the others transmissive; CFL 0.3."""
    nx, ny = dims if dims is not None else (n, n)
    case = Case("bubble_collapse_2d", [nx, ny], [0.0] * 2, [1.0] * 2,
                [TRANSMISSIVE, TRANSMISSIVE], [REFLECTIVE, TRANSMISSIVE],
                [WATER[0], AIR[0]], [WATER[1], AIR[1]], cfl=0.3, steps=steps)
    X, Y, _ = _centres(case)
    r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2)
    eps = 1e-6
    h = case.dx(0)
    a_water = eps + (1.0 - 2.0 * eps) * 0.5 * (1.0 + np.tanh((r - 0.1) / h))
    shp = case.shape[1:]
    # pressure follows the volume fraction across the smeared interface
    p = 1.0e4 + (1.0e7 - 1.0e4) * (a_water - eps) / (1.0 - 2.0 * eps)
    zero = np.zeros(shp)
    W = _assemble(case, [a_water, 1.0 - a_water], [np.full(shp, 1000.0), np.full(shp, 1.0)],
                  [zero, zero], p)
    return case, W


# ---------------------------------------------------------------------------
# Verification problems
# ---------------------------------------------------------------------------

def gresho_vortex(n: int, mach: float, R: float = 0.2, gamma: float = 1.4) -> tuple:
    """Gresho vortex (the low-Mach test of Sec. 4.2.4), one ideal gas, on the
    periodic unit square centred at (0.5, 0.5): u_phi = u_r (r/R, 2 - r/R, 0)
    on [0, R), [R, 2R), [2R, inf); p = p_r + rho_r u_r^2 ((r/R)^2/2,
    (r/R)^2/2 + 4 (1 - r/R + ln(r/R)), -2 + 4 ln 2) on the same intervals;
    rho_r = 1, u_r = 2 pi R M_r and p_r from M_r = u_r / sqrt(gamma (p_r/rho_r
    + u_r^2/2)).  One turn takes t_r = 2 pi R / u_r = 1/M_r.  Point values at
    the cell centres."""
    case = Case("gresho", [n, n], [0.0, 0.0], [1.0, 1.0], [PERIODIC, PERIODIC], [PERIODIC, PERIODIC],
                [gamma], [0.0], cfl=0.4, steps=0)
    X, Y, _ = _centres(case)
    x, y = X - 0.5, Y - 0.5
    r = np.sqrt(x * x + y * y)
    s = r / R
    rho_r = 1.0
    u_r = 2.0 * math.pi * R * mach
    p_r = rho_r * (u_r * u_r / (gamma * mach * mach) - 0.5 * u_r * u_r)
    uphi = u_r * np.where(s < 1.0, s, np.where(s < 2.0, 2.0 - s, 0.0))
    with np.errstate(divide="ignore"):
        mid = 0.5 * s * s + 4.0 * (1.0 - s + np.log(np.where(s > 0, s, 1.0)))
    p = p_r + rho_r * u_r * u_r * np.where(s < 1.0, 0.5 * s * s, np.where(s < 2.0, mid, -2.0 + 4.0 * math.log(2.0)))
    with np.errstate(invalid="ignore", divide="ignore"):
        ux = np.where(r > 0, -uphi * y / r, 0.0)
        uy = np.where(r > 0, uphi * x / r, 0.0)
    shp = case.shape[1:]
    W = _assemble(case, [np.ones(shp)], [np.full(shp, rho_r)], [ux, uy], p)
    return case, W


def riemann_1d(n: int, left, right, x0: float, gamma, pi_inf, t_end: float = 0.0,
               bc=TRANSMISSIVE, cfl: float = 0.4, alpha_left: float = 1.0 - 1e-6,
               alpha_right: float = 1e-6, rho2_left: Optional[float] = None,
               rho2_right: Optional[float] = None) -> tuple:
    """1D Riemann problem on [0,1].  left / right = (rho, u, p) of the fluid
    that fills that side.  With one fluid, alpha is unused.  With two fluids,
    fluid 1 fills the left (alpha_left) and fluid 2 the right; the minority
    phase keeps the density given by rho2_* (default: the majority density of
    its own side)."""
    nf = len(gamma)
    case = Case("riemann_1d", [n], [0.0], [1.0], [bc], [bc], list(gamma), list(pi_inf),
                cfl=cfl, steps=0)
    X, _, _ = _centres(case)
    L = X < x0
    u = np.where(L, left[1], right[1])
    p = np.where(L, left[2], right[2])
    if nf == 1:
        rho = np.where(L, left[0], right[0])
        return case, _assemble(case, [np.ones_like(rho)], [rho], [u], p)
    a1 = np.where(L, alpha_left, alpha_right)
    r1 = np.full_like(a1, left[0])
    r2 = np.full_like(a1, right[0] if rho2_right is None else rho2_right)
    if rho2_left is not None:
        r1 = np.where(L, left[0], rho2_left)
    return case, _assemble(case, [a1, 1.0 - a1], [r1, r2], [u], p)


def two_component_advection_1d(n: int, amp: float = 0.25, gamma=(1.4, 1.6)) -> tuple:
    """Two-component advection (Sec. 3.5) on the periodic unit interval with
    p = u = 1 and alpha_i = alpha_i rho_i = 0.5 + (-1)^i amp sin(2 pi x).  The
    printed amplitude (1) gives alpha outside [0, 1]; amp = 0.25 is used.
    Values are point values at cell centres; see `two_component_advection_avg`
    for exact cell averages."""
    case = Case("advection_1d", [n], [0.0], [1.0], [PERIODIC], [PERIODIC],
                list(gamma), [0.0, 0.0], cfl=0.4, steps=0)
    X, _, _ = _centres(case)
    s = np.sin(2 * math.pi * X)
    a1 = 0.5 - amp * s
    a2 = 0.5 + amp * s
    one = np.ones_like(X)
    return case, _assemble(case, [a1, a2], [one, one], [one], one)


def two_component_advection_avg(n: int, amp: float = 0.25, gamma=(1.4, 1.6), shift: float = 0.0):
    """Exact cell averages of the two-component advection state translated by
    `shift` (alpha averages integrate sin exactly)."""
    case = Case("advection_1d", [n], [0.0], [1.0], [PERIODIC], [PERIODIC],
                list(gamma), [0.0, 0.0], cfl=0.4, steps=0)
    h = 1.0 / n
    xl = np.arange(n) * h - shift
    # average of sin(2 pi x) over [xl, xl + h]
    avg_s = (np.cos(2 * math.pi * xl) - np.cos(2 * math.pi * (xl + h))) / (2 * math.pi * h)
    a1 = (0.5 - amp * avg_s)[None, None, :]
    a2 = (0.5 + amp * avg_s)[None, None, :]
    one = np.ones_like(a1)
    return case, _assemble(case, [a1, a2], [one, one], [one], one)


def isentropic_vortex_point(x, y, t: float = 0.0, strength: float = 5.0, gamma: float = 1.4,
                            centre=(5.0, 5.0), uinf=(1.0, 1.0), period: float = 10.0):
    """Point values (rho, u, v, p) of the isentropic vortex (Shu) on the
    periodic square [0, period]^2, advected with uinf for time t."""
    cx = (centre[0] + uinf[0] * t) % period
    cy = (centre[1] + uinf[1] * t) % period
    dxv = (x - cx + period / 2) % period - period / 2
    dyv = (y - cy + period / 2) % period - period / 2
    r2 = dxv ** 2 + dyv ** 2
    f = np.exp(0.5 * (1.0 - r2))
    du = -strength / (2 * math.pi) * f * dyv
    dv = strength / (2 * math.pi) * f * dxv
    T = 1.0 - (gamma - 1.0) * strength ** 2 / (8.0 * gamma * math.pi ** 2) * f * f
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho * T
    return rho, uinf[0] + du, uinf[1] + dv, p


def interface_advection(n, gamma, pi_inf, rho, u, p, smear: Optional[float] = None,
                        bc=PERIODIC) -> tuple:
    """Material interface(s) advected at uniform velocity u and pressure p:
    fluid 1 occupies the middle half of each axis span [0.25, 0.75) in x (a
    slab), with a sharp (smear=None) or tanh (width smear * dx) profile.
    `rho` gives the phasic densities; `u` one velocity per active axis."""
    nd = len(n)
    case = Case("interface_advection", list(n), [0.0] * nd, [1.0] * nd, [bc] * nd, [bc] * nd,
                list(gamma), list(pi_inf), cfl=0.4, steps=0)
    X, _, _ = _centres(case)
    shp = case.shape[1:]
    eps = 1e-6
    if smear is None:
        inside = (X >= 0.25) & (X < 0.75)
        a1 = np.where(inside, 1.0 - eps, eps)
    else:
        w = smear * case.dx(0)
        a1 = eps + (1 - 2 * eps) * 0.25 * (1 + np.tanh((X - 0.25) / w)) * (1 + np.tanh((0.75 - X) / w))
    a1 = np.broadcast_to(a1, shp)
    vel = [np.full(shp, float(u[d])) for d in range(nd)]
    return case, _assemble(case, [a1, 1.0 - a1], [np.full(shp, rho[0]), np.full(shp, rho[1])],
                           vel, np.full(shp, float(p)))


def random_smooth_state(case: Case, seed: int = 0, amp: float = 0.05) -> np.ndarray:
    """A smooth, positive random primitive state on any grid: a few Fourier
    modes on top of rho = 1, p = 1, alpha = 0.5, u = 0.3 per axis."""
    X, Y, Z = _centres(case)
    span = [case.hi[a] - case.lo[a] for a in range(case.ndim)] + [1.0] * (3 - case.ndim)
    Xs, Ys, Zs = X / span[0], Y / span[1], Z / span[2]
    shp = case.shape[1:]
    fields = []
    for s in range(case.nq + case.nf):
        fields.append(np.broadcast_to(_fourier_field(1000 * seed + s, Xs, Ys, Zs, modes=4, kmax=2), shp))
    nf, nd = case.nf, case.ndim
    raw_a = [np.exp(amp * 4 * fields[i]) for i in range(nf)]
    tot = sum(raw_a)
    alpha = [a / tot for a in raw_a]
    rho = [1.0 + amp * fields[nf + i] + 0.3 * i for i in range(nf)]
    vel = [0.3 + amp * fields[2 * nf + d] for d in range(nd)]
    p = 1.0 + amp * fields[2 * nf + nd]
    return _assemble(case, alpha, rho, vel, p)


# ---------------------------------------------------------------------------
# Viscous workloads (the stress of Sec. 2.1.1)
# ---------------------------------------------------------------------------

def taylor_green(n: int = 256, ndim: int = 3, re: float = 1600.0, mach: float = 0.1, gamma: float = 1.4,
                 steps: int = 100, dims=None) -> tuple:
    """Taylor-Green vortex, the paper's viscous example (Sec. 5.3: Re 1600,
    Ma 0.1).  One fluid (gamma 1.4), the periodic cube [0, 2 pi)^ndim, rho0 = 1,
    V0 = 1, L = 1, so eta = rho0 V0 L / Re and p0 = rho0 V0^2 / (gamma Ma^2).
    3D: u = V0 sin x cos y cos z, v = -V0 cos x sin y cos z, w = 0,
    p = p0 + rho0 V0^2 / 16 (cos 2x + cos 2y)(cos 2z + 2); 2D: u = V0 sin x
    cos y, v = -V0 cos x sin y, p = p0 + rho0 V0^2 / 4 (cos 2x + cos 2y).
    Reading (the paper cites the initial condition without printing it): an
    isothermal start, rho = rho0 p / p0.  CFL 0.4, WENO5-M, HLLC."""
    if dims is None:
        dims = [n] * ndim
    ndim = len(dims)
    two_pi = 2.0 * math.pi
    rho0, V0 = 1.0, 1.0
    p0 = rho0 * V0 ** 2 / (gamma * mach ** 2)
    case = Case(f"taylor_green_{ndim}d", list(dims), [0.0] * ndim, [two_pi] * ndim, [PERIODIC] * ndim,
                [PERIODIC] * ndim, [gamma], [0.0], cfl=0.4, steps=steps, eta=[rho0 * V0 / re])
    X, Y, Z = _centres(case)
    if ndim == 3:
        u = V0 * np.sin(X) * np.cos(Y) * np.cos(Z)
        v = -V0 * np.cos(X) * np.sin(Y) * np.cos(Z)
        w = np.zeros_like(u)
        p = p0 + rho0 * V0 ** 2 / 16.0 * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0)
        vel = [u, v, w]
    else:
        u = V0 * np.sin(X) * np.cos(Y)
        v = -V0 * np.cos(X) * np.sin(Y)
        p = p0 + rho0 * V0 ** 2 / 4.0 * (np.cos(2 * X) + np.cos(2 * Y))
        vel = [u, v]
    rho = rho0 * p / p0
    W = _assemble(case, [np.ones_like(rho)], [rho], vel, p)
    return case, W


def shear_wave_2d(n: int = 32, amp: float = 1e-3, eta: float = 0.02, p0: float = 100.0, gamma: float = 1.4,
                  k: int = 1) -> tuple:
    """A decaying shear wave: v = amp sin(2 pi k x), u = 0, rho = 1, p = p0 on
    the periodic unit square, one fluid of viscosity eta.  It is an exact
    solution of the compressible Navier-Stokes equations up to the viscous
    heating, of relative size amp^2: v decays as exp(-eta (2 pi k)^2 t / rho),
    with no pressure or density change."""
    case = Case("shear_wave_2d", [n, 4], [0.0, 0.0], [1.0, 4.0 / n], [PERIODIC] * 2, [PERIODIC] * 2,
                [gamma], [0.0], cfl=0.4, steps=0, eta=[eta])
    X, Y, _ = _centres(case)
    v = amp * np.sin(2.0 * math.pi * k * X) + 0.0 * Y
    W = _assemble(case, [np.ones_like(v)], [np.ones_like(v)], [np.zeros_like(v), v], np.full_like(v, p0))
    return case, W
