"""Python access to the plain FP64 CPU oracle (``mfc_oracle.cpp``).

Test infrastructure only: ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference legs of ``bench.py`` may import this package.
The product path never does, and this package imports nothing from it.

Arrays exchanged with the oracle are float64, C-contiguous, interior cells
only, shaped ``(n_fields, nz, ny, nx)`` (``ny = nz = 1`` in 1D, ``nz = 1`` in
2D).  Field order: partial densities alpha_i rho_i, momenta rho u_d, total
energy rho E, volume fractions alpha_1 .. alpha_{N_f - 1} (Sec. 2.1.1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mfc_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
# the same source built with OpenMP: the loops over grid lines and cells run
# on all host cores (used to time the CPU baseline; results are identical)
_SO_OMP = os.path.join(_BUILD, "liboracle_omp.so")

BC_PERIODIC, BC_TRANSMISSIVE, BC_REFLECTIVE = 0, 1, 2
WENO_JS, WENO_M, WENO_Z, WENO_TENO = 0, 1, 2, 3
MAXF = 4

_lock = threading.Lock()
_libs = {}
_parallel = False


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with g++ (no FMA contraction, no fast-math);
    openmp=True builds the multi-threaded copy."""
    os.makedirs(_BUILD, exist_ok=True)
    so = _SO_OMP if openmp else _SO
    if not force and os.path.exists(so) and os.path.getmtime(so) >= os.path.getmtime(_SRC):
        return so
    tmp = so + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    if openmp:
        cmd.append("-fopenmp")
    cmd += [_SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, so)
    return so


def set_parallel(on: bool) -> None:
    """Route the module's calls to the OpenMP build (True) or to the
    single-threaded build (False, the default)."""
    global _parallel
    _parallel = bool(on)


def threads() -> int:
    """Host threads the current build's loops use."""
    return int(_load().oc_threads())


class _Problem(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int32), ("nf", ctypes.c_int32), ("n", ctypes.c_int32 * 3),
        ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
        ("bc_lo", ctypes.c_int32 * 3), ("bc_hi", ctypes.c_int32 * 3),
        ("gamma", ctypes.c_double * MAXF), ("pi_inf", ctypes.c_double * MAXF),
        ("weno", ctypes.c_int32), ("eps", ctypes.c_double), ("teno_ct", ctypes.c_double),
        ("model", ctypes.c_int32), ("riemann", ctypes.c_int32), ("low_mach", ctypes.c_int32),
        ("eta", ctypes.c_double * MAXF), ("viscous_dt", ctypes.c_int32),
    ]


def _load():
    with _lock:
        key = "omp" if _parallel else "serial"
        if key not in _libs:
            lib = ctypes.CDLL(build(openmp=_parallel))
            P = ctypes.POINTER(_Problem)
            dp = ctypes.POINTER(ctypes.c_double)
            i64p = ctypes.POINTER(ctypes.c_int64)
            sig = {
                "oc_threads": (ctypes.c_int, []),
                "oc_nfields": (ctypes.c_int, [P]),
                "oc_prim_to_cons": (ctypes.c_int, [P, dp, dp]),
                "oc_cons_to_prim": (ctypes.c_int, [P, dp, dp]),
                "oc_dt": (ctypes.c_double, [P, dp, ctypes.c_double]),
                "oc_rhs": (ctypes.c_int, [P, dp, dp]),
                "oc_viscous_rhs": (ctypes.c_int, [P, dp, dp]),
                "oc_rk3_step": (ctypes.c_int, [P, dp, ctypes.c_double]),
                "oc_rk3_run": (ctypes.c_int, [P, dp, ctypes.c_int, ctypes.c_double, dp, dp]),
                "oc_rhs_jvp": (ctypes.c_int, [P, dp, dp, dp, dp]),
                "oc_rk3_step_jvp": (ctypes.c_int, [P, dp, dp, ctypes.c_double]),
                "oc_rk3_step_sampled": (ctypes.c_int, [P, dp, ctypes.c_double, ctypes.c_int64, i64p, dp]),
                "oc_rk3_step_count": (ctypes.c_int, [P, dp, ctypes.c_double, i64p]),
                "oc_block_counts": (ctypes.c_int, [P, dp, dp, i64p]),
                "oc_weno5_detail": (None, [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp]),
                "oc_hllc_face": (ctypes.c_int, [P, ctypes.c_int, dp, dp, dp, dp]),
                "oc_rk3_linear": (ctypes.c_double, [ctypes.c_double, ctypes.c_double, ctypes.c_double]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _libs[key] = lib
    return _libs[key]


@dataclass
class Problem:
    """Grid, boundary conditions, fluids and WENO options of one case."""
    n: Sequence[int]                      # cells per active axis (len = ndim)
    gamma: Sequence[float]
    pi_inf: Sequence[float]
    lo: Sequence[float] = None
    hi: Sequence[float] = None
    bc_lo: Sequence[int] = None           # per axis; default transmissive
    bc_hi: Sequence[int] = None
    weno: int = WENO_M
    eps: float = 1e-40
    teno_ct: float = 1e-6
    model: int = 0                        # 0: K = 0 (Allaire); 1: Kapila K div u (two fluids)
    riemann: int = 0                      # 0: HLLC; 1: HLL
    low_mach: int = 0                     # 0: none; 1: Thornber; 2: anti-dissipation pressure correction
    eta: Sequence[float] = None           # shear viscosity per fluid; None or zeros: inviscid
    viscous_dt: int = 0                   # 1: the CFL dt also respects the explicit viscous limit
    _c: _Problem = field(default=None, repr=False)

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
    def shape(self):
        n3 = list(self.n) + [1] * (3 - self.ndim)
        return (self.nq, n3[2], n3[1], n3[0])

    def cstruct(self) -> _Problem:
        p = _Problem()
        p.ndim, p.nf = self.ndim, self.nf
        nd = self.ndim
        lo = list(self.lo) if self.lo is not None else [0.0] * nd
        hi = list(self.hi) if self.hi is not None else [1.0] * nd
        bl = list(self.bc_lo) if self.bc_lo is not None else [BC_TRANSMISSIVE] * nd
        bh = list(self.bc_hi) if self.bc_hi is not None else [BC_TRANSMISSIVE] * nd
        for a in range(3):
            p.n[a] = int(self.n[a]) if a < nd else 1
            p.lo[a] = float(lo[a]) if a < nd else 0.0
            p.hi[a] = float(hi[a]) if a < nd else 1.0
            p.bc_lo[a] = int(bl[a]) if a < nd else BC_TRANSMISSIVE
            p.bc_hi[a] = int(bh[a]) if a < nd else BC_TRANSMISSIVE
        for i in range(MAXF):
            p.gamma[i] = float(self.gamma[i]) if i < self.nf else 0.0
            p.pi_inf[i] = float(self.pi_inf[i]) if i < self.nf else 0.0
            p.eta[i] = float(self.eta[i]) if (self.eta is not None and i < self.nf) else 0.0
        p.weno, p.eps, p.teno_ct = int(self.weno), float(self.eps), float(self.teno_ct)
        p.model, p.riemann, p.low_mach = int(self.model), int(self.riemann), int(self.low_mach)
        p.viscous_dt = int(self.viscous_dt)
        return p

    def dx(self, axis: int) -> float:
        lo = self.lo[axis] if self.lo is not None else 0.0
        hi = self.hi[axis] if self.hi is not None else 1.0
        return (hi - lo) / self.n[axis]


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _arr(P: Problem, a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != P.shape:
        a = a.reshape(P.shape)
    return a


def _check(rc: int, what: str):
    if rc < 0:
        raise ValueError(f"oracle {what}: bad problem description")
    return rc


def prim_to_cons(P: Problem, w) -> np.ndarray:
    lib = _load(); c = P.cstruct(); w = _arr(P, w); q = np.empty_like(w)
    _check(lib.oc_prim_to_cons(ctypes.byref(c), _dp(w), _dp(q)), "prim_to_cons")
    return q


def cons_to_prim(P: Problem, q) -> np.ndarray:
    lib = _load(); c = P.cstruct(); q = _arr(P, q); w = np.empty_like(q)
    _check(lib.oc_cons_to_prim(ctypes.byref(c), _dp(q), _dp(w)), "cons_to_prim")
    return w


def cfl_dt(P: Problem, q, cfl: float) -> float:
    lib = _load(); c = P.cstruct(); q = _arr(P, q)
    dt = lib.oc_dt(ctypes.byref(c), _dp(q), float(cfl))
    if dt < 0:
        raise ValueError("oracle dt: bad problem description")
    return dt


def rhs(P: Problem, q, return_bad: bool = False):
    lib = _load(); c = P.cstruct(); q = _arr(P, q); L = np.empty_like(q)
    bad = _check(lib.oc_rhs(ctypes.byref(c), _dp(q), _dp(L)), "rhs")
    return (L, bad) if return_bad else L


def viscous_rhs(P: Problem, q) -> np.ndarray:
    """The viscous part of L(q) alone."""
    lib = _load(); c = P.cstruct(); q = _arr(P, q); V = np.empty_like(q)
    _check(lib.oc_viscous_rhs(ctypes.byref(c), _dp(q), _dp(V)), "viscous_rhs")
    return V


def rk3_step(P: Problem, q, dt: float, return_bad: bool = False):
    lib = _load(); c = P.cstruct(); q = _arr(P, q).copy()
    bad = _check(lib.oc_rk3_step(ctypes.byref(c), _dp(q), float(dt)), "rk3_step")
    return (q, bad) if return_bad else q


def rk3_run(P: Problem, q, nsteps: int, cfl: float = 0.0, dts=None, return_bad: bool = False):
    """nsteps RK3 steps; dts (fixed per-step dt) or else the CFL dt per step.
    Returns (q, dts_used[, n_bad])."""
    lib = _load(); c = P.cstruct(); q = _arr(P, q).copy()
    out = np.empty(nsteps, dtype=np.float64)
    dtp = None
    if dts is not None:
        dts = np.ascontiguousarray(dts, dtype=np.float64)
        assert dts.shape == (nsteps,)
        dtp = _dp(dts)
    bad = _check(lib.oc_rk3_run(ctypes.byref(c), _dp(q), int(nsteps), float(cfl), dtp, _dp(out)), "rk3_run")
    return (q, out, bad) if return_bad else (q, out)


def rhs_jvp(P: Problem, q, dq):
    lib = _load(); c = P.cstruct(); q = _arr(P, q); dq = _arr(P, dq)
    L = np.empty_like(q); dL = np.empty_like(q)
    _check(lib.oc_rhs_jvp(ctypes.byref(c), _dp(q), _dp(dq), _dp(L), _dp(dL)), "rhs_jvp")
    return L, dL


def rk3_step_jvp(P: Problem, q, dq, dt: float):
    lib = _load(); c = P.cstruct(); q = _arr(P, q).copy(); dq = _arr(P, dq).copy()
    _check(lib.oc_rk3_step_jvp(ctypes.byref(c), _dp(q), _dp(dq), float(dt)), "rk3_step_jvp")
    return q, dq


def rk3_step_sampled(P: Problem, q, dt: float, cells) -> np.ndarray:
    """One RK3 step evaluated at the given interior cells ((i, j, k) rows)
    through their domain of dependence.  Returns (n_cells, n_fields)."""
    lib = _load(); c = P.cstruct(); q = _arr(P, q)
    cells = np.ascontiguousarray(np.asarray(cells, dtype=np.int64).reshape(-1, 3))
    out = np.empty((cells.shape[0], P.nq), dtype=np.float64)
    _check(lib.oc_rk3_step_sampled(ctypes.byref(c), _dp(q), float(dt), cells.shape[0],
                                   cells.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(out)),
           "rk3_step_sampled")
    return out


def rk3_step_counts(P: Problem, q, dt: float) -> dict:
    lib = _load(); c = P.cstruct(); q = _arr(P, q)
    cnt = np.zeros(5, dtype=np.int64)
    _check(lib.oc_rk3_step_count(ctypes.byref(c), _dp(q), float(dt),
                                 cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))), "count")
    return dict(zip(("add", "mul", "div", "sqrt", "cmp"), cnt.tolist()))


def block_counts(P: Problem, qa, qb) -> dict:
    """Operation counts of one call of each building block (see the C source)."""
    lib = _load(); c = P.cstruct()
    qa = np.ascontiguousarray(qa, dtype=np.float64); qb = np.ascontiguousarray(qb, dtype=np.float64)
    out = np.zeros((8, 5), dtype=np.int64)
    _check(lib.oc_block_counts(ctypes.byref(c), _dp(qa), _dp(qb),
                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))), "block_counts")
    names = ("c2p", "weno_edge", "hllc", "cell_term", "rk_update", "cfl_cell", "weno_beta", "face_check")
    keys = ("add", "mul", "div", "sqrt", "cmp")
    return {n: dict(zip(keys, out[i].tolist())) for i, n in enumerate(names)}


def weno5_detail(f, variant: int = WENO_M, eps: float = 1e-40, teno_ct: float = 1e-6) -> dict:
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    assert f.shape == (5,)
    out = np.zeros(17)
    lib.oc_weno5_detail(int(variant), float(eps), float(teno_ct), _dp(f), _dp(out))
    return {"p_right": out[0:3].copy(), "beta": out[3:6].copy(), "w_right": out[6:9].copy(),
            "v_right": out[9], "p_left": out[10:13].copy(), "w_left": out[13:16].copy(), "v_left": out[16]}


def hllc_face(P: Problem, direction: int, WL, WR):
    lib = _load(); c = P.cstruct()
    WL = np.ascontiguousarray(WL, dtype=np.float64); WR = np.ascontiguousarray(WR, dtype=np.float64)
    F = np.zeros(P.nq); uf = ctypes.c_double(0.0)
    bad = _check(lib.oc_hllc_face(ctypes.byref(c), int(direction), _dp(WL), _dp(WR), _dp(F),
                                  ctypes.byref(uf)), "hllc_face")
    return F, uf.value, bad


def rk3_linear(lam: float, y0: float, dt: float) -> float:
    return _load().oc_rk3_linear(float(lam), float(y0), float(dt))
