"""Thin Python binding of the C ABI in include/mfc.h.

Argument marshalling only: every numerical step runs in the CUDA kernels of
``libmfcgb.so``.  PyTorch supplies device memory and the current stream.
If the library has not been built the binding raises; there is no CPU
fallback.

The ``mfc_*`` functions mirror the C entry points one to one (pointers are
passed as integers, streams as ``cudaStream_t`` integers).  ``Solver`` wraps
a context for use with torch tensors laid out as in the header:
``[field][nz + 2g][ny + 2g][nx + 2g]`` float64 on the context's device.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmfcgb.so")

MFC_OK, MFC_ERR_ARG, MFC_ERR_ALLOC, MFC_ERR_CUDA, MFC_ERR_NONPHYSICAL, MFC_ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5
MFC_BC_PERIODIC, MFC_BC_TRANSMISSIVE, MFC_BC_REFLECTIVE, MFC_BC_HALO = 0, 1, 2, 3
MFC_FP64, MFC_MIXED, MFC_FP64_FAST, MFC_DF64 = 0, 1, 2, 3
MFC_WENO_JS, MFC_WENO_M, MFC_WENO_Z, MFC_WENO_TENO = 0, 1, 2, 3
MFC_MODEL_K0, MFC_MODEL_KAPILA = 0, 1
MFC_RIEMANN_HLLC, MFC_RIEMANN_HLL = 0, 1
MFC_LOW_MACH_NONE, MFC_LOW_MACH_THORNBER, MFC_LOW_MACH_APC = 0, 1, 2

_STATUS = {0: "MFC_OK", -1: "MFC_ERR_ARG", -2: "MFC_ERR_ALLOC", -3: "MFC_ERR_CUDA",
           -4: "MFC_ERR_NONPHYSICAL", -5: "MFC_ERR_UNSUPPORTED"}


class MfcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class mfc_grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("n", ctypes.c_int64 * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("ghost", ctypes.c_int32), ("bc_lo", ctypes.c_int32 * 3),
                ("bc_hi", ctypes.c_int32 * 3)]


class mfc_eos(ctypes.Structure):
    _fields_ = [("nfluids", ctypes.c_int32), ("gamma", ctypes.c_double * 4), ("pi_inf", ctypes.c_double * 4),
                ("eta", ctypes.c_double * 4)]


class mfc_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("weno", ctypes.c_int32), ("weno_eps", ctypes.c_double),
                ("cfl", ctypes.c_double), ("teno_ct", ctypes.c_double), ("model", ctypes.c_int32),
                ("riemann", ctypes.c_int32), ("low_mach", ctypes.c_int32), ("viscous_dt", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()

_VP = ctypes.c_void_p
_SIGS = {
    "mfc_init": (ctypes.c_int, [ctypes.POINTER(mfc_grid), ctypes.POINTER(mfc_eos), ctypes.POINTER(mfc_opts),
                               ctypes.POINTER(_VP)]),
    "mfc_destroy": (ctypes.c_int, [_VP]),
    "mfc_field_stride": (ctypes.c_int64, [_VP]),
    "mfc_num_fields": (ctypes.c_int32, [_VP]),
    "mfc_prim_to_cons": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "mfc_cons_to_prim": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "mfc_compute_dt": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_double), _VP]),
    "mfc_rhs": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "mfc_rk3_step": (ctypes.c_int, [_VP, _VP, ctypes.c_double, _VP, _VP]),
    "mfc_rk3_stage": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, _VP, _VP, ctypes.c_double, _VP]),
    "mfc_rk3_run": (ctypes.c_int, [_VP, _VP, ctypes.c_int32, ctypes.c_double, _VP, _VP]),
    "mfc_rk3_step_batch_host": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                                               ctypes.c_double, _VP, _VP]),
    "mfc_rhs_vjp": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "mfc_rk3_step_vjp": (ctypes.c_int, [_VP, _VP, ctypes.c_double, _VP, _VP, _VP]),
    "mfc_check": (ctypes.c_int, [_VP, _VP]),
    "mfc_last_error": (ctypes.c_char_p, [_VP]),
    "mfc_rk3_step_noalloc": (ctypes.c_int, [ctypes.POINTER(mfc_grid), ctypes.POINTER(mfc_eos),
                                            ctypes.POINTER(mfc_opts), _VP, ctypes.c_double, _VP, _VP]),
}
EXPORTED = tuple(_SIGS)


def lib() -> ctypes.CDLL:
    """Load libmfcgb.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                                   "(run paper_2503_07953_gb300.build.build())")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _err(ctx, status: int) -> None:
    if status != MFC_OK:
        msg = lib().mfc_last_error(ctx)
        raise MfcError(status, msg.decode() if msg else "")


# --- one-to-one wrappers of the C entry points ------------------------------

def mfc_init(grid: mfc_grid, eos: mfc_eos, opts: mfc_opts) -> int:
    out = _VP()
    _err(None, lib().mfc_init(ctypes.byref(grid), ctypes.byref(eos), ctypes.byref(opts), ctypes.byref(out)))
    return out.value


def mfc_destroy(ctx) -> None:
    _err(None, lib().mfc_destroy(ctx))


def mfc_field_stride(ctx) -> int:
    return lib().mfc_field_stride(ctx)


def mfc_num_fields(ctx) -> int:
    return lib().mfc_num_fields(ctx)


def mfc_prim_to_cons(ctx, w, q, stream) -> None:
    _err(ctx, lib().mfc_prim_to_cons(ctx, w, q, stream))


def mfc_cons_to_prim(ctx, q, w, stream) -> None:
    _err(ctx, lib().mfc_cons_to_prim(ctx, q, w, stream))


def mfc_compute_dt(ctx, q, stream) -> float:
    dt = ctypes.c_double(0.0)
    _err(ctx, lib().mfc_compute_dt(ctx, q, ctypes.byref(dt), stream))
    return dt.value


def mfc_rhs(ctx, q, rhs, stream) -> None:
    _err(ctx, lib().mfc_rhs(ctx, q, rhs, stream))


def mfc_rk3_step(ctx, q, dt, dt_used, stream) -> None:
    _err(ctx, lib().mfc_rk3_step(ctx, q, float(dt), dt_used, stream))


def mfc_rk3_stage(ctx, stage, q_in, q_n, q_out, dt, stream) -> None:
    _err(ctx, lib().mfc_rk3_stage(ctx, int(stage), q_in, q_n, q_out, float(dt), stream))


def mfc_rk3_run(ctx, q, nsteps, dt, dt_log, stream) -> None:
    _err(ctx, lib().mfc_rk3_run(ctx, q, int(nsteps), float(dt), dt_log, stream))


def mfc_rk3_step_batch_host(ctx, count, q_in, q_out, dt, dt_used, stream) -> None:
    """q_in, q_out: sequences of `count` host addresses (ints); dt_used: a host
    address of `count` doubles or None."""
    ins = (_VP * max(int(count), 1))(*q_in)
    outs = (_VP * max(int(count), 1))(*q_out)
    _err(ctx, lib().mfc_rk3_step_batch_host(ctx, int(count), ins, outs, float(dt), dt_used, stream))


def mfc_rhs_vjp(ctx, q, rhs_bar, q_bar, stream) -> None:
    _err(ctx, lib().mfc_rhs_vjp(ctx, q, rhs_bar, q_bar, stream))


def mfc_rk3_step_vjp(ctx, q_n, dt, qnp1_bar, qn_bar, stream) -> None:
    _err(ctx, lib().mfc_rk3_step_vjp(ctx, q_n, float(dt), qnp1_bar, qn_bar, stream))


def mfc_check(ctx, stream) -> None:
    _err(ctx, lib().mfc_check(ctx, stream))


def mfc_rk3_step_noalloc(grid: mfc_grid, eos: mfc_eos, opts: mfc_opts, q, dt, dt_used, stream) -> None:
    """One RK3 step without a context or any device allocation (see mfc.h)."""
    _err(None, lib().mfc_rk3_step_noalloc(ctypes.byref(grid), ctypes.byref(eos), ctypes.byref(opts), q,
                                          float(dt), dt_used, stream))


def mfc_last_error(ctx) -> str:
    m = lib().mfc_last_error(ctx)
    return m.decode() if m else ""


# --- torch convenience -------------------------------------------------------

def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else t.data_ptr()


class Solver:
    """A context plus helpers for torch tensors on its device."""

    def __init__(self, n: Sequence[int], gamma: Sequence[float], pi_inf: Sequence[float],
                 lo: Optional[Sequence[float]] = None, hi: Optional[Sequence[float]] = None,
                 bc_lo: Optional[Sequence[int]] = None, bc_hi: Optional[Sequence[int]] = None,
                 ghost: int = 3, precision: int = MFC_FP64, weno: int = MFC_WENO_M,
                 weno_eps: Optional[float] = None, cfl: float = 0.4, teno_ct: float = 1e-6,
                 model: int = MFC_MODEL_K0, riemann: int = MFC_RIEMANN_HLLC,
                 low_mach: int = MFC_LOW_MACH_NONE, eta: Optional[Sequence[float]] = None,
                 viscous_dt: bool = False, device=None):
        nd = len(n)
        self.ndim, self.nf = nd, len(gamma)
        self.n = [int(x) for x in n] + [1] * (3 - nd)
        self.ghost = int(ghost)
        self.precision = int(precision)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        g = mfc_grid()
        g.ndim = nd
        for a in range(3):
            g.n[a] = self.n[a]
            g.lo[a] = float(lo[a]) if (lo is not None and a < nd) else 0.0
            g.hi[a] = float(hi[a]) if (hi is not None and a < nd) else 1.0
            g.bc_lo[a] = int(bc_lo[a]) if (bc_lo is not None and a < nd) else MFC_BC_TRANSMISSIVE
            g.bc_hi[a] = int(bc_hi[a]) if (bc_hi is not None and a < nd) else MFC_BC_TRANSMISSIVE
        g.ghost = self.ghost
        e = mfc_eos()
        e.nfluids = self.nf
        for i in range(min(4, self.nf)):
            e.gamma[i] = float(gamma[i])
            e.pi_inf[i] = float(pi_inf[i])
            e.eta[i] = float(eta[i]) if eta is not None else 0.0
        o = mfc_opts()
        o.precision = self.precision
        o.weno = int(weno)
        o.weno_eps = float(weno_eps if weno_eps is not None else (1e-6 if weno == MFC_WENO_JS else 1e-40))
        o.cfl = float(cfl)
        o.teno_ct = float(teno_ct)
        o.model = int(model)
        o.riemann = int(riemann)
        o.low_mach = int(low_mach)
        o.viscous_dt = int(bool(viscous_dt))
        with torch.cuda.device(self.device):
            self.ctx = mfc_init(g, e, o)
        self.nq = mfc_num_fields(self.ctx)
        pad = [self.n[a] + (2 * self.ghost if a < nd else 0) for a in range(3)]
        self.shape = (self.nq, pad[2], pad[1], pad[0])
        self.interior_shape = (self.nq, self.n[2], self.n[1], self.n[0])
        assert mfc_field_stride(self.ctx) == pad[0] * pad[1] * pad[2]

    @classmethod
    def from_case(cls, case, **kw):
        return cls(case.n, case.gamma, case.pi_inf, lo=case.lo, hi=case.hi, bc_lo=case.bc_lo,
                   bc_hi=case.bc_hi, weno=case.weno, weno_eps=case.eps, cfl=case.cfl, teno_ct=case.teno_ct,
                   model=case.model, riemann=case.riemann, low_mach=case.low_mach,
                   eta=getattr(case, "eta", None), viscous_dt=getattr(case, "viscous_dt", False), **kw)

    # layout helpers
    def empty(self) -> torch.Tensor:
        return torch.zeros(self.shape, dtype=torch.float64, device=self.device)

    def _slices(self):
        g = self.ghost
        sl = []
        for a in (2, 1, 0):
            sl.append(slice(g, g + self.n[a]) if a < self.ndim else slice(0, 1))
        return (slice(None), *sl)

    def interior(self, t: torch.Tensor) -> torch.Tensor:
        return t[self._slices()]

    def from_interior(self, arr) -> torch.Tensor:
        t = self.empty()
        src = torch.as_tensor(np.ascontiguousarray(arr) if isinstance(arr, np.ndarray) else arr,
                              dtype=torch.float64).reshape(self.interior_shape)
        t[self._slices()] = src.to(self.device)
        return t

    def _check(self, *ts):
        for t in ts:
            if t is None:
                continue
            if t.dtype != torch.float64 or t.device != self.device or not t.is_contiguous() \
                    or tuple(t.shape) != self.shape:
                raise ValueError(f"expected a contiguous float64 tensor of shape {self.shape} on {self.device}")

    @staticmethod
    def _stream():
        return torch.cuda.current_stream().cuda_stream

    # numerics
    def prim_to_cons(self, w: torch.Tensor, q: Optional[torch.Tensor] = None) -> torch.Tensor:
        q = self.empty() if q is None else q
        self._check(w, q)
        mfc_prim_to_cons(self.ctx, _ptr(w), _ptr(q), self._stream())
        return q

    def cons_to_prim(self, q: torch.Tensor, w: Optional[torch.Tensor] = None) -> torch.Tensor:
        w = self.empty() if w is None else w
        self._check(q, w)
        mfc_cons_to_prim(self.ctx, _ptr(q), _ptr(w), self._stream())
        return w

    def compute_dt(self, q: torch.Tensor) -> float:
        self._check(q)
        return mfc_compute_dt(self.ctx, _ptr(q), self._stream())

    def rhs(self, q: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        out = self.empty() if out is None else out
        self._check(q, out)
        mfc_rhs(self.ctx, _ptr(q), _ptr(out), self._stream())
        return out

    def rk3_step(self, q: torch.Tensor, dt: float = 0.0, dt_used: Optional[torch.Tensor] = None) -> torch.Tensor:
        self._check(q)
        mfc_rk3_step(self.ctx, _ptr(q), dt, _ptr(dt_used), self._stream())
        return q

    def rk3_stage(self, stage: int, q_in: torch.Tensor, q_n: Optional[torch.Tensor], q_out: torch.Tensor,
                  dt: float) -> torch.Tensor:
        """Stage 1, 2 or 3 of the RK3 step at the step's dt > 0 (mfc_rk3_stage)."""
        self._check(q_in, q_n, q_out)
        mfc_rk3_stage(self.ctx, stage, _ptr(q_in), _ptr(q_n), _ptr(q_out), dt, self._stream())
        return q_out

    def rk3_run(self, q: torch.Tensor, nsteps: int, dt: float = 0.0,
                dt_log: Optional[torch.Tensor] = None) -> torch.Tensor:
        self._check(q)
        if dt_log is not None:
            assert dt_log.dtype == torch.float64 and dt_log.is_cuda and dt_log.numel() >= nsteps
        mfc_rk3_run(self.ctx, _ptr(q), nsteps, dt, _ptr(dt_log), self._stream())
        return q

    def rk3_step_batch_host(self, q_in, q_out, dt: float = 0.0) -> torch.Tensor:
        """One RK3 step of each host state q_in[b] into q_out[b] (CPU float64
        tensors of the state shape; pinned ones let the copies overlap the
        steps).  Returns the dt each state took (a CPU tensor)."""
        if len(q_in) != len(q_out):
            raise ValueError("q_in and q_out must have the same length")
        for t in (*q_in, *q_out):
            if t.dtype != torch.float64 or t.device.type != "cpu" or not t.is_contiguous() \
                    or tuple(t.shape) != self.shape:
                raise ValueError(f"expected contiguous float64 CPU tensors of shape {self.shape}")
        dts = torch.zeros(max(len(q_in), 1), dtype=torch.float64)
        mfc_rk3_step_batch_host(self.ctx, len(q_in), [t.data_ptr() for t in q_in], [t.data_ptr() for t in q_out],
                                dt, dts.data_ptr(), self._stream())
        return dts[:len(q_in)]

    def rhs_vjp(self, q: torch.Tensor, rhs_bar: torch.Tensor, q_bar: Optional[torch.Tensor] = None) -> torch.Tensor:
        q_bar = self.empty() if q_bar is None else q_bar
        self._check(q, rhs_bar, q_bar)
        mfc_rhs_vjp(self.ctx, _ptr(q), _ptr(rhs_bar), _ptr(q_bar), self._stream())
        return q_bar

    def rk3_step_vjp(self, q_n: torch.Tensor, dt: float, qnp1_bar: torch.Tensor,
                     qn_bar: Optional[torch.Tensor] = None) -> torch.Tensor:
        qn_bar = self.empty() if qn_bar is None else qn_bar
        self._check(q_n, qnp1_bar, qn_bar)
        mfc_rk3_step_vjp(self.ctx, _ptr(q_n), dt, _ptr(qnp1_bar), _ptr(qn_bar), self._stream())
        return qn_bar

    def check(self) -> None:
        mfc_check(self.ctx, self._stream())

    def close(self) -> None:
        if getattr(self, "ctx", None):
            mfc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
