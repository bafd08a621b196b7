"""The C-ABI library builds, loads and exports every entry point the header
declares; descriptions are validated on the host before any CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(mfc_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for required in ("mfc_init", "mfc_destroy", "mfc_rhs", "mfc_rk3_step", "mfc_rhs_vjp",
                     "mfc_rk3_step_vjp", "mfc_compute_dt", "mfc_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(mfc_lib):
    lib = ctypes.CDLL(mfc_lib.LIB_PATH)
    for name in declared_entry_points():
        assert hasattr(lib, name), name
    # and the binding covers them all
    assert set(declared_entry_points()) <= set(mfc_lib.EXPORTED)


def _desc(mfc_lib, **over):
    g = mfc_lib.mfc_grid()
    g.ndim = 3
    for a in range(3):
        g.n[a] = 8
        g.lo[a] = 0.0
        g.hi[a] = 1.0
        g.bc_lo[a] = g.bc_hi[a] = mfc_lib.MFC_BC_TRANSMISSIVE
    g.ghost = 3
    e = mfc_lib.mfc_eos()
    e.nfluids = 2
    e.gamma[0], e.gamma[1] = 1.4, 1.67
    o = mfc_lib.mfc_opts()
    o.precision, o.weno, o.weno_eps, o.cfl = 0, 1, 1e-40, 0.4
    for k, v in sorted(over.items()):
        obj, field, val = v
        target = {"g": g, "e": e, "o": o}[obj]
        if isinstance(field, tuple):
            getattr(target, field[0])[field[1]] = val
        else:
            setattr(target, field, val)
    return g, e, o


@pytest.mark.parametrize("case,why", [
    ({"x": ("g", "ndim", 4)}, "ndim"),
    ({"x": ("g", ("n", 0), 0)}, "n >= 1"),
    ({"x": ("g", ("n", 2), 2)}, "inactive"),
    ({"x": ("g", ("bc_lo", 0), 0)}, "periodic must be set on both ends"),
    ({"x": ("g", ("hi", 1), -1.0)}, "lo < hi"),
    ({"x": ("g", "ghost", -1)}, "ghost"),
    ({"x": ("e", "nfluids", 5)}, "nfluids"),
    ({"x": ("e", ("gamma", 1), 1.0)}, "gamma"),
    ({"x": ("e", ("pi_inf", 0), -1.0)}, "pi_inf"),
    ({"x": ("o", "precision", 7)}, "precision"),
    ({"x": ("o", "precision", 4)}, "precision"),
    ({"x": ("o", "weno", 4)}, "WENO"),
    ({"x": ("o", "weno", 3), "y": ("o", "teno_ct", 1.5)}, "teno_ct"),
    ({"x": ("o", "weno_eps", 0.0)}, "weno_eps"),
    ({"x": ("o", "cfl", -0.1)}, "cfl"),
    ({"x": ("o", "model", 2)}, "unknown model"),
    ({"x": ("o", "riemann", 2)}, "Riemann"),
    ({"x": ("o", "low_mach", 3)}, "low-Mach"),
    ({"x": ("o", "low_mach", 2), "y": ("o", "riemann", 1)}, "needs HLLC"),
    ({"x": ("o", "model", 1), "y": ("e", "nfluids", 3), "z": ("e", ("gamma", 2), 1.6)}, "Kapila"),
])
def test_invalid_descriptions_rejected_on_host(mfc_lib, case, why):
    g, e, o = _desc(mfc_lib, **case)
    if case["x"][1] == ("n", 2):
        g.ndim = 2
        g.n[2] = 2
    with pytest.raises(mfc_lib.MfcError) as ei:
        mfc_lib.mfc_init(g, e, o)
    assert ei.value.status == mfc_lib.MFC_ERR_ARG
    assert why in mfc_lib.mfc_last_error(None)


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_every_precision_passes_the_host_checks(mfc_lib, precision):
    """MFC_FP64, MFC_MIXED, MFC_FP64_FAST and MFC_DF64 are valid: mfc_init
    gets past the host-side checks (without a GPU it then fails on the
    device with MFC_ERR_CUDA; with one it returns a context)."""
    g, e, o = _desc(mfc_lib)
    o.precision = precision
    try:
        ctx = mfc_lib.mfc_init(g, e, o)
    except mfc_lib.MfcError as err:
        assert err.status != mfc_lib.MFC_ERR_ARG, mfc_lib.mfc_last_error(None)
    else:
        mfc_lib.mfc_destroy(ctx)


def test_null_context_is_an_argument_error(mfc_lib):
    lib = mfc_lib.lib()
    assert lib.mfc_rhs(None, None, None, None) == mfc_lib.MFC_ERR_ARG
    assert lib.mfc_rk3_step(None, None, 0.0, None, None) == mfc_lib.MFC_ERR_ARG
    assert lib.mfc_rhs_vjp(None, None, None, None, None) == mfc_lib.MFC_ERR_ARG
    assert lib.mfc_destroy(None) == mfc_lib.MFC_OK
    assert lib.mfc_field_stride(None) == -1
    assert lib.mfc_num_fields(None) == -1


def test_product_path_fails_loudly_without_the_library(mfc_lib, monkeypatch):
    monkeypatch.setattr(mfc_lib, "_lib", None)
    monkeypatch.setattr(mfc_lib, "LIB_PATH", "/nonexistent/libmfcgb.so")
    with pytest.raises(RuntimeError, match="not built"):
        mfc_lib.lib()
