"""Pins of the oracle's WENO5 reconstruction (Sec. 3.2.1, Sec. 4.2.2)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def load_golden():
    path = os.path.join(HERE, "golden", "weno5_coeffs.txt")
    out = {}
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            tok = line.split()
            if tok[0] in ("chat_right", "chat_left"):
                out[(tok[0], int(tok[1]))] = [float(Fraction(t)) for t in tok[2:]]
            elif tok[0] == "bhat":
                out[("bhat", int(tok[1]))] = {(int(t[0]), int(t[1])): float(Fraction(t.split(":")[1]))
                                              for t in tok[2:]}
            else:
                out[tok[0]] = [float(Fraction(t)) for t in tok[1:]]
    return out


def test_golden_matches_paper_formula():
    """The stored constants are what the Sec. 4.2.2 construction gives."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("mk", os.path.join(HERE, "golden", "make_weno5_coeffs.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    res = mk.derive()
    g = load_golden()
    for r in range(3):
        assert [float(x) for x in res[("chat_right", r)]] == g[("chat_right", r)]
        assert [float(x) for x in res[("chat_left", r)]] == g[("chat_left", r)]
        assert {k: float(v) for k, v in res[("bhat", r)].items()} == g[("bhat", r)]
    assert [float(x) for x in res[("d", "right")]] == g["d_right"]
    assert [float(x) for x in res[("d", "left")]] == g["d_left"]


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_candidates_and_smoothness_match_generic_construction(oracle_lib, variant):
    g = load_golden()
    rng = np.random.default_rng(1)
    for _ in range(200):
        f = rng.normal(size=5) * 10.0 ** rng.integers(-3, 4)
        det = oracle_lib.weno5_detail(f, variant, 1e-6 if variant == 0 else 1e-40)
        scale = np.abs(f).max()
        for r in range(3):
            loc = f[r:r + 3]
            df = np.diff(loc)
            pr = loc[0] + sum(c * d for c, d in zip(g[("chat_right", r)], df))
            pl = loc[0] + sum(c * d for c, d in zip(g[("chat_left", r)], df))
            assert abs(det["p_right"][r] - pr) <= 1e-14 * scale
            assert abs(det["p_left"][r] - pl) <= 1e-14 * scale
            b = sum(v * df[j] * df[m] for (j, m), v in g[("bhat", r)].items())
            assert abs(det["beta"][r] - b) <= 1e-13 * scale ** 2


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_constant_data_gives_ideal_weights_and_exact_value(oracle_lib, variant):
    g = load_golden()
    for c in (0.0, 1.0, -3.5, 1e9, 1e-7):
        det = oracle_lib.weno5_detail(np.full(5, c), variant, 1e-6 if variant == 0 else 1e-40)
        assert det["v_right"] == pytest.approx(c, rel=1e-15, abs=0)
        assert det["v_left"] == pytest.approx(c, rel=1e-15, abs=0)
        np.testing.assert_allclose(det["w_right"], g["d_right"], rtol=1e-14)
        np.testing.assert_allclose(det["w_left"], g["d_left"], rtol=1e-14)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_linear_data_is_reconstructed_exactly(oracle_lib, variant):
    # cell averages of a linear function equal its centre values
    for a, b in ((1.0, 2.0), (-4.0, 0.5), (1e5, -3e3)):
        f = a + b * np.arange(-2, 3, dtype=float)
        det = oracle_lib.weno5_detail(f, variant, 1e-6 if variant == 0 else 1e-40)
        assert det["v_right"] == pytest.approx(a + 0.5 * b, rel=1e-13, abs=1e-13 * abs(a))
        assert det["v_left"] == pytest.approx(a - 0.5 * b, rel=1e-13, abs=1e-13 * abs(a))


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_mirror_symmetry(oracle_lib, variant):
    rng = np.random.default_rng(2)
    for _ in range(100):
        f = rng.normal(size=5)
        a = oracle_lib.weno5_detail(f, variant)
        b = oracle_lib.weno5_detail(f[::-1].copy(), variant)
        assert a["v_left"] == pytest.approx(b["v_right"], rel=1e-14, abs=1e-15)


@pytest.mark.parametrize("variant,eps", [(1, 1e-40), (2, 1e-40), (0, 1e-6), (3, 1e-40)])
def test_fifth_order_on_smooth_data(oracle_lib, variant, eps):
    """Edge value from exact cell averages of exp(x): error ~ h^5."""
    errs = []
    hs = [0.2 / 2 ** i for i in range(4)]
    for h in hs:
        x0 = 0.3
        # cell c spans [x0 - h/2, x0 + h/2]; averages of exp over the 5 cells
        lefts = x0 - 2.5 * h + h * np.arange(5)
        f = (np.exp(lefts + h) - np.exp(lefts)) / h
        det = oracle_lib.weno5_detail(f, variant, eps)
        errs.append(abs(det["v_right"] - math.exp(x0 + 0.5 * h)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > 4.5, rates


def test_mapped_weights_closer_to_ideal_than_js(oracle_lib):
    g = load_golden()
    d = np.array(g["d_right"])
    for h in (0.1, 0.05):
        lefts = 0.1 - 2.5 * h + h * np.arange(5)
        f = (np.sin(lefts + h) - np.sin(lefts)) / h
        js = oracle_lib.weno5_detail(f, 0, 1e-40)["w_right"]
        m = oracle_lib.weno5_detail(f, 1, 1e-40)["w_right"]
        assert np.abs(m - d).max() < np.abs(js - d).max()


def test_discontinuity_weights_avoid_crossing_stencil(oracle_lib):
    # a jump between cells c+1 and c+2: stencil 2 (c..c+2) crosses it
    f = np.array([1.0, 1.0, 1.0, 1.0, 100.0])
    for v in (0, 1, 2):
        det = oracle_lib.weno5_detail(f, v, 1e-6 if v == 0 else 1e-40)
        assert det["w_right"][2] < 1e-6
        assert det["v_right"] == pytest.approx(1.0, abs=1e-4)


def test_teno_smooth_data_is_the_linear_fifth_order_scheme(oracle_lib):
    """TENO (Sec. 4.2.2) keeps every stencil on smooth data (chi_r >= C_T),
    so its weights are the ideal weights and the edge value is the linear
    upwind-biased fifth-order reconstruction sum_r d_r p_r."""
    g = load_golden()
    for h in (0.2, 0.1, 0.05):
        for x0 in (0.1, 0.7, 2.0):
            lefts = x0 - 2.5 * h + h * np.arange(5)
            f = (np.sin(lefts + h) - np.sin(lefts)) / h + 2.0
            det = oracle_lib.weno5_detail(f, 3, 1e-40, 1e-6)
            np.testing.assert_allclose(det["w_right"], g["d_right"], rtol=1e-15)
            np.testing.assert_allclose(det["w_left"], g["d_left"], rtol=1e-15)
            lin = sum(d * p for d, p in zip(g["d_right"], det["p_right"]))
            assert det["v_right"] == pytest.approx(lin, rel=1e-15)


def test_teno_discontinuity_switches_the_crossing_stencil_off(oracle_lib):
    """Across a jump the stencil that contains it gets chi ~ 0 < C_T and a
    weight of exactly zero; the others keep their ideal weights
    renormalised, so a step is reconstructed without any contribution of
    the far side (WENO-JS/M/Z only make that weight small)."""
    g = load_golden()
    f = np.array([1.0, 1.0, 1.0, 1.0, 100.0])
    det = oracle_lib.weno5_detail(f, 3, 1e-40, 1e-6)
    d = np.array(g["d_right"])
    assert det["w_right"][2] == 0.0
    np.testing.assert_allclose(det["w_right"][:2], d[:2] / d[:2].sum(), rtol=1e-15)
    assert det["v_right"] == 1.0
    # the mirrored jump switches off the mirrored stencil of the other edge
    det = oracle_lib.weno5_detail(f[::-1].copy(), 3, 1e-40, 1e-6)
    assert det["w_left"][0] == 0.0 and det["v_left"] == 1.0


def test_teno_threshold_selects_by_chi(oracle_lib):
    """Brute force over random stencils: the stencils the oracle switches
    off are exactly those whose relative indicator chi_r is below C_T, and
    raising C_T never switches a stencil back on."""
    rng = np.random.default_rng(5)
    for _ in range(300):
        f = rng.normal(size=5) * np.array([1, 1, 1, 1, 1]) + np.where(rng.random(5) < 0.3, 50.0, 0.0)
        prev = None
        for ct in (1e-12, 1e-6, 1e-3, 0.2):
            det = oracle_lib.weno5_detail(f, 3, 1e-40, ct)
            beta = det["beta"]
            tau = abs(beta[0] - beta[2])
            A = 1.0 + tau / (beta + 1e-40)
            dR = np.array([0.1, 0.6, 0.3])
            gam = dR * (A / A.max()) ** 6
            chi = gam / gam.sum()
            off = det["w_right"] == 0.0
            # away from the threshold itself the selection follows chi
            clear = np.abs(chi - ct) > 1e-9 * ct
            assert np.array_equal(off[clear], (chi < ct)[clear])
            if prev is not None:
                assert np.all(off | ~prev)
            prev = off
