"""Pins of the oracle's twiddle tables against the values the paper prints
(Table I, Table II, Theorem 1, Section V) and against trigonometric closed
forms."""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables_n1024.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = line.split()
            out[k] = float(v)
    return out


def test_dual_select_ratio_bound_table1(orc):
    """Theorem 1 / Table I: dual-select |t| <= 1, max exactly 1.0 at k = N/8
    once rounded to FP32 or FP16."""
    g = golden()
    N = 1024
    t64, m64, p = orc.table(N, orc.DS, orc.FP64)
    assert np.all(np.abs(t64) <= 1.0)
    assert int(np.argmax(np.abs(t64))) == int(g["ds_tmax_k"])
    assert abs(np.max(np.abs(t64)) - g["ds_tmax"]) < 1e-12
    for fmt in (orc.FP32, orc.FP16, orc.BF16):
        t, m, _ = orc.table(N, orc.DS, fmt)
        assert np.max(np.abs(t)) == 1.0
        assert np.all(np.abs(t) <= 1.0)
    # the outer multiplier never drops below 1/sqrt(2): the larger of |cos|, |sin|
    assert np.min(np.abs(m64)) >= 1 / math.sqrt(2) - 1e-15
    assert int(np.sum(np.isinf(t64))) == int(g["ds_singularities"])


def test_linzer_feig_ratio_table1(orc):
    """Table I: LF |t|max = |cot(pi/512)| = 163.0 over k >= 1, at k = 1; one
    singular twiddle (k = 0) that needs the epsilon clamp."""
    g = golden()
    N = 1024
    t, m, p = orc.table(N, orc.LF, orc.FP64, eps=1e-7)
    assert np.all(p == orc.PATH_SIN)
    tk = np.abs(t[1:])
    assert int(np.argmax(tk)) + 1 == int(g["lf_tmax_k"])
    assert round(float(np.max(tk)), 1) == g["lf_tmax"]
    assert abs(np.max(tk) - 1 / math.tan(math.pi / 512)) < 1e-9
    # the clamped W^0 entry: multiplier -eps, ratio 1/(-eps)
    assert m[0] == -1e-7 and abs(t[0] + 1e7) < 1e-3
    # exactly one twiddle has sin(theta) == 0 before clamping
    th = -2 * np.pi * np.arange(N // 2) / N
    assert int(np.sum(np.sin(th) == 0)) == int(g["lf_singularities"])


def test_cosine_ratio_table1(orc):
    """Table I: cosine |t| > 1e16 at k = N/4 where |cos theta| ~ 6e-17."""
    g = golden()
    N = 1024
    t, m, p = orc.table(N, orc.COS, orc.FP64)
    assert np.all(p == orc.PATH_COS)
    k = int(np.argmax(np.abs(t)))
    assert k == int(g["cos_tmax_k"])
    assert abs(t[k]) > g["cos_tmax_lower"]
    assert 1e-17 < abs(m[k]) < 1e-16 and round(abs(m[k]), 17) == g["cos_abs_cos_at_quarter"]
    # FP16 rounding of that entry is non-finite / zero: the "divergent" column
    t16, m16, _ = orc.table(N, orc.COS, orc.FP16)
    assert math.isinf(t16[k]) and m16[k] == 0.0


def test_path_distribution_section5(orc):
    """Section V: 256 cosine / 256 sine at N = 1024 (ties at k = N/8 and
    3N/8 resolved by FP64 cos/sin of theta = (-2 pi k)/N and the >= rule)."""
    g = golden()
    _, _, p = orc.table(1024, orc.DS, orc.FP64)
    assert int(np.sum(p == orc.PATH_COS)) == int(g["ds_cos_count"])
    assert int(np.sum(p == orc.PATH_SIN)) == int(g["ds_sin_count"])
    # cosine near 0 and pi, sine near -pi/2
    assert p[0] == orc.PATH_COS and p[511] == orc.PATH_COS and p[256] == orc.PATH_SIN


def test_error_bounds_tables1_2(orc):
    """Table I per-butterfly FP16 bound |t|max * eps and Table II cumulative
    bound (1 + |t|max eps)^m - 1 (Eq. 11) with m = 10, from the oracle's
    ratios."""
    g = golden()
    # the paper evaluates the bounds with the printed eps = 4.88e-4 (2^-11
    # rounded to three digits)
    assert abs(2.0 ** -11 - g["fp16_eps"]) < 1e-6
    eps = g["fp16_eps"]
    lf = orc.table(1024, orc.LF, orc.FP64)[0][1:]
    ds = orc.table(1024, orc.DS, orc.FP16)[0]
    lf_max, ds_max = float(np.max(np.abs(lf))), float(np.max(np.abs(ds)))
    assert round(lf_max * eps, 4) == g["lf_fp16_bound"]
    assert round(ds_max * eps, 6) == g["ds_fp16_bound"]
    lf_cum = (1 + lf_max * eps) ** 10 - 1
    ds_cum = (1 + ds_max * eps) ** 10 - 1
    assert round(lf_cum, 2) == g["lf_cumulative"]
    assert round(ds_cum, 5) == g["ds_cumulative"]
    assert round(lf_cum / ds_cum) == g["improvement"]


@pytest.mark.parametrize("N", [2, 4, 8, 64, 4096, 1 << 16])
def test_table_matches_trig_closed_form(orc, N):
    """FP64 tables reproduce cos/sin: m * (1, t) or m * (t, 1) rebuilds W^k."""
    k = np.arange(N // 2)
    wr, wi = np.cos(-2 * np.pi * k / N), np.sin(-2 * np.pi * k / N)
    for fac in (orc.DS, orc.COS):
        t, m, p = orc.table(N, fac, orc.FP64)
        rr = np.where(p == orc.PATH_COS, m, m * t)
        ii = np.where(p == orc.PATH_COS, m * t, m)
        ok = np.isfinite(t)
        np.testing.assert_allclose(rr[ok], wr[ok], atol=3e-16)
        np.testing.assert_allclose(ii[ok], wi[ok], atol=3e-16)
    t, m, p = orc.table(N, orc.DS, orc.FP64)
    assert np.all(np.abs(t) <= 1) and np.all(np.isfinite(t))


def test_inverse_table_is_conjugate(orc):
    """Inverse twiddles are conj(W): ratio negated everywhere, multiplier
    negated on the sine path, path flags unchanged."""
    for fac in (orc.DS, orc.LF, orc.COS):
        for fmt in (orc.FP32, orc.FP16):
            tf, mf, pf = orc.table(1024, fac, fmt, direction=-1)
            ti, mi, pi = orc.table(1024, fac, fmt, direction=+1)
            np.testing.assert_array_equal(pf, pi)
            np.testing.assert_array_equal(ti, -tf)
            np.testing.assert_array_equal(mi, np.where(pf == orc.PATH_SIN, -mf, mf))


def test_scaled_multiplier_is_half(orc):
    """The x0.5-per-pass table stores RN(m/2): exactly half the unscaled
    multiplier for dual-select (|m| >= 1/sqrt(2) keeps it normal)."""
    for fmt in (orc.FP32, orc.FP16, orc.BF16):
        t0, m0, _ = orc.table(4096, orc.DS, fmt)
        t1, m1, _ = orc.table(4096, orc.DS, fmt, scaled=True)
        np.testing.assert_array_equal(t0, t1)
        np.testing.assert_array_equal(m1, m0 / 2)


def test_table_prefix_property(orc):
    """theta = (-2 pi k)/N scales exactly with N, so the table of N is every
    (Nmax/N)-th entry of the table of Nmax, bit for bit."""
    big = orc.table(1 << 14, orc.DS, orc.FP16)
    for N in (2, 16, 1024, 1 << 13):
        small = orc.table(N, orc.DS, orc.FP16)
        st = (1 << 14) // N
        for a, b in zip(small, big):
            np.testing.assert_array_equal(a, b[::st])
