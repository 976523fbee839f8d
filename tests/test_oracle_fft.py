"""Pins of the oracle's transforms: the FP64 DFT against numpy's FFT, the FP64
radix-2 FFT against the DFT, the 6-FMA butterflies against the 10-op
butterfly of Eqs. 2-3, and the emulated FFT against closed forms (impulse,
constant, tone), Parseval, linearity and the FP32 round trip of Section V."""
import math

import numpy as np
import pytest

from paper_2604_00567_b300 import signals


def _sig(seed, batch, N, prec="fp64"):
    return signals.signal(seed, batch, N, prec)


@pytest.mark.parametrize("N", [1, 2, 3, 8, 60, 256, 1024])
def test_dft_matches_numpy(orc, N):
    x = _sig(3, 2, N)
    np.testing.assert_allclose(orc.dft(x), np.fft.fft(x, axis=-1), rtol=0, atol=1e-12 * N)
    np.testing.assert_allclose(orc.dft(x, sign=+1), np.fft.ifft(x, axis=-1) * N, rtol=0, atol=1e-12 * N)


@pytest.mark.parametrize("N", [2, 4, 16, 512, 4096])
def test_fft_fp64_matches_dft(orc, N):
    x = _sig(4, 3, N)
    for sign in (-1, +1):
        ref = orc.dft(x, sign=sign)
        assert orc.rel_l2(orc.fft_fp64(x, sign=sign), ref) < 1e-13


def test_dft_bin_matches_dft(orc):
    x = _sig(5, 1, 1024)[0]
    ref = orc.dft(x)
    for k in (0, 1, 77, 512, 1023):
        assert abs(orc.dft_bin(x, k) - ref[k]) < 1e-11


def _ten_op(wr, wi, a, b):
    """Eqs. 2-3 in FP64."""
    pr = wr * b.real - wi * b.imag
    pi = wi * b.real + wr * b.imag
    return complex(a.real + pr, a.imag + pi), complex(a.real - pr, a.imag - pi)


@pytest.mark.parametrize("fac", ["DS", "COS", "LF"])
def test_six_fma_forms_reproduce_ten_op_butterfly(orc, fac):
    """Each 6-FMA form (FP64 arithmetic, unrounded FP64 table) equals the
    10-op butterfly up to a few ulp for every twiddle of N = 64, except where
    the factorization itself is singular (cos at k = N/4) or clamped (LF k=0)."""
    N = 64
    f = {"DS": orc.DS, "COS": orc.COS, "LF": orc.LF}[fac]
    t, m, p = orc.table(N, f, orc.FP64)
    rng = np.random.default_rng(6)
    for k in range(N // 2):
        if (fac == "COS" and k == N // 4) or (fac == "LF" and k == 0):
            continue
        th = -2 * math.pi * k / N
        wr, wi = math.cos(th), math.sin(th)
        for _ in range(20):
            a = complex(*rng.uniform(-1, 1, 2))
            b = complex(*rng.uniform(-1, 1, 2))
            A, B = orc.butterfly(orc.FP64, False, t[k], m[k], p[k], a, b)
            A0, B0 = _ten_op(wr, wi, a, b)
            tol = 8e-16 * max(1.0, abs(t[k]))
            assert abs(A - A0) < tol and abs(B - B0) < tol, (k, A, A0, B, B0)


def test_printed_eq4_s2_is_a_misprint(orc):
    """Eq. 4 as printed (s2 = (w_r/w_i) b_r + b_i) gives the wrong A_i; the
    corrected s2 = b_r + (w_r/w_i) b_i, used by the oracle, gives Eq. 2."""
    N, k = 16, 3
    th = -2 * math.pi * k / N
    wr, wi = math.cos(th), math.sin(th)
    t = wr / wi
    a, b = complex(0.3, -0.2), complex(0.7, 0.4)
    A_ref, _ = _ten_op(wr, wi, a, b)
    s2_printed = t * b.real + b.imag
    s2_fixed = b.real + t * b.imag
    assert abs((a.imag + s2_printed * wi) - A_ref.imag) > 1e-2
    assert abs((a.imag + s2_fixed * wi) - A_ref.imag) < 1e-15
    A, _ = orc.butterfly(orc.FP64, False, t, wi, orc.PATH_SIN, a, b)
    assert abs(A - A_ref) < 1e-15


@pytest.mark.parametrize("N", [2, 8, 64, 1024, 4096])
@pytest.mark.parametrize("fac", ["DS", "COS"])
def test_emulator_fp64_is_an_fft(orc, N, fac):
    """With FP64 arithmetic the emulated 6-FMA Stockham FFT is the DFT."""
    f = {"DS": orc.DS, "COS": orc.COS}[fac]
    x = _sig(7, 2, N)
    for d in (-1, +1):
        t, m, p = orc.table(N, f, orc.FP64, direction=d)
        y = orc.emulate_fft(x, orc.FP64, t, m, p)
        assert orc.rel_l2(y, orc.dft(x, sign=d)) < 1e-13 * (1 if fac == "DS" else 1e3)


def test_emulator_lf_clamp_perturbs(orc):
    """The epsilon clamp perturbs W^0 by about eps per pass (Section I), so the
    FP64 Linzer-Feig FFT is off by ~1e-7 while dual-select is exact to FP64."""
    N = 1024
    x = _sig(8, 2, N)
    ref = orc.dft(x)
    t, m, p = orc.table(N, orc.LF, orc.FP64, eps=1e-7)
    err = orc.rel_l2(orc.emulate_fft(x, orc.FP64, t, m, p), ref)
    assert 1e-8 < err < 1e-6


@pytest.mark.parametrize("fmt", ["FP32", "FP16", "BF16"])
@pytest.mark.parametrize("scaled", [False, True])
def test_impulse_gives_ones_exactly(orc, fmt, scaled):
    """delta[0] -> all ones (or all 1/N with x0.5 per pass), bit-exact."""
    f = getattr(orc, fmt)
    N = 256
    x = np.zeros((1, N), dtype=np.complex128)
    x[0, 0] = 1.0
    t, m, p = orc.table(N, orc.DS, f, scaled=scaled)
    y = orc.emulate_fft(x, f, t, m, p, scaled=scaled)
    want = 1.0 / N if scaled else 1.0
    assert np.all(y.real == want) and np.all(y.imag == 0)


@pytest.mark.parametrize("fmt", ["FP32", "FP16", "BF16"])
def test_constant_gives_scaled_delta_exactly(orc, fmt):
    """Constant c -> (N c, 0, ..., 0) bit-exact for dual-select (W^0 is exact:
    t = 0, m = 1); with x0.5 per pass the DC bin is exactly c."""
    f = getattr(orc, fmt)
    N = 1024
    c = complex(0.375, -0.25)
    x = np.full((1, N), c)
    t, m, p = orc.table(N, orc.DS, f)
    y = orc.emulate_fft(x, f, t, m, p)
    assert y[0, 0] == N * c and np.all(y[0, 1:] == 0)
    t, m, p = orc.table(N, orc.DS, f, scaled=True)
    y = orc.emulate_fft(x, f, t, m, p, scaled=True)
    assert y[0, 0] == c and np.all(y[0, 1:] == 0)


def test_constant_leaks_with_lf_clamp(orc):
    """The clamped W^0 of Linzer-Feig leaks the real part into the imaginary
    part of the DC bin (the precision loss Section I describes)."""
    N = 1024
    x = np.full((1, N), complex(0.375, 0.0))
    t, m, p = orc.table(N, orc.LF, orc.FP32, eps=1e-7)
    y = orc.emulate_fft(x, orc.FP32, t, m, p)
    assert y[0, 0].imag != 0.0


def test_tone(orc):
    """A single tone exp(+j 2 pi k0 n/N) transforms to N delta[k - k0]."""
    N, k0 = 512, 37
    n = np.arange(N)
    x = np.exp(2j * np.pi * k0 * n / N)[None, :]
    x32 = orc.round_array(x, orc.FP32)
    t, m, p = orc.table(N, orc.DS, orc.FP32)
    y = orc.emulate_fft(x32, orc.FP32, t, m, p)
    want = np.zeros(N, dtype=np.complex128)
    want[k0] = N
    assert np.max(np.abs(y[0] - want)) < 5e-4


def test_parseval_and_linearity(orc):
    N = 1024
    x = _sig(9, 4, N, "fp32")
    t, m, p = orc.table(N, orc.DS, orc.FP64)
    y = orc.emulate_fft(x, orc.FP64, t, m, p)
    np.testing.assert_allclose(np.sum(np.abs(y) ** 2, axis=1), N * np.sum(np.abs(x) ** 2, axis=1), rtol=1e-12)
    z = orc.emulate_fft(2 * x[:2] - 0.5 * x[2:], orc.FP64, t, m, p)
    np.testing.assert_allclose(z, 2 * y[:2] - 0.5 * y[2:], atol=1e-11)


@pytest.mark.parametrize("fac", ["DS", "LF"])
def test_fp32_round_trip_section5(orc, fac):
    """Section V: FP32 round trip (forward, inverse, /N) has relative L2 error
    ~1e-7 for both Linzer-Feig and dual-select."""
    f = {"DS": orc.DS, "LF": orc.LF}[fac]
    N = 1024
    x = _sig(10, 8, N, "fp32")
    tf, mf, pf = orc.table(N, f, orc.FP32, direction=-1)
    ti, mi, pi = orc.table(N, f, orc.FP32, direction=+1)
    y = orc.emulate_fft(x, orc.FP32, tf, mf, pf)
    z = orc.emulate_fft(y, orc.FP32, ti, mi, pi) / N
    err = orc.rel_l2(z, x)
    assert 2e-8 < err < 5e-7, err


@pytest.mark.parametrize("fmt,tol", [("FP32", 2e-6), ("FP16", 4e-3)])
def test_emulated_accuracy_vs_fp64(orc, fmt, tol):
    """The emulated dual-select FFT meets the stated FP64 tolerances (FP32 on
    raw values, FP16 with x0.5 per pass against DFT/N)."""
    f = getattr(orc, fmt)
    N = 1024
    x = _sig(11, 8, N, fmt.lower())
    scaled = fmt == "FP16"
    t, m, p = orc.table(N, orc.DS, f, scaled=scaled)
    y = orc.emulate_fft(x, f, t, m, p, scaled=scaled)
    ref = orc.dft(x) / (N if scaled else 1)
    assert orc.rel_l2(y, ref) < tol


def test_fp16_lf_and_cosine_are_non_finite(orc):
    """LF (t = 1/eps overflows FP16) and cosine (t = tan at k = N/4 overflows)
    produce non-finite FP16 results: the 'divergent' of Table I."""
    N = 1024
    x = _sig(12, 1, N, "fp16")
    for fac in (orc.LF, orc.COS):
        t, m, p = orc.table(N, fac, orc.FP16, scaled=True)
        y = orc.emulate_fft(x, orc.FP16, t, m, p, scaled=True)
        assert not np.all(np.isfinite(y))


def test_threads_split_is_identical(orc):
    N = 256
    x = _sig(13, 9, N, "fp16")
    t, m, p = orc.table(N, orc.DS, orc.FP16, scaled=True)
    a = orc.emulate_fft(x, orc.FP16, t, m, p, scaled=True, threads=1)
    b = orc.emulate_fft(x, orc.FP16, t, m, p, scaled=True, threads=4)
    np.testing.assert_array_equal(a, b)
