"""Pins of the oracle's emulated FP32/FP16/BF16 arithmetic.

Each emulated operation must equal the IEEE 754 correctly rounded result:
checked against exact rational arithmetic (tests/exact.py), against numpy's
float32/float16 casts, and (FP32) against the C library's fmaf.
"""
import ctypes
import ctypes.util
import math

import numpy as np
import pytest

from exact import exact_fma, rn

FMTS = {"fp32": 1, "fp16": 2, "bf16": 3}


def _random_values(rng, fmt, n):
    """Random finite values of the format, drawn from bit patterns (covers
    subnormals, tiny and huge magnitudes)."""
    if fmt == "fp16":
        bits = rng.integers(0, 1 << 16, size=4 * n, dtype=np.uint32).astype(np.uint16)
        v = bits.view(np.float16).astype(np.float64)
    elif fmt == "bf16":
        bits = rng.integers(0, 1 << 16, size=4 * n, dtype=np.uint32) << np.uint32(16)
        v = bits.astype(np.uint32).view(np.float32).astype(np.float64)
    else:
        bits = rng.integers(0, 1 << 32, size=4 * n, dtype=np.uint64).astype(np.uint32)
        v = bits.view(np.float32).astype(np.float64)
    v = v[np.isfinite(v)]
    return v[:n]


def _near_values(rng, fmt, n, scale_exp):
    """Values of moderate magnitude so that products and sums interact
    (cancellation, ties, carries)."""
    x = rng.uniform(-2, 2, size=n) * 2.0 ** rng.integers(-scale_exp, scale_exp, size=n)
    if fmt == "fp16":
        return x.astype(np.float16).astype(np.float64)
    if fmt == "fp32":
        return x.astype(np.float32).astype(np.float64)
    return np.array([rn(__import__("fractions").Fraction(float(v)), "bf16") for v in x])


@pytest.mark.parametrize("fmt", ["fp16", "fp32"])
def test_round_matches_numpy_cast(orc, fmt):
    rng = np.random.default_rng(1)
    # doubles spanning subnormal, normal and overflow ranges of the format
    x = rng.uniform(-1, 1, 200000) * 2.0 ** rng.integers(-30 if fmt == "fp16" else -160, 20 if fmt == "fp16" else 140, 200000)
    # exact ties: midpoints between adjacent fp16 values
    if fmt == "fp16":
        h = rng.integers(0, 0x7BFF, 5000).astype(np.uint16)
        lo = h.view(np.float16).astype(np.float64)
        hi = (h + 1).astype(np.uint16).view(np.float16).astype(np.float64)
        x = np.concatenate([x, 0.5 * (lo + hi), -0.5 * (lo + hi), [65504.0, 65519.99, 65520.0, 2.0 ** -25, 3 * 2.0 ** -26]])
    ref = x.astype(np.float16 if fmt == "fp16" else np.float32).astype(np.float64)
    got = orc.round_array(x, FMTS[fmt])
    np.testing.assert_array_equal(got, ref)
    # sign of zero survives
    assert math.copysign(1.0, orc.round_to(-1e-30, FMTS[fmt])) == -1.0


def test_round_bf16_matches_exact(orc):
    from fractions import Fraction
    rng = np.random.default_rng(2)
    x = rng.uniform(-1, 1, 20000) * 2.0 ** rng.integers(-140, 128, 20000)
    got = orc.round_array(x, FMTS["bf16"])
    ref = np.array([rn(Fraction(float(v)), "bf16") for v in x])
    np.testing.assert_array_equal(got, ref)


def test_round_bf16_matches_torch_on_fp32_inputs(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    bits = rng.integers(0, 1 << 32, 100000, dtype=np.uint64).astype(np.uint32)
    f = bits.view(np.float32)
    f = f[np.isfinite(f)]
    ref = torch.from_numpy(f.copy()).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    got = orc.round_array(f.astype(np.float64), FMTS["bf16"])
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("fmt", ["fp16", "bf16", "fp32"])
def test_fma_matches_exact_rational(orc, fmt):
    rng = np.random.default_rng(10 + FMTS[fmt])
    n = 3000
    sets = [
        (_random_values(rng, fmt, n), _random_values(rng, fmt, n), _random_values(rng, fmt, n)),
        (_near_values(rng, fmt, n, 6), _near_values(rng, fmt, n, 6), _near_values(rng, fmt, n, 6)),
    ]
    for a, b, c in sets:
        for i in range(min(len(a), len(b), len(c))):
            want = exact_fma(a[i], b[i], c[i], fmt)
            got = orc.fma(a[i], b[i], c[i], FMTS[fmt])
            assert (got == want and math.copysign(1, got) == math.copysign(1, want)) or (
                math.isnan(got) and math.isnan(want)), (fmt, a[i], b[i], c[i], got, want)


def test_fma_fp32_matches_libm_fmaf(orc):
    libm = ctypes.CDLL(ctypes.util.find_library("m"))
    libm.fmaf.restype = ctypes.c_float
    libm.fmaf.argtypes = [ctypes.c_float] * 3
    rng = np.random.default_rng(20)
    a = _near_values(rng, "fp32", 50000, 20)
    b = _near_values(rng, "fp32", 50000, 20)
    c = _near_values(rng, "fp32", 50000, 20)
    for i in range(len(a)):
        want = libm.fmaf(a[i], b[i], c[i])
        got = orc.fma(a[i], b[i], c[i], FMTS["fp32"])
        assert got == want, (a[i], b[i], c[i], got, want)


@pytest.mark.parametrize("fmt", ["fp16", "bf16", "fp32"])
def test_fma_special_values(orc, fmt):
    f = FMTS[fmt]
    inf = math.inf
    assert orc.fma(inf, 1.0, 1.0, f) == inf
    assert math.isnan(orc.fma(inf, 0.0, 1.0, f))
    assert math.isnan(orc.fma(inf, 1.0, -inf, f))
    assert math.isnan(orc.fma(math.nan, 1.0, 1.0, f))
    # exact cancellation gives +0 under round-to-nearest
    z = orc.fma(2.0, 3.0, -6.0, f)
    assert z == 0.0 and math.copysign(1, z) == 1.0
    z = orc.fma(-0.0, 1.0, -0.0, f)
    assert z == 0.0 and math.copysign(1, z) == -1.0
    # overflow of the rounded result
    big = {"fp16": 65504.0, "bf16": 3.3895313892515355e38, "fp32": 3.4028234663852886e38}[fmt]
    assert orc.fma(big, 2.0, 0.0, f) == inf
    assert orc.mul(big, 0.5, f) == big / 2


def test_mul_half_is_exact_except_subnormal(orc):
    """x * 0.5 is exact for normal fp16 values (the per-pass scaling step) and
    rounds to even for the smallest subnormals."""
    h = np.arange(0, 0x7C00, dtype=np.uint16).view(np.float16).astype(np.float64)
    got = np.array([orc.mul(v, 0.5, FMTS["fp16"]) for v in h])
    normal = h >= 2.0 ** -13
    np.testing.assert_array_equal(got[normal], h[normal] / 2)
    ref = (h / 2).astype(np.float16).astype(np.float64)
    np.testing.assert_array_equal(got, ref)
