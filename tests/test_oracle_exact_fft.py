"""Independent pin of the oracle's rounded operation sequence.

The emulator (``orc.emulate_fft``) is checked elsewhere against closed forms
(impulse, constant) in which every product is exact, so a slip in its
rounding sequence (an FMA done as a rounded multiply plus a rounded add, a
missing RN(a/2), a rounding in the wrong format) could survive those pins.
Here whole transforms at N = 2, 4, 8, 16 are recomputed with exact rational
arithmetic (``tests/exact.py``: Fraction products and sums, one
round-to-nearest-even per operation at the target format, gradual
underflow) and must equal the emulator bit for bit.

The reference is written independently of the oracle's Stockham loop: a
recursive radix-2 decimation in time, X[j] = E[j] + W^j O[j] and
X[j + M/2] = E[j] - W^j O[j] for the length-M sub-transforms of the even
and odd samples, which applies the same butterflies (same operands, same
twiddle index j N/M) as the passes of Section IV.  The butterflies are the
paper's branched forms: the cosine path of Eqs. 7-9 (t = w_i/w_r, m = w_r)
and the sine path of Eqs. 4-6 with the corrected s2 = b_r + t b_i
(t = w_r/w_i, m = w_i).  With x0.5 per pass the a operand is RN(a/2) and the
table multiplier is the halved entry.  The table entries are the oracle's
rounded table (pinned by test_oracle_table.py).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from exact import exact_fma, rn
from paper_2604_00567_b300 import signals

FMTS = ("fp16", "bf16", "fp32")


INEXACT_HALVES = [0]


def _half(a: float, fmt: str) -> float:
    """RN(a / 2) in ``fmt`` (the x0.5 of a scaled pass; inexact only when the
    result is subnormal).  Counts the inexact ones."""
    r = rn(Fraction(a) / 2, fmt, zero_sign=a)
    if Fraction(r) != Fraction(a) / 2:
        INEXACT_HALVES[0] += 1
    return r


def _butterfly(a: complex, b: complex, t: float, m: float, path: int, scaled: bool, fmt: str, fused=True):
    """Branched 6-FMA butterfly, each operation rounded once.  ``fused=False``
    rounds every product before its addition (a deliberately wrong sequence,
    used only to show that this comparison can tell the two apart)."""
    def fma(x, y, z):
        if fused:
            return exact_fma(x, y, z, fmt)
        p = rn(Fraction(x) * Fraction(y), fmt, zero_sign=math.copysign(1.0, x) * math.copysign(1.0, y))
        return exact_fma(p, 1.0, z, fmt)

    ar, ai, br, bi = a.real, a.imag, b.real, b.imag
    if scaled:
        ar, ai = _half(ar, fmt), _half(ai, fmt)
    if path == 0:
        # cosine path, Eq. 7: s1 = b_r - t b_i, s2 = t b_r + b_i; Eqs. 8-9
        s1 = fma(-t, bi, br)
        s2 = fma(t, br, bi)
        A = (fma(s1, m, ar), fma(s2, m, ai))
        B = (fma(-s1, m, ar), fma(-s2, m, ai))
    else:
        # sine path, Eq. 4 (s2 corrected): s1 = b_i - t b_r, s2 = b_r + t b_i;
        # Eqs. 5-6: A_r = a_r - s1 w_i, A_i = a_i + s2 w_i
        s1 = fma(-t, br, bi)
        s2 = fma(t, bi, br)
        A = (fma(-s1, m, ar), fma(s2, m, ai))
        B = (fma(s1, m, ar), fma(-s2, m, ai))
    return A, B


def _fft_exact(x, N, t, m, path, scaled, fmt, fused=True):
    """Recursive radix-2 DIT on the list ``x`` (length M dividing N): the
    sub-transform butterflies use table index j N/M."""
    M = len(x)
    if M == 1:
        return [(x[0].real, x[0].imag)]
    E = _fft_exact(x[0::2], N, t, m, path, scaled, fmt, fused)
    O = _fft_exact(x[1::2], N, t, m, path, scaled, fmt, fused)
    out = [None] * M
    for j in range(M // 2):
        k = j * (N // M)
        A, B = _butterfly(complex(*E[j]), complex(*O[j]), float(t[k]), float(m[k]), int(path[k]), scaled, fmt,
                          fused)
        out[j] = A
        out[j + M // 2] = B
    return out


def _to_array(pairs):
    y = np.empty(len(pairs), dtype=np.complex128)
    y.real = [p[0] for p in pairs]      # assigned, not computed: keeps -0
    y.imag = [p[1] for p in pairs]
    return y


def _assert_same_bits(y, ref, what):
    for part in ("real", "imag"):
        a, b = getattr(y, part), getattr(ref, part)
        bad = (a != b) | (np.signbit(a) != np.signbit(b))
        assert not np.any(bad), f"{what} {part}: oracle {a[bad][:4]} vs exact {b[bad][:4]}"


def _cases():
    for fmt in FMTS:
        for fac in ("DS", "LF", "COS"):
            if fmt == "fp16" and fac == "COS":
                continue   # t = tan(theta) overflows FP16 at k = N/4 (non-finite table)
            yield fmt, fac


@pytest.mark.parametrize("fmt,fac", list(_cases()))
@pytest.mark.parametrize("N", [2, 4, 8, 16])
def test_emulator_equals_exact_rational_fft(orc, fmt, fac, N):
    """Uniform inputs, both directions, scaled and unscaled."""
    ofmt = {"fp32": orc.FP32, "fp16": orc.FP16, "bf16": orc.BF16}[fmt]
    f = {"DS": orc.DS, "LF": orc.LF, "COS": orc.COS}[fac]
    # LF in FP16 needs a clamp whose ratio 1/eps stays finite (reading of the
    # Section I clamp); FP32/BF16 use the default eps = 1e-7
    eps = 2.0 ** -14 if (fac == "LF" and fmt == "fp16") else 1e-7
    x = signals.signal(9100 + N, 3, N, fmt)
    for direction in (-1, 1):
        for scaled in (False, True):
            t, m, p = orc.table(N, f, ofmt, direction=direction, scaled=scaled, eps=eps)
            assert np.all(np.isfinite(t)) and np.all(np.isfinite(m))
            y = orc.emulate_fft(x, ofmt, t, m, p, scaled=scaled)
            for r in range(x.shape[0]):
                ref = _to_array(_fft_exact(list(x[r]), N, t, m, p, scaled, fmt))
                _assert_same_bits(y[r], ref, f"N={N} {fmt} {fac} dir={direction} scaled={scaled} row {r}")


@pytest.mark.parametrize("fmt", FMTS)
def test_emulator_equals_exact_rational_fft_near_underflow(orc, fmt):
    """Inputs scaled towards the subnormal range, so that RN(a/2) and the
    FMAs round at gradual underflow (the cases where x0.5 is inexact)."""
    ofmt = {"fp32": orc.FP32, "fp16": orc.FP16, "bf16": orc.BF16}[fmt]
    shift = {"fp16": -12, "bf16": -124, "fp32": -124}[fmt]
    N = 16
    x = signals.signal(9200, 4, N, "fp64") * 2.0 ** shift
    x = signals.round_storage(x.real, fmt) + 1j * signals.round_storage(x.imag, fmt)
    INEXACT_HALVES[0] = 0
    for direction in (-1, 1):
        for scaled in (False, True):
            t, m, p = orc.table(N, orc.DS, ofmt, direction=direction, scaled=scaled)
            y = orc.emulate_fft(x, ofmt, t, m, p, scaled=scaled)
            for r in range(x.shape[0]):
                ref = _to_array(_fft_exact(list(x[r]), N, t, m, p, scaled, fmt))
                _assert_same_bits(y[r], ref, f"underflow N={N} {fmt} dir={direction} scaled={scaled} row {r}")
    assert INEXACT_HALVES[0] > 0, "the inputs did not reach the range where x0.5 rounds"


def test_signed_zero_inputs(orc):
    """Zeros of both signs on both operands: the sign rules of exact zero
    results are those of IEEE round-to-nearest."""
    N = 8
    base = np.array([0.0, -0.0, 0.5, -0.0, 0.0, -0.25, -0.0, 0.0])
    x = np.empty((1, N), dtype=np.complex128)
    x.real = base
    x.imag = base[::-1].copy()
    for fmt in FMTS:
        ofmt = {"fp32": orc.FP32, "fp16": orc.FP16, "bf16": orc.BF16}[fmt]
        for scaled in (False, True):
            t, m, p = orc.table(N, orc.DS, ofmt, scaled=scaled)
            y = orc.emulate_fft(x, ofmt, t, m, p, scaled=scaled)
            ref = _to_array(_fft_exact(list(x[0]), N, t, m, p, scaled, fmt))
            _assert_same_bits(y[0], ref, f"signed zeros {fmt} scaled={scaled}")


def test_comparison_detects_unfused_rounding(orc):
    """The comparison above has the power to catch a rounding slip: the same
    recursive FFT with every product rounded before its addition differs
    from the emulator (FP16, N = 16), while the fused one agrees."""
    N = 16
    x = signals.signal(9300, 2, N, "fp16")
    t, m, p = orc.table(N, orc.DS, orc.FP16, scaled=True)
    y = orc.emulate_fft(x, orc.FP16, t, m, p, scaled=True)
    differs = 0
    for r in range(x.shape[0]):
        good = _to_array(_fft_exact(list(x[r]), N, t, m, p, True, "fp16"))
        bad = _to_array(_fft_exact(list(x[r]), N, t, m, p, True, "fp16", fused=False))
        _assert_same_bits(y[r], good, "fused")
        differs += int(np.sum((y[r] != bad)))
    assert differs > 0
