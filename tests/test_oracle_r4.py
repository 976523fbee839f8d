"""Pins of the oracle's radix-4 dual-select FFT (orc_emulate_fft_r4, the
radix-4 extension the paper's Discussion proposes): with FP64 arithmetic it is
the DFT (any index, sign, twiddle or operand mistake breaks this), closed
forms come out bit-exact, the rounded forms stay within the accuracy of the
radix-2 form and of Eq. 11, and forward/inverse round-trip."""
import numpy as np
import pytest

from paper_2604_00567_b300 import signals


def _sig(seed, batch, N, prec="fp64"):
    return signals.signal(seed, batch, N, prec)


def _tables(orc, N, fac, fmt, direction=-1, scaled=False):
    t4, m4, p4 = orc.table4(N, fac, fmt, direction=direction, scaled=scaled)
    t2, m2, p2 = orc.table(N, fac, fmt, direction=direction, scaled=scaled)
    return (t4, m4, p4), (t2[0], m2[0], p2[0])


def _run(orc, x, fmt, fac=None, direction=-1, scaled=False):
    N = x.shape[-1]
    fac = orc.DS if fac is None else fac
    (t4, m4, p4), e0 = _tables(orc, N, fac, fmt, direction, scaled)
    return orc.emulate_fft_r4(x, fmt, t4, m4, p4, e0, scaled=scaled, inverse=direction > 0)


def test_table4_extends_table(orc):
    """The first N/2 radix-4 entries are the radix-2 table; beyond N/2 the
    angles pass -pi and the selection still follows |cos| >= |sin|."""
    N = 1024
    for fmt in (orc.FP64, orc.FP16):
        t4, m4, p4 = orc.table4(N, orc.DS, fmt)
        t2, m2, p2 = orc.table(N, orc.DS, fmt)
        assert np.array_equal(t4[:N // 2], t2) and np.array_equal(m4[:N // 2], m2)
        assert np.array_equal(p4[:N // 2], p2)
        k = np.arange(3 * N // 4)
        th = (-2.0 * np.pi * k) / N
        want = (np.abs(np.cos(th)) >= np.abs(np.sin(th))).astype(np.int32)
        assert np.array_equal(p4 == orc.PATH_COS, want == 1)
    t4, m4, _ = orc.table4(N, orc.DS, orc.FP64)
    assert np.max(np.abs(t4)) <= 1.0 + 1e-15                       # Theorem 1 over the whole range
    k = np.arange(3 * N // 4)
    w = np.exp(-2j * np.pi * k / N)
    # W = m (1 + i t) on the cosine path, m (t + i) on the sine path
    _, _, p4 = orc.table4(N, orc.DS, orc.FP64)
    rebuilt = np.where(p4 == orc.PATH_COS, m4 * (1 + 1j * t4), m4 * (t4 + 1j))
    np.testing.assert_allclose(rebuilt, w, rtol=0, atol=1e-15)
    ts, ms, _ = orc.table4(N, orc.DS, orc.FP16, scaled=True)
    tu, mu, _ = orc.table4(N, orc.DS, orc.FP16, scaled=False)
    assert np.array_equal(ts, tu) and np.array_equal(ms, mu / 4)    # RN(m/4) = RN(m)/4 (normal range)


@pytest.mark.parametrize("N", [2, 4, 8, 16, 32, 64, 128, 1024, 2048, 4096])
@pytest.mark.parametrize("fac", ["DS", "COS"])
def test_r4_fp64_is_the_dft(orc, N, fac):
    """Odd and even log2 N (radix-2 first pass or not), both directions."""
    f = {"DS": orc.DS, "COS": orc.COS}[fac]
    x = _sig(11, 3, N)
    for d in (-1, +1):
        y = _run(orc, x, orc.FP64, f, direction=d)
        tol = 1e-13 if fac == "DS" else 1e-10
        assert orc.rel_l2(y, orc.dft(x, sign=d)) < tol, (N, d)


def test_r4_hand_example_n4(orc):
    """N = 4: one radix-4 butterfly with W^0: X = [10, -2+2i, -2, -2-2i] for
    x = [1, 2, 3, 4] (forward), and the conjugate pattern inverse."""
    x = np.array([[1, 2, 3, 4]], dtype=np.complex128)
    for fmt in (orc.FP32, orc.FP16, orc.BF16):
        y = _run(orc, x, fmt)
        assert np.array_equal(y[0], np.array([10, -2 + 2j, -2, -2 - 2j]))
        y = _run(orc, x, fmt, direction=+1)
        assert np.array_equal(y[0], np.array([10, -2 - 2j, -2, -2 + 2j]))


@pytest.mark.parametrize("fmt", ["FP32", "FP16", "BF16"])
@pytest.mark.parametrize("N", [256, 512])
@pytest.mark.parametrize("scaled", [False, True])
def test_r4_impulse_gives_ones_exactly(orc, fmt, N, scaled):
    f = getattr(orc, fmt)
    x = np.zeros((1, N), dtype=np.complex128)
    x[0, 0] = 1.0
    y = _run(orc, x, f, scaled=scaled)
    want = 1.0 / N if scaled else 1.0
    assert np.all(y.real == want) and np.all(y.imag == 0)


@pytest.mark.parametrize("fmt", ["FP32", "FP16", "BF16"])
@pytest.mark.parametrize("N", [1024, 2048])
def test_r4_constant_gives_delta_exactly(orc, fmt, N):
    f = getattr(orc, fmt)
    c = complex(0.375, -0.25)
    x = np.full((1, N), c)
    y = _run(orc, x, f)
    assert y[0, 0] == N * c and np.all(y[0, 1:] == 0)
    y = _run(orc, x, f, scaled=True)
    assert y[0, 0] == c and np.all(y[0, 1:] == 0)


@pytest.mark.parametrize("fmt,tol", [("FP32", 3e-7), ("FP16", 2.5e-3), ("BF16", 2e-2)])
@pytest.mark.parametrize("N", [1024, 2048, 4096])
def test_r4_accuracy_matches_radix2(orc, fmt, tol, N):
    """Rounded radix-4 error vs the FP64 DFT: same order as the radix-2 form
    (within a factor 1.5) and inside the tolerance of the format."""
    f = getattr(orc, fmt)
    prec = {"FP32": "fp32", "FP16": "fp16", "BF16": "bf16"}[fmt]
    scaled = fmt != "FP32"
    x = _sig(5, 4, N, prec)
    ref = orc.dft(x) / (N if scaled else 1)
    e4 = orc.rel_l2(_run(orc, x, f, scaled=scaled), ref)
    t, m, p = orc.table(N, orc.DS, f, scaled=scaled)
    e2 = orc.rel_l2(orc.emulate_fft(x, f, t, m, p, scaled=scaled), ref)
    assert e4 < tol and e4 < 1.5 * e2 and e2 < 1.5 * e4 * 1.5


@pytest.mark.parametrize("N", [1024, 2048])
def test_r4_fp32_round_trip(orc, N):
    x = _sig(9, 2, N, "fp32")
    y = _run(orc, x, orc.FP32)
    z = _run(orc, y, orc.FP32, direction=+1)
    assert orc.rel_l2(z / N, x) < 3e-7


def test_r4_threads_split_is_identical(orc):
    N = 512
    x = _sig(4, 9, N, "fp16")
    (t4, m4, p4), e0 = _tables(orc, N, orc.DS, orc.FP16, scaled=True)
    a = orc.emulate_fft_r4(x, orc.FP16, t4, m4, p4, e0, scaled=True, threads=1)
    b = orc.emulate_fft_r4(x, orc.FP16, t4, m4, p4, e0, scaled=True, threads=4)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
