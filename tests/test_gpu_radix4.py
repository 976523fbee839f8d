"""Radix-4 dual-select plans (the radix-4 extension of the Discussion): the
fused radix-4 kernel is bit-exact against the oracle's radix-4 emulation fed
with the plan's own downloaded tables, for every N = 2..2^14, all precisions,
both directions, scaled and unscaled; its radix-4 table matches the oracle's
and its accuracy matches the radix-2 plans'."""
import numpy as np
import pytest

import oracle as orc
from gpu_util import FMT, FAC, assert_bitexact, gpu_fft
from paper_2604_00567_b300 import signals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dsfft():
    import paper_2604_00567_b300 as m
    m.lib()
    return m


def emulate_r4(plan, x, direction=-1):
    t4, m4, p4 = plan.table4(direction)
    t2, m2, p2 = plan.table(direction)
    scaled = plan.scale_forward if direction < 0 else plan.scale_inverse
    return orc.emulate_fft_r4(x, FMT[plan.precision], t4, m4, p4, (t2[0], m2[0], p2[0]), scaled=scaled,
                              inverse=direction > 0, threads=8)


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("log2n", list(range(1, 15)))
def test_radix4_bitexact(dsfft, prec, log2n):
    n = 1 << log2n
    batch = max(3, min(64, (1 << 16) // n)) + 1        # ragged tail of the last block
    x = signals.signal(100 + log2n, batch, n, prec)
    plan = dsfft.Plan(n, prec, "dual_select", radix=4)
    assert plan.info()["radix"] == 4
    for d in (-1, 1):
        y = gpu_fft(plan, x, direction=d)
        assert_bitexact(y, emulate_r4(plan, x, d), f"radix-4 {prec} N=2^{log2n} d={d}")


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("log2n", [5, 10, 13])
def test_radix4_unscaled_and_inverse_scaled(dsfft, prec, log2n):
    n = 1 << log2n
    x = signals.signal(7, 5, n, prec, dist="gaussian")
    plan = dsfft.Plan(n, prec, "dual_select", radix=4, scale_forward=False, scale_inverse=True)
    for d in (-1, 1):
        assert_bitexact(gpu_fft(plan, x, direction=d), emulate_r4(plan, x, d), f"{prec} 2^{log2n} d={d}")


@pytest.mark.parametrize("fac", ["linzer_feig_clamped", "cosine"])
def test_radix4_other_tables_fp32(dsfft, fac):
    n = 4096
    x = signals.signal(3, 4, n, "fp32")
    plan = dsfft.Plan(n, "fp32", fac, radix=4)
    assert_bitexact(gpu_fft(plan, x), emulate_r4(plan, x), f"fp32 {fac}")


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_radix4_table_matches_oracle(dsfft, prec):
    """The GPU's radix-4 table (k < 3N/4) equals the oracle's rounding of the
    host FP64 values except where the two FP64 sin/cos differ across a
    rounding boundary (at most a handful of entries)."""
    n = 1 << 14
    plan = dsfft.Plan(n, prec, "dual_select", radix=4)
    for d in (-1, 1):
        t, m, p = plan.table4(d)
        scaled = plan.scale_forward if d < 0 else plan.scale_inverse
        ot, om, op = orc.table4(n, orc.DS, FMT[prec], direction=d, scaled=scaled)
        assert len(t) == 3 * n // 4
        diff = (t != ot) | (m != om) | (p != op)
        assert diff.sum() <= 4, int(diff.sum())
        assert np.max(np.abs(t)) <= 1.0


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-6), ("fp16", 4e-3)])
def test_radix4_accuracy_vs_fp64(dsfft, prec, tol):
    n = 1 << 14
    x = signals.signal(21, 8, n, prec)
    plan = dsfft.Plan(n, prec, "dual_select", radix=4)
    y = gpu_fft(plan, x)
    ref = np.fft.fft(x, axis=-1) / (n if plan.scale_forward else 1)
    err = orc.rel_l2(y, ref)
    assert err < tol


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("log2n", [15, 16, 17, 18, 19, 20])
def test_radix4_sweeps_bitexact(dsfft, prec, log2n):
    """N > 2^14: two HBM sweeps of whole radix-4 passes (sweep 1 also holds
    the radix-2 pass of an odd log2 N)."""
    n = 1 << log2n
    batch = 3 if log2n <= 17 else 1
    x = signals.signal(300 + log2n, batch, n, prec)
    plan = dsfft.Plan(n, prec, "dual_select", radix=4)
    info = plan.info()
    assert info["radix"] == 4 and info["kernel"] == 1 and info["launches"] == 2
    for d in (-1, 1):
        y = gpu_fft(plan, x, direction=d)
        assert_bitexact(y, emulate_r4(plan, x, d), f"radix-4 sweeps {prec} N=2^{log2n} d={d}")


def test_radix4_sweeps_largest(dsfft):
    n = 1 << 22
    x = signals.signal(5, 1, n, "fp16")
    plan = dsfft.Plan(n, "fp16", "dual_select", radix=4)
    assert_bitexact(gpu_fft(plan, x), emulate_r4(plan, x), "radix-4 fp16 N=2^22")
