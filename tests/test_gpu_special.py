"""IEEE special values through every kernel path: inputs with +-inf, NaN,
-0, subnormals and values near the format's maximum (overflow to inf in the
unscaled direction) give the oracle's results: equal finite values, equal
signs of zeros and infinities, NaN in the same positions."""
import numpy as np
import pytest

import oracle as orc
from gpu_util import FMT, assert_bitexact, emulate, gpu_fft
from paper_2604_00567_b300 import signals

pytestmark = pytest.mark.gpu

MAXV = {"fp32": 3.4028234663852886e38, "fp16": 65504.0, "bf16": 3.3895313892515355e38}


@pytest.fixture(scope="module")
def dsfft():
    import paper_2604_00567_b300 as m
    m.lib()
    return m


def _special_inputs(prec, batch, n, seed):
    rng = np.random.default_rng(seed)
    x = signals.signal(seed, batch, n, prec)
    specials = np.array([np.inf, -np.inf, np.nan, -0.0, 0.0, MAXV[prec], -MAXV[prec],
                         MAXV[prec] / 2, 2.0 ** -24 if prec == "fp16" else 1e-40])
    re = x.real.copy()
    im = x.imag.copy()
    # transform 0: clean; 1: one inf; 2: one NaN; 3: large values (overflow when unscaled);
    # others: a sprinkle of every special value
    re[1, n // 3] = np.inf
    im[2, 5] = np.nan
    re[3, :] = MAXV[prec] * np.sign(re[3, :] + 0.5)
    for b in range(4, batch):
        idx = rng.integers(0, n, 6)
        re[b, idx] = rng.choice(specials, 6)
        im[b, idx[::-1]] = rng.choice(specials, 6)
    y = np.empty_like(x)
    y.real = signals.round_storage(re, prec)
    y.imag = signals.round_storage(im, prec)
    return y


@pytest.mark.parametrize("prec,log2n,variant", [("fp16", 10, "auto"), ("bf16", 12, "auto"), ("fp32", 11, "auto"),
                                                ("fp16", 15, "cluster"), ("fp16", 16, "sweeps"),
                                                ("fp32", 15, "cluster")])
def test_special_values_bitexact(dsfft, prec, log2n, variant):
    n = 1 << log2n
    x = _special_inputs(prec, 7, n, 40 + log2n)
    for scale in (True, False):
        plan = dsfft.Plan(n, prec, "dual_select", variant=variant, scale_forward=scale)
        for d in (-1, 1):
            assert_bitexact(gpu_fft(plan, x, d), emulate(plan, x, d), f"{prec} 2^{log2n} {variant} s={scale} d={d}")


@pytest.mark.parametrize("prec,log2n", [("fp16", 11), ("fp32", 15)])
def test_special_values_radix4(dsfft, prec, log2n):
    n = 1 << log2n
    x = _special_inputs(prec, 6, n, 90 + log2n)
    plan = dsfft.Plan(n, prec, "dual_select", radix=4)
    for d in (-1, 1):
        t4, m4, p4 = plan.table4(d)
        t2, m2, p2 = plan.table(d)
        scaled = plan.scale_forward if d < 0 else plan.scale_inverse
        ref = orc.emulate_fft_r4(x, FMT[prec], t4, m4, p4, (t2[0], m2[0], p2[0]), scaled=scaled, inverse=d > 0,
                                 threads=6)
        assert_bitexact(gpu_fft(plan, x, d), ref, f"radix-4 {prec} 2^{log2n} d={d}")
