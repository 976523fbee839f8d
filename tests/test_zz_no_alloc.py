"""fft_exec_batch_noalloc: the mixed-batch entry point that allocates no
device memory, for callers that cannot call cudaMalloc where they transform
(programs that own all device memory through their own pool, latency-bound
loops that must not stall on the allocator).  Its work descriptors live in
one fixed array of the library shared by every call, so this file runs last
and checks two calls in a row against fft_exec on the same plans."""
import numpy as np
import pytest

from gpu_util import assert_bitexact
from paper_2604_00567_b300 import signals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dsfft():
    import paper_2604_00567_b300 as m
    m.lib()
    return m


def _items(dsfft, plans, seed, count):
    """`count` transforms over the given plans with seeded inputs; returns
    (items for the no-alloc call, reference outputs from fft_exec)."""
    import torch
    rng = np.random.default_rng(seed)
    items, refs = [], []
    for k in range(count):
        plan = plans[int(rng.integers(0, len(plans)))]
        d = -1 if rng.random() < 0.6 else 1
        x = signals.signal(seed * 7919 + k, 1, plan.n, plan.precision)
        xt = signals.to_torch(x, plan.precision, "cuda")
        refs.append(signals.from_torch(plan.exec(xt, direction=d), plan.precision))
        items.append((plan, d, xt, torch.empty_like(xt)))
    return items, refs


def test_noalloc_two_calls_match_fft_exec(dsfft):
    import torch
    plans = [dsfft.Plan(1 << l, p, "dual_select")
             for l, p in ((4, "fp32"), (10, "fp16"), (12, "bf16"), (13, "fp32"), (14, "fp16"),
                          (16, "fp16"), (15, "fp32"), (18, "fp16"))]
    for call, seed in enumerate((1, 2)):
        items, refs = _items(dsfft, plans, seed, 40 + 17 * call)
        dsfft.exec_batch_noalloc(items)
        torch.cuda.synchronize()
        for k, ((plan, d, _, out), ref) in enumerate(zip(items, refs)):
            got = signals.from_torch(out, plan.precision)
            assert_bitexact(got, ref, f"call {call} item {k} N={plan.n} {plan.precision} dir={d}")


def test_noalloc_rejects_more_than_the_maximum(dsfft):
    import torch
    plan = dsfft.Plan(64, "fp16", "dual_select")
    x = torch.zeros((1, 64, 2), dtype=torch.float16, device="cuda")
    with pytest.raises(dsfft.DsfftError) as e:
        dsfft.exec_batch_noalloc([(plan, -1, x, x)] * (dsfft.NOALLOC_MAX_ITEMS + 1))
    assert e.value.status == 2
    assert "4096" in str(e.value)
