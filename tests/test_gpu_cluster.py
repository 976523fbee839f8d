"""The cluster kernel (N = 2^15 .. 2^17) on contiguous batches and through
gathered per-transform pointers (mixed batches) gives identical bytes, and a
transform matches the oracle's emulation."""
import pytest

from gpu_util import assert_bitexact, emulate
from paper_2604_00567_b300 import signals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dsfft():
    import paper_2604_00567_b300 as m
    m.lib()
    return m


@pytest.mark.parametrize("prec,log2n", [("fp16", 15), ("fp16", 16), ("fp16", 17), ("bf16", 16), ("fp32", 15),
                                        ("fp32", 16)])
def test_cluster_contiguous_vs_gathered(dsfft, prec, log2n):
    import torch
    n = 1 << log2n
    batch = 300 if log2n < 17 else 160
    x = signals.device_signal(batch, n, prec, seed=log2n)
    plan = dsfft.Plan(n, prec, "dual_select", variant="cluster")
    y = plan.exec(x)
    yb = torch.empty_like(x)
    b = dsfft.Batch([(n, prec, "dual_select", -1, x[i:i + 1], yb[i:i + 1]) for i in range(0, batch, 37)])
    b.exec()
    torch.cuda.synchronize()
    word = torch.int32 if prec == "fp32" else torch.int16
    for i in range(0, batch, 37):
        assert torch.equal(y[i].view(word), yb[i].view(word)), i
    xs = signals.from_torch(x[batch - 1:batch], prec)
    assert_bitexact(signals.from_torch(y[batch - 1:batch], prec), emulate(plan, xs, -1), f"{prec} 2^{log2n} last")
