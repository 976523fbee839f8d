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
    plan.device_status()            # no bounded wait gave up


@pytest.mark.parametrize("prec,log2n", [("fp16", 16), ("bf16", 17)])
def test_cluster_wait_limit_sets_status(dsfft, monkeypatch, prec, log2n):
    """Fault injection: each CTA's mbarrier expects 16 bytes more than the
    other CTAs send, so the wait for the phase-1 data runs out (about 1 s);
    the CTA records it in the plan's status word and skips phase 2, and the
    cluster still leaves together.  No GPU fault: the context stays usable."""
    import torch
    n = 1 << log2n
    monkeypatch.setenv("DSFFT_FAULT_WAIT", "1")
    bad = dsfft.Plan(n, prec, "dual_select", variant="cluster")
    monkeypatch.delenv("DSFFT_FAULT_WAIT")
    x = signals.device_signal(4, n, prec, seed=7)
    bad.exec(x)
    with pytest.raises(dsfft.DsfftError) as e:
        bad.device_status()
    assert e.value.status == 6
    bad.device_status()             # cleared by the read
    good = dsfft.Plan(n, prec, "dual_select", variant="cluster")
    y = good.exec(x)
    torch.cuda.synchronize()
    xs = signals.from_torch(x[3:4], prec)
    assert_bitexact(signals.from_torch(y[3:4], prec), emulate(good, xs, -1), "after the injected timeout")
    good.device_status()
