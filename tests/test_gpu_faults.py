"""Failure paths without a GPU fault: injected allocation failures
(DSFFT_FAULT_ALLOC) make plan, batch, pipeline and server creation return
FFT_ERR_OOM, free what they had allocated and leave the library usable; and
guard bands around output buffers stay untouched by every kernel path."""
import os

import pytest

from paper_2604_00567_b300 import signals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dsfft():
    import paper_2604_00567_b300 as m
    m.lib()
    return m


@pytest.fixture
def fault():
    def set_k(k):
        if k is None:
            os.environ.pop("DSFFT_FAULT_ALLOC", None)
        else:
            os.environ["DSFFT_FAULT_ALLOC"] = str(k)
    yield set_k
    os.environ.pop("DSFFT_FAULT_ALLOC", None)


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_plan_creation_oom_is_clean(dsfft, fault, k):
    n = 1 << 20                                   # 16 MB + 8 MB of tables per direction
    before = _free_bytes()
    fault(k)
    with pytest.raises(dsfft.DsfftError) as ei:
        dsfft.Plan(n, "fp16", "dual_select")
    assert ei.value.status == 4
    fault(None)
    assert abs(_free_bytes() - before) < (4 << 20)  # nothing left allocated
    p = dsfft.Plan(n, "fp16", "dual_select")       # the library still works
    assert p.info()["n"] == n


def test_other_creators_oom(dsfft, fault):
    import torch
    plan = dsfft.Plan(1024, "fp16", "dual_select")
    fault(1)
    with pytest.raises(dsfft.DsfftError) as ei:
        dsfft.Pipeline(plan, 16, 2)
    assert ei.value.status == 4
    fault(2)
    with pytest.raises(dsfft.DsfftError) as ei:
        dsfft.Server(memory_budget=1 << 24)
    assert ei.value.status == 4
    fault(None)
    x = torch.zeros(1, 1024, 2, dtype=torch.float16, device="cuda")
    y = torch.zeros_like(x)
    fault(7)                                       # the batch's own plan is created first
    with pytest.raises(dsfft.DsfftError) as ei:
        dsfft.Batch([(1024, "fp16", "dual_select", -1, x, y)])
    assert ei.value.status == 4
    fault(None)
    dsfft.Batch([(1024, "fp16", "dual_select", -1, x, y)]).exec()
    torch.cuda.synchronize()


@pytest.mark.parametrize("prec,log2n,variant,radix", [
    ("fp16", 5, "auto", 2), ("fp16", 10, "auto", 2), ("fp32", 12, "fused_narrow", 2), ("bf16", 14, "auto", 2),
    ("fp16", 15, "cluster", 2), ("fp16", 16, "cluster", 2), ("fp32", 16, "sweeps", 2), ("fp16", 17, "sweeps", 2),
    ("fp16", 17, "cluster", 2), ("fp32", 16, "cluster", 2), ("fp32", 15, "cluster", 2),
    ("fp16", 11, "auto", 4), ("fp32", 16, "auto", 4)])
def test_guard_bands_untouched(dsfft, prec, log2n, variant, radix):
    """The output lies between two guard transforms filled with a pattern;
    after the transform the guards are unchanged."""
    import torch
    n = 1 << log2n
    batch = 5 if log2n <= 14 else 3
    x = signals.device_signal(batch, n, prec, seed=log2n)
    plan = dsfft.Plan(n, prec, "dual_select", variant=variant, radix=radix)
    buf = torch.empty((batch + 2,) + tuple(x.shape[1:]), dtype=x.dtype, device="cuda")
    word = torch.int32 if prec == "fp32" else torch.int16
    buf.view(word).fill_(0x5A5A)
    guard = buf.view(word)[0].clone()
    out = buf[1:batch + 1]
    plan.exec(x, out=out)
    plan.exec(x, direction=1, out=out)
    torch.cuda.synchronize()
    assert torch.equal(buf.view(word)[0], guard) and torch.equal(buf.view(word)[batch + 1], guard)
