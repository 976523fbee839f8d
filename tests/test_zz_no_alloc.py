"""fft_exec_batch_noalloc: the mixed-batch entry point that allocates no
device memory, for callers that cannot call cudaMalloc where they transform
(programs that own all device memory through their own pool, latency-bound
loops that must not stall on the allocator).  Its work descriptors live in
one fixed array of the library shared by every call, so this file runs last.

Checked: two calls in a row against fft_exec on the same plans; that a call
returns while earlier work on its stream is still running (it does not wait
for the stream); that it succeeds with every library allocation made to fail
and leaves the device's free memory unchanged; and each refusal path."""
import time

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


@pytest.fixture(scope="module")
def plans(dsfft):
    return [dsfft.Plan(1 << l, p, "dual_select")
            for l, p in ((4, "fp32"), (10, "fp16"), (12, "bf16"), (13, "fp32"), (14, "fp16"),
                         (16, "fp16"), (15, "fp32"), (18, "fp16"))]


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
    torch.cuda.synchronize()
    return items, refs


def _check(items, refs, what):
    for k, ((plan, d, _, out), ref) in enumerate(zip(items, refs)):
        got = signals.from_torch(out, plan.precision)
        assert_bitexact(got, ref, f"{what} item {k} N={plan.n} {plan.precision} dir={d}")


def test_noalloc_two_calls_match_fft_exec(dsfft, plans):
    import torch
    for call, seed in enumerate((1, 2)):
        items, refs = _items(dsfft, plans, seed, 40 + 17 * call)
        dsfft.exec_batch_noalloc(items)
        torch.cuda.synchronize()
        _check(items, refs, f"call {call}")


def test_noalloc_does_not_wait_for_the_stream(dsfft, plans):
    """A call queued behind about half a second of GPU work returns while
    that work is still running: the descriptors go to the device as kernel
    parameters, so nothing waits for the stream.  The work ahead is torch's
    clock-cycle delay kernel, which ends by itself."""
    import torch
    items, refs = _items(dsfft, plans, 3, 30)
    dsfft.exec_batch_noalloc(items)            # same kernels once first: set-up, modules loaded
    torch.cuda.synchronize()
    for _, _, _, out in items:
        out.zero_()
    stream = torch.cuda.current_stream()
    torch.cuda._sleep(1_000_000_000)            # ~0.5 s at 2 GHz on this stream
    ahead = torch.cuda.Event()
    ahead.record(stream)
    t0 = time.perf_counter()
    dsfft.exec_batch_noalloc(items, stream=stream)
    dt = time.perf_counter() - t0
    still_running = not ahead.query()
    torch.cuda.synchronize()
    assert still_running, "the call returned only after the earlier work on its stream had finished"
    assert dt < 0.25, f"the call took {dt:.3f} s"
    _check(items, refs, "behind a long kernel")


def test_noalloc_allocates_nothing(dsfft, plans, monkeypatch):
    """With every library allocation made to fail (DSFFT_FAULT_ALLOC=1: the
    next cudaMalloc the library attempts returns out-of-memory) the call still
    succeeds and is bit-exact, and the device's free memory is the same
    before and after it."""
    import torch
    items, refs = _items(dsfft, plans, 5, 50)
    dsfft.exec_batch_noalloc(items)            # same kernels once first: set-up, modules loaded
    torch.cuda.synchronize()
    for _, _, _, out in items:
        out.zero_()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    monkeypatch.setenv("DSFFT_FAULT_ALLOC", "1")
    dsfft.exec_batch_noalloc(items)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    monkeypatch.delenv("DSFFT_FAULT_ALLOC")
    assert free1 == free0
    _check(items, refs, "fault-injected")
    # the injection is live: a plan creation (which allocates) now fails
    monkeypatch.setenv("DSFFT_FAULT_ALLOC", "1")
    with pytest.raises(dsfft.DsfftError) as e:
        dsfft.Plan(256, "fp16", "dual_select")
    assert e.value.status == 4
    monkeypatch.delenv("DSFFT_FAULT_ALLOC")


def _raw_call(dsfft, entries):
    """Direct C-ABI call with hand-filled items: (plan, direction, reserved,
    in_ptr, out_ptr) tuples."""
    arr = (dsfft.NoAllocItemC * max(1, len(entries)))()
    for i, (plan, d, reserved, pin, pout) in enumerate(entries):
        arr[i].plan = plan.handle.value
        arr[i].direction = d
        arr[i].reserved = reserved
        arr[i].in_ = pin
        arr[i].out = pout
    return dsfft.lib().fft_exec_batch_noalloc(arr, len(entries), None)


def test_noalloc_refusals(dsfft, plans):
    import torch
    sweep = [p for p in plans if p.n == 1 << 18][0]
    assert sweep.info()["kernel"] == 1
    y = torch.zeros((1, 1 << 18, 2), dtype=torch.float16, device="cuda")
    # in place on the HBM-sweep path
    assert _raw_call(dsfft, [(sweep, -1, 0, y.data_ptr(), y.data_ptr())]) == 3
    # radix-4 plans are not batched
    p4 = dsfft.Plan(1024, "fp16", "dual_select", radix=4)
    a = torch.ones((1, 1024, 2), dtype=torch.float16, device="cuda")
    b = torch.zeros_like(a)
    assert _raw_call(dsfft, [(p4, -1, 0, a.data_ptr(), b.data_ptr())]) == 3
    small = [p for p in plans if p.n == 1024][0]
    # nonzero reserved field, bad direction, null pointer, misaligned element
    assert _raw_call(dsfft, [(small, -1, 7, a.data_ptr(), b.data_ptr())]) == 1
    assert _raw_call(dsfft, [(small, 0, 0, a.data_ptr(), b.data_ptr())]) == 1
    assert _raw_call(dsfft, [(small, -1, 0, a.data_ptr(), 0)]) == 1
    assert _raw_call(dsfft, [(small, -1, 0, a.data_ptr() + 2, b.data_ptr())]) == 1
    # an empty list is a no-op; a negative count is refused
    lib = dsfft.lib()
    assert lib.fft_exec_batch_noalloc(None, 0, None) == 0
    assert lib.fft_exec_batch_noalloc(None, -1, None) == 1
    torch.cuda.synchronize()
    # refused calls launch nothing
    assert torch.count_nonzero(y) == 0 and torch.count_nonzero(b) == 0


def test_noalloc_rejects_more_than_the_maximum(dsfft):
    import torch
    plan = dsfft.Plan(64, "fp16", "dual_select")
    x = torch.zeros((1, 64, 2), dtype=torch.float16, device="cuda")
    with pytest.raises(dsfft.DsfftError) as e:
        dsfft.exec_batch_noalloc([(plan, -1, x, x)] * (dsfft.NOALLOC_MAX_ITEMS + 1))
    assert e.value.status == 2
    assert "4096" in str(e.value)


def test_noalloc_full_size_list(dsfft, plans):
    """The maximum item count (descriptors spread over several parameter
    launches) against fft_exec."""
    import torch
    small = [p for p in plans if p.n <= 1 << 12]
    rng = np.random.default_rng(8)
    x = {p.n: signals.to_torch(signals.signal(8000 + p.n, 64, p.n, p.precision), p.precision, "cuda")
         for p in small}
    items, refs = [], []
    outs = {p.n: torch.empty((dsfft.NOALLOC_MAX_ITEMS,) + tuple(x[p.n].shape[1:]), dtype=x[p.n].dtype,
                             device="cuda") for p in small}
    for k in range(dsfft.NOALLOC_MAX_ITEMS):
        p = small[int(rng.integers(0, len(small)))]
        r = int(rng.integers(0, 64))
        items.append((p, -1, x[p.n][r:r + 1], outs[p.n][k:k + 1]))
        refs.append((p, r))
    dsfft.exec_batch_noalloc(items)
    torch.cuda.synchronize()
    expect = {p.n: signals.from_torch(p.exec(x[p.n]), p.precision) for p in small}
    for k, ((p, _, _, out), (_, r)) in enumerate(zip(items, refs)):
        assert_bitexact(signals.from_torch(out, p.precision), expect[p.n][r:r + 1], f"item {k} N={p.n}")
