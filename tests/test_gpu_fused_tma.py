"""The persistent fused kernel fed by bulk asynchronous copies (variant
fused_tma, 2^8 <= N <= 2^14): bit-exact against the oracle's emulation,
equal to the wide fused kernel on batches that give every block several
tiles (double-buffer refills, ragged last tile), in place, with an
unaligned input (the wide kernel runs), and its bounded copy wait reported
through the plan's device status word."""
import numpy as np
import pytest

from gpu_util import assert_bitexact, emulate, gpu_fft
from paper_2604_00567_b300 import signals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dsfft():
    import paper_2604_00567_b300 as m
    m.lib()
    return m


@pytest.mark.parametrize("prec", ["fp16", "fp32", "bf16"])
@pytest.mark.parametrize("log2n", [8, 9, 10, 11, 12, 13, 14])
def test_tma_bitexact_vs_oracle(dsfft, prec, log2n):
    N = 1 << log2n
    if prec == "fp32" and log2n == 14:      # two buffers would exceed a block's shared memory
        with pytest.raises(dsfft.DsfftError) as e:
            dsfft.Plan(N, prec, "dual_select", variant="fused_tma")
        assert e.value.status == 3
        return
    plan = dsfft.Plan(N, prec, "dual_select", variant="fused_tma")
    info = plan.info()
    assert info["variant_name"] == "fused_tma" and info["kernel"] == 0
    batch = 3 * info["transforms_per_block"] + 1          # ragged last tile
    x = signals.signal(1100 + log2n, batch, N, prec)
    for d in (-1, 1):
        assert_bitexact(gpu_fft(plan, x, d), emulate(plan, x, d), f"tma N=2^{log2n} {prec} dir={d}")


@pytest.mark.parametrize("prec,log2n", [("fp16", 8), ("fp16", 10), ("fp16", 12), ("fp32", 12), ("bf16", 14),
                                        ("fp16", 14)])
def test_tma_many_tiles_per_block_equal_wide(dsfft, prec, log2n):
    """A batch of about 2.5 grids of tiles: every block refills both buffers
    at least once and the last tile is partial."""
    import torch
    N = 1 << log2n
    tma = dsfft.Plan(N, prec, "dual_select", variant="fused_tma")
    wide = dsfft.Plan(N, prec, "dual_select", variant="fused_wide")
    tpc = tma.info()["transforms_per_block"]
    blocks = torch.cuda.get_device_properties(0).multi_processor_count * 8
    batch = int(2.5 * blocks) * tpc + tpc // 2 + 1
    g = torch.Generator(device="cuda").manual_seed(1200 + log2n)
    if prec == "fp32":
        xt = torch.randn((batch, N), dtype=torch.complex64, device="cuda", generator=g)
    else:
        dt = torch.float16 if prec == "fp16" else torch.bfloat16
        xt = (torch.rand((batch, N, 2), device="cuda", generator=g) * 2 - 1).to(dt)
    for d in (-1, 1):
        a = tma.exec(xt, direction=d)
        b = wide.exec(xt, direction=d)
        torch.cuda.synchronize()
        assert torch.equal(a.view(torch.int32) if prec != "fp32" else torch.view_as_real(a).view(torch.int32),
                           b.view(torch.int32) if prec != "fp32" else torch.view_as_real(b).view(torch.int32)), \
            f"tma vs wide N=2^{log2n} {prec} dir={d} batch={batch}"
    tma.device_status()


@pytest.mark.parametrize("prec,log2n", [("fp16", 12), ("fp32", 10)])
def test_tma_in_place(dsfft, prec, log2n):
    N = 1 << log2n
    plan = dsfft.Plan(N, prec, "dual_select", variant="fused_tma")
    x = signals.signal(1300 + log2n, 2 * plan.info()["transforms_per_block"] + 3, N, prec)
    assert_bitexact(gpu_fft(plan, x, inplace=True), emulate(plan, x), f"in-place tma N=2^{log2n} {prec}")


def test_tma_unaligned_input_runs_wide_kernel(dsfft):
    """An input 4 bytes off a 16-byte boundary cannot be bulk-copied; the
    plan runs the wide kernel, with the same result."""
    import torch
    N, batch = 4096, 5
    plan = dsfft.Plan(N, "fp16", "dual_select", variant="fused_tma")
    x = signals.signal(1310, batch, N, "fp16")
    xt = signals.to_torch(x, "fp16", "cuda")
    buf = torch.empty((batch * N + 1, 2), dtype=torch.float16, device="cuda")
    shifted = buf[1:].view(batch, N, 2)
    shifted.copy_(xt)
    assert shifted.data_ptr() % 16 == 4
    y = plan.exec(shifted)
    torch.cuda.synchronize()
    assert_bitexact(signals.from_torch(y, "fp16"), emulate(plan, x), "unaligned input")


def test_tma_wait_limit_sets_status(dsfft, monkeypatch):
    """Fault injection: the copy barrier expects 16 bytes more than the
    copies deliver, so each block's first wait runs out (about 1 s), the
    block records it in the status word, waits (bounded) for its copies and
    returns.  No GPU fault: the context stays usable."""
    import torch
    monkeypatch.setenv("DSFFT_FAULT_WAIT", "1")
    bad = dsfft.Plan(1024, "fp16", "dual_select", variant="fused_tma")
    monkeypatch.delenv("DSFFT_FAULT_WAIT")
    x = signals.to_torch(signals.signal(1320, 64, 1024, "fp16"), "fp16", "cuda")
    bad.exec(x)
    with pytest.raises(dsfft.DsfftError) as e:
        bad.device_status()
    assert e.value.status == 6
    bad.device_status()                     # cleared by the read
    good = dsfft.Plan(1024, "fp16", "dual_select", variant="fused_tma")
    xs = signals.signal(1321, 9, 1024, "fp16")
    assert_bitexact(gpu_fft(good, xs), emulate(good, xs), "after the injected timeout")
    good.device_status()
    torch.cuda.synchronize()
