"""Large transforms (N = 2^21 .. 2^24, grouped HBM sweeps) bit for bit
against the oracle's op-by-op emulation (fed the plan's own table).

Covered: radix-2 plans at every N from 2^21 to 2^24 in complex64 (FP32) and
complex-FP16, forward and inverse, each with the split of passes between
the two sweeps that the plan runs by default (10 + 11 / 12 + 9, 11 + 11 /
12 + 10, 12 + 11, 12 + 12); the first and last transform of batch-8 runs at 2^20
and 2^24 in both formats; a forward + inverse round trip at 2^24 in both
formats (Section V's round-trip check); every sweep length LS = 7..12
as the first and as the second sweep; and small batches (every transform)
with contiguous and gathered pointers.

The emulation of one 2^24-point transform takes tens of seconds of one
host core, so the module computes every GPU output first and runs all the
emulations concurrently on a thread pool (ctypes releases the GIL)."""
import os
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle as orc
from gpu_util import assert_bitexact, emulate_async
from paper_2604_00567_b300 import signals

pytestmark = pytest.mark.gpu

LARGE = (21, 22, 23, 24)
PRECS = ("fp32", "fp16")
# passes in sweep 1 / sweep 2 of the built-in plans
DEFAULT_SPLIT = {("fp32", 21): (10, 11), ("fp16", 21): (12, 9), ("fp32", 22): (11, 11), ("fp16", 22): (12, 10),
                 ("fp32", 23): (12, 11), ("fp16", 23): (12, 11), ("fp32", 24): (12, 12), ("fp16", 24): (12, 12)}


@pytest.fixture(scope="module")
def dsfft():
    import paper_2604_00567_b300 as m
    m.lib()
    return m


def _row_signal(seed, N, prec, row):
    """Transform ``row`` of a seeded batch (regenerated alone)."""
    return signals.signal(seed, 1, N, prec, start_transform=row)


@pytest.fixture(scope="module")
def large(dsfft):
    """GPU outputs and the matching emulation futures of every case."""
    import torch
    workers = max(2, min(16, os.cpu_count() or 2))
    pool = ThreadPoolExecutor(max_workers=workers)
    res = {}
    try:
        for l in LARGE:
            N = 1 << l
            for prec in PRECS:
                plan = dsfft.Plan(N, prec, "dual_select")
                x = _row_signal(2100 + l, N, prec, 0)
                xt = signals.to_torch(x, prec, "cuda")
                yf = plan.exec(xt)
                yi = plan.exec(xt, direction=1)
                torch.cuda.synchronize()
                res[("single", prec, l)] = dict(
                    info=plan.info(), x=x,
                    fwd=(signals.from_torch(yf, prec), emulate_async(pool, plan, x, -1)),
                    inv=(signals.from_torch(yi, prec), emulate_async(pool, plan, x, 1)))
                if l == 24:
                    # round trip: inverse of the GPU's forward output
                    z = plan.exec(yf, direction=1)
                    torch.cuda.synchronize()
                    yfh = signals.from_torch(yf, prec)
                    res[("round_trip", prec, l)] = dict(
                        x=x, scaled_forward=plan.scale_forward,
                        out=(signals.from_torch(z, prec), emulate_async(pool, plan, yfh, 1)))
                del xt, yf, yi
        for l in (20, 24):
            N = 1 << l
            for prec in PRECS:
                plan = dsfft.Plan(N, prec, "dual_select")
                rows = [_row_signal(2400 + l, N, prec, b) for b in range(8)]
                xt = torch.cat([signals.to_torch(r, prec, "cuda") for r in rows], dim=0)
                y = plan.exec(xt)
                torch.cuda.synchronize()
                res[("batch8", prec, l)] = {
                    b: (signals.from_torch(y[b:b + 1], prec), emulate_async(pool, plan, rows[b], -1))
                    for b in (0, 7)}
                del xt, y
        torch.cuda.empty_cache()
        yield res
    finally:
        pool.shutdown(wait=True, cancel_futures=True)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("log2n", LARGE)
def test_large_radix2_bitexact(large, prec, log2n):
    case = large[("single", prec, log2n)]
    info = case["info"]
    assert info["kernel"] == 1 and info["launches"] == 2
    ls1, ls2 = DEFAULT_SPLIT[(prec, log2n)]
    assert info["sweep_passes"] == ls1 and ls1 + ls2 == log2n
    for d in ("fwd", "inv"):
        got, fut = case[d]
        assert_bitexact(got, fut.result(), f"N=2^{log2n} {prec} {d} (sweeps {ls1} + {ls2})")


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("log2n", (20, 24))
def test_batch_of_eight_first_and_last(large, prec, log2n):
    for b, (got, fut) in large[("batch8", prec, log2n)].items():
        assert_bitexact(got, fut.result(), f"batch 8 N=2^{log2n} {prec} transform {b}")


@pytest.mark.parametrize("prec,tol", [("fp32", 5e-7), ("fp16", 4e-3)])
def test_round_trip_n2pow24(large, prec, tol):
    """Forward (x0.5 per pass for FP16: DFT/N) then inverse (unscaled) on the
    GPU: bit-exact against the emulated inverse of the same spectrum, and
    back to the input within the FP64 tolerance of the format."""
    case = large[("round_trip", prec, 24)]
    got, fut = case["out"]
    assert_bitexact(got, fut.result(), f"round trip N=2^24 {prec}")
    back = got if case["scaled_forward"] else got / (1 << 24)
    assert orc.rel_l2(back, case["x"]) < tol


# sweep lengths LS1 + LS2: every LS in 7..12 appears as the first and as the
# second sweep
SPLITS = [(15, 7), (15, 8), (18, 9), (19, 7), (19, 12), (20, 9), (20, 10), (21, 11)]


@pytest.mark.parametrize("prec", ("fp32", "fp16", "bf16"))
@pytest.mark.parametrize("log2n,ls1", SPLITS)
def test_every_sweep_length_bitexact(dsfft, prec, log2n, ls1):
    import torch
    N = 1 << log2n
    plan = dsfft.Plan(N, prec, "dual_select", sweep_passes=ls1)
    info = plan.info()
    assert info["variant_name"] == "sweeps" and info["sweep_passes"] == ls1
    x = _row_signal(2600 + log2n, N, prec, ls1)
    xt = signals.to_torch(x, prec, "cuda")
    with ThreadPoolExecutor(max_workers=2) as pool:
        futs = {d: emulate_async(pool, plan, x, d) for d in (-1, 1)}
        for d in (-1, 1):
            y = plan.exec(xt, direction=d)
            torch.cuda.synchronize()
            assert_bitexact(signals.from_torch(y, prec), futs[d].result(),
                            f"N=2^{log2n} {prec} sweeps {ls1} + {log2n - ls1} dir={d}")


# small batches of the two-sweep path (odd counts, every transform checked;
# the second sweep runs its blocks group-major across the batch), with
# contiguous and with gathered (fft_batch) pointers
@pytest.mark.parametrize("prec,log2n,batch", [("fp16", 18, 5), ("fp16", 18, 8), ("fp16", 20, 3), ("fp32", 17, 6),
                                              ("fp32", 18, 5), ("bf16", 19, 4), ("fp32", 20, 2)])
def test_sweep_small_batches_bitexact(dsfft, prec, log2n, batch):
    import torch
    N = 1 << log2n
    plan = dsfft.Plan(N, prec, "dual_select")
    assert plan.info()["kernel"] == 1
    rows = [_row_signal(2700 + log2n, N, prec, b) for b in range(batch)]
    xt = torch.cat([signals.to_torch(r, prec, "cuda") for r in rows], dim=0)
    with ThreadPoolExecutor(max_workers=8) as pool:
        futs = {d: [emulate_async(pool, plan, r, d) for r in rows] for d in (-1, 1)}
        for d in (-1, 1):
            y = plan.exec(xt, direction=d)
            torch.cuda.synchronize()
            for b in range(batch):
                assert_bitexact(signals.from_torch(y[b:b + 1], prec), futs[d][b].result(),
                                f"N=2^{log2n} {prec} batch {batch} transform {b} dir={d}")


def test_sweep_gathered_batch(dsfft):
    """Six 2^18 FP16 transforms with their own buffers through fft_batch
    (gathered pointers) against the oracle."""
    import torch
    N = 1 << 18
    rows = [_row_signal(2800, N, "fp16", b) for b in range(6)]
    ins = [signals.to_torch(r, "fp16", "cuda") for r in rows]
    outs = [torch.empty_like(x) for x in ins]
    batch = dsfft.Batch([(N, "fp16", "dual_select", -1, x, o) for x, o in zip(ins, outs)])
    assert batch.info()["large_groups"] == 1
    batch.exec()
    torch.cuda.synchronize()
    plan = dsfft.Plan(N, "fp16", "dual_select")
    with ThreadPoolExecutor(max_workers=6) as pool:
        futs = [emulate_async(pool, plan, r, -1) for r in rows]
        for b in range(6):
            assert_bitexact(signals.from_torch(outs[b], "fp16"), futs[b].result(), f"gathered transform {b}")
    batch.close()
