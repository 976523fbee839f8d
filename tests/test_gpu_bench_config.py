"""Parity at the benchmark's full sizes and launch configuration: for every
N of the timed workload (FP16 dual-select, x0.5 per pass, 1 GiB batch per N,
inputs drawn on the GPU as bench.py draws them, the plan's built-in kernel),
sampled transforms — first, last and the tail of the last block among them —
are bit-exact against the oracle's emulation; likewise the FP32 and radix-4
comparison runs, and the host pipeline of the end-to-end leg returns the
device results."""
import numpy as np
import pytest

import bench
from gpu_util import assert_bitexact, emulate
from paper_2604_00567_b300 import signals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dsfft():
    import paper_2604_00567_b300 as m
    m.lib()
    return m


def _samples(batch):
    return sorted({0, 1, batch // 3, batch // 2 + 1, batch - 2, batch - 1})


@pytest.mark.parametrize("log2n", list(bench.LOG2NS))
def test_bench_workload_sampled_bitexact(dsfft, log2n):
    import torch
    n = 1 << log2n
    batch = bench.batch_for(log2n)
    x = signals.device_signal(batch, n, bench.PRECISION, seed=log2n)
    plan = dsfft.Plan(n, bench.PRECISION, bench.FACTORIZATION)
    y = plan.exec(x)
    torch.cuda.synchronize()
    idx = torch.as_tensor(_samples(batch), device="cuda")
    xs = signals.from_torch(x.index_select(0, idx), bench.PRECISION)
    ys = signals.from_torch(y.index_select(0, idx), bench.PRECISION)
    assert_bitexact(ys, emulate(plan, xs, -1), f"bench N=2^{log2n} ({plan.info()['variant_name']})")


@pytest.mark.parametrize("log2n", list(bench.LOG2NS))
def test_bench_fp32_and_radix4_sampled_bitexact(dsfft, log2n):
    import torch
    import oracle as orc
    n = 1 << log2n
    batch = bench.batch_for(log2n, "fp32")
    x = signals.device_signal(batch, n, "fp32", seed=77 + log2n)
    plan = dsfft.Plan(n, "fp32", bench.FACTORIZATION)
    y = plan.exec(x)
    torch.cuda.synchronize()
    idx = torch.as_tensor(_samples(batch), device="cuda")
    xs = signals.from_torch(x.index_select(0, idx), "fp32")
    assert_bitexact(signals.from_torch(y.index_select(0, idx), "fp32"), emulate(plan, xs, -1), f"fp32 2^{log2n}")
    del x, y
    if log2n > 14:
        return
    batch = bench.batch_for(log2n)
    x = signals.device_signal(batch, n, bench.PRECISION, seed=log2n)
    p4 = dsfft.Plan(n, bench.PRECISION, bench.FACTORIZATION, radix=4)
    y = p4.exec(x)
    torch.cuda.synchronize()
    idx = torch.as_tensor(_samples(batch), device="cuda")
    xs = signals.from_torch(x.index_select(0, idx), bench.PRECISION)
    t4, m4, q4 = p4.table4(-1)
    t2, m2, q2 = p4.table(-1)
    ref = orc.emulate_fft_r4(xs, orc.FP16, t4, m4, q4, (t2[0], m2[0], q2[0]), scaled=True, threads=8)
    assert_bitexact(signals.from_torch(y.index_select(0, idx), bench.PRECISION), ref, f"radix-4 2^{log2n}")


def test_e2e_pipeline_returns_device_results(dsfft):
    """The end-to-end leg's configuration (64 MiB chunks, 3 streams) at the
    largest N of the workload."""
    import torch
    log2n = max(bench.LOG2NS)
    n = 1 << log2n
    batch = bench.batch_for(log2n)
    x = signals.device_signal(batch, n, bench.PRECISION, seed=log2n)
    plan = dsfft.Plan(n, bench.PRECISION, bench.FACTORIZATION)
    pipe = dsfft.Pipeline(plan, max(1, (64 << 20) // (4 << log2n)), 3)
    hin = x.cpu().pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    pipe.exec(hin, hout)
    y = plan.exec(x)
    torch.cuda.synchronize()
    assert torch.equal(hout.view(torch.int16), y.cpu().view(torch.int16))
    assert np.isfinite(signals.from_torch(y[:2], bench.PRECISION)).all()
