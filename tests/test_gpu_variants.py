"""Kernel variants (all bit-identical) and the autotuner that picks among
them: every variant equals the oracle's emulation; autotuning times the
candidates once per GPU model and caches the choice in JSON."""
import json
import os

import pytest

from gpu_util import assert_bitexact, emulate, gpu_fft
from paper_2604_00567_b300 import signals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dsfft():
    import paper_2604_00567_b300 as m
    m.lib()
    return m


@pytest.mark.parametrize("prec,log2n", [("fp16", 5), ("fp16", 10), ("bf16", 11), ("fp16", 12), ("fp16", 13),
                                        ("fp16", 14), ("fp32", 5), ("fp32", 9), ("fp32", 12), ("fp32", 13)])
def test_fused_narrow_bitexact(dsfft, prec, log2n):
    N = 1 << log2n
    x = signals.signal(950 + log2n, 7, N, prec)
    plan = dsfft.Plan(N, prec, "dual_select", variant="fused_narrow")
    info = plan.info()
    assert info["variant_name"] == "fused_narrow"
    wide = dsfft.Plan(N, prec, "dual_select", variant="fused_wide").info()["points_per_thread"]
    assert info["points_per_thread"] == wide // 2
    for d in (-1, 1):
        assert_bitexact(gpu_fft(plan, x, d), emulate(plan, x, d), f"narrow N=2^{log2n} {prec} dir={d}")


@pytest.mark.parametrize("prec,log2n", [("fp16", 15), ("fp32", 16), ("bf16", 17)])
def test_cluster_and_sweeps_agree(dsfft, prec, log2n):
    N = 1 << log2n
    x = signals.signal(960 + log2n, 2, N, prec)
    a = dsfft.Plan(N, prec, "dual_select", variant="cluster")
    b = dsfft.Plan(N, prec, "dual_select", variant="sweeps")
    assert a.info()["kernel"] == 2 and b.info()["kernel"] == 1
    ya = gpu_fft(a, x)
    assert_bitexact(ya, gpu_fft(b, x), f"cluster vs sweeps N=2^{log2n} {prec}")
    assert_bitexact(ya, emulate(a, x), "vs oracle")


def test_autotune_and_cache(dsfft, tmp_path, monkeypatch):
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("DSFFT_AUTOTUNE_CACHE", str(cache))
    p1 = dsfft.Plan(4096, "fp16", "dual_select", autotune=True)
    i1 = p1.info()
    assert i1["autotuned"] == 1 and i1["variant_name"] in ("fused_wide", "fused_narrow", "fused_tma")
    data = json.loads(cache.read_text())
    keys = [k for k in data if k != "format"]
    assert len(keys) == 1 and keys[0].endswith("|1|12|2") and data[keys[0]] == i1["variant"]
    p2 = dsfft.Plan(4096, "fp16", "dual_select", autotune=True)
    assert p2.info()["autotuned"] == 2 and p2.info()["variant"] == i1["variant"]
    p3 = dsfft.Plan(1 << 16, "fp32", "dual_select", autotune=True)
    assert p3.info()["autotuned"] == 1 and p3.info()["variant_name"] in ("cluster", "sweeps")
    assert len([k for k in json.loads(cache.read_text()) if k != "format"]) == 2
    x = signals.signal(970, 3, 4096, "fp16")
    assert_bitexact(gpu_fft(p2, x), emulate(p2, x), "autotuned plan")
    # a single-candidate size needs no tuning
    p4 = dsfft.Plan(16, "fp16", "dual_select", autotune=True)
    assert p4.info()["autotuned"] == 0


@pytest.mark.parametrize("prec,log2n,splits", [("fp16", 18, (8, 9, 10)), ("fp32", 17, (8, 9, 10)),
                                               ("bf16", 20, (9, 10, 11))])
def test_sweep_splits_agree(dsfft, prec, log2n, splits):
    """Any split of the passes between the two sweeps runs the same
    butterflies: identical bytes; the plan reports the split it runs."""
    import torch
    N = 1 << log2n
    x = signals.device_signal(2, N, prec, seed=log2n)
    outs = []
    for sp in splits:
        plan = dsfft.Plan(N, prec, "dual_select", sweep_passes=sp)
        info = plan.info()
        assert info["variant_name"] == "sweeps" and info["sweep_passes"] == sp
        outs.append(plan.exec(x))
    torch.cuda.synchronize()
    word = torch.int32 if prec == "fp32" else torch.int16
    for y in outs[1:]:
        assert torch.equal(y.view(word), outs[0].view(word))


def test_autotune_sweep_split_cached(dsfft, tmp_path, monkeypatch):
    """The autotuner also times the sweep splits; a cached split is reused."""
    import json
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("DSFFT_AUTOTUNE_CACHE", str(cache))
    p1 = dsfft.Plan(1 << 18, "fp16", "dual_select", autotune=True)
    i1 = p1.info()
    assert i1["autotuned"] == 1 and i1["variant_name"] == "sweeps" and 7 <= i1["sweep_passes"] <= 11
    data = json.loads(cache.read_text())
    key = [k for k in data if k.endswith("|1|18|2")][0]
    data[key] = 4 * 100 + 10          # sweeps with 10 passes in sweep 1
    cache.write_text(json.dumps(data))
    p2 = dsfft.Plan(1 << 18, "fp16", "dual_select", autotune=True)
    i2 = p2.info()
    assert i2["autotuned"] == 2 and i2["sweep_passes"] == 10
