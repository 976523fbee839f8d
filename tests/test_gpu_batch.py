"""Mixed batches (one persistent launch + large-size groups, optionally
through a CUDA graph): every transform's output is bit-exact against the
oracle's op-by-op emulation of that transform (fed its plan's table), and
bit-identical to transforming it alone with the same plan."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from gpu_util import assert_bitexact, emulate_async
from paper_2604_00567_b300 import signals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dsfft():
    import paper_2604_00567_b300 as m
    m.lib()
    return m


def _mixed_items(seed, count, log2_lo, log2_hi, facs=("dual_select",), inplace_every=0):
    """Transforms with log-uniform sizes 2^e, e ~ U{log2_lo..log2_hi},
    random precision and direction (seeded), each with its own buffers."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        e = int(rng.integers(log2_lo, log2_hi + 1))
        prec = ["fp32", "fp16", "bf16"][int(rng.integers(0, 3))]
        fac = facs[int(rng.integers(0, len(facs)))]
        d = -1 if rng.random() < 0.7 else 1
        rows = int(rng.integers(1, 3))
        out.append((e, prec, fac, d, rows, bool(inplace_every and i % inplace_every == 0)))
    return out


def _run(dsfft, spec, seed, graph=False, repeat=1):
    """Returns (batch, items, batch outputs, fft_exec outputs, oracle
    emulations), one entry per transform."""
    import torch
    items, inputs, refs, emus = [], [], [], []
    plans = {}
    with ThreadPoolExecutor(max_workers=8) as pool:
        for k, (e, prec, fac, d, rows, inplace) in enumerate(spec):
            n = 1 << e
            x = signals.signal(seed * 1000 + k, rows, n, prec)
            for r in range(rows):
                xt = signals.to_torch(x[r:r + 1], prec, "cuda")
                key = (n, prec, fac)
                if key not in plans:
                    plans[key] = dsfft.Plan(n, prec, fac)
                refs.append(signals.from_torch(plans[key].exec(xt.clone(), direction=d), prec))
                emus.append(emulate_async(pool, plans[key], x[r:r + 1], d))
                out = xt if (inplace and plans[key].info()["kernel"] != 1) else torch.empty_like(xt)
                items.append((n, prec, fac, d, xt, out))
                inputs.append(xt)
        batch = dsfft.Batch(items)
        for _ in range(repeat):
            if graph:
                batch.exec_graph()
            else:
                batch.exec()
        torch.cuda.synchronize()
        outs = [signals.from_torch(it[5], it[1]) for it in items]
        emus = [f.result() for f in emus]
    return batch, items, outs, refs, emus


def _check(items, outs, refs, emus, what=""):
    for k, (o, r, em) in enumerate(zip(outs, refs, emus)):
        tag = f"{what}item {k} N={items[k][0]} {items[k][1]} {items[k][2]} dir={items[k][3]}"
        assert_bitexact(o, em, tag + " vs oracle")
        assert_bitexact(o, r, tag + " vs fft_exec")


def test_mixed_small_sizes_bitexact(dsfft):
    spec = _mixed_items(1, 120, 1, 14)
    batch, items, outs, refs, emus = _run(dsfft, spec, 11)
    info = batch.info()
    assert info["large_groups"] == 0 and info["launches"] == 1 and info["tiles"] >= 1
    _check(items, outs, refs, emus)


def test_mixed_with_large_sizes_and_graph(dsfft):
    """Sizes 2^6..2^16 (the mixed-batch study's range) through the captured
    graph, replayed twice."""
    spec = _mixed_items(2, 60, 6, 16)
    batch, items, outs, refs, emus = _run(dsfft, spec, 12, graph=True, repeat=2)
    info = batch.info()
    assert info["graph_ready"] == 1
    _check(items, outs, refs, emus, "graph ")


def test_mixed_factorizations_and_in_place(dsfft):
    spec = _mixed_items(3, 48, 3, 13, facs=("dual_select", "linzer_feig_clamped", "cosine"), inplace_every=3)
    batch, items, outs, refs, emus = _run(dsfft, spec, 13)
    _check(items, outs, refs, emus)


def test_sweep_sizes_in_batch(dsfft):
    spec = [(18, "fp16", "dual_select", -1, 1, False), (17, "fp32", "dual_select", 1, 1, False),
            (10, "fp16", "dual_select", -1, 2, False)]
    batch, items, outs, refs, emus = _run(dsfft, spec, 14)
    assert batch.info()["large_groups"] == 2
    _check(items, outs, refs, emus)


def test_sweep_sizes_in_graph(dsfft):
    """Two-sweep groups (sweep 2 a programmatic dependent launch of sweep 1)
    inside the captured graph, replayed twice."""
    spec = [(18, "fp16", "dual_select", -1, 2, False), (19, "fp32", "dual_select", 1, 1, False),
            (12, "bf16", "dual_select", -1, 3, False)]
    batch, items, outs, refs, emus = _run(dsfft, spec, 15, graph=True, repeat=2)
    info = batch.info()
    assert info["large_groups"] == 2 and info["graph_ready"] == 1
    _check(items, outs, refs, emus, "graph ")


def test_batch_argument_errors(dsfft):
    import torch
    x = torch.zeros((1, 1000), dtype=torch.complex64, device="cuda")
    with pytest.raises(dsfft.DsfftError) as e:
        dsfft.Batch([(1000, "fp32", "dual_select", -1, x, x)])
    assert e.value.status == 2
    y = torch.zeros((1, 1 << 18, 2), dtype=torch.float16, device="cuda")
    with pytest.raises(dsfft.DsfftError) as e:
        dsfft.Batch([(1 << 18, "fp16", "dual_select", -1, y, y)])   # in-place sweep size
    assert e.value.status == 3
    empty = dsfft.Batch([])
    empty.exec()
    assert empty.info()["launches"] == 0
