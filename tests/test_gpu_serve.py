"""The serving loop (fft_server_*): requests of mixed size, precision,
factorization and direction, batched by the library's scheduler into ticks,
give outputs bit-identical to fft_exec of each request alone (which the
other GPU tests pin to the oracle); admission respects the arena budget;
waits time out instead of hanging; an open-loop replay completes."""
import numpy as np
import pytest

from gpu_util import assert_bitexact, emulate
from paper_2604_00567_b300 import signals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dsfft():
    import paper_2604_00567_b300 as m
    m.lib()
    return m


def _out_tensor(x):
    import torch
    return torch.empty_like(x)


def _alone(dsfft, plans, n, prec, fac, d, x):
    key = (n, prec, fac)
    if key not in plans:
        plans[key] = dsfft.Plan(n, prec, fac)
    return plans[key].exec(x, direction=d)


def _spec(seed, count, lo, hi):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        e = int(rng.integers(lo, hi + 1))
        prec = ["fp32", "fp16", "bf16"][int(rng.integers(0, 3))]
        fac = ["dual_select", "dual_select", "linzer_feig_clamped", "cosine"][int(rng.integers(0, 4))]
        if prec != "fp32" and fac != "dual_select":
            fac = "dual_select"      # LF / cosine tables overflow in FP16 (non-finite by design)
        d = -1 if rng.random() < 0.7 else 1
        rows = int(rng.integers(1, 6))
        out.append((e, prec, fac, d, rows))
    return out


def test_mixed_requests_match_exec_alone(dsfft):
    """Sizes 2^2 .. 2^18 (fused, cluster and sweep paths in one tick)."""
    import torch
    srv = dsfft.Server(memory_budget=1 << 30)
    try:
        spec = _spec(11, 40, 2, 18)
        tickets, inputs = [], []
        for k, (e, prec, fac, d, rows) in enumerate(spec):
            n = 1 << e
            x = signals.device_signal(rows, n, prec, seed=500 + k)
            inputs.append(x)
            tickets.append(srv.submit(x, n, prec, fac, d, tag=k))
        plans = {}
        for k, ((e, prec, fac, d, rows), t) in enumerate(zip(spec, tickets)):
            c = srv.wait(t, 60.0)
            assert c["status"] == 0 and c["tag"] == k
            assert c["t_submit_ns"] <= c["t_admit_ns"] <= c["t_launch_ns"] <= c["t_done_ns"]
            got = srv.copy_out(t, _out_tensor(inputs[k]))
            torch.cuda.synchronize()
            srv.release(t)
            ref = _alone(dsfft, plans, 1 << e, prec, fac, d, inputs[k])
            torch.cuda.synchronize()
            assert_bitexact(signals.from_torch(got, prec), signals.from_torch(ref, prec),
                            f"request {k} N=2^{e} {prec} {fac} d={d}")
        st = srv.stats()
        assert st["completed"] == len(spec) and st["released"] == len(spec) and st["arena_used"] == 0
        assert st["ticks"] >= 1
    finally:
        srv.close()


def test_one_request_against_oracle(dsfft):
    """Direct parity of a served FP16 request with the oracle's emulation."""
    import torch
    n, prec = 1024, "fp16"
    x = signals.signal(77, 3, n, prec)
    xt = signals.to_torch(x, prec, device="cuda")
    with dsfft.Server(memory_budget=1 << 26) as srv:
        t = srv.submit(xt, n, prec)
        assert srv.wait(t, 30.0)["status"] == 0
        y = srv.copy_out(t, torch.empty_like(xt))
        torch.cuda.synchronize()
        srv.release(t)
    plan = dsfft.Plan(n, prec, "dual_select")
    assert_bitexact(signals.from_torch(y, prec), emulate(plan, x, -1), "served fp16 N=1024")


def test_same_result_alone_and_in_mix(dsfft):
    """A request served alone and served among 30 others: identical bytes."""
    import torch
    n, prec = 4096, "fp16"
    x = signals.device_signal(7, n, prec, seed=42)
    with dsfft.Server(memory_budget=1 << 28) as srv:
        t = srv.submit(x, n, prec)
        srv.wait(t)
        alone = srv.copy_out(t, _out_tensor(x))
        torch.cuda.synchronize()
        srv.release(t)
    with dsfft.Server(memory_budget=1 << 28, max_ticks_in_flight=1) as srv:
        others = []
        for k, (e, p2, fac, d, rows) in enumerate(_spec(5, 30, 3, 16)):
            y = signals.device_signal(rows, 1 << e, p2, seed=900 + k)
            others.append((srv.submit(y, 1 << e, p2, fac, d), y))
        t = srv.submit(x, n, prec)
        c = srv.wait(t)
        mixed = srv.copy_out(t, _out_tensor(x))
        torch.cuda.synchronize()
        srv.release(t)
        srv.drain(60.0)
        for tk, _ in others:
            srv.release(tk)
    assert torch.equal(alone.view(torch.int16), mixed.view(torch.int16))
    assert c["tick"] >= 1


def test_admission_under_budget(dsfft):
    """Outputs held until release: a budget of 4 MiB admits the FIFO prefix
    that fits, the rest waits (wait/drain time out), releases admit more."""
    import torch
    n, prec = 1 << 14, "fp32"                 # 128 KiB per signal
    budget = 4 << 20
    with dsfft.Server(memory_budget=budget) as srv:
        xs = [signals.device_signal(8, n, prec, seed=k) for k in range(6)]   # 1 MiB each
        ts = [srv.submit(x, n, prec) for x in xs]
        for t in ts[:4]:
            assert srv.wait(t, 30.0)["status"] == 0
        st = srv.stats()
        assert st["queued"] == 2 and st["arena_used"] == budget and st["arena_peak"] == budget
        with pytest.raises(dsfft.DsfftError) as ei:
            srv.wait(ts[4], 0.2)
        assert ei.value.status == 6
        with pytest.raises(dsfft.DsfftError) as ei:
            srv.drain(0.2)
        assert ei.value.status == 6
        srv.release(ts[0])
        srv.release(ts[1])
        for t in ts[4:]:
            assert srv.wait(t, 30.0)["status"] == 0
        srv.drain(10.0)
        for t in ts[2:]:
            srv.release(t)
        assert srv.stats()["arena_used"] == 0
        # a request larger than the whole arena is refused at submit
        big = signals.device_signal(40, n, prec, seed=99)
        with pytest.raises(dsfft.DsfftError) as ei:
            srv.submit(big, n, prec)
        assert ei.value.status == 4
        torch.cuda.synchronize()


def test_submit_validation(dsfft):
    import torch
    with dsfft.Server(memory_budget=1 << 24, max_tick_transforms=16) as srv:
        x = torch.zeros(2, 1000, dtype=torch.complex64, device="cuda")
        with pytest.raises(dsfft.DsfftError) as ei:
            srv.submit(x, 1000, "fp32")
        assert ei.value.status == 2
        y = signals.device_signal(32, 64, "fp16", seed=2)
        with pytest.raises(dsfft.DsfftError) as ei:    # more than max_tick_transforms small signals
            srv.submit(y, 64, "fp16")
        assert ei.value.status == 2
        with pytest.raises(dsfft.DsfftError):
            srv.release(12345)
        with pytest.raises(dsfft.DsfftError):
            srv.wait(12345, 0.1)
        torch.cuda.synchronize()


def test_replay_poisson_trace(dsfft):
    """Open-loop replay of a short Poisson trace (release at completion):
    every request completes, ticks batch several requests, latencies are
    ordered."""
    rng = np.random.default_rng(2)
    count = 400
    arrivals = np.cumsum(rng.exponential(1e9 / 20000, count)).astype(np.int64)
    pools = {p: signals.device_signal(64, 1 << 14, p, seed=3) for p in ("fp32", "fp16")}
    reqs = []
    with dsfft.Server(memory_budget=1 << 30, release_on_complete=True) as srv:
        for k in range(count):
            e = int(rng.integers(8, 15))
            prec = "fp32" if rng.random() < 0.5 else "fp16"
            rows = int(rng.integers(1, 33))
            srv.prepare(1 << e, prec)
            x = pools[prec]
            r = dsfft.Server.request(x, 1 << e, prec, tag=k)
            r.count = rows
            reqs.append(r)
        tickets = srv.replay(reqs, arrivals, keep=pools)
        srv.drain(60.0)
        done = []
        while True:
            got = srv.poll(1024)
            if not got:
                break
            done += got
    assert len(done) == count and sorted(c["ticket"] for c in done) == sorted(tickets)
    assert all(c["status"] == 0 for c in done)
    lat = np.array([c["t_done_ns"] - c["t_submit_ns"] for c in done])
    assert np.all(lat > 0)
    assert len({c["tick"] for c in done}) < count


def test_tick_byte_limit(dsfft):
    """max_tick_bytes splits the admitted requests into ticks of at most that
    many output bytes (a single larger request still forms its own tick)."""
    n, prec = 1 << 14, "fp32"                 # 128 KiB per signal
    xs = [signals.device_signal(8, n, prec, seed=k) for k in range(10)]   # 1 MiB each
    with dsfft.Server(memory_budget=64 << 20, max_ticks_in_flight=1, max_tick_bytes=2 << 20) as srv:
        ts = [srv.submit(x, n, prec) for x in xs]
        cs = [srv.wait(t, 30.0) for t in ts]
        for t in ts:
            srv.release(t)
    ticks = {}
    for c in cs:
        assert c["status"] == 0
        ticks.setdefault(c["tick"], 0)
        ticks[c["tick"]] += c["bytes"]
    assert all(b <= 2 << 20 for b in ticks.values()) and len(ticks) >= 5
