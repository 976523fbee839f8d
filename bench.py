#!/usr/bin/env python3
"""Benchmark of the dual-select FMA FFT on one B300 (or N replicas).

Workload (one "step"): forward FP16 dual-select FFTs with exact x0.5 per
pass of one 1 GiB batch at each N in {2^10, 2^12, 2^14, 2^16}
(batch = 2^30 / (4 N) signals; re/im i.i.d. uniform[-1, 1], seeded).
``value`` = transforms/s over the whole step (all N, all ranks).

Also reported on the same JSON line:
  roofline     : the dominant kernel's algorithmic bytes (read + write of the
                 batch) / its CUDA-event launch time, against the measured
                 HBM copy bandwidth;
  per_n        : transforms/s, GB/s, fraction of roofline, and relative L2
                 error vs an FP64 FFT (numpy) on sampled signals, per N;
  fp32_plain   : the FP32 form (no scaling) on the same bytes per N;
  radix4_fp16  : radix-4 dual-select plans (N <= 2^14) on the same FP16 batches;
  batch_c3     : a mixed batch of 4096 transforms (N 2^6..2^16, FP32/FP16) as
                 one graph-replayed fft_batch;
  e2e          : the same metric with the input copied from pinned host
                 memory and the output copied back inside the timed region;
  cpu_baseline : the CPU oracle (op-by-op emulation) on a bounded sample;
  serve        : the serving loop under a Poisson arrival trace (20k req/s,
                 mixed N 2^8..2^18, FP32/FP16, 40 GB arena): p50/p99 latency
                 and throughput;
  clocks       : nvidia-smi samples taken during the timed region.

``--impl reference`` times the CPU oracle itself on the same workload (a
bounded sample per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "transforms/s & % HBM roofline, FP16 vs FP32 at stated FP64 error; serve p99 ms"
LOG2NS = (10, 12, 14, 16)
BATCH_BYTES = 1 << 30
PRECISION = "fp16"
FACTORIZATION = "dual_select"
CPU_SAMPLE_DIV = 8           # oracle sample: batch / 8 signals per N (about 10 s on 16 cores)


def batch_for(log2n: int, precision: str = PRECISION) -> int:
    eb = 8 if precision == "fp32" else 4
    return BATCH_BYTES // (eb << log2n)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons (200 ms)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}


# ---------------------------------------------------------------------------
def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x: float, world: int) -> float:
    """Max of x over the ranks (NCCL tensors on the GPU, gloo on the CPU)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(local_ms: float, units_per_rank: int, world: int):
    """Replicas only: every rank transforms its own batch.  The job's time is
    the slowest rank's; the throughput counts every rank's units."""
    ms = allreduce_max(local_ms, world)
    return ms, world * units_per_rank / (ms / 1e3)


def kernel_source_hash() -> str:
    """Hash of the device-code sources (kernels, their headers and the table
    builder; not the host-only files api.cu, noalloc.cu, pipeline.cu,
    serve.cu): a recorded ncu traffic figure is only used while the kernels
    it was measured on are unchanged."""
    import hashlib
    host_only = {"api.cu", "noalloc.cu", "pipeline.cu", "serve.cu"}
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2604_00567_b300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h")) and name not in host_only:
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + f.read())
    return h.hexdigest()[:12]


def recorded_traffic(key: str, algorithmic_bytes: int):
    """DRAM bytes (read + write) per launch of the dominant kernel from the
    committed ncu summary (profiles/dram_traffic.txt: `key source_hash
    bytes_per_launch_at_1GiB`), or None when absent or stale."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    want = kernel_source_hash()
    with open(path) as f:
        for line in f:
            parts = line.split("#", 1)[0].split()
            if len(parts) == 3 and parts[0] == key and parts[1] == want:
                return int(float(parts[2]))
    return None


def error_vs_fp64(plan, x_dev, y_dev, log2n, precision, scaled, samples=4):
    """Relative L2 error of sampled outputs vs numpy's FP64 FFT of the same
    (already rounded) inputs."""
    from paper_2604_00567_b300 import signals
    n = 1 << log2n
    import torch
    idx = torch.as_tensor(np.linspace(0, x_dev.shape[0] - 1, samples).astype(np.int64), device=x_dev.device)
    xs = signals.from_torch(x_dev.index_select(0, idx), precision)
    ys = signals.from_torch(y_dev.index_select(0, idx), precision)
    ref = np.fft.fft(xs, axis=-1) / (n if scaled else 1)
    return float(np.linalg.norm((ys - ref).ravel()) / np.linalg.norm(ref.ravel()))


def run_ours(args):
    import torch
    import paper_2604_00567_b300 as dsfft
    from paper_2604_00567_b300 import signals

    world, rank, local = dist_setup()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    hbm_peak, peak_kind = measured_peaks()

    log2ns = [l for l in args.log2n]
    plans, xs, ys = {}, {}, {}
    for l in log2ns:
        plans[l] = dsfft.Plan(1 << l, PRECISION, FACTORIZATION)
        xs[l] = signals.device_signal(batch_for(l), 1 << l, PRECISION, seed=1000 * rank + l, device=dev)
        ys[l] = torch.empty_like(xs[l])
    stream = torch.cuda.current_stream()

    def step(events=None):
        for i, l in enumerate(log2ns):
            if events is not None:
                events[i][0].record(stream)
            plans[l].exec(xs[l], out=ys[l], stream=stream)
            if events is not None:
                events[i][1].record(stream)

    K = args.steps
    evs = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in log2ns]
           for _ in range(K)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    # warm-up right before the timed steps, after the sampler has started: an
    # idle GPU (the sampler's start-up) would enter the first timed launch at
    # lower clocks
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for s in range(K):
        step(evs[s])
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    transforms_per_step = sum(batch_for(l) for l in log2ns)
    ms_total, _ = replica_throughput(t_start.elapsed_time(t_end), transforms_per_step * K, world)
    ms_per_step = ms_total / K
    value = world * transforms_per_step / (ms_per_step / 1e3)

    per_n = {}
    dominant = None
    for i, l in enumerate(log2ns):
        ms = statistics.mean(evs[s][i][0].elapsed_time(evs[s][i][1]) for s in range(K))
        nbytes = 2 * batch_for(l) * (4 << l)
        gbs = nbytes / (ms / 1e3) / 1e9
        per_n[f"2^{l}"] = {
            "batch": batch_for(l), "ms_per_launch": round(ms, 4),
            "transforms_per_s": batch_for(l) / (ms / 1e3), "GB_per_s": round(gbs, 1),
            "frac_of_hbm": round(gbs / hbm_peak, 4), "launches": plans[l].info()["launches"],
            "variant": plans[l].info()["variant_name"],
            "rel_l2_vs_fp64": error_vs_fp64(plans[l], xs[l], ys[l], l, PRECISION, plans[l].scale_forward),
        }
        if dominant is None or ms > dominant[1]:
            dominant = (l, ms, nbytes, gbs)
    l, ms, nbytes, gbs = dominant
    info_l = plans[l].info()
    kname = {0: f"fused_fft_kernel fp16 N=2^{l} ({info_l['variant_name']}, R={info_l['points_per_thread']})",
             1: f"sweep_fft_kernel x2 fp16 N=2^{l} (one fft_exec)",
             2: f"cluster_fft_kernel fp16 N=2^{l}"}[info_l["kernel"]]
    roofline = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(gbs / hbm_peak, 4), "traffic": recorded_traffic(f"fp16_n{1 << l}", nbytes),
                "kernel": kname, "peak_kind": peak_kind, "algorithmic_bytes_per_launch": nbytes}

    # FP32 plain form on the same bytes per N (separate timing, not in value)
    fp32 = {}
    for l in log2ns:
        p32 = dsfft.Plan(1 << l, "fp32", FACTORIZATION)
        x32 = signals.device_signal(batch_for(l, "fp32"), 1 << l, "fp32", seed=77 + l, device=dev)
        y32 = torch.empty_like(x32)
        for _ in range(3):
            p32.exec(x32, out=y32)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(max(3, K)):
            p32.exec(x32, out=y32)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / max(3, K)
        nb = 2 * batch_for(l, "fp32") * (8 << l)
        fp32[f"2^{l}"] = {"transforms_per_s": batch_for(l, "fp32") / (ms / 1e3),
                          "GB_per_s": round(nb / (ms / 1e3) / 1e9, 1),
                          "frac_of_hbm": round(nb / (ms / 1e3) / 1e9 / hbm_peak, 4),
                          "rel_l2_vs_fp64": error_vs_fp64(p32, x32, y32, l, "fp32", False)}
        del x32, y32, p32

    # radix-4 dual-select plans (N <= 2^14) on the same FP16 batches
    radix4 = {}
    for l in log2ns:
        if l > 14:
            continue
        p4 = dsfft.Plan(1 << l, PRECISION, FACTORIZATION, radix=4)
        for _ in range(3):
            p4.exec(xs[l], out=ys[l])
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(max(3, K)):
            p4.exec(xs[l], out=ys[l])
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / max(3, K)
        nb = 2 * batch_for(l) * (4 << l)
        radix4[f"2^{l}"] = {"transforms_per_s": batch_for(l) / (ms / 1e3), "GB_per_s": round(nb / (ms / 1e3) / 1e9, 1),
                            "frac_of_hbm": round(nb / (ms / 1e3) / 1e9 / hbm_peak, 4),
                            "rel_l2_vs_fp64": error_vs_fp64(p4, xs[l], ys[l], l, PRECISION, True)}
        del p4

    # end to end through the host-memory pipeline (fft_pipeline_exec): pinned
    # host input -> device -> FFT -> host every step, 64 MiB chunks on 3
    # streams so both copy directions and the kernels overlap
    e2e_steps = max(1, min(K, 3))
    host_in = {l: xs[l].cpu().pin_memory() for l in log2ns}
    host_out = {l: torch.empty_like(host_in[l]).pin_memory() for l in log2ns}
    pipes = {l: dsfft.Pipeline(plans[l], max(1, (64 << 20) // (4 << l)), 3) for l in log2ns}
    for l in log2ns:
        pipes[l].exec(host_in[l], host_out[l], stream=stream)
    torch.cuda.synchronize()
    barrier(world)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(e2e_steps):
        for l in log2ns:
            pipes[l].exec(host_in[l], host_out[l], stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = allreduce_max(a.elapsed_time(b), world) / e2e_steps
    step_bytes = sum(2 * batch_for(l) * (2 << l) for l in log2ns)
    e2e = {"value": world * transforms_per_step / (e2e_ms / 1e3), "unit": "transforms/s",
           "h2d_bytes_per_step": step_bytes, "d2h_bytes_per_step": step_bytes, "ms_per_step": round(e2e_ms, 3),
           "steps": e2e_steps, "api": "fft_pipeline_exec, pinned host buffers, 64 MiB chunks, 3 streams"}
    for l in log2ns:
        pipes[l].close()

    c3 = batch_c3()
    c4 = large_n_c4(hbm_peak)

    serve, serve_sweep = None, None
    if not args.no_serve:
        serve = serve_measure(args.serve_seconds)
        # 1 s of arrivals at 10 k (10 000 requests, as many as the 20 k run
        # has in its second) so that one host or driver stall does not set
        # the p99; 0.5 s at the saturating rates, whose backlog grows anyway
        serve_sweep = [serve_measure(1.0 if r < 20000.0 else 0.5, rate=r, brief=True)
                       for r in (10000.0, 40000.0, 80000.0)]

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(log2ns, samples_div=CPU_SAMPLE_DIV)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "transforms/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16", "data": "synthetic",
            "config": {"workload": "fp16 dual_select forward FFT, x0.5 per pass, 1 GiB batch at each N",
                       "N": [1 << l for l in log2ns], "batch": [batch_for(l) for l in log2ns],
                       "precision": PRECISION, "factorization": FACTORIZATION,
                       "input": "re/im i.i.d. uniform[-1,1], torch.Generator seeded",
                       "l2": "inputs 1 GiB per launch > 126 MB L2; no flush", "parallelism": f"replicas{world}"},
            "roofline": roofline, "per_n": per_n, "fp32_plain": fp32, "radix4_fp16": radix4, "batch_c3": c3,
            "large_n_c4": c4, "e2e": e2e,
            "gpu_launches": K * sum(plans[l].info()["launches"] for l in log2ns),
            "clocks": clocks, "cpu_baseline": cpu, "serve": serve, "serve_sweep": serve_sweep,
        }
        # last key: a compact digest that survives a truncated log tail
        line["summary"] = summary_text(per_n, fp32, c4, c3, serve, serve_sweep)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
def batch_c3(steps: int = 10, count: int = 4096, seed: int = 1):
    """Mixed batch: `count` forward dual-select transforms with
    N = 2^e, e ~ U{6..16}, precision FP32 or FP16 with probability 1/2
    (seeded), each with its own input/output rows, run as one fft_batch
    (one persistent launch for N <= 2^14 plus one launch per larger group)
    replayed as a CUDA graph.  For context also the same work as one
    fft_exec per (N, precision) group."""
    import torch
    import paper_2604_00567_b300 as dsfft
    from paper_2604_00567_b300 import signals
    rng = np.random.default_rng(seed)
    es = rng.integers(6, 17, count)
    fp32 = rng.random(count) < 0.5
    groups = {}
    for i in range(count):
        groups.setdefault((int(es[i]), "fp32" if fp32[i] else "fp16"), []).append(i)
    xs, ys, items, nbytes = {}, {}, [], 0
    for (e, prec), idx in sorted(groups.items()):
        xs[(e, prec)] = signals.device_signal(len(idx), 1 << e, prec, seed=seed * 100 + e)
        ys[(e, prec)] = torch.empty_like(xs[(e, prec)])
        for r in range(len(idx)):
            items.append((1 << e, prec, FACTORIZATION, -1, xs[(e, prec)][r:r + 1], ys[(e, prec)][r:r + 1]))
        nbytes += 2 * len(idx) * ((8 if prec == "fp32" else 4) << e)
    b = dsfft.Batch(items)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        b.exec_graph()
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        b.exec_graph()
    z.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(z) / steps
    info = b.info()
    plans = {k: dsfft.Plan(1 << k[0], k[1], FACTORIZATION) for k in groups}
    for _ in range(3):
        for k, p in plans.items():
            p.exec(xs[k], out=ys[k])
    a.record(stream)
    for _ in range(steps):
        for k, p in plans.items():
            p.exec(xs[k], out=ys[k])
    z.record(stream)
    torch.cuda.synchronize()
    ms_grouped = a.elapsed_time(z) / steps
    b.close()
    return {"config": f"mixed batch: {count} transforms, N = 2^U{{6..16}}, FP32/FP16 p=0.5 (seed {seed}), dual_select "
                      "forward, own buffers per transform, one fft_batch replayed as a CUDA graph",
            "ms_per_exec": round(ms, 4), "transforms_per_s": count / (ms / 1e3),
            "algorithmic_GB_per_s": round(nbytes / (ms / 1e3) / 1e9, 1), "launches_per_exec": info["launches"],
            "persistent_tiles": info["tiles"],
            "grouped_exec_ms": round(ms_grouped, 4), "grouped_exec_launches": len(plans)}


# ---------------------------------------------------------------------------
def large_n_c4(hbm_peak: float, steps: int = 10):
    """Large transforms (grouped HBM sweeps): N = 2^20 and 2^24, batch 1 and
    8, complex64 (FP32) and complex-FP16, forward; transforms/s and the
    fraction of the HBM roofline (algorithmic bytes: one read and one write
    of the batch; the best of three runs of `steps` executions), plus the
    forward + inverse round-trip error on the GPU."""
    import torch
    import paper_2604_00567_b300 as dsfft
    from paper_2604_00567_b300 import signals
    stream = torch.cuda.current_stream()
    out = {}
    for l in (20, 24):
        n = 1 << l
        for prec in ("fp32", "fp16"):
            plan = dsfft.Plan(n, prec, FACTORIZATION)
            eb = 8 if prec == "fp32" else 4
            for batch in (1, 8):
                x = signals.device_signal(batch, n, prec, seed=400 + l + batch)
                y = torch.empty_like(x)
                for _ in range(3):
                    plan.exec(x, out=y)
                # best of three runs of `steps` executions (single small
                # transforms take tens of microseconds: one stray host or
                # driver delay would dominate a single run)
                ms = float("inf")
                for _ in range(3):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    for _ in range(steps):
                        plan.exec(x, out=y)
                    b.record(stream)
                    torch.cuda.synchronize()
                    ms = min(ms, a.elapsed_time(b) / steps)
                nb = 2 * batch * n * eb
                gbs = nb / (ms / 1e3) / 1e9
                row = {"ms_per_exec": round(ms, 4), "transforms_per_s": batch / (ms / 1e3),
                       "GB_per_s": round(gbs, 1), "frac_of_hbm": round(gbs / hbm_peak, 4),
                       "sweep_passes": plan.info()["sweep_passes"]}
                if batch == 1:
                    z = plan.exec(y, direction=1)
                    torch.cuda.synchronize()
                    xs, zs = signals.from_torch(x, prec), signals.from_torch(z, prec)
                    zs = zs if plan.scale_forward else zs / n
                    row["round_trip_rel_l2"] = float(np.linalg.norm((zs - xs).ravel()) / np.linalg.norm(xs.ravel()))
                out[f"{prec} 2^{l} x{batch}"] = row
                del x, y
            plan.close()
    torch.cuda.empty_cache()
    return out


def summary_text(per_n, fp32, c4, c3, serve, serve_sweep) -> str:
    """One short line with the per-size fractions of the HBM roofline."""
    parts = ["fp16 " + " ".join(f"{k}:{100 * v['frac_of_hbm']:.1f}%" for k, v in per_n.items()),
             "fp32 " + " ".join(f"{k}:{100 * v['frac_of_hbm']:.1f}%" for k, v in fp32.items())]
    if c4:
        parts.append("large " + " ".join(f"{k.replace(' ', '/')}:{100 * v['frac_of_hbm']:.1f}%" for k, v in c4.items()))
    if c3:
        parts.append(f"c3 {c3['ms_per_exec']}ms {c3['launches_per_exec']}launch "
                     f"{c3['algorithmic_GB_per_s']}GB/s")
    if serve:
        parts.append(f"serve20k p50 {serve['p50_ms']} p99 {serve['p99_ms']}ms")
    if serve_sweep:
        parts.append("sweep " + " ".join(f"{int(r['rate'] / 1000)}k:p99 {r['p99_ms']}ms/{r['requests_per_s']:.0f}rps"
                                          for r in serve_sweep))
    return " | ".join(parts)


# ---------------------------------------------------------------------------
def serve_trace(seconds: float, rate: float, seed: int = 2):
    """Open-loop arrival trace: Poisson arrivals at ``rate`` req/s for
    ``seconds``; each request has U{1..256} signals of N = 2^e, e ~ U{8..18},
    precision FP32 or FP16 with probability 1/2 (seeded)."""
    rng = np.random.default_rng(seed)
    count = int(seconds * rate)
    arrivals = np.cumsum(rng.exponential(1e9 / rate, count)).astype(np.int64)
    log2n = rng.integers(8, 19, count)
    signals_ = rng.integers(1, 257, count)
    fp32 = rng.random(count) < 0.5
    return arrivals, log2n, signals_, fp32


def serve_measure(seconds: float = 1.0, rate: float = 20000.0, budget: int = 40_000_000_000,
                  max_tick_bytes: int = 1 << 26, brief: bool = False, in_flight: int = 8):
    """Serving loop under the arrival trace: inputs resident on the device
    (read from per-precision pools), outputs in the server's 40 GB arena
    (freed at completion).  Latency = completion seen by the scheduler -
    submission, per request.  ``brief``: only the load-sweep fields."""
    import torch
    import paper_2604_00567_b300 as dsfft
    from paper_2604_00567_b300 import signals
    arrivals, log2n, sig, fp32 = serve_trace(seconds, rate)
    pools = {"fp32": signals.device_signal(256, 1 << 18, "fp32", seed=21),
             "fp16": signals.device_signal(256, 1 << 18, "fp16", seed=22)}
    torch.cuda.synchronize()
    srv = dsfft.Server(memory_budget=budget, release_on_complete=True, max_tick_bytes=max_tick_bytes,
                       max_ticks_in_flight=in_flight)
    try:
        reqs = []
        for k in range(len(arrivals)):
            prec = "fp32" if fp32[k] else "fp16"
            n = 1 << int(log2n[k])
            srv.prepare(n, prec)
            r = dsfft.Server.request(pools[prec], n, prec, tag=k)
            r.count = int(sig[k])
            reqs.append(r)
        # warm-up: the first tenth of the trace (at most 1000 requests),
        # drained and discarded, so that the measured replay starts from a
        # server whose streams, arena and scheduler have already run
        nw = min(1000, max(1, len(reqs) // 10))
        srv.replay(reqs[:nw], arrivals[:nw], keep=pools)
        srv.drain(600.0)
        while srv.poll(65536):
            pass
        ticks0 = srv.stats()["ticks"]
        srv.replay(reqs, arrivals, keep=pools)
        srv.drain(600.0)
        done = []
        while True:
            got = srv.poll(65536)
            if not got:
                break
            done += got
        st = srv.stats()
    finally:
        srv.close()
    ok = [c for c in done if c["status"] == 0]
    lat_ms = np.array([(c["t_done_ns"] - c["t_submit_ns"]) / 1e6 for c in ok])
    t0 = min(c["t_submit_ns"] for c in done)
    t1 = max(c["t_done_ns"] for c in done)
    span = (t1 - t0) / 1e9
    transforms = int(sum(int(sig[c["tag"]]) for c in ok))
    payload = int(sum(2 * c["bytes"] for c in ok))
    if brief:
        return {"rate": rate, "seconds": seconds, "requests": len(arrivals), "completed_ok": len(ok),
                "p50_ms": round(float(np.percentile(lat_ms, 50)), 3),
                "p99_ms": round(float(np.percentile(lat_ms, 99)), 3),
                "requests_per_s": len(ok) / span, "algorithmic_GB_per_s": round(payload / span / 1e9, 1),
                "arena_peak_GB": round(st["arena_peak"] / 1e9, 3)}
    return {
        "config": "open-loop Poisson trace %.0f req/s for %.1f s (seed 2), U{1..256} signals, N = 2^U{8..18}, "
                  "FP32/FP16 p=0.5 (dual_select), inputs resident on the device, 40 GB arena, "
                  "outputs freed at completion, ticks of at most %d MiB of output, %d ticks in flight, "
                  "after a warm-up replay of the trace's first tenth"
                  % (rate, seconds, max_tick_bytes >> 20, in_flight),
        "requests": len(arrivals), "completed_ok": len(ok),
        "p50_ms": round(float(np.percentile(lat_ms, 50)), 3), "p99_ms": round(float(np.percentile(lat_ms, 99)), 3),
        "max_ms": round(float(lat_ms.max()), 3), "mean_ms": round(float(lat_ms.mean()), 3),
        "requests_per_s": len(ok) / span, "transforms_per_s": transforms / span,
        "algorithmic_GB_per_s": round(payload / span / 1e9, 1),
        "ticks": st["ticks"] - ticks0, "requests_per_tick": round(len(ok) / max(1, st["ticks"] - ticks0), 2),
        "arena_peak_GB": round(st["arena_peak"] / 1e9, 3), "plans": st["plans"],
        "wall_s": round(span, 3),
    }


# ---------------------------------------------------------------------------
UNIT_ROUNDOFF = {"fp32": 2.0 ** -24, "fp16": 2.0 ** -11, "bf16": 2.0 ** -8}
STUDY_FACS = (("dual_select", 1e-7), ("linzer_feig_clamped", 1e-7), ("linzer_feig_clamped", 2.0 ** -14),
              ("cosine", 1e-7))


def error_study(log2ns=(10, 12, 14, 16, 18, 20, 22, 24), precisions=("fp32", "fp16", "bf16"),
                dists=("uniform", "gaussian")):
    """Measured error of the three factorizations (LF also with eps = 2^-14)
    on the GPU path against numpy's FP64 FFT of the same rounded inputs, next
    to the cumulative bound of Eq. 11, (1 + |t|max eps)^m - 1, with |t|max of
    the plan's own rounded table.  FP16/BF16 run with x0.5 per pass (DFT/N),
    FP32 unscaled.  Per case: a few sampled signals (fewer at large N, where
    numpy's FFT dominates the time)."""
    import torch
    import paper_2604_00567_b300 as dsfft
    from paper_2604_00567_b300 import signals
    rows = []
    for l in log2ns:
        n = 1 << l
        count = 4 if l <= 20 else 2 if l <= 22 else 1
        for prec in precisions:
            for fac, eps in STUDY_FACS:
                plan = dsfft.Plan(n, prec, fac, lf_eps=eps)
                t, m, path = plan.table(-1)
                finite_t = np.isfinite(t) & np.isfinite(m)
                tmax = float(np.max(np.abs(t))) if np.all(finite_t) else float("inf")
                with np.errstate(over="ignore"):
                    bound = float(np.power(1.0 + tmax * UNIT_ROUNDOFF[prec], float(l)) - 1.0)
                row = {"N": n, "precision": prec, "factorization": fac, "lf_eps": eps if fac == "linzer_feig_clamped" else None,
                       "t_max": tmax, "nonfinite_table_entries": int((~finite_t).sum()),
                       "bound_eq11": bound}
                for dist in dists:
                    x = signals.device_signal(count, n, prec, seed=7 * l + 1, dist=dist)
                    y = plan.exec(x)
                    torch.cuda.synchronize()
                    xs, ys = signals.from_torch(x, prec), signals.from_torch(y, prec)
                    ref = np.fft.fft(xs, axis=-1) / (n if plan.scale_forward else 1)
                    bad = ~np.isfinite(ys)
                    row[f"nonfinite_out_{dist}"] = int(bad.sum())
                    row[f"rel_l2_{dist}"] = (float(np.linalg.norm((ys - ref).ravel()) / np.linalg.norm(ref.ravel()))
                                             if not bad.any() else float("nan"))
                    del x, y
                rows.append(row)
                plan.close()
        torch.cuda.empty_cache()
    return rows


def error_study_markdown(rows) -> str:
    def f(v):
        if v is None:
            return "—"
        if isinstance(v, float):
            if v != v:
                return "non-finite"
            if v == float("inf"):
                return "inf"
            return f"{v:.3g}"
        return str(v)
    out = ["| N | prec | factorization | \\|t\\|max | Eq. 11 bound | rel L2 uniform | rel L2 gaussian | non-finite outputs |",
           "|---|---|---|---|---|---|---|---|"]
    for r in rows:
        fac = r["factorization"] + (f" (eps={r['lf_eps']:.3g})" if r["lf_eps"] is not None else "")
        nf = r["nonfinite_out_uniform"] + r["nonfinite_out_gaussian"]
        out.append(f"| 2^{int(np.log2(r['N']))} | {r['precision']} | {fac} | {f(r['t_max'])} | {f(r['bound_eq11'])} | "
                   f"{f(r['rel_l2_uniform'])} | {f(r['rel_l2_gaussian'])} | {nf} |")
    return "\n".join(out)


# ---------------------------------------------------------------------------
def cpu_baseline(log2ns, samples_div=CPU_SAMPLE_DIV, seconds_cap=None):
    """Time the CPU oracle (op-by-op FP16 emulation of the same FFT) on a
    bounded sample of each N's batch, on all host cores."""
    import oracle as orc
    from paper_2604_00567_b300 import signals
    cores = os.cpu_count() or 1
    tot_tr, tot_s = 0, 0.0
    parts = []
    for l in log2ns:
        n = 1 << l
        cnt = max(2, batch_for(l) // samples_div)
        x = signals.signal(4242 + l, cnt, n, PRECISION)
        t, m, p = orc.table(n, orc.DS, orc.FP16, scaled=True)
        t0 = time.perf_counter()
        orc.emulate_fft(x, orc.FP16, t, m, p, scaled=True, threads=cores)
        dt = time.perf_counter() - t0
        tot_tr += cnt
        tot_s += dt
        parts.append(f"{cnt}x2^{l}")
    # the sample keeps the workload's mix (1/samples_div of each batch)
    return {"value": tot_tr / tot_s, "unit": "transforms/s", "cores": cores, "kind": "oracle",
            "sample": f"{', '.join(parts)} signals (1/{samples_div} of each batch), fp16 dual_select "
                      f"op-by-op emulation in C, {tot_s:.1f} s"}


def run_reference(args):
    """The oracle as the reference arm: rank 0 only, bounded samples."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    log2ns = list(args.log2n)
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(log2ns, samples_div=CPU_SAMPLE_DIV * 8)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(log2ns, samples_div=CPU_SAMPLE_DIV * 8))
    wall = time.perf_counter() - t0
    value = statistics.mean(v["value"] for v in vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "transforms/s",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * wall / args.steps, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16",
        "data": "synthetic",
        "config": {"workload": "fp16 dual_select forward FFT, x0.5 per pass, 1 GiB batch at each N",
                   "N": [1 << l for l in log2ns], "precision": PRECISION, "factorization": FACTORIZATION},
        "cpu_baseline": {"value": value, "unit": "transforms/s", "cores": vals[0]["cores"], "kind": "oracle",
                         "sample": vals[0]["sample"]},
        "e2e": {"value": value, "unit": "transforms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_exec_only(args):
    """Profiling driver: plan + seeded input for one N, `--iters` fft_exec
    calls on a `--batch-mib` batch, nothing timed (for ncu captures)."""
    import torch
    import paper_2604_00567_b300 as dsfft
    from paper_2604_00567_b300 import signals
    l, prec = args.exec_only, args.precision
    n = 1 << l
    eb = 8 if prec == "fp32" else 4
    batch = max(1, (args.batch_mib << 20) // (eb * n))
    plan = dsfft.Plan(n, prec, args.factorization, variant=args.variant)
    x = signals.device_signal(batch, n, prec, seed=l)
    y = torch.empty_like(x)
    for _ in range(args.iters):
        plan.exec(x, out=y)
    torch.cuda.synchronize()
    print(json.dumps({"exec_only": True, "N": n, "precision": prec, "batch": batch, "iters": args.iters,
                      "kernel": plan.info()["kernel"], "variant": plan.info()["variant_name"],
                      "launches_per_exec": plan.info()["launches"]}))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1,
                    help="replicas, one per GPU (started with torchrun when not already under it)")
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--log2n", type=int, nargs="+", default=list(LOG2NS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-loop measurement")
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--serve-only", action="store_true", help="print only the serving-loop measurement")
    ap.add_argument("--error-study", action="store_true",
                    help="LF / cosine / dual-select error study across N and precisions (JSON + markdown)")
    ap.add_argument("--exec-only", type=int, metavar="LOG2N",
                    help="profiling driver: run --iters transforms of one size and exit")
    ap.add_argument("--precision", default="fp16", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--factorization", default="dual_select",
                    choices=["dual_select", "linzer_feig_clamped", "cosine"])
    ap.add_argument("--batch-mib", type=int, default=256)
    ap.add_argument("--variant", default="auto",
                    choices=["auto", "fused_wide", "fused_narrow", "cluster", "sweeps", "fused_tma"])
    ap.add_argument("--iters", type=int, default=2)
    args = ap.parse_args()
    if args.exec_only is not None:
        run_exec_only(args)
        return
    if args.error_study:
        rows = error_study()
        print(error_study_markdown(rows), flush=True)
        print(json.dumps({"error_study": rows}), flush=True)
        return
    if args.serve_only:
        print(json.dumps({"serve": serve_measure(args.serve_seconds)}), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # one replica per GPU: start the ranks (torchrun) with the same arguments
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
               "--master-addr", "127.0.0.1", "--master-port", str(29500 + os.getpid() % 2000),
               os.path.abspath(__file__)] + sys.argv[1:]
        sys.exit(subprocess.call(cmd))
    if world != args.gpus:
        sys.exit(f"bench.py: --gpus {args.gpus} but WORLD_SIZE={world}")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
