"""Replica (multi-GPU) bookkeeping of bench.py on CPU: two gloo ranks, the
job time is the slowest rank's and the throughput counts both ranks."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value = bench.replica_throughput(10.0 * (rank + 1), 1000, world)
    q.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_throughput():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in res:
        assert ms == 20.0                      # the slowest rank's time
        assert value == pytest.approx(2 * 1000 / 0.020)


def test_single_rank_is_local():
    import bench
    ms, value = bench.replica_throughput(5.0, 100, 1)
    assert ms == 5.0 and value == pytest.approx(100 / 0.005)
