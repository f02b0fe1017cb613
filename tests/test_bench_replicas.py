"""Replica aggregation of bench.py over two gloo ranks on the CPU: the job's
throughput is all ranks' pixels over the slowest rank's time."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, port, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    total_ms = [100.0, 250.0][rank]  # rank 1 is the slow one
    val, ms = bench.aggregate(total_ms, px_per_step=1000, steps=10, world_size=2)
    q.put((rank, val, ms))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, val, ms in res:
        assert ms == 250.0
        # 2 ranks x 1000 px x 10 steps in 0.25 s = 80,000 px/s = 0.08 Mpix/s
        assert abs(val - 0.08) < 1e-12


def test_single_rank_is_plain_rate():
    import bench
    val, ms = bench.aggregate(50.0, px_per_step=2_000_000, steps=5, world_size=1)
    assert ms == 50.0 and abs(val - 200.0) < 1e-9
