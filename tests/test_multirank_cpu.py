"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own
problem time; the job time is the slowest rank and the value aggregates the
points of every rank (weak scaling, no data-path collective)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = 10.0 + 5.0 * rank
    mx = bench.reduce_max_ms(local, world, device="cpu")
    val = bench.aggregate_value(128.0 ** 3, world, mx)
    dist.barrier()
    q.put((rank, mx, val))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, val in out:
        assert mx == 15.0
        assert abs(val - 2 * 128.0 ** 3 / 15e-3 / 1e6) < 1e-6


def test_single_rank_passthrough():
    import bench
    assert bench.reduce_max_ms(3.5, 1) == 3.5
    assert bench.aggregate_value(1e6, 1, 1.0) == pytest.approx(1000.0)
