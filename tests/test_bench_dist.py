"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own
timing; the job time is the slowest rank's and the throughput counts every
rank's replica.  (The GPU runs use NCCL; the reduction code is the same.)"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.5, 40.0][rank]  # rank 1 is the slower one
        t = bench.reduce_max(ms, dist, "cpu")
        v = bench.job_throughput(1000, world, 10, t * 1e-3)
        out[rank] = (t, v)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        t, v = out[r]
        assert t == 40.0
        assert v == pytest.approx(1000 * 2 * 10 / 0.040)


def test_single_process_needs_no_group():
    import bench
    assert bench.reduce_max(3.5, None, "cpu") == 3.5
    assert bench.job_throughput(5, 1, 2, 0.5) == 20.0
