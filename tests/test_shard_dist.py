"""Replicate sharding on CPU with two gloo ranks: each rank takes its share of
an ensemble (paper_2306_11544_gb300.shard), advances its replicates with the
oracle, and the per-replicate positions gathered from both ranks, put back in
the ensemble's order, equal a single-process run of every replicate bit for
bit.  The ranks exchange nothing but the results gathered for the check."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

STEPS = 3


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _ensemble():
    from paper_2306_11544_gb300 import synth
    return synth.ensemble_256(seed=4, scale=0.01, n_rep=6)


def _advance(p):
    import oracle
    dims = oracle.grid_dims(p.lo, p.hi, p.h)
    x, _, _ = oracle.run(p.xyz, p.R, p.ccr, p.cca, p.A, p.lo, p.h, dims, p.dt, STEPS)
    return x


def _rank(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import oracle
    from paper_2306_11544_gb300 import shard
    oracle.set_threads(1)
    ws, r, _ = shard.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=ws)
    try:
        ens = _ensemble()
        sub, mine = shard.local_ensemble(ens, r, ws)
        pieces = [_advance(p) for p in sub.reps]
        gathered = [None] * ws
        dist.all_gather_object(gathered, (mine, pieces))
        if r == 0:
            idx = [g[0] for g in gathered]
            res = shard.reassemble([g[1] for g in gathered], idx, len(ens.reps))
            out["idx"] = idx
            out["res"] = [x.tolist() for x in res]
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_single_process_ensemble():
    import oracle
    oracle.build()
    world = 2
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    ens = _ensemble()
    idx = out["idx"]
    assert sorted(i for x in idx for i in x) == list(range(len(ens.reps)))
    assert all(len(x) > 0 for x in idx)
    for k, p in enumerate(ens.reps):
        assert np.array_equal(np.asarray(out["res"][k]), _advance(p)), k


def test_reassembly_rejects_missing_and_duplicate_replicates():
    from paper_2306_11544_gb300 import shard
    a, b = np.zeros((2, 3)), np.ones((1, 3))
    assert [x.shape[0] for x in shard.reassemble([[a], [b]], [[1], [0]], 2)] == [1, 2]
    with pytest.raises(ValueError):
        shard.reassemble([[a], [b]], [[0], [0]], 2)
    with pytest.raises(ValueError):
        shard.reassemble([[a], []], [[0], []], 2)
    with pytest.raises(ValueError):
        shard.reassemble([[a, b]], [[0]], 2)
    rows = np.arange(12).reshape(6, 2)
    parts = shard.split_rows(rows, [2, 0, 4])
    assert [x.shape[0] for x in parts] == [2, 0, 4] and np.array_equal(np.vstack(parts), rows)
