"""Replicate sharding across GPUs (one process per GPU).

An ensemble's replicates are independent populations (the paper averages
its runs over 5 seeds, Sec. 5.5; an ABM study runs many such replicates), so
they shard across ranks with no exchange at all on the data path: every rank
advances its own replicates in its own batch handle on its own GPU, and the
only collective a job needs is the timing reduction.  A single population is
not split (that would need a halo exchange and cell migration every step).

Host logic only: the split, the per-rank sub-ensemble and the reassembly of
per-replicate results in the ensemble's order.  `rank_handle` builds the
rank's batch handle.
"""
from __future__ import annotations

import os

import numpy as np

from . import synth


def shard_replicates(counts, world: int):
    """Replicates split over `world` ranks: largest first, each to the rank
    with the fewest cells so far (ties to the lower rank).  Returns each
    rank's replicate indices in ascending order.  Every replicate lands on
    exactly one rank; no rank exceeds the mean load by more than the largest
    replicate."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if world > len(counts):
        raise ValueError(f"{world} ranks for {len(counts)} replicates")
    load = [0] * world
    out = [[] for _ in range(world)]
    for r in sorted(range(len(counts)), key=lambda i: (-int(counts[i]), i)):
        k = min(range(world), key=lambda w: (load[w], w))
        out[k].append(r)
        load[k] += int(counts[r])
    return [sorted(x) for x in out]


def dist_env():
    """(world size, rank, local rank) from the launcher's environment."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def local_ensemble(ens: synth.Ensemble, rank: int, world: int):
    """The sub-ensemble of `rank` and the global indices of its replicates."""
    parts = shard_replicates([p.n for p in ens.reps], world)
    mine = parts[rank]
    sub = synth.Ensemble(ens.name, [ens.reps[i] for i in mine], ens.steps, dict(ens.meta))
    return sub, mine


def split_rows(rows: np.ndarray, counts) -> list:
    """Per-replicate blocks of a concatenated per-cell array."""
    edges = np.concatenate([[0], np.cumsum(np.asarray(counts, dtype=np.int64))])
    return [rows[edges[k]:edges[k + 1]] for k in range(len(counts))]


def reassemble(pieces_by_rank, indices_by_rank, n_replicates: int) -> list:
    """Per-replicate results gathered from every rank (pieces_by_rank[k] is
    rank k's list of per-replicate arrays, for its replicate indices
    indices_by_rank[k]), back in the ensemble's replicate order."""
    out = [None] * n_replicates
    for pieces, idx in zip(pieces_by_rank, indices_by_rank):
        if len(pieces) != len(idx):
            raise ValueError("a rank returned a different number of replicates than it holds")
        for p, i in zip(pieces, idx):
            if out[i] is not None:
                raise ValueError(f"replicate {i} returned by two ranks")
            out[i] = p
    missing = [i for i, p in enumerate(out) if p is None]
    if missing:
        raise ValueError(f"replicates {missing[:5]} returned by no rank")
    return out


def rank_handle(ens: synth.Ensemble, rank: int, world: int, mode: str = "mixed"):
    """This rank's batch handle (on the current CUDA device) and the global
    indices of its replicates."""
    from .mech import Mech
    sub, mine = local_ensemble(ens, rank, world)
    return Mech.from_ensemble(sub, mode=mode), mine
