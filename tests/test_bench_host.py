"""Host logic of bench.py (no GPU): the turnover mode's precomputed death and
division events keep the cell count, place each daughter half a radius from a
survivor of that event, give it that cell's parameters, and are
reproducible; the ensemble's replicates are split over ranks once each and
in balance."""
import numpy as np
import pytest

import bench
from paper_2306_11544_gb300 import shard, synth


def replay(pop, events):
    """Apply the events to the initial indices, as the handle sees them."""
    orig = np.arange(pop.n)
    out = []
    for alive, xyz, R, ccr, cca in events:
        assert len(alive) == len(orig) == pop.n  # the count is kept
        orig = orig[alive]
        # each daughter sits half a radius from one survivor of this event
        d = np.linalg.norm(xyz[:, None, :] - pop.xyz[orig][None, :, :], axis=2)
        j = np.argmin(np.abs(d - 0.5 * pop.R[orig][None, :]), axis=1)
        parents = orig[j]
        assert np.allclose(np.linalg.norm(xyz - pop.xyz[parents], axis=1), 0.5 * pop.R[parents])
        assert np.array_equal(R, pop.R[parents]) and np.array_equal(ccr, pop.ccr[parents])
        assert np.array_equal(cca, pop.cca[parents])
        assert len(xyz) == pop.n - len(orig)  # as many daughters as deaths
        out.append(len(xyz))
        orig = np.concatenate([orig, parents])
    return out


def test_turnover_events_keep_the_count_and_follow_survivors():
    pop = synth.spheroid_1m(seed=3, scale=0.0005)  # 500 cells, three types
    events = bench.turnover_events(pop, 4, 0.05)
    counts = replay(pop, events)
    assert all(c > 0 for c in counts)
    again = bench.turnover_events(pop, 4, 0.05)
    for a, b in zip(events, again):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_replicate_sharding_covers_every_replicate_once_and_balances():
    counts = [p.n for p in synth.ensemble_256(seed=0, scale=0.01).reps]
    for world in (1, 2, 3, 8):
        parts = shard.shard_replicates(counts, world)
        flat = sorted(i for x in parts for i in x)
        assert flat == list(range(len(counts)))  # each replicate on exactly one rank
        loads = [sum(counts[i] for i in x) for x in parts]
        # greedy largest-first: no rank exceeds the mean by more than the largest replicate
        assert max(loads) - sum(counts) / world <= max(counts)
        assert shard.shard_replicates(counts, world) == parts  # deterministic
    with pytest.raises(ValueError):
        shard.shard_replicates([5, 6], 3)


def test_issue_roofline_only_for_the_counted_configuration():
    """The bench line's issue roofline scales the committed instruction count
    by the cell count and divides by the kernel time and SMs x 4 schedulers x
    clock; for any other configuration than the one counted it is absent."""
    import argparse
    tr = {"tile_kernel": {"warp_instructions_per_launch": 1000, "cells": 10, "source": "test"}}
    args = argparse.Namespace(workload="clustered_20m", mode="kahan", tile="4,4,4", dense_min=12,
                              dense_kernel="block_per_tile")
    r = bench.issue_roofline(tr, args, 20, 2e-3, 10, 1000.0)
    assert r["instructions_per_launch"] == 2000
    assert r["achieved"] == pytest.approx(1e6) and r["peak"] == pytest.approx(4e10)
    assert r["frac"] == pytest.approx(2.5e-5)
    for change in ({"mode": "mixed"}, {"tile": "4,4,8"}, {"dense_min": 16}, {"workload": "spheroid_1m"},
                   {"dense_kernel": "warp_per_voxel"}):
        other = argparse.Namespace(**{**vars(args), **change})
        assert bench.issue_roofline(tr, other, 20, 2e-3, 10, 1000.0) is None
    assert bench.issue_roofline(None, args, 20, 2e-3, 10, 1000.0) is None
    assert bench.issue_roofline({}, args, 20, 2e-3, 10, 1000.0) is None
