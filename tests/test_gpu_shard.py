"""Replicate sharding on one GPU: the batch handles of two ranks' shares
(built one after the other; the ranks never wait on each other) advance
their replicates exactly as the whole ensemble's batch handle does, replicate
by replicate and bit for bit."""
import numpy as np
import pytest

from paper_2306_11544_gb300 import shard, synth
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", ["mixed", "kahan"])
def test_rank_handles_reproduce_the_whole_batch(mode):
    H.lib()
    from paper_2306_11544_gb300 import mech
    ens = synth.ensemble_256(seed=5, scale=0.01, n_rep=7)
    with mech.Mech.from_ensemble(ens, mode=mode) as m:
        m.step(8)
        whole = shard.split_rows(m.positions(), [p.n for p in ens.reps])
    pieces, idx = [], []
    for rank in range(2):
        h, mine = shard.rank_handle(ens, rank, 2, mode=mode)
        with h:
            h.step(8)
            pieces.append(shard.split_rows(h.positions(), [ens.reps[i].n for i in mine]))
        idx.append(mine)
    got = shard.reassemble(pieces, idx, len(ens.reps))
    for k in range(len(ens.reps)):
        assert np.array_equal(got[k], whole[k]), k
