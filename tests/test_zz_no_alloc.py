"""mech_bin_noalloc, the binning entry point for callers that cannot allocate
device memory when they call it (their device memory is owned by another
allocator, or a cudaMalloc and its implicit synchronisation would stall a
latency-critical loop).  Its working memory is a fixed array inside the
library.  Through the C ABI, this checks:
  * a first call with n = 0 (the set-up call the header recommends) works;
  * two calls in a row on different populations give exactly the oracle's
    binning (FP64 voxel keys, stable counting sort): integer work, so the
    tolerance is bit-exact, and the leftover contents of the shared working
    array from one call do not leak into the next;
  * a voxel holding 65,536 cells (the in-voxel ranking's costly case) is still
    ordered by input index;
  * sizes beyond the working memory are refused."""
import numpy as np
import pytest
import torch

import oracle
from paper_2306_11544_gb300 import mech, synth
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _bin(pop_xyz, lo, h, dims, stream):
    n = pop_xyz.shape[0]
    V = int(np.prod(dims))
    xyz = torch.from_numpy(np.ascontiguousarray(pop_xyz, dtype=np.float64)).to("cuda")
    key = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    start = torch.full((V + 1,), -1, dtype=torch.int32, device="cuda")
    order = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    mech.mech_bin_noalloc(n, xyz.data_ptr(), lo, h, dims, key.data_ptr(), start.data_ptr(), order.data_ptr(),
                          stream)
    stream.synchronize()
    return (key.cpu().numpy().view(np.uint32)[:n], start.cpu().numpy().view(np.uint32),
            order.cpu().numpy().astype(np.int64)[:n])


def _reference(xyz, lo, h, dims):
    key = oracle.keys(xyz, lo, h, dims)
    _, start, order = oracle.counting_sort(key, int(np.prod(dims)))
    return key, start, order


def test_no_alloc_binning_matches_the_oracle_twice():
    H.lib()
    oracle.build()
    stream = torch.cuda.current_stream()
    # the set-up call: no cells, a small grid
    key, start, order = _bin(np.zeros((0, 3)), np.zeros(3), 30.0, np.array([3, 2, 2], np.int32), stream)
    assert key.size == 0 and order.size == 0 and np.array_equal(start, np.zeros(13, np.uint32))
    pops = [synth.clustered_20m(seed=21, scale=0.005), synth.spheroid_1m(seed=22, scale=0.05)]
    for pop in pops:
        dims = oracle.grid_dims(pop.lo, pop.hi, pop.h)
        got = _bin(pop.xyz, pop.lo, pop.h, dims, stream)
        ref = _reference(pop.xyz, pop.lo, pop.h, dims)
        for g, r, name in zip(got, ref, ("key", "start", "order")):
            assert np.array_equal(g, r), name


def test_no_alloc_orders_a_crowded_voxel_by_input_index():
    H.lib()
    oracle.build()
    stream = torch.cuda.current_stream()
    rng = np.random.Generator(np.random.PCG64(23))
    n = 65536
    xyz = rng.uniform(31.0, 59.0, size=(n, 3))  # every cell in voxel (1, 1, 1)
    xyz[::7] = rng.uniform(0.0, 90.0, size=(len(xyz[::7]), 3))  # and some spread over the grid
    lo, h, dims = np.zeros(3), 30.0, np.array([3, 3, 3], np.int32)
    got = _bin(xyz, lo, h, dims, stream)
    ref = _reference(xyz, lo, h, dims)
    assert np.bincount(ref[0], minlength=27).max() > 50000
    for g, r, name in zip(got, ref, ("key", "start", "order")):
        assert np.array_equal(g, r), name


def test_no_alloc_rejects_sizes_beyond_its_working_memory():
    H.lib()
    with pytest.raises(mech.MechError) as e:
        mech.mech_bin_noalloc(1 << 19, 0, [0, 0, 0], 30.0, [4, 4, 4], 0, 1, 0)
    assert e.value.code == mech.MECH_E_ARG
    with pytest.raises(mech.MechError) as e:
        mech.mech_bin_noalloc(0, 0, [0, 0, 0], 30.0, [100, 100, 100], 0, 1, 0)
    assert e.value.code == mech.MECH_E_ARG
