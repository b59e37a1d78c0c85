"""mech_bin_noalloc, the binning entry point for callers that cannot allocate
device memory when they call it (their device memory is owned by another
allocator, or a cudaMalloc and its implicit synchronisation would stall a
latency-critical loop).  Its working memory is a fixed array inside the
library; this test checks, through the C ABI, that two calls in a row give
exactly the binning of the handle-based entry point (mech_debug_bins in FP64
mode): integer work, so the tolerance is bit-exact.  The second call also
shows that the leftover contents of the shared working array from the first
call do not leak into the next result."""
import numpy as np
import pytest
import torch

from paper_2306_11544_gb300 import mech, synth
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def test_no_alloc_binning_matches_handle_binning_twice():
    H.lib()
    stream = torch.cuda.current_stream()
    pops = [synth.clustered_20m(seed=21, scale=0.005), synth.spheroid_1m(seed=22, scale=0.05)]
    for pop in pops:
        with mech.Mech.from_population(pop, mode="fp64") as m:
            key_ref, _, start_ref, order_ref = m.bins()
            lo, dims, _ = m.grid(0)
        n = pop.n
        V = int(np.prod(dims))
        xyz = torch.from_numpy(np.ascontiguousarray(pop.xyz)).to("cuda")
        key = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        start = torch.full((V + 1,), -1, dtype=torch.int32, device="cuda")
        order = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        mech.mech_bin_noalloc(n, xyz.data_ptr(), lo, pop.h, dims, key.data_ptr(), start.data_ptr(),
                              order.data_ptr(), stream)
        stream.synchronize()
        assert np.array_equal(key.cpu().numpy().view(np.uint32), key_ref)
        assert np.array_equal(start.cpu().numpy().view(np.uint32), start_ref)
        assert np.array_equal(order.cpu().numpy().astype(np.int64), order_ref)


def test_no_alloc_rejects_sizes_beyond_its_working_memory():
    H.lib()
    with pytest.raises(mech.MechError) as e:
        mech.mech_bin_noalloc(1 << 19, 0, [0, 0, 0], 30.0, [4, 4, 4], 0, 1, 0)
    assert e.value.code == mech.MECH_E_ARG
    with pytest.raises(mech.MechError) as e:
        mech.mech_bin_noalloc(0, 0, [0, 0, 0], 30.0, [100, 100, 100], 0, 1, 0)
    assert e.value.code == mech.MECH_E_ARG
