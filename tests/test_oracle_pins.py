"""The oracle against its pins (CPU only)."""
import pytest

import oracle
from tests import oracle_pins


@pytest.fixture(scope="module")
def o():
    oracle.build()
    return oracle._load()


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(o, pin):
    pin(o)


def test_thread_count_independence(o):
    """Each cell's sum is taken in a fixed order, so the thread count cannot
    change a single bit of the result."""
    import numpy as np
    from paper_2306_11544_gb300 import synth
    p = synth.spheroid_2k(seed=3)
    dims = oracle.grid_dims(p.lo, p.hi, p.h)
    t0 = o.num_threads()
    try:
        o.set_threads(1)
        v1 = o.velocities(p.xyz, p.R, p.ccr, p.cca, p.A, p.lo, p.h, dims)
        o.set_threads(max(2, t0))
        v2 = o.velocities(p.xyz, p.R, p.ccr, p.cca, p.A, p.lo, p.h, dims)
    finally:
        o.set_threads(t0)
    assert np.array_equal(v1, v2)
