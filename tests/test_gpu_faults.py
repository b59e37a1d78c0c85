"""Failure paths, made on the host (nothing here faults, traps or hangs a
GPU): a tile-kernel copy barrier armed to expect more bytes than are copied
(its bounded wait gives up after 1 ms and the kernel returns an error status),
and an injected device-allocation failure."""
import numpy as np
import pytest

import oracle
from paper_2306_11544_gb300 import mech, synth
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    H.lib()
    oracle.build()


def test_tile_wait_timeout_is_reported_and_state_recovers():
    pop = synth.clustered_20m(seed=14, scale=0.002)
    hmin = 2 * pop.A * pop.R.max() * (1 + 1e-5)
    with H.make(pop, "kahan", voxel=hmin) as m:
        m.set_tiling((4, 4, 4), 16)
        m.step(2)
        saved = m.read_state()
        mech.mech_debug_inject(m.h, mech.MECH_FAULT_TILE_WAIT)
        m.step(1)
        with pytest.raises(mech.MechError) as e:
            m.sync()
        assert e.value.code == mech.MECH_E_TIMEOUT
        with pytest.raises(mech.MechError) as e:
            m.step(1)  # the state is inconsistent until it is reloaded
        assert e.value.code == mech.MECH_E_STATE
        with pytest.raises(mech.MechError) as e:
            m.write_positions(saved["xyz"])  # positions alone do not repair the previous velocities
        assert e.value.code == mech.MECH_E_STATE
        mech.mech_debug_inject(m.h, mech.MECH_FAULT_NONE)
        m.load_state(saved)
        x = m.positions()
        m.step(1)
        v = m.velocities()
    vref = oracle.velocities(x, pop.R, pop.ccr, pop.cca, pop.A, pop.lo, pop.h, H.dims_of(pop))
    assert H.rel_err(v, vref) <= H.TOL_V_MIXED


def test_injected_allocation_failure_is_reported_once():
    pop = synth.spheroid_2k(seed=15, n=500)
    mech.mech_debug_inject(None, mech.MECH_FAULT_ALLOC)
    try:
        with pytest.raises(mech.MechError) as e:
            H.make(pop, "mixed")
        assert e.value.code == mech.MECH_E_OOM
    finally:
        mech.mech_debug_inject(None, mech.MECH_FAULT_NONE)
    with H.make(pop, "mixed") as m:  # the injected failure fired once
        m.step(2)
        assert np.all(np.isfinite(m.positions()))
