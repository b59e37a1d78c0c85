"""Velocity variants on the GPU (per-type adhesion affinity, domain walls)
against the variant oracle: FP64 mode bit for bit (velocities and
trajectories), the FP32 modes within the stated tolerances, with every dense
kernel; an affinity matrix of ones reproduces the base law bit for bit;
invalid settings are refused."""
import numpy as np
import pytest

import oracle
from paper_2306_11544_gb300 import mech, synth
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

AFF = np.array([[1.0, 0.3, 2.0],
                [0.3, 0.0, 1.5],
                [2.0, 1.5, 0.7]])


@pytest.fixture(scope="module", autouse=True)
def _lib():
    H.lib()
    oracle.build()


def walled_population(seed=5, scale=0.004):
    """A three-type spheroid (the 1M-cell recipe at a small scale) in a box
    that cuts through it: many cells overlap a face or lie beyond it."""
    pop = synth.spheroid_1m(seed=seed, scale=scale)
    r = np.abs(pop.xyz).max()
    half = 0.8 * r
    pop.lo = np.full(3, -half)
    pop.hi = np.full(3, half)
    return pop


def walls_of(pop, mask=0b111111, cw=5.0):
    return (pop.lo, pop.hi, mask, cw)


def configure(m, pop, aff=AFF, mask=0b111111, cw=5.0):
    m.set_affinity(aff)
    m.set_walls(mask, cw)


def test_population_exercises_the_variants():
    pop = walled_population()
    assert set(np.unique(pop.ctype)) == {0, 1, 2}
    outside = (pop.xyz < pop.lo).any(axis=1) | (pop.xyz > pop.hi).any(axis=1)
    assert outside.sum() > 10


def test_fp64_velocities_and_trajectory_are_bit_identical():
    pop = walled_population()
    dims = H.dims_of(pop)
    with H.make(pop, "fp64") as m:
        configure(m, pop)
        v = m.compute_velocities()
        m.step(20)
        x = m.positions()
    vref = oracle.velocities_ext(pop.xyz, pop.R, pop.ccr, pop.cca, pop.A, pop.lo, pop.h, dims, pop.ctype, AFF,
                                 walls_of(pop))
    assert np.array_equal(v, vref), float(np.abs(v - vref).max())
    xr, _, _ = oracle.run_ext(pop.xyz, pop.R, pop.ccr, pop.cca, pop.A, pop.lo, pop.h, dims, pop.dt, 20, pop.ctype,
                              AFF, walls_of(pop))
    assert np.array_equal(x, xr), float(np.abs(x - xr).max())


@pytest.mark.parametrize("kernel", [None, "block_per_tile", "warp_per_voxel"])
@pytest.mark.parametrize("mode", ["mixed", "kahan"])
def test_fp32_modes_match_the_oracle(mode, kernel):
    pop = walled_population(seed=6)
    dims = H.dims_of(pop)
    with H.make(pop, mode) as m:
        configure(m, pop)
        if kernel is None:
            m.set_tiling(None)  # every cell through the thread-per-cell kernel
        else:
            m.set_dense_kernel(kernel)
            m.set_tiling((4, 4, 4), 1)  # every tile dense
        for _ in range(2):
            x = m.positions()
            m.step(1)
            v = m.velocities()
            vref = oracle.velocities_ext(x, pop.R, pop.ccr, pop.cca, pop.A, pop.lo, pop.h, dims, pop.ctype, AFF,
                                         walls_of(pop))
            assert H.rel_err(v, vref) <= H.TOL_V_MIXED
        m.step(38)
        xg = m.positions()
    xr, _, _ = oracle.run_ext(pop.xyz, pop.R, pop.ccr, pop.cca, pop.A, pop.lo, pop.h, dims, pop.dt, 40, pop.ctype,
                              AFF, walls_of(pop))
    assert np.abs(xg - xr).max() <= H.TOL_X_MIXED


@pytest.mark.parametrize("mode", ["fp64", "mixed", "kahan"])
def test_affinity_of_ones_is_the_base_law(mode):
    pop = walled_population(seed=7)
    states = []
    for aff in (None, np.ones((3, 3))):
        with H.make(pop, mode) as m:
            m.set_affinity(aff)
            m.step(5)
            states.append(m.read_state())
    for k in ("xyz", "vprev", "comp"):
        assert np.array_equal(states[0][k], states[1][k]), k


def test_walls_on_some_faces_only():
    pop = walled_population(seed=8)
    dims = H.dims_of(pop)
    for mask in (0b000001, 0b100100):
        with H.make(pop, "fp64") as m:
            m.set_walls(mask, 2.5)
            v = m.compute_velocities()
        vref = oracle.velocities_ext(pop.xyz, pop.R, pop.ccr, pop.cca, pop.A, pop.lo, pop.h, dims, None, None,
                                     walls_of(pop, mask, 2.5))
        assert np.array_equal(v, vref)


def test_batch_with_variants_equals_plain_handles():
    reps = [walled_population(seed=s, scale=0.002) for s in (11, 12)]
    ens = synth.Ensemble("walled", reps, 10, {})
    with mech.Mech.from_ensemble(ens, mode="kahan") as mb:
        for r, p in enumerate(reps):
            mb.set_domain(r, p.lo, p.hi)
        mb.set_affinity(AFF)
        mb.set_walls(0b111111, 5.0)
        mb.step(6)
        xb = mb.positions()
    off = 0
    for p in reps:
        with H.make(p, "kahan") as m:
            configure(m, p)
            m.step(6)
            x = m.positions()
        assert np.array_equal(xb[off:off + p.n], x)
        off += p.n


def test_added_cells_carry_their_types():
    """Division with types: daughters of type 2 next to survivors; FP64 stays
    bit-identical to the oracle applying the same change."""
    pop = walled_population(seed=9)
    dims = H.dims_of(pop)
    rng = np.random.Generator(np.random.PCG64(3))
    with H.make(pop, "fp64") as m:
        configure(m, pop)
        m.step(3)
        x = m.positions()
        par = rng.choice(pop.n, size=40, replace=False)
        xn = x[par] + rng.normal(0.0, 2.0, size=(40, 3))
        tn = np.full(40, 2, np.int32)
        m.add_cells(xn, pop.R[par], pop.ccr[par], pop.cca[par], tn)
        m.step(3)
        xg = m.positions()
    xr, vp, _ = oracle.run_ext(pop.xyz, pop.R, pop.ccr, pop.cca, pop.A, pop.lo, pop.h, dims, pop.dt, 3, pop.ctype,
                               AFF, walls_of(pop))
    xyz2 = np.vstack([xr, xn])
    R2 = np.concatenate([pop.R, pop.R[par]])
    ccr2 = np.concatenate([pop.ccr, pop.ccr[par]])
    cca2 = np.concatenate([pop.cca, pop.cca[par]])
    t2 = np.concatenate([pop.ctype, tn])
    vp2 = np.vstack([vp, np.zeros((40, 3))])
    xr2, _, _ = oracle.run_ext(xyz2, R2, ccr2, cca2, pop.A, pop.lo, pop.h, dims, pop.dt, 3, t2, AFF, walls_of(pop),
                               vprev=vp2)
    assert np.array_equal(xg, xr2)


def test_invalid_variant_settings_are_refused():
    pop = walled_population()
    with H.make(pop, "kahan") as m:
        def sym3(a01):
            a = np.ones((3, 3))
            a[0, 1] = a[1, 0] = a01
            return a
        asym = np.ones((3, 3))
        asym[0, 2] = 0.4
        for bad, code in ((asym, mech.MECH_E_ARG),                                 # asymmetric
                          (sym3(-0.1), mech.MECH_E_ARG),                           # negative
                          (sym3(np.inf), mech.MECH_E_NONFINITE),
                          (np.ones((2, 2)), mech.MECH_E_ARG),                      # type 2 outside a 2 x 2 table
                          (np.ones((17, 17)), mech.MECH_E_ARG)):
            with pytest.raises(mech.MechError) as e:
                m.set_affinity(bad)
            assert e.value.code == code
        for mask, cw, code in ((64, 1.0, mech.MECH_E_ARG), (-1, 1.0, mech.MECH_E_ARG), (3, -1.0, mech.MECH_E_ARG),
                               (3, np.nan, mech.MECH_E_NONFINITE)):
            with pytest.raises(mech.MechError) as e:
                m.set_walls(mask, cw)
            assert e.value.code == code
        m.set_affinity(AFF)
        with pytest.raises(mech.MechError) as e:  # a new cell of a type outside the table
            m.add_cells(np.zeros((1, 3)), [8.4], [10.0], [0.4], np.array([3], np.int32))
        assert e.value.code == mech.MECH_E_ARG


@pytest.mark.parametrize("mode", ["mixed", "kahan"])
def test_graph_replay_with_variants_is_bitwise(mode):
    """Setting the variants invalidates a captured graph; the replayed steps
    equal direct launches bit for bit."""
    pop = walled_population(seed=10)
    states = []
    for graph in (0, 4):
        with H.make(pop, mode) as m:
            if graph:
                m.set_graph(graph)
                m.step(4)  # captured without the variants
            else:
                m.step(4)
            configure(m, pop)
            m.step(8)
            states.append(m.read_state())
    for k in ("xyz", "vprev", "comp"):
        assert np.array_equal(states[0][k], states[1][k]), k
