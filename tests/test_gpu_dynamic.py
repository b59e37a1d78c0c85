"""Dynamic population: cells removed (death) and added (division) between
steps, against the oracle run on the same changed population.  The oracle
side applies the change to its own FP64 state: survivors keep their position
and previous velocity in caller order, new cells start with a zero previous
velocity (as at creation)."""
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


def daughters(pop_R, x, alive, rng, m):
    """m new cells, each half a radius from a random survivor, with its
    parent's radius and coefficients."""
    parents = rng.choice(np.flatnonzero(alive), size=m)
    u = rng.normal(size=(m, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    return parents, x[parents] + 0.5 * pop_R[parents][:, None] * u


class OracleState:
    """The oracle's FP64 state of a population whose cells change."""

    def __init__(self, pop):
        self.pop = pop
        self.x = pop.xyz.copy()
        self.vprev = np.zeros_like(self.x)
        self.R, self.ccr, self.cca = pop.R.copy(), pop.ccr.copy(), pop.cca.copy()
        self.v = None

    def run(self, steps):
        p = self.pop
        self.x, self.vprev, self.v = oracle.run(self.x, self.R, self.ccr, self.cca, p.A, p.lo, p.h, H.dims_of(p),
                                                p.dt, steps, vprev=self.vprev)

    def remove(self, alive):
        self.x, self.vprev = self.x[alive], self.vprev[alive]
        self.R, self.ccr, self.cca = self.R[alive], self.ccr[alive], self.cca[alive]

    def add(self, xyz, R, ccr, cca):
        self.x = np.vstack([self.x, xyz])
        self.vprev = np.vstack([self.vprev, np.zeros_like(xyz)])
        self.R, self.ccr, self.cca = (np.concatenate([self.R, R]), np.concatenate([self.ccr, ccr]),
                                      np.concatenate([self.cca, cca]))


def check(mode, x, v, ref):
    if mode == "fp64":
        assert np.array_equal(x, ref.x)  # same operations in the same order
        assert np.array_equal(v, ref.v)
    else:
        assert np.abs(x - ref.x).max() <= H.TOL_X_MIXED
        assert H.rel_err(v, ref.v) <= H.TOL_V_MIXED


@pytest.mark.parametrize("mode", ["fp64", "mixed", "kahan"])
def test_death_and_division_match_oracle(mode):
    """2,000 cells: 5 steps, 10 % of the cells die and 150 divide, 5 steps,
    again, 5 steps."""
    pop = synth.spheroid_2k(seed=21)
    rng = np.random.Generator(np.random.PCG64(22))
    ref = OracleState(pop)
    with H.make(pop, mode) as m:
        for _ in range(2):
            m.step(5)
            ref.run(5)
            alive = rng.random(m.n) >= 0.1
            parents, xyz = daughters(ref.R, ref.x, alive, rng, 150)
            R, ccr, cca = ref.R[parents], ref.ccr[parents], ref.cca[parents]
            m.remove_cells(alive)
            ref.remove(alive)
            m.add_cells(xyz, R, ccr, cca)
            ref.add(xyz, R, ccr, cca)
            assert m.n == m.info()["n_cells"] == len(ref.x)
        m.step(5)
        ref.run(5)
        x, v = m.positions(), m.velocities()
    check(mode, x, v, ref)


@pytest.mark.parametrize("mode", ["fp64", "kahan"])
def test_growth_beyond_capacity(mode):
    """500 cells grow to 2,300 in three additions (the device buffers grow
    twice), with steps in between."""
    pop = synth.spheroid_2k(seed=23, n=500)
    rng = np.random.Generator(np.random.PCG64(24))
    ref = OracleState(pop)
    with H.make(pop, mode) as m:
        for m_new in (300, 700, 800):
            m.step(3)
            ref.run(3)
            parents, xyz = daughters(ref.R, ref.x, np.ones(m.n, bool), rng, m_new)
            R, ccr, cca = ref.R[parents], ref.ccr[parents], ref.cca[parents]
            m.add_cells(xyz, R, ccr, cca)
            ref.add(xyz, R, ccr, cca)
        m.step(4)
        ref.run(4)
        x, v = m.positions(), m.velocities()
    check(mode, x, v, ref)


@pytest.mark.parametrize("mode", ["mixed", "kahan"])
def test_turnover_with_tiles_and_graphs(mode):
    """Clustered population with dense tiles and 4-step graphs: the handle
    changes between graph launches (the graphs are re-captured for the new
    population) and matches a handle without graphs bit for bit, and the
    oracle within the mixed-mode bound."""
    pop = synth.clustered_20m(seed=25, scale=0.002)
    rng = np.random.Generator(np.random.PCG64(26))
    ref = OracleState(pop)
    with H.make(pop, mode, graph=4) as g, H.make(pop, mode) as p:
        for m in (g, p):
            m.set_tiling((4, 4, 4), 12)
        for _ in range(2):
            for m in (g, p):
                m.step(8)
            ref.run(8)
            alive = rng.random(g.n) >= 0.05
            parents, xyz = daughters(ref.R, ref.x, alive, rng, 2000)
            R, ccr, cca = ref.R[parents], ref.ccr[parents], ref.cca[parents]
            for m in (g, p):
                m.remove_cells(alive)
                m.add_cells(xyz, R, ccr, cca)
            ref.remove(alive)
            ref.add(xyz, R, ccr, cca)
        for m in (g, p):
            m.step(8)
        ref.run(8)
        sg, sp = g.read_state(), p.read_state()
        x, v = g.positions(), g.velocities()
    for k in ("xyz", "vprev", "comp"):
        assert np.array_equal(sg[k], sp[k]), k
    check(mode, x, v, ref)


def test_remove_all_then_add():
    pop = synth.spheroid_2k(seed=27, n=300)
    rng = np.random.Generator(np.random.PCG64(28))
    with H.make(pop, "fp64") as m:
        m.step(2)
        m.remove_cells(np.zeros(m.n, bool))
        assert m.n == 0 and m.positions().shape == (0, 3)
        m.step(3)  # nothing to do
        xyz = pop.xyz[:120] + rng.normal(0, 0.1, size=(120, 3))
        m.add_cells(xyz, pop.R[:120], pop.ccr[:120], pop.cca[:120])
        m.step(4)
        x = m.positions()
    ref = OracleState(pop)
    ref.remove(np.zeros(pop.n, bool))
    ref.add(xyz, pop.R[:120], pop.ccr[:120], pop.cca[:120])
    ref.run(4)
    assert np.array_equal(x, ref.x)


@pytest.mark.parametrize("mode", ["fp64", "kahan"])
def test_remove_none_and_add_nothing_change_nothing(mode):
    pop = synth.spheroid_2k(seed=29, n=400)
    with H.make(pop, mode) as m:
        m.step(3)
        before = m.read_state()
        m.remove_cells(np.ones(m.n, bool))
        m.add_cells(np.zeros((0, 3)), [], [], [])
        after = m.read_state()
        m.step(2)
    for k in ("xyz", "vprev", "comp"):
        assert np.array_equal(before[k], after[k]), k


def test_invalid_changes_are_refused_before_anything_changes():
    pop = synth.spheroid_2k(seed=31, n=200)
    with H.make(pop, "mixed") as m:
        m.step(2)
        before = m.read_state()
        big = 30.0 / (2 * pop.A) * 1.01  # needs a voxel above the workload's 30 um
        with pytest.raises(mech.MechError) as e:
            m.add_cells([[0.0, 0.0, 0.0]], [big], [10.0], [0.4])
        assert e.value.code == mech.MECH_E_VOXEL_TOO_SMALL
        with pytest.raises(mech.MechError) as e:
            m.add_cells([[np.nan, 0.0, 0.0]], [8.0], [10.0], [0.4])
        assert e.value.code == mech.MECH_E_NONFINITE
        with pytest.raises(mech.MechError) as e:
            m.add_cells([[0.0, 0.0, 0.0]], [-1.0], [10.0], [0.4])
        assert e.value.code == mech.MECH_E_ARG
        assert m.n == 200 and m.info()["n_cells"] == 200
        after = m.read_state()
    for k in ("xyz", "vprev", "comp"):
        assert np.array_equal(before[k], after[k]), k
    ens = synth.ensemble_256(seed=32, scale=0.01, n_rep=3)
    with mech.Mech.from_ensemble(ens, mode="mixed") as b:
        with pytest.raises(mech.MechError) as e:  # a batch needs the per-replicate counts
            b.add_cells([[0.0, 0.0, 0.0]], [8.0], [10.0], [0.4])
        assert e.value.code == mech.MECH_E_ARG
        with pytest.raises(ValueError):
            b.add_cells([[0.0, 0.0, 0.0]], [8.0], [10.0], [0.4], counts=[1, 1, 0])


@pytest.mark.parametrize("mode", ["fp64", "mixed", "kahan"])
def test_batch_turnover_equals_separate_handles(mode):
    """Four replicates in one batch (one of them emptied, one growing from
    nothing) and four separate handles take the same deaths and divisions:
    the batch gives, replicate by replicate, exactly the separate handles'
    positions and velocities (every replicate stays one range of caller
    indices)."""
    ens = synth.ensemble_256(seed=33, scale=0.02, n_rep=4)
    rng = np.random.Generator(np.random.PCG64(34))
    reps = ens.reps
    with mech.Mech.from_ensemble(ens, mode=mode) as b:
        singles = [H.make(p, mode) for p in reps]
        try:
            for event in range(2):
                b.step(4)
                for s in singles:
                    s.step(4)
                xs = [s.positions() for s in singles]
                masks = [rng.random(s.n) >= 0.1 for s in singles]
                if event == 0:
                    masks[1][:] = False  # replicate 1 dies out
                add = [int(rng.integers(0, 30)) for _ in singles]
                if event == 1:
                    add[1] = 25  # and grows again
                new = []
                for r, (s, mk, k) in enumerate(zip(singles, masks, add)):
                    src = xs[r][mk] if mk.any() else reps[r].xyz
                    j = rng.integers(0, len(src), size=k)
                    xyz = src[j] + rng.normal(0, 2.0, size=(k, 3))
                    new.append((xyz, np.full(k, reps[r].R.max()), np.full(k, reps[r].ccr[0]),
                                np.full(k, reps[r].cca[0])))
                b.remove_cells(np.concatenate(masks))
                b.add_cells(*(np.concatenate([x[f] for x in new]) for f in range(4)), counts=add)
                for s, mk, (xyz, R, ccr, cca) in zip(singles, masks, new):
                    s.remove_cells(mk)
                    s.add_cells(xyz, R, ccr, cca)
                assert list(b.counts) == [s.n for s in singles]
            b.step(5)
            xb, vb = b.positions(), b.velocities()
            off = 0
            for r, s in enumerate(singles):
                s.step(5)
                x, v = s.positions(), s.velocities()
                assert np.array_equal(xb[off:off + s.n], x), r
                assert np.array_equal(vb[off:off + s.n], v), r
                off += s.n
        finally:
            for s in singles:
                s.close()
