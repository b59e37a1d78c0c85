"""CUDA path against the oracle, element by element, on seeded inputs.

Binning (keys, histogram, scan, permutation) must be bit-exact; FP64-mode
velocities must match to 1e-5 (they are expected to be bit-identical, since
the kernel evaluates the same operations in the same order); the FP32 pair
arithmetic of the mixed modes must match to TOL_V_MIXED; final positions of
the mixed modes to 1e-3 um."""
import numpy as np
import pytest

import oracle
from paper_2306_11544_gb300 import synth
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

MODES = ["fp64", "mixed", "kahan"]
DENSE_KERNELS = ["warp_per_voxel", "block_per_tile"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    H.lib()
    oracle.build()


def oracle_keys_for(m, pop, mode):
    dims = H.dims_of(pop)
    if mode == "fp64":
        return oracle.keys(m.positions(), pop.lo, pop.h, dims)
    if mode == "mixed":
        return oracle.keys_f32(m.positions().astype(np.float32), pop.lo, pop.h, dims)
    st = m.read_state()  # Kahan: the FP32 x_hi values decide the voxel
    return oracle.keys_f32(st["xyz"].astype(np.float32), pop.lo, pop.h, dims)


def check_bins(m, pop, mode):
    key, count, start, order = m.bins()
    kref = oracle_keys_for(m, pop, mode)
    V = int(np.prod(H.dims_of(pop)))
    cref, sref, oref = oracle.counting_sort(kref, V)
    assert np.array_equal(key, kref)
    assert np.array_equal(count, cref)
    assert np.array_equal(start, sref)
    assert np.array_equal(order, oref)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("name", list(H.parity_populations().keys()))
def test_binning_bit_exact(name, mode):
    pop = H.parity_populations()[name]
    with H.make(pop, mode) as m:
        check_bins(m, pop, mode)
        m.step(3)  # and again after the fused next-step histogram
        check_bins(m, pop, mode)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("name", list(H.edge_populations().keys()))
def test_edge_cases(name, mode):
    pop = H.edge_populations()[name]
    with H.make(pop, mode) as m:
        check_bins(m, pop, mode)
        x0 = m.positions()
        v = m.compute_velocities()
        vref = oracle.velocities(x0, pop.R, pop.ccr, pop.cca, pop.A, pop.lo, pop.h, H.dims_of(pop))
        tol = H.TOL_V_FP64 if mode == "fp64" else H.TOL_V_MIXED
        assert H.rel_err(v, vref) <= tol, (name, mode, H.rel_err(v, vref))
        if np.abs(vref).max() == 0:
            assert np.abs(v).max() == 0
        assert np.all(np.isfinite(v))


@pytest.mark.parametrize("name", list(H.parity_populations().keys()))
def test_fp64_velocity(name):
    pop = H.parity_populations()[name]
    with H.make(pop, "fp64") as m:
        v = m.compute_velocities()
        vref = oracle.velocities(pop.xyz, pop.R, pop.ccr, pop.cca, pop.A, pop.lo, pop.h, H.dims_of(pop))
        err = H.rel_err(v, vref)
        print(f"fp64 {name}: rel err {err:.3e}, bitwise equal: {np.array_equal(v, vref)}")
        assert err <= H.TOL_V_FP64
        assert np.array_equal(v, vref)  # same operations, same order


@pytest.mark.parametrize("mode", ["mixed", "kahan"])
@pytest.mark.parametrize("name", list(H.parity_populations().keys()))
def test_mixed_velocity_per_step(name, mode):
    """A7: per-step velocity on identical input positions (the GPU state fed
    to the oracle), over a few steps."""
    pop = H.parity_populations()[name]
    with H.make(pop, mode) as m:
        for _ in range(3):
            x = m.positions()
            m.step(1)
            v = m.velocities()
            vref = oracle.velocities(x, pop.R, pop.ccr, pop.cca, pop.A, pop.lo, pop.h, H.dims_of(pop))
            err = H.rel_err(v, vref)
            print(f"{mode} {name}: per-step velocity rel err {err:.3e}")
            assert err <= H.TOL_V_MIXED


def test_fp64_trajectory_spheroid_2k():
    """2,000 cells, FP64, the configuration's 100 steps, against the oracle."""
    pop = synth.spheroid_2k(seed=0)
    with H.make(pop, "fp64") as m:
        m.step(pop.steps)
        x = m.positions()
        v = m.velocities()
    xr, vpr, vr = oracle.run(pop.xyz, pop.R, pop.ccr, pop.cca, pop.A, pop.lo, pop.h, H.dims_of(pop), pop.dt, pop.steps)
    err = np.abs(x - xr).max()
    print(f"fp64 spheroid_2k 100 steps: max |dx| = {err:.3e} um, bitwise: {np.array_equal(x, xr)}")
    assert err <= 1e-9
    assert H.rel_err(v, vr) <= H.TOL_V_FP64


@pytest.mark.parametrize("mode", ["mixed", "kahan"])
def test_mixed_trajectory_spheroid_2k(mode):
    pop = synth.spheroid_2k(seed=0)
    with H.make(pop, mode) as m:
        m.step(pop.steps)
        x = m.positions()
    xr, _, _ = oracle.run(pop.xyz, pop.R, pop.ccr, pop.cca, pop.A, pop.lo, pop.h, H.dims_of(pop), pop.dt, pop.steps)
    err = np.abs(x - xr).max()
    print(f"{mode} spheroid_2k 100 steps: max |dx| = {err:.3e} um")
    assert err <= H.TOL_X_MIXED


@pytest.mark.parametrize("mode", ["mixed", "kahan"])
def test_mixed_trajectory_spheroid_1m_scaled(mode):
    """Three cell types with lognormal radii (20k cells, same density as the
    1M-cell spheroid), 300 steps."""
    pop = synth.spheroid_1m(seed=1, scale=0.02)
    steps = 300
    with H.make(pop, mode) as m:
        m.step(steps)
        x = m.positions()
    xr, _, _ = oracle.run(pop.xyz, pop.R, pop.ccr, pop.cca, pop.A, pop.lo, pop.h, H.dims_of(pop), pop.dt, steps)
    err = np.abs(x - xr).max()
    print(f"{mode} spheroid_1m x0.02 {steps} steps: max |dx| = {err:.3e} um")
    assert err <= H.TOL_X_MIXED


@pytest.mark.parametrize("mode", MODES)
def test_graph_replay_is_bitwise_identical(mode):
    pop = synth.clustered_20m(seed=3, scale=0.0005)
    with H.make(pop, mode) as a, H.make(pop, mode, graph=4) as b:
        a.step(11)
        b.step(11)
        sa, sb = a.read_state(), b.read_state()
    for k in ("xyz", "vprev", "comp"):
        assert np.array_equal(sa[k], sb[k]), k


@pytest.mark.parametrize("mode", MODES)
def test_checkpoint_resume_is_bitwise(mode):
    pop = synth.spheroid_1m(seed=4, scale=0.005)
    with H.make(pop, mode) as a:
        a.step(7)
        saved = a.read_state()
        a.step(6)
        full = a.read_state()
    with H.make(pop, mode) as b:
        b.load_state(saved)
        b.step(6)
        resumed = b.read_state()
    assert resumed["step"] == full["step"] == 13
    for k in ("xyz", "vprev", "comp"):
        assert np.array_equal(resumed[k], full[k]), k


@pytest.mark.parametrize("offset", [0.0, 1.0e6, 3.0e7])
@pytest.mark.parametrize("mode", ["fp64", "mixed", "kahan"])
def test_domains_far_from_the_origin(mode, offset):
    """The 2k spheroid and its domain translated far from the origin: the
    record build's integer split of FP64 positions (and, at 3e7 um, its
    fallback to FP64 arithmetic, whose fixed-point centre would pass 2^61),
    and the integer conversions between FP64 and the compensated FP32 pair
    at large exponents, over three steps against the oracle (FP64 mode bit
    for bit; the FP32 modes at the mixed tolerance, relative to the largest
    velocity)."""
    base = synth.spheroid_2k(seed=5)
    shift = np.array([offset, -0.5 * offset, 0.25 * offset])
    pop = synth.Population("far", base.xyz + shift, base.R, base.ccr, base.cca, base.ctype, base.lo + shift,
                           base.hi + shift, A=base.A, h=base.h, dt=base.dt, steps=3)
    dims = H.dims_of(pop)
    xr, _, _ = oracle.run(pop.xyz, pop.R, pop.ccr, pop.cca, pop.A, pop.lo, pop.h, dims, pop.dt, 3)
    with H.make(pop, mode) as m:
        m.step(3)
        x = m.positions()
        v = m.compute_velocities()
    vref = oracle.velocities(xr, pop.R, pop.ccr, pop.cca, pop.A, pop.lo, pop.h, dims)
    if mode == "fp64":
        assert np.array_equal(x, xr)
        assert np.array_equal(v, vref)
    else:
        assert np.abs(x - xr).max() <= H.TOL_X_MIXED
        assert H.rel_err(v, vref) <= H.TOL_V_MIXED


@pytest.mark.parametrize("mode", ["mixed", "kahan"])
def test_internal_voxel_keeps_the_pair_set(mode):
    """A finer internal voxel (>= 2 A max R) changes only the FP32 order."""
    pop = synth.clustered_20m(seed=5, scale=0.001)
    with H.make(pop, mode) as m:
        v30 = m.compute_velocities()
    hmin = 2 * pop.A * pop.R.max() * (1 + 1e-5)
    with H.make(pop, mode, voxel=hmin) as m:
        vmin = m.compute_velocities()
    vref = oracle.velocities(pop.xyz, pop.R, pop.ccr, pop.cca, pop.A, pop.lo, pop.h, H.dims_of(pop))
    assert H.rel_err(v30, vref) <= H.TOL_V_MIXED
    assert H.rel_err(vmin, vref) <= H.TOL_V_MIXED


def test_empty_population():
    pop = H.tiny_population(np.zeros((0, 3)), [-60] * 3, [60] * 3)
    with H.make(pop, "mixed") as m:
        m.step(5)
        assert m.positions().shape == (0, 3)
        assert m.info()["step"] == 5


def test_precision_switch_round_trip():
    pop = synth.spheroid_2k(seed=6)
    with H.make(pop, "fp64") as m:
        m.step(3)
        x = m.positions()
        m.set_precision("kahan")
        assert np.abs(m.positions() - x).max() <= 1e-4
        m.set_precision("fp64")
        assert np.abs(m.positions() - x).max() <= 1e-4


def test_write_positions_then_step_matches_fresh_handle():
    pop = synth.spheroid_2k(seed=7)
    rng = np.random.Generator(np.random.PCG64(8))
    moved = pop.xyz + rng.normal(0, 0.5, size=pop.xyz.shape)
    with H.make(pop, "fp64") as m:
        m.write_positions(moved)
        v = m.compute_velocities()
    vref = oracle.velocities(moved, pop.R, pop.ccr, pop.cca, pop.A, pop.lo, pop.h, H.dims_of(pop))
    assert np.array_equal(v, vref)


@pytest.mark.parametrize("pinned", [False, True])
@pytest.mark.parametrize("mode", ["fp64", "mixed", "kahan"])
def test_position_transfers_are_exact(mode, pinned):
    """1.3M cells, from pageable and from pinned host memory: after steps have
    reordered the cells into voxel order, the position read matches the state
    read bit for bit, and a write is read back exactly (Kahan mode: as the
    FP32 value and compensation it stores)."""
    import torch
    pop = synth.clustered_20m(seed=31, scale=0.065)
    n = pop.n
    assert 2 * 2**19 < n < 3 * 2**19
    buf = (torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy() if pinned
           else np.empty((n, 3)))
    with H.make(pop, mode) as m:
        m.set_tiling((4, 4, 8), 48)
        m.step(3)
        st = m.read_state()
        x = m.positions(out=buf).copy()
        assert np.array_equal(x, st["xyz"] - st["comp"] if mode == "kahan" else st["xyz"])
        rng = np.random.Generator(np.random.PCG64(32))
        buf[:] = x + rng.normal(0, 0.3, size=x.shape)
        w = buf.copy()
        m.write_positions(buf)
        back = m.positions()
    if mode == "kahan":
        hi = w.astype(np.float32).astype(np.float64)
        w = hi - (hi - w).astype(np.float32).astype(np.float64)
    assert np.array_equal(back, w)


def test_nonfinite_state_raises_device_flag():
    """A cell pushed to a non-finite position is reported, not hidden (the
    fault is made on the host: positions written with a huge value overflow
    in the update)."""
    from paper_2306_11544_gb300 import mech
    pop = H.tiny_population([[0.0, 0.0, 0.0], [1e-30, 0.0, 0.0]], [-60] * 3, [60] * 3)
    with H.make(pop, "fp64") as m:
        m.write_positions(np.array([[0.0, 0.0, 0.0], [1.7e308, 0.0, 0.0]]))
        m.set_params(1.25, 30.0, 1e308)
        m.load_state({"xyz": np.array([[0.0, 0.0, 0.0], [1.7e308, 0.0, 0.0]]),
                      "vprev": np.array([[0.0, 0.0, 0.0], [-1e308, 0.0, 0.0]]), "step": 0})
        m.step(1)
        with pytest.raises(mech.MechError) as e:
            m.sync()
        assert e.value.code == mech.MECH_E_DEVICE_FLAG


@pytest.mark.parametrize("kernel", DENSE_KERNELS)
@pytest.mark.parametrize("mode", ["mixed", "kahan"])
@pytest.mark.parametrize("tiling", [None, ((4, 4, 4), 32), ((4, 4, 4), 1), ((4, 4, 8), 32), ((4, 4, 8), 1),
                                    ((8, 4, 4), 32), ((8, 4, 4), 1)],
                         ids=["cells_only", "t444", "t444_all_dense", "t448", "t448_all_dense", "t844",
                              "t844_all_dense"])
def test_tiled_force_matches_oracle(mode, tiling, kernel):
    """Either dense-tile kernel (warp per voxel, or block per tile with the
    halo in shared memory) and the thread-per-cell kernel (the rest) give the
    same velocities as the oracle, for every tile shape and density
    threshold, including every tile treated as dense (the warp-per-voxel
    kernel then also takes the tiles at the grid faces)."""
    pop = synth.clustered_20m(seed=9, scale=0.002)
    with H.make(pop, mode) as m:
        m.set_dense_kernel(kernel)
        m.set_tiling(*tiling) if tiling else m.set_tiling(None)
        for _ in range(2):
            x = m.positions()
            m.step(1)
            v = m.velocities()
            vref = oracle.velocities(x, pop.R, pop.ccr, pop.cca, pop.A, pop.lo, pop.h, H.dims_of(pop))
            assert H.rel_err(v, vref) <= H.TOL_V_MIXED
        check_bins(m, pop, mode)


@pytest.mark.parametrize("mode", ["mixed", "kahan"])
def test_tile_passes_of_few_targets_split_lists(mode):
    """Interior tiles holding 1 to 40 cells: a warp pass of the block-per-tile
    kernel with g <= 16 targets splits each target's candidate list over
    32 / g lanes (2 to 32) and combines the parts' Kahan sums by a tree of
    shuffles; with 17 to 32 targets it is one lane per target, and 33 or
    more take a second pass.  Every count is present, each cluster packed
    tightly enough that most cells interact, and the velocities match the
    oracle."""
    rng = np.random.Generator(np.random.PCG64(41))
    h = 30.0
    counts = [1, 2, 3, 4, 5, 7, 8, 9, 15, 16, 17, 31, 32, 33, 40]
    xyz = []
    k = 0
    for bz in range(1, 4):
        for by in range(1, 4):
            for bx in range(1, 3):
                if k == len(counts):
                    break
                c = (np.array([bx, by, bz]) * 4 + 2) * h  # centre of the tile
                xyz.append(c + rng.uniform(-20.0, 20.0, size=(counts[k], 3)))
                k += 1
    xyz = np.concatenate(xyz)
    pop = H.tiny_population(xyz, [0.0] * 3, [4 * 5 * h] * 3, h=h)
    with H.make(pop, mode) as m:
        m.set_dense_kernel("block_per_tile")
        m.set_tiling((4, 4, 4), 1)
        v = m.compute_velocities()
    vref = oracle.velocities(xyz, pop.R, pop.ccr, pop.cca, pop.A, pop.lo, pop.h, H.dims_of(pop))
    assert np.abs(vref).max() > 1.0  # the clusters interact
    assert H.rel_err(v, vref) <= H.TOL_V_MIXED


@pytest.mark.parametrize("kernel", DENSE_KERNELS)
@pytest.mark.parametrize("tile", [(4, 4, 4), (4, 4, 8), (8, 4, 4)])
@pytest.mark.parametrize("mode", ["mixed", "kahan"])
def test_tile_halo_overflow_falls_back(mode, tile, kernel):
    """A crowd far denser than a tissue (3,000 cells in two voxels' width):
    the block-per-tile kernel's halo exceeds its shared-memory capacity and
    the tile is handed back to the thread-per-cell kernel; the warp-per-voxel
    kernel takes it with more than 64 targets per voxel and more candidates
    than its registers hold (the reloading path)."""
    rng = np.random.Generator(np.random.PCG64(31))
    xyz = rng.uniform(250.0, 305.0, size=(3000, 3))  # inside an interior tile of either shape
    pop = H.tiny_population(xyz, [0] * 3, [720] * 3)
    with H.make(pop, mode) as m:
        m.set_dense_kernel(kernel)
        m.set_tiling(tile, 32)
        v = m.compute_velocities()
    vref = oracle.velocities(xyz, pop.R, pop.ccr, pop.cca, pop.A, pop.lo, pop.h, H.dims_of(pop))
    assert H.rel_err(v, vref) <= H.TOL_V_MIXED


@pytest.mark.parametrize("kernel", DENSE_KERNELS)
@pytest.mark.parametrize("radii", ["uniform", "spread"])
@pytest.mark.parametrize("tile", [(4, 4, 4), (4, 4, 8), (8, 4, 4)])
@pytest.mark.parametrize("mode", ["mixed", "kahan"])
def test_tile_scan_keeps_pairs_at_the_cutoff(mode, tile, radii, kernel):
    """Every interacting pair of a jittered cubic lattice (13,824 cells, every
    tile dense) sits just inside the adhesion cutoff, 1 - d/(A S) between
    6e-4 and 5.4e-3, and all diagonal pairs are out of range: each velocity is
    a sum of six of the smallest possible terms, so a pair dropped by the tile
    kernel's cutoff test anywhere in a tile changes a velocity by its whole
    size.  "spread": the lattice radius lies between the smallest and the
    largest radius of the population (two isolated cells), which loosens the
    test through its R_max and C0 bounds."""
    rng = np.random.Generator(np.random.PCG64(41))
    R0 = 7.5 if radii == "spread" else 8.41
    AS = 1.25 * 2 * R0
    g = (np.arange(24) - 11.5) * AS * (1 - 3e-3)
    xyz = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    xyz += rng.uniform(-1.2e-3 * AS, 1.2e-3 * AS, size=xyz.shape)
    R = np.full(len(xyz), R0)
    if radii == "spread":
        xyz = np.vstack([xyz, [[285.0, 285.0, 285.0], [-285.0, 285.0, -285.0]]])
        R = np.append(R, [6.0, 9.0])
    pop = H.tiny_population(xyz, [-300] * 3, [300] * 3, R=R)
    hmin = 2 * pop.A * pop.R.max() * (1 + 1e-5)
    with H.make(pop, mode, voxel=hmin) as m:
        m.set_dense_kernel(kernel)
        m.set_tiling(tile, 1)
        v = m.compute_velocities()
    vref = oracle.velocities(xyz, pop.R, pop.ccr, pop.cca, pop.A, pop.lo, pop.h, H.dims_of(pop))
    assert (np.abs(vref[:13824]).max(axis=1) > 0).all()
    assert H.rel_err(v, vref) <= 1e-4


def test_internal_voxel_with_tiles_over_steps():
    """Autotuner-style setting: minimum internal voxel, 4x4x4 tiles, Kahan,
    20 steps against the FP64 oracle trajectory."""
    pop = synth.clustered_20m(seed=10, scale=0.001)
    hmin = 2 * pop.A * pop.R.max() * (1 + 1e-5)
    with H.make(pop, "kahan", voxel=hmin) as m:
        m.set_tiling((4, 4, 4), 32)
        m.step(20)
        x = m.positions()
    xr, _, _ = oracle.run(pop.xyz, pop.R, pop.ccr, pop.cca, pop.A, pop.lo, pop.h, H.dims_of(pop), pop.dt, 20)
    assert np.abs(x - xr).max() <= H.TOL_X_MIXED


@pytest.mark.parametrize("mode", MODES)
def test_batched_equals_plain_per_replicate(mode):
    """Replicates advanced together in one batched handle (graph replay) give,
    replicate by replicate, exactly the positions of separate handles."""
    from paper_2306_11544_gb300 import mech
    ens = synth.ensemble_256(seed=5, scale=0.05, n_rep=6)
    with mech.Mech.from_ensemble(ens, mode=mode) as b:
        b.set_graph(4)
        b.step(9)
        xb = b.positions()
        vb = b.velocities()
    off = 0
    for p in ens.reps:
        with H.make(p, mode) as m:
            m.step(9)
            x = m.positions()
            v = m.velocities()
        assert np.array_equal(xb[off:off + p.n], x), p.name
        assert np.array_equal(vb[off:off + p.n], v), p.name
        off += p.n


def test_batch_with_empty_and_tiny_replicates():
    from paper_2306_11544_gb300 import mech
    a = H.tiny_population([[0.0, 0.0, 0.0], [15.0, 0.0, 0.0]], [-60] * 3, [60] * 3)
    b = H.tiny_population(np.zeros((0, 3)), [-60] * 3, [60] * 3)
    c = synth.spheroid_2k(seed=12, n=300)
    xyz = np.concatenate([a.xyz, b.xyz, c.xyz])
    cat = lambda f: np.concatenate([getattr(a, f), getattr(b, f), getattr(c, f)])
    with mech.Mech(xyz, cat("R"), cat("ccr"), cat("cca"), counts=[a.n, b.n, c.n]) as m:
        m.set_params(1.25, 30.0, 0.1)
        for r, p in enumerate((a, b, c)):
            m.set_domain(r, p.lo, p.hi)
        m.set_precision("fp64")
        v = m.compute_velocities()
    va = oracle.velocities(a.xyz, a.R, a.ccr, a.cca, 1.25, a.lo, 30.0, H.dims_of(a))
    vc = oracle.velocities(c.xyz, c.R, c.ccr, c.cca, 1.25, c.lo, 30.0, H.dims_of(c))
    assert np.array_equal(v, np.concatenate([va, vc]))


def test_autotuner_restores_state_and_stays_correct():
    from paper_2306_11544_gb300 import autotune
    pop = synth.clustered_20m(seed=13, scale=0.002)
    hmin = 2 * pop.A * pop.R.max() * (1 + 1e-5)
    cfgs = [{"voxel": hmin, "tile": (4, 4, 4), "dense_min": 16, "dense_kernel": "block_per_tile", "block": 128},
            {"voxel": hmin, "tile": (4, 4, 4), "dense_min": 16, "dense_kernel": "warp_per_voxel", "block": 128},
            {"voxel": pop.h, "tile": None, "dense_min": 0, "dense_kernel": "block_per_tile", "block": 256}]
    with H.make(pop, "kahan") as m:
        m.step(2)
        before = m.read_state()
        res = autotune.autotune(m, hmin, pop.h, steps=2, warmup=1, cache_path=None, configs=cfgs)
        after = m.read_state()
        for k in ("xyz", "vprev", "comp"):
            assert np.array_equal(before[k], after[k]), k
        assert res["best"] in cfgs and len(res["trials"]) == 6
        assert m.info()["voxel"] == pytest.approx(res["best"]["voxel"])
        x = m.positions()
        m.step(1)
        v = m.velocities()
    vref = oracle.velocities(x, pop.R, pop.ccr, pop.cca, pop.A, pop.lo, pop.h, H.dims_of(pop))
    assert H.rel_err(v, vref) <= H.TOL_V_MIXED


def candidates_from_bins(m):
    """Ordered candidate pairs of the 27-voxel stencil, from the binning itself."""
    key, count, _, _ = m.bins()
    _, dims, _ = m.grid(0)
    dims = dims.astype(np.int64)
    k = key.astype(np.int64)
    ix, iy, iz = k % dims[0], (k // dims[0]) % dims[1], k // (dims[0] * dims[1])
    total = 0
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                jx, jy, jz = ix + dx, iy + dy, iz + dz
                ok = (jx >= 0) & (jx < dims[0]) & (jy >= 0) & (jy < dims[1]) & (jz >= 0) & (jz < dims[2])
                vk = jx[ok] + dims[0] * (jy[ok] + dims[1] * jz[ok])
                total += int(count[vk].astype(np.int64).sum())
    return total - key.size


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("name,voxel", [("spheroid_2k", None), ("clustered_small", "min")])
def test_pair_stats_match_oracle(name, voxel, mode):
    """Interacting pairs are the oracle's pair set (bit-exact count, FP64
    decision); candidates are the 27-voxel stencil of the binning."""
    pop = synth.spheroid_2k(seed=21) if name == "spheroid_2k" else synth.clustered_20m(seed=22, scale=0.002)
    hv = 2 * pop.A * pop.R.max() * (1 + 1e-5) if voxel == "min" else None
    with H.make(pop, mode, voxel=hv) as m:
        m.step(3)
        cand, pairs = m.pair_stats()
        x = m.positions()
        assert cand == candidates_from_bins(m)
    pref = oracle.pairs(x, pop.R, pop.A, pop.lo, pop.h, H.dims_of(pop))
    assert pairs == pref.shape[0]
    assert pairs > 0 and cand > 2 * pairs


@pytest.mark.parametrize("kernel", DENSE_KERNELS)
@pytest.mark.parametrize("tile", [(4, 4, 4), (4, 4, 8), (8, 4, 4)])
def test_runs_are_bitwise_reproducible(tile, kernel):
    """The slot order the scatter takes from atomics never reaches the result:
    two handles advanced the same way end bitwise equal (dense tiles, sparse
    cells and hand-back paths all active)."""
    pop = synth.clustered_20m(seed=23, scale=0.002)
    hmin = 2 * pop.A * pop.R.max() * (1 + 1e-5)
    xs = []
    for _ in range(2):
        with H.make(pop, "kahan", voxel=hmin) as m:
            m.set_dense_kernel(kernel)
            m.set_tiling(tile, 16)
            m.step(12)
            xs.append(m.read_state())
    for k in ("xyz", "vprev", "comp"):
        assert np.array_equal(xs[0][k], xs[1][k]), k


def test_pair_stats_of_a_batch_sum_over_replicates():
    """Neighbour statistics of a batched handle are the sums of its replicates'
    statistics, and the pairs are the oracle's pairs replicate by replicate."""
    from paper_2306_11544_gb300 import mech
    ens = synth.ensemble_256(seed=24, scale=0.02, n_rep=5)
    with mech.Mech.from_ensemble(ens, mode="mixed") as b:
        b.step(2)
        cand_b, pairs_b = b.pair_stats()
        xb = b.positions()
    cand, pairs, pref, off = 0, 0, 0, 0
    for p in ens.reps:
        x = xb[off:off + p.n]
        off += p.n
        with H.make(p, "mixed") as m:
            m.load_state({"xyz": x, "vprev": np.zeros_like(x), "step": 0})
            c, q = m.pair_stats()
        cand += c
        pairs += q
        pref += oracle.pairs(x, p.R, p.A, p.lo, p.h, H.dims_of(p)).shape[0]
    assert (cand_b, pairs_b) == (cand, pairs)
    assert pairs_b == pref
