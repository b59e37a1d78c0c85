"""Pins for the oracle: checks against facts fixed by the mathematics, not by
the oracle's own code.

Each ``pin_*`` takes an ``oracle.OracleLib`` and raises AssertionError when the
oracle it is given is wrong.  ``test_oracle_pins.py`` runs them on the real
oracle; ``test_oracle_mutants.py`` runs them on copies of the oracle with a
planted mistake and checks that every mistake is caught by at least one pin.

What pins what:
  * voxel keys      -> exact rational floor of (x - lo)/h away from faces; faces
                       on a dyadic grid go to the higher voxel; clamping.
  * counting sort   -> numpy's stable argsort, bincount and cumsum.
  * neighbour set   -> O(n^2) all-pairs search (exact set equality).
  * binned velocity -> all-pairs velocity (same terms, other order).
  * force law       -> analytic equilibrium distance of two cells, the value at
                       d = S where the repulsion vanishes, the d -> 0 limit,
                       continuity of value and slope at both cutoffs.
  * geometry        -> zero net velocity, translation by whole voxels (bitwise
                       on a dyadic grid), 90-degree rotations, the equilibrium
                       of a simple cubic lattice at the two-cell equilibrium
                       spacing.
  * FP32 keys       -> the same faces on a dyadic grid decided in FP32 (every
                       operation exact there, so a cell on a face goes to the
                       higher voxel in FP32 too).
  * subset velocity -> its rows equal the full binned velocity's rows of the
                       listed cells (any order, repeats, empty list).
  * force law       -> the scalar force of two like cells evaluated by hand
                       at d = 10, 18, 20 um with the 2,000-cell spheroid's
                       parameters (R 8.41, ccr 10, cca 0.4, A 1.25):
                       1.534069, -0.0082802, -0.00095068 um/min.
  * integrator      -> the linear contraction rate of two cells relaxing to
                       equilibrium equals the dominant root of the AB2
                       characteristic polynomial built from the analytic
                       slope of the force at equilibrium; the separation of
                       two cells follows the scalar two-step recursion
                       s_{n+1} = s_n + dt (3 f(s_n) - f(s_{n-1})), f(s_{-1}) = 0,
                       with f written out here from the force law.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

A_CFG = 1.25
R_CFG, CCR_CFG, CCA_CFG = 8.41, 10.0, 0.4


def equilibrium_distance(S, Cr, Ca, A):
    """Root of Cr (1 - d/S)^2 = Ca (1 - d/(A S)) ^2 with d < S: taking square
    roots of both sides gives a linear equation in d."""
    return S * (math.sqrt(Cr) - math.sqrt(Ca)) / (math.sqrt(Cr) - math.sqrt(Ca) / A)


def force_slope(d, S, Cr, Ca, A):
    """Analytic derivative of the scalar pair force for d < S."""
    return -2.0 * Cr * (1.0 - d / S) / S + 2.0 * Ca * (1.0 - d / (A * S)) / (A * S)


def _two_cells(d, direction=(1.0, 0.0, 0.0), Ri=R_CFG, Rj=R_CFG, ccr=(CCR_CFG, CCR_CFG),
               cca=(CCA_CFG, CCA_CFG), center=(3.0, -2.0, 1.0)):
    e = np.asarray(direction, dtype=np.float64)
    e = e / np.linalg.norm(e)
    c = np.asarray(center, dtype=np.float64)
    xyz = np.stack([c + 0.5 * d * e, c - 0.5 * d * e])
    return xyz, np.array([Ri, Rj]), np.array(ccr, float), np.array(cca, float), e


def _scalar_force(o, d, **kw):
    """Velocity of cell 0 projected on the unit vector from cell 1 to cell 0."""
    xyz, R, ccr, cca, _ = _two_cells(d, **kw)
    v = o.velocities_allpairs(xyz, R, ccr, cca, A_CFG)
    u = (xyz[0] - xyz[1]) / np.linalg.norm(xyz[0] - xyz[1])
    return float(v[0] @ u), v, u


# ---------------------------------------------------------------- binning ---

def pin_keys(o):
    rng = np.random.Generator(np.random.PCG64(11))
    lo = np.array([-100.0, -40.0, 7.0])
    h = 30.0
    dims = np.array([7, 5, 4], np.int32)
    xyz = rng.uniform(lo - 20.0, lo + dims * h + 20.0, size=(400, 3))
    k = o.keys(xyz, lo, h, dims).astype(np.int64)
    ix, iy, iz = k % dims[0], (k // dims[0]) % dims[1], k // (dims[0] * dims[1])
    got = np.stack([ix, iy, iz], axis=1)
    for i in range(xyz.shape[0]):
        for d in range(3):
            q = (Fraction(xyz[i, d]) - Fraction(lo[d])) / Fraction(h)
            exact = math.floor(q)
            clamped = min(max(exact, 0), dims[d] - 1)
            dist = abs(q - round(q))
            if dist > Fraction(1, 10**9):
                assert got[i, d] == clamped, (i, d, got[i, d], clamped)
            else:
                assert abs(got[i, d] - clamped) <= 1
    # faces on a dyadic grid are exact: a cell on a face belongs to the higher voxel
    h2 = 0.5
    lo2 = np.zeros(3)
    dims2 = np.array([4, 4, 4], np.int32)
    faces = np.array([[0.5, 1.0, 1.5], [0.0, 0.0, 0.0], [1.5, 0.5, 1.0], [1.999, 0.49, 0.25]])
    k2 = o.keys(faces, lo2, h2, dims2).astype(np.int64)
    expect = [(1, 2, 3), (0, 0, 0), (3, 1, 2), (3, 0, 0)]
    for kk, (ex, ey, ez) in zip(k2, expect):
        assert kk == ex + 4 * (ey + 4 * ez), (kk, ex, ey, ez)
    # clamping: far outside on either side lands in the edge voxels
    far = np.array([[-1e6, 1e6, 0.1], [1e9, -1e9, 1.9]])
    k3 = o.keys(far, lo2, h2, dims2).astype(np.int64)
    assert list(k3) == [0 + 4 * (3 + 4 * 0), 3 + 4 * (0 + 4 * 3)]


def pin_keys_f32(o):
    rng = np.random.Generator(np.random.PCG64(12))
    lo = np.array([-500.0, -500.0, -500.0])
    h = 30.0
    dims = np.array([34, 34, 34], np.int32)
    xyz = rng.uniform(-520.0, 540.0, size=(2000, 3))
    t = (xyz - lo) / h
    away = np.all(np.abs(t - np.round(t)) > 1e-4, axis=1)
    k64 = o.keys(xyz[away], lo, h, dims)
    k32 = o.keys_f32(xyz[away].astype(np.float32), lo, h, dims)
    assert np.array_equal(k64, k32)


def pin_keys_f32_faces(o):
    """FP32 decision at exact faces: with lo and h powers of two (times small
    integers) every FP32 operation of the index is exact, so a coordinate on
    a face lands in the higher voxel, as the FP64 rule does."""
    h = 0.5
    lo = np.array([-2.0, 0.0, 4.0])
    dims = np.array([16, 8, 6], np.int32)
    pts = np.array([[-2.0, 0.0, 4.0], [-1.5, 0.5, 4.5], [0.0, 3.5, 6.5], [5.5, 0.25, 5.0],
                    [-1.75, 3.75, 6.75], [1.0, 1.0, 5.5]], np.float32)
    expect = [(0, 0, 0), (1, 1, 1), (4, 7, 5), (15, 0, 2), (0, 7, 5), (6, 2, 3)]
    k32 = o.keys_f32(pts, lo, h, dims).astype(np.int64)
    k64 = o.keys(pts.astype(np.float64), lo, h, dims).astype(np.int64)
    for kk, kd, (ex, ey, ez) in zip(k32, k64, expect):
        want = ex + int(dims[0]) * (ey + int(dims[1]) * ez)
        assert kk == want, (kk, want)
        assert kd == want, (kd, want)
    # one FP32 ulp below a face stays in the lower voxel (lo = 0, so the
    # subtraction cannot round it up onto the face)
    below = np.nextafter(np.float32(1.5), np.float32(0.0))
    kb = o.keys_f32(np.array([[below, 0.75, 1.25]], np.float32), np.zeros(3), h, dims)
    assert int(kb[0]) == 2 + int(dims[0]) * (1 + int(dims[1]) * 2), int(kb[0])


def pin_counting_sort(o):
    rng = np.random.Generator(np.random.PCG64(13))
    for n, V in [(0, 5), (1, 1), (1000, 37), (5000, 4000)]:
        key = rng.integers(0, V, size=n).astype(np.uint32)
        if n == 1000:
            key[:300] = 3  # a crowded bin
        count, start, order = o.counting_sort(key, V)
        assert np.array_equal(count, np.bincount(key, minlength=V))
        assert np.array_equal(start, np.concatenate([[0], np.cumsum(count)]).astype(np.uint32))
        assert np.array_equal(order, np.argsort(key, kind="stable"))


def _pin_populations():
    """Tiny populations covering dense clusters, cells outside the domain, a
    single crowded voxel, cells on voxel faces and heterogeneous radii."""
    rng = np.random.Generator(np.random.PCG64(14))
    pops = []
    n = 300
    xyz = rng.uniform(-50.0, 50.0, size=(n, 3))
    pops.append((xyz, np.full(n, R_CFG), np.full(n, CCR_CFG), np.full(n, CCA_CFG), np.full(3, -60.0), 30.0, np.array([4, 4, 4])))
    n = 200
    xyz = rng.uniform(-100.0, 100.0, size=(n, 3))
    pops.append((xyz, np.full(n, R_CFG), np.full(n, CCR_CFG), np.full(n, CCA_CFG), np.full(3, -45.0), 30.0, np.array([3, 3, 3])))
    n = 80
    xyz = rng.uniform(1.0, 26.0, size=(n, 3))
    pops.append((xyz, np.full(n, R_CFG), np.full(n, CCR_CFG), np.full(n, CCA_CFG), np.zeros(3), 30.0, np.array([3, 3, 3])))
    g = np.arange(0.0, 121.0, 30.0)
    face = np.array([[a, b, c] for a in g for b in g for c in (0.0, 15.0, 30.0)])
    face = face + rng.choice([0.0, 1e-9, -1e-9, 8.0, -8.0], size=face.shape)
    n = face.shape[0]
    pops.append((face, np.full(n, R_CFG), np.full(n, CCR_CFG), np.full(n, CCA_CFG), np.zeros(3), 30.0, np.array([5, 5, 3])))
    n = 400
    xyz = rng.uniform(-60.0, 60.0, size=(n, 3))
    R = rng.uniform(6.0, 11.0, size=n)
    ccr = rng.uniform(5.0, 15.0, size=n)
    cca = rng.uniform(0.1, 0.8, size=n)
    h = 2.0 * A_CFG * R.max() + 0.1
    dims = np.ceil(120.0 / h).astype(int) * np.ones(3, int)
    pops.append((xyz, R, ccr, cca, np.full(3, -60.0), h, dims))
    return pops


def pin_neighbour_set(o):
    for xyz, R, ccr, cca, lo, h, dims in _pin_populations():
        p_bin = o.pairs(xyz, R, A_CFG, lo, h, dims)
        p_all = o.pairs_allpairs(xyz, R, A_CFG)
        a = set(map(tuple, p_bin.tolist()))
        b = set(map(tuple, p_all.tolist()))
        assert len(a) == p_bin.shape[0]
        assert a == b, (len(a), len(b))
        assert len(b) > 0


def pin_velocities_subset(o):
    """Rows of the subset routine are the full routine's rows of the listed
    cells, for an unsorted list with repeats, and for an empty list."""
    xyz, R, ccr, cca, lo, h, dims = _pin_populations()[4]
    full = o.velocities(xyz, R, ccr, cca, A_CFG, lo, h, dims)
    rng = np.random.Generator(np.random.PCG64(19))
    idx = rng.integers(0, xyz.shape[0], size=57)
    idx[3] = idx[10]
    idx[-1] = xyz.shape[0] - 1
    sub = o.velocities_subset(xyz, R, ccr, cca, A_CFG, lo, h, dims, idx)
    assert sub.shape == (idx.size, 3)
    assert np.array_equal(sub, full[idx])
    empty = o.velocities_subset(xyz, R, ccr, cca, A_CFG, lo, h, dims, np.zeros(0, np.int64))
    assert empty.shape == (0, 3)


def pin_binned_velocity(o):
    for xyz, R, ccr, cca, lo, h, dims in _pin_populations():
        v_bin = o.velocities(xyz, R, ccr, cca, A_CFG, lo, h, dims)
        v_all = o.velocities_allpairs(xyz, R, ccr, cca, A_CFG)
        scale = np.abs(v_all).max()
        assert scale > 0
        assert np.abs(v_bin - v_all).max() <= 1e-12 * scale


# -------------------------------------------------------------- force law ---

def pin_two_cell(o):
    S = 2 * R_CFG
    AS = A_CFG * S
    ds = equilibrium_distance(S, CCR_CFG, CCA_CFG, A_CFG)
    assert abs(ds - S * 20.0 / 21.0) < 1e-12  # sqrt(cca/ccr) = 1/5 makes it S*20/21
    rng = np.random.Generator(np.random.PCG64(15))
    for _ in range(4):
        e = rng.standard_normal(3)
        f, v, u = _scalar_force(o, ds, direction=e)
        assert abs(f) < 1e-12, f
        # pair terms are equal and opposite, along the line of centres
        assert np.array_equal(v[0], -v[1])
        f, v, u = _scalar_force(o, ds - 0.5, direction=e)
        assert f > 0.01  # repulsion pushes the cells apart
        assert np.linalg.norm(np.cross(v[0], u)) < 1e-12 * np.linalg.norm(v[0])
        f, v, u = _scalar_force(o, ds + 0.5, direction=e)
        assert f < -1e-3  # adhesion pulls them together
    # at d = S the repulsion term is zero and only adhesion is left
    f, _, _ = _scalar_force(o, S)
    assert abs(f - (-CCA_CFG * (1.0 - 1.0 / A_CFG) ** 2)) < 1e-13
    # d -> 0: both brackets tend to one
    f, _, _ = _scalar_force(o, 1e-7)
    assert abs(f - (CCR_CFG - CCA_CFG)) < 1e-6
    # no interaction at or beyond A*S; some just inside it
    for d in (AS, AS + 1e-9, AS + 3.0, 1e3):
        f, v, _ = _scalar_force(o, d)
        assert np.all(v == 0.0)
    f, _, _ = _scalar_force(o, AS - 1e-3)
    assert -1e-7 < f < 0.0
    # coincident cells are skipped (d = 0): no NaN, no force
    xyz = np.array([[1.0, 2.0, 3.0], [1.0, 2.0, 3.0]])
    v = o.velocities_allpairs(xyz, [R_CFG] * 2, [CCR_CFG] * 2, [CCA_CFG] * 2, A_CFG)
    assert np.all(v == 0.0)
    # unlike cells: S = Ri + Rj, coefficients are geometric means
    Ri, Rj, ccr, cca = 6.0, 11.0, (8.0, 12.0), (0.2, 0.6)
    Cr, Ca = math.sqrt(ccr[0] * ccr[1]), math.sqrt(cca[0] * cca[1])
    S2 = Ri + Rj
    d2 = equilibrium_distance(S2, Cr, Ca, A_CFG)
    f, v, _ = _scalar_force(o, d2, Ri=Ri, Rj=Rj, ccr=ccr, cca=cca)
    assert abs(f) < 1e-12
    assert np.array_equal(v[0], -v[1])
    f, _, _ = _scalar_force(o, S2, Ri=Ri, Rj=Rj, ccr=ccr, cca=cca)
    assert abs(f - (-Ca * (1.0 - 1.0 / A_CFG) ** 2)) < 1e-13


# f(d) of two like cells with R 8.41 um, ccr 10, cca 0.4 (um/min), A 1.25,
# evaluated by hand from the force law: S = 16.82, A S = 21.025;
# f(10) = 10 (1 - 10/16.82)^2 - 0.4 (1 - 10/21.025)^2, f(18) and f(20) have
# d > S, so only the adhesion bracket is left.
TWO_CELL_VALUES = [(10.0, 1.534069, 5e-7), (18.0, -0.0082802, 5e-8), (20.0, -0.00095068, 5e-9)]


def pin_two_cell_values(o):
    for d, f_ref, tol in TWO_CELL_VALUES:
        for e in ((1.0, 0.0, 0.0), (0.0, -1.0, 0.0), (0.48, 0.6, -0.64)):
            f, v, _ = _scalar_force(o, d, direction=e)
            assert abs(f - f_ref) <= tol, (d, f, f_ref)
            assert np.array_equal(v[0], -v[1])


def pin_c1_at_cutoffs(o):
    S = 2 * R_CFG
    AS = A_CFG * S
    eps = 1e-5
    for c in (S, AS):
        fl, _, _ = _scalar_force(o, c - eps)
        fr, _, _ = _scalar_force(o, c + eps)
        fll, _, _ = _scalar_force(o, c - 2 * eps)
        frr, _, _ = _scalar_force(o, c + 2 * eps)
        # value at the cutoff extrapolated linearly from each side
        assert abs((2 * fl - fll) - (2 * fr - frr)) < 1e-8, (c, fl, fr)  # continuous
        sl = (fl - fll) / eps
        sr = (frr - fr) / eps
        assert abs(sl - sr) < 1e-4, (c, sl, sr)  # slope continuous


# --------------------------------------------------------------- geometry ---

def pin_zero_net_velocity(o):
    rng = np.random.Generator(np.random.PCG64(16))
    n = 1500
    xyz = rng.uniform(-70.0, 70.0, size=(n, 3))
    R = rng.uniform(6.0, 11.0, size=n)
    ccr = rng.uniform(5.0, 15.0, size=n)
    cca = rng.uniform(0.1, 0.8, size=n)
    v = o.velocities(xyz, R, ccr, cca, A_CFG, np.full(3, -90.0), 30.0, np.array([6, 6, 6]))
    assert np.abs(v).sum() > 10.0
    assert np.abs(v.sum(axis=0)).max() <= 1e-12 * np.abs(v).sum()


def pin_translation(o):
    rng = np.random.Generator(np.random.PCG64(17))
    n = 800
    h = 32.0  # a power of two: every coordinate below stays exact under the shift
    xyz = np.round(rng.uniform(-90.0, 90.0, size=(n, 3)) * 2**20) / 2**20
    R, ccr, cca = np.full(n, R_CFG), np.full(n, CCR_CFG), np.full(n, CCA_CFG)
    lo = np.full(3, -96.0)
    dims = np.array([6, 6, 6])
    v0 = o.velocities(xyz, R, ccr, cca, A_CFG, lo, h, dims)
    k0 = o.keys(xyz, lo, h, dims)
    shift = np.array([3.0, -5.0, 7.0]) * h
    v1 = o.velocities(xyz + shift, R, ccr, cca, A_CFG, lo + shift, h, dims)
    k1 = o.keys(xyz + shift, lo + shift, h, dims)
    assert np.array_equal(k0, k1)
    assert np.array_equal(v0, v1)
    # a general shift on a non-dyadic voxel keeps the result to rounding level
    h3 = 30.0
    dims3 = np.array([7, 7, 7])
    lo3 = np.full(3, -105.0)
    v2 = o.velocities(xyz, R, ccr, cca, A_CFG, lo3, h3, dims3)
    s3 = np.array([4.0, 1.0, -2.0]) * h3
    v3 = o.velocities(xyz + s3, R, ccr, cca, A_CFG, lo3 + s3, h3, dims3)
    assert np.abs(v2 - v3).max() <= 1e-10 * np.abs(v2).max()


def pin_rotation(o):
    rng = np.random.Generator(np.random.PCG64(18))
    n = 700
    xyz = rng.uniform(-80.0, 80.0, size=(n, 3))
    R = rng.uniform(6.0, 11.0, size=n)
    ccr = rng.uniform(5.0, 15.0, size=n)
    cca = rng.uniform(0.1, 0.8, size=n)
    lo = np.full(3, -90.0)
    dims = np.array([6, 6, 6])
    v = o.velocities(xyz, R, ccr, cca, A_CFG, lo, 30.0, dims)
    scale = np.abs(v).max()
    rots = [np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]], float),
            np.array([[1, 0, 0], [0, 0, -1], [0, 1, 0]], float),
            np.array([[0, 0, 1], [0, 1, 0], [-1, 0, 0]], float)]
    for Q in rots:
        vr = o.velocities(xyz @ Q.T, R, ccr, cca, A_CFG, lo, 30.0, dims)
        assert np.abs(vr - v @ Q.T).max() <= 1e-12 * scale


def pin_lattice(o):
    S = 2 * R_CFG
    ds = equilibrium_distance(S, CCR_CFG, CCA_CFG, A_CFG)
    assert ds * math.sqrt(2.0) > A_CFG * S  # diagonals do not interact
    g = np.arange(6) * ds
    xyz = np.array([[a, b, c] for a in g for b in g for c in g]) - 2.5 * ds
    n = xyz.shape[0]
    R, ccr, cca = np.full(n, R_CFG), np.full(n, CCR_CFG), np.full(n, CCA_CFG)
    v = o.velocities(xyz, R, ccr, cca, A_CFG, np.full(3, -60.0), 30.0, np.array([4, 4, 4]))
    assert np.abs(v).max() < 1e-12
    # a stretched lattice is cohesive: the corner cell is pulled towards the centre
    v2 = o.velocities(xyz * 1.02, R, ccr, cca, A_CFG, np.full(3, -60.0), 30.0, np.array([4, 4, 4]))
    corner = int(np.argmax(np.linalg.norm(xyz, axis=1)))
    assert float(v2[corner] @ xyz[corner]) < 0.0


# ------------------------------------------------------------- integrator ---

def pin_ab2_relaxation_rate(o):
    S = 2 * R_CFG
    ds = equilibrium_distance(S, CCR_CFG, CCA_CFG, A_CFG)
    dt = 0.1
    mu = 2.0 * force_slope(ds, S, CCR_CFG, CCA_CFG, A_CFG)  # d(separation)/dt = 2 f(separation)
    b = 1.0 + 1.5 * mu * dt
    lam = 0.5 * (b + math.sqrt(b * b - 4.0 * 0.5 * mu * dt))  # dominant root of x^2 - b x + mu dt/2
    xyz, R, ccr, cca, e = _two_cells(ds - 2.0, direction=(0.3, -0.5, 0.8))
    lo = np.full(3, -60.0)
    dims = np.array([4, 4, 4])
    seps = []
    vprev = None
    x = xyz
    for _ in range(12):
        x, vprev, _ = o.run(x, R, ccr, cca, A_CFG, lo, 30.0, dims, dt, 100, vprev=vprev)
        seps.append(float(np.linalg.norm(x[0] - x[1])))
    err = np.array(seps) - ds
    assert np.all(err < 0.0)  # approached from the compressed side without overshoot
    assert abs(err[-1]) < 1e-3 * 2.0
    rate = (err[-1] / err[-2]) ** (1.0 / 100.0)
    assert abs(rate - lam) < 2e-6, (rate, lam)
    # the cell pair moved symmetrically: the midpoint never moves
    mid = 0.5 * (x[0] + x[1])
    assert np.abs(mid - 0.5 * (xyz[0] + xyz[1])).max() < 1e-12


def _f_scalar(s, S, Cr, Ca, A):
    """Scalar pair force of the force law, written out independently here."""
    if not (0.0 < s < A * S):
        return 0.0
    rep = Cr * (1.0 - s / S) ** 2 if s < S else 0.0
    return rep - Ca * (1.0 - s / (A * S)) ** 2


def pin_ab2_scalar_recursion(o):
    """Two like cells on the x axis, symmetric about the origin: each moves by
    dt (1.5 v_n - 0.5 v_{n-1}) with v = +-f(s) along the axis, so the
    separation obeys s_{n+1} = s_n + dt (3 f(s_n) - f(s_{n-1})), f(s_{-1}) = 0.
    Started from both sides of the equilibrium (and from beyond S); the
    oracle's separation must follow the recursion to rounding."""
    S = 2 * R_CFG
    dt = 0.1
    lo = np.full(3, -60.0)
    dims = np.array([4, 4, 4])
    for s0, steps in ((12.0, 60), (19.5, 60), (16.5, 25)):
        xyz = np.array([[0.5 * s0, 0.0, 0.0], [-0.5 * s0, 0.0, 0.0]])
        R, ccr, cca = np.full(2, R_CFG), np.full(2, CCR_CFG), np.full(2, CCA_CFG)
        x, _, _ = o.run(xyz, R, ccr, cca, A_CFG, lo, 30.0, dims, dt, steps)
        s, f_prev = s0, 0.0
        for _ in range(steps):
            f_now = _f_scalar(s, S, CCR_CFG, CCA_CFG, A_CFG)
            s, f_prev = s + dt * (3.0 * f_now - f_prev), f_now
        got = x[0, 0] - x[1, 0]
        assert abs(got - s) <= 1e-14 * s, (s0, got, s, got - s)
        assert np.all(x[:, 1:] == 0.0)
        assert abs(x[0, 0] + x[1, 0]) <= 1e-13


def pin_ab2_start(o):
    """First step of AB2 with v_{-1} = 0, second step with the stored v."""
    xyz, R, ccr, cca, e = _two_cells(14.0)
    lo = np.full(3, -60.0)
    dims = np.array([4, 4, 4])
    v0 = o.velocities_allpairs(xyz, R, ccr, cca, A_CFG)
    x1, vp1, vl = o.run(xyz, R, ccr, cca, A_CFG, lo, 30.0, dims, 0.1, 1)
    assert np.array_equal(vl, v0) and np.array_equal(vp1, v0)
    step1 = x1 - xyz
    assert np.allclose(step1, 0.15 * v0, rtol=1e-14, atol=1e-15)
    v1 = o.velocities_allpairs(x1, R, ccr, cca, A_CFG)
    x2, _, _ = o.run(x1, R, ccr, cca, A_CFG, lo, 30.0, dims, 0.1, 1, vprev=vp1)
    assert np.allclose(x2 - x1, 0.1 * (1.5 * v1 - 0.5 * v0), rtol=1e-14, atol=1e-15)


def pin_special_sizes(o):
    lo, dims = np.full(3, -60.0), np.array([4, 4, 4])
    v = o.velocities(np.zeros((0, 3)), [], [], [], A_CFG, lo, 30.0, dims)
    assert v.shape == (0, 3)
    v = o.velocities(np.array([[1.0, 2.0, 3.0]]), [R_CFG], [CCR_CFG], [CCA_CFG], A_CFG, lo, 30.0, dims)
    assert np.all(v == 0.0)


ALL_PINS = [pin_keys, pin_keys_f32, pin_keys_f32_faces, pin_counting_sort, pin_neighbour_set,
            pin_velocities_subset, pin_binned_velocity, pin_two_cell, pin_two_cell_values, pin_c1_at_cutoffs,
            pin_zero_net_velocity, pin_translation, pin_rotation, pin_lattice, pin_ab2_relaxation_rate,
            pin_ab2_scalar_recursion, pin_ab2_start, pin_special_sizes]
