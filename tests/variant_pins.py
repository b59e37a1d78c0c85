"""Pins of the velocity-variant oracle (per-type adhesion affinity, domain
walls): checks against what the statement fixes without the oracle's code,
each a function of an oracle library object `o`, so that planted mistakes in
copies of the oracle can be run against them too.

* Reduction: an affinity matrix of ones and no walls is the base law, bit for
  bit (the same operations in the same order).
* Brute force: the binned velocities equal an all-pairs sum with the same
  variants (types, a non-trivial affinity matrix, walls on some faces, cells
  overlapping and outside the walls).
* Two cells of types a, b: the scalar force written out here,
  f(d) = Cr (1 - d/S)^2 [d < S] - a_ab Ca (1 - d/(A S))^2, and its zero at
  d* = S (sqrt Cr - sqrt(a_ab Ca)) / (sqrt Cr - sqrt(a_ab Ca) / A); a zero
  affinity leaves no force between S and A S; both orders of the types give
  the same force (symmetric matrix).
* Walls: one cell at inward distance d_w from a face gets c_w (1 - d_w/R)^2
  along the inward normal for 0 < d_w < R, c_w at or beyond the face, nothing
  from R on; value and slope continuous at d_w = R; a corner cell gets the sum
  of its two faces; a disabled face gives nothing; mirrored faces give
  mirrored velocities.
* Integration: a cell leaving a wall follows the scalar two-step recursion
  s_{n+1} = s_n + dt (1.5 g(s_n) - 0.5 g(s_{n-1})), g(s) = c_w (1 - s/R)^2.
"""
import math

import numpy as np

A = 1.25
R0, CR0, CA0 = 8.41, 10.0, 0.4
AFF = np.array([[1.0, 0.3, 2.0],
                [0.3, 0.0, 1.5],
                [2.0, 1.5, 0.7]])


def scalar_force(d, S, Cr, Ca, a):
    """The variant's pair force along the line of centres, written out here."""
    if not (0.0 < d < A * S):
        return 0.0
    rep = Cr * (1.0 - d / S) ** 2 if d < S else 0.0
    return rep - a * Ca * (1.0 - d / (A * S)) ** 2


def two_cells(d, direction=(1.0, 0.0, 0.0), center=(2.0, -1.0, 3.0)):
    e = np.asarray(direction, float)
    e = e / np.linalg.norm(e)
    c = np.asarray(center, float)
    return np.stack([c + 0.5 * d * e, c - 0.5 * d * e]), e


def population(seed, n=400, walls=True):
    rng = np.random.Generator(np.random.PCG64(seed))
    xyz = rng.uniform(-62.0, 62.0, size=(n, 3))
    R = rng.uniform(6.0, 11.0, size=n)
    ccr = rng.uniform(5.0, 15.0, size=n)
    cca = rng.uniform(0.1, 0.8, size=n)
    types = rng.integers(0, 3, size=n).astype(np.int32)
    h = 2.0 * A * R.max() + 0.1
    lo = np.full(3, -65.0)
    dims = np.ceil(130.0 / h).astype(int) * np.ones(3, int)
    w = ((np.array([-55.0, -58.0, -60.0]), np.array([57.0, 55.0, 60.0]), 0b101011, 6.0) if walls else None)
    return xyz, R, ccr, cca, types, lo, h, dims, w


def pin_reduces_to_base(o):
    xyz, R, ccr, cca, types, lo, h, dims, _ = population(1, walls=False)
    ones = np.ones((3, 3))
    v_base = o.velocities(xyz, R, ccr, cca, A, lo, h, dims)
    v_ext = o.velocities_ext(xyz, R, ccr, cca, A, lo, h, dims, types, ones, None)
    assert np.array_equal(v_base, v_ext)
    x1, vp1, _ = o.run(xyz, R, ccr, cca, A, lo, h, dims, 0.1, 3)
    x2, vp2, _ = o.run_ext(xyz, R, ccr, cca, A, lo, h, dims, 0.1, 3, types, ones, None)
    assert np.array_equal(x1, x2) and np.array_equal(vp1, vp2)


def pin_binned_equals_allpairs(o):
    for seed in (2, 3):
        xyz, R, ccr, cca, types, lo, h, dims, w = population(seed)
        v_bin = o.velocities_ext(xyz, R, ccr, cca, A, lo, h, dims, types, AFF, w)
        v_all = o.velocities_allpairs_ext(xyz, R, ccr, cca, A, types, AFF, w)
        scale = np.abs(v_all).max()
        assert scale > 0
        assert np.abs(v_bin - v_all).max() <= 1e-12 * scale
        # the walls act: cells beyond a face are pushed back inward
        wlo, whi, mask, cw = w
        out = xyz[:, 0] < wlo[0] - 1.0
        assert out.any()


def pin_two_cell_types(o):
    S = 2 * R0
    lo = np.full(3, -60.0)
    dims = np.array([4, 4, 4])
    for ta in range(3):
        for tb in range(3):
            a = AFF[ta, tb]
            types = np.array([ta, tb], np.int32)
            for d in (9.0, 14.5, 16.3, 18.0, 20.5, 21.5):
                for e in ((1.0, 0.0, 0.0), (0.3, -0.4, 0.866)):
                    xyz, u = two_cells(d, e)
                    v = o.velocities_ext(xyz, [R0, R0], [CR0, CR0], [CA0, CA0], A, lo, 30.0, dims, types, AFF)
                    f = float(v[0] @ u)
                    ref = scalar_force(d, S, CR0, CA0, a)
                    assert abs(f - ref) <= 1e-13 * max(1.0, abs(ref)), (ta, tb, d, f, ref)
                    assert np.array_equal(v[0], -v[1])
                    # swapped types: the same force
                    v2 = o.velocities_ext(xyz, [R0, R0], [CR0, CR0], [CA0, CA0], A, lo, 30.0, dims, types[::-1],
                                          AFF)
                    assert np.array_equal(v2, v)
            if a > 0:
                dstar = S * (math.sqrt(CR0) - math.sqrt(a * CA0)) / (math.sqrt(CR0) - math.sqrt(a * CA0) / A)
                xyz, u = two_cells(dstar)
                v = o.velocities_ext(xyz, [R0, R0], [CR0, CR0], [CA0, CA0], A, lo, 30.0, dims, types, AFF)
                assert abs(float(v[0] @ u)) < 1e-12
            else:
                for d in (S + 0.01, 0.5 * (S + A * S), A * S - 0.01):
                    xyz, u = two_cells(d)
                    v = o.velocities_ext(xyz, [R0, R0], [CR0, CR0], [CA0, CA0], A, lo, 30.0, dims, types, AFF)
                    assert np.all(v == 0.0)


def pin_zero_net_without_walls(o):
    xyz, R, ccr, cca, types, lo, h, dims, _ = population(4, n=900, walls=False)
    v = o.velocities_ext(xyz, R, ccr, cca, A, lo, h, dims, types, AFF, None)
    assert np.abs(v).sum() > 10.0
    assert np.abs(v.sum(axis=0)).max() <= 1e-12 * np.abs(v).sum()


def _one_cell(o, x, walls, R=R0):
    lo = np.full(3, -60.0)
    return o.velocities_ext(np.asarray(x, float).reshape(1, 3), [R], [CR0], [CA0], A, lo, 30.0,
                            np.array([4, 4, 4]), None, None, walls)[0]


def pin_walls(o):
    wlo, whi, cw = np.array([-50.0, -40.0, -30.0]), np.array([45.0, 35.0, 25.0]), 3.0
    allf = (wlo, whi, 0b111111, cw)
    mid = 0.5 * (wlo + whi)
    for f in range(6):
        axis, high = f // 2, f % 2
        n = np.zeros(3)
        n[axis] = -1.0 if high else 1.0
        for dw in (-3.0, 0.0, 0.5, 4.0, 8.0, R0 - 1e-3, R0, R0 + 0.5):
            x = mid.copy()
            x[axis] = whi[axis] - dw if high else wlo[axis] + dw
            v = _one_cell(o, x, allf)
            t = 1.0 if dw <= 0 else max(0.0, 1.0 - dw / R0)
            ref = cw * t * t * n if dw < R0 else np.zeros(3)
            assert np.abs(v - ref).max() <= 1e-13, (f, dw, v, ref)
            # only this face enabled: the same; its mirror face disabled: nothing
            assert np.array_equal(_one_cell(o, x, (wlo, whi, 1 << f, cw)), v)
            assert np.all(_one_cell(o, x, (wlo, whi, 0b111111 & ~(1 << f), cw)) == 0.0)
    # value and slope continuous at d_w = R
    eps = 1e-5
    def fx(dw):
        x = mid.copy()
        x[0] = wlo[0] + dw
        return float(_one_cell(o, x, allf)[0])
    assert abs(2 * fx(R0 - eps) - fx(R0 - 2 * eps)) < 1e-8
    assert abs((fx(R0 - eps) - fx(R0 - 2 * eps)) / eps) < 1e-4
    # a corner cell: the sum of its two faces
    x = np.array([wlo[0] + 2.0, whi[1] - 5.0, mid[2]])
    v = _one_cell(o, x, allf)
    ref = np.array([cw * (1 - 2.0 / R0) ** 2, -cw * (1 - 5.0 / R0) ** 2, 0.0])
    assert np.abs(v - ref).max() <= 1e-13
    # mirrored faces give mirrored velocities (symmetric box)
    sym = (np.full(3, -40.0), np.full(3, 40.0), 0b111111, cw)
    a = _one_cell(o, [-36.5, 2.0, 1.0], sym)
    b = _one_cell(o, [36.5, 2.0, 1.0], sym)
    assert a[0] > 0 and a[0] == -b[0] and a[1] == b[1] == 0.0
    # a wall and a neighbour superpose
    xyz = np.array([[wlo[0] + 3.0, 0.0, 0.0], [wlo[0] + 3.0 + 15.0, 0.0, 0.0]])
    v = o.velocities_ext(xyz, [R0, R0], [CR0, CR0], [CA0, CA0], A, np.full(3, -60.0), 30.0, np.array([4, 4, 4]),
                         None, None, (wlo, whi, 1, cw))
    assert abs(v[0, 0] - (cw * (1 - 3.0 / R0) ** 2 - scalar_force(15.0, 2 * R0, CR0, CA0, 1.0))) <= 1e-13
    assert abs(v[1, 0] - scalar_force(15.0, 2 * R0, CR0, CA0, 1.0)) <= 1e-13


def pin_wall_recursion(o):
    wlo, whi, cw, dt = np.full(3, -50.0), np.full(3, 50.0), 4.0, 0.1
    for s0, steps in ((1.0, 40), (-2.0, 25), (7.9, 10)):
        x0 = np.array([[wlo[0] + s0, 0.0, 0.0]])
        x, _, _ = o.run_ext(x0, [R0], [CR0], [CA0], A, np.full(3, -60.0), 30.0, np.array([4, 4, 4]), dt, steps,
                            None, None, (wlo, whi, 0b000001, cw))
        s, g_prev = s0, 0.0
        for _ in range(steps):
            t = 1.0 if s <= 0 else (1.0 - s / R0 if s < R0 else 0.0)
            g = cw * t * t
            s, g_prev = s + dt * (1.5 * g - 0.5 * g_prev), g
        got = x[0, 0] - wlo[0]
        assert abs(got - s) <= 1e-13 * max(1.0, abs(s)), (s0, got, s)


ALL_VARIANT_PINS = [pin_reduces_to_base, pin_binned_equals_allpairs, pin_two_cell_types,
                    pin_zero_net_without_walls, pin_walls, pin_wall_recursion]
