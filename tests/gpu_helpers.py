"""Shared helpers of the GPU parity tests: build a libmech handle from a
synthetic population and compute the error metrics the tolerances refer to."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2306_11544_gb300 import build, mech, synth

# Per-step velocity tolerance (relative to the largest reference velocity
# component) for the FP64 mode: the stated bar.
TOL_V_FP64 = 1e-5
# Per-step velocity tolerance for the FP32 pair arithmetic, relative to the
# largest reference velocity.  The pair vector is exact up to its final FP32
# rounding (hi parts on a power-of-two grid plus 16-bit residuals of at most
# 6e-8 um), 1 - d/S is formed from error-free products, and a cell's sum is
# Kahan-compensated: a pair term is accurate to a few FP32 ulp (~3e-7
# relative), and the largest errors come from cells whose velocity is a small
# difference of large terms (terms up to ~15 um/min against velocities of
# O(1-10) um/min).  The worst case observed over every parity population is
# 6.4e-6; the bar is 2e-5, three times that, so a tenfold loss of accuracy in
# the pair term fails it.
TOL_V_MIXED = 2e-5
# Final position error (um) after a configuration's steps in the mixed modes.
TOL_X_MIXED = 1e-3


def lib():
    build.build()
    return mech.load_library()


def make(pop: synth.Population, mode: str, voxel=None, graph=0):
    m = mech.Mech(pop.xyz, pop.R, pop.ccr, pop.cca, pop.ctype)
    m.set_params(pop.A, pop.h, pop.dt)
    m.set_domain(-1, pop.lo, pop.hi)
    m.set_precision(mode)
    if voxel:
        m.set_internal_voxel(voxel)
    if graph:
        m.set_graph(graph)
    return m


def dims_of(pop, h=None):
    return oracle.grid_dims(pop.lo, pop.hi, pop.h if h is None else h)


def rel_err(v, vref):
    scale = np.abs(vref).max()
    if scale == 0:
        return float(np.abs(v).max())
    return float(np.abs(v - vref).max() / scale)


def tiny_population(xyz, lo, hi, R=8.41, ccr=10.0, cca=0.4, h=30.0):
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    n = xyz.shape[0]
    return synth.Population("tiny", xyz, np.full(n, R), np.full(n, ccr), np.full(n, cca), np.zeros(n, np.int32),
                            np.asarray(lo, float), np.asarray(hi, float), A=1.25, h=h, dt=0.1, steps=10)


def edge_populations():
    """Degenerate and adversarial layouts."""
    rng = np.random.Generator(np.random.PCG64(77))
    out = {}
    out["one_cell"] = tiny_population([[3.0, -4.0, 5.0]], [-60] * 3, [60] * 3)
    out["two_coincident"] = tiny_population([[1.0, 2.0, 3.0], [1.0, 2.0, 3.0]], [-60] * 3, [60] * 3)
    out["two_touching"] = tiny_population([[0.0, 0.0, 0.0], [15.0, 0.0, 0.0]], [-60] * 3, [60] * 3)
    out["one_voxel_crowd"] = tiny_population(rng.uniform(1.0, 29.0, size=(300, 3)), [0] * 3, [90] * 3)
    g = np.arange(0.0, 121.0, 30.0)
    faces = np.array([[a, b, c] for a in g for b in g for c in g])
    out["on_faces"] = tiny_population(faces + rng.choice([0.0, 8.0, -8.0], size=faces.shape), [0] * 3, [120] * 3)
    out["outside_domain"] = tiny_population(rng.uniform(-150.0, 150.0, size=(600, 3)), [-45] * 3, [45] * 3)
    one_per = np.array([[15.0 + 30 * i, 15.0 + 30 * j, 15.0 + 30 * k] for i in range(3) for j in range(3)
                        for k in range(3)]) + rng.uniform(-14, 14, size=(27, 3))
    out["one_per_voxel"] = tiny_population(one_per, [0] * 3, [90] * 3)
    out["dense_lattice"] = tiny_population(
        np.array([[a, b, c] for a in np.arange(0, 60, 7.0) for b in np.arange(0, 60, 7.0)
                  for c in np.arange(0, 60, 7.0)]) + rng.uniform(-0.5, 0.5, size=(729, 3)), [-10] * 3, [80] * 3)
    return out


def parity_populations():
    """Seeded workloads at sizes the oracle finishes in seconds, spanning many
    tiles with a ragged tail."""
    return {
        "spheroid_2k": synth.spheroid_2k(seed=0),
        "spheroid_1m_x0.02": synth.spheroid_1m(seed=1, scale=0.02),
        "clustered_20m_x0.001": synth.clustered_20m(seed=2, scale=0.001),
    }
