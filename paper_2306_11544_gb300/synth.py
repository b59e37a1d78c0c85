"""Seeded synthetic cell populations shaped like the paper's workloads.

The paper's own inputs (the PhysiCell ``heterogeneity`` sample, Sec. 3.2, and
the 12-day organoid run of Sec. 5.5) are not available, so every input is a
synthetic spheroid drawn here: cell centres uniform in a ball (rejection
sampling from the bounding cube), per-cell radius and repulsion/adhesion
coefficients, and a cubic domain centred at the origin.

This module holds no arithmetic of the mechanics step.  Both the CUDA library
tests and the oracle tests draw their inputs from it; nothing here depends on
either side.

Recipes (all lengths in um, times in min):

* ``spheroid_2k``  2,000 cells, ball radius 100, R = 8.41, ccr = 10,
  cca = 0.4, A = 1.25, voxel 30, domain [-500, 500]^3, dt = 0.1, 100 steps.
* ``spheroid_1m``  1,000,000 cells, ball radius 1100, three types with
  probabilities 0.6/0.3/0.1 (ccr 10/8/12, cca 0.4/0.2/0.6), radius lognormal
  with median 8.4 and log-sd 0.1 clipped to [6, 11], voxel 30, dt = 0.1,
  1,000 steps; domain side ceil(3 * 1100 / 30) * 30.
* ``clustered_20m``  16M cells uniform in a core ball of radius 2500 plus 4M
  uniform in the cube [-5000, 5000]^3, R = 8.41, ccr = 10, cca = 0.4,
  voxel 30, 200 steps.
* ``ensemble_256``  256 replicates, N_r log-uniform in [1e3, 2e5], ccr_r ~
  U[5, 15], cca_r ~ U[0.1, 0.8], R = 8.41, ball radius 8.41 (N_r/0.466)^(1/3)
  (the packing fraction of ``spheroid_1m``), 100 steps.
* ``ensemble_32_long``  32 replicates, N_r log-uniform in [5e5, 5e6], cell
  types and radii as ``spheroid_1m``, ball radius 8.4 (N_r/0.466)^(1/3),
  10,000 steps.

Every recipe takes a ``scale`` that shrinks the cell counts while keeping the
number density (lengths scale by scale^(1/3)), for test-sized cases.
Random streams: replicate r of an ensemble draws its cells from PCG64 seeded
with ``seed + r``; the per-replicate counts and coefficients come from a
separate PCG64 stream seeded with ``SeedSequence((seed, 1))``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PACKING = 0.466  # packing fraction of the 1M-cell spheroid (1M cells, radius 1.1 mm)


@dataclass
class Population:
    """One independent cell population (one replicate)."""

    name: str
    xyz: np.ndarray  # (n, 3) float64, um
    R: np.ndarray  # (n,) float64 radius, um
    ccr: np.ndarray  # (n,) float64 repulsion coefficient, um/min
    cca: np.ndarray  # (n,) float64 adhesion coefficient, um/min
    ctype: np.ndarray  # (n,) int32 cell type (carried, not used by the force)
    lo: np.ndarray  # (3,) domain lower corner
    hi: np.ndarray  # (3,) domain upper corner
    A: float = 1.25
    h: float = 30.0
    dt: float = 0.1
    steps: int = 100
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])


@dataclass
class Ensemble:
    name: str
    reps: list
    steps: int
    meta: dict = field(default_factory=dict)

    @property
    def n_total(self) -> int:
        return int(sum(p.n for p in self.reps))


def ball_uniform(rng: np.random.Generator, n: int, radius: float, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """n points uniform in a ball: uniform in the bounding cube, keep the ones inside."""
    out = np.empty((n, 3), dtype=np.float64)
    got = 0
    while got < n:
        need = n - got
        batch = int(need / 0.5236 * 1.05) + 64  # acceptance rate pi/6
        p = rng.uniform(-radius, radius, size=(batch, 3))
        p = p[np.einsum("ij,ij->i", p, p) < radius * radius]
        take = min(need, p.shape[0])
        out[got:got + take] = p[:take]
        got += take
    out += np.asarray(center, dtype=np.float64)
    return out


def cube_uniform(rng: np.random.Generator, n: int, half: float) -> np.ndarray:
    return rng.uniform(-half, half, size=(n, 3))


def centred_domain(radius: float, h: float):
    """Cube centred at the origin with side ceil(2 * 1.5 * radius / h) * h."""
    L = math.ceil(2.0 * 1.5 * radius / h) * h
    return np.full(3, -L / 2.0), np.full(3, L / 2.0)


def three_types(rng: np.random.Generator, n: int):
    """Types 0/1/2 with probabilities 0.6/0.3/0.1 by inverse CDF of one uniform;
    ccr and cca per type; radius lognormal (median 8.4, log-sd 0.1) in [6, 11]."""
    u = rng.uniform(size=n)
    t = np.where(u < 0.6, 0, np.where(u < 0.9, 1, 2)).astype(np.int32)
    ccr = np.array([10.0, 8.0, 12.0])[t]
    cca = np.array([0.4, 0.2, 0.6])[t]
    R = np.clip(np.exp(np.log(8.4) + 0.1 * rng.standard_normal(n)), 6.0, 11.0)
    return t, R, ccr, cca


def _scaled(n: int, scale: float) -> int:
    return max(1, int(round(n * scale)))


def spheroid_2k(seed: int = 0, scale: float = 1.0, n: int | None = None) -> Population:
    rng = np.random.Generator(np.random.PCG64(seed))
    n = _scaled(2000, scale) if n is None else n
    s = (n / 2000.0) ** (1.0 / 3.0)
    xyz = ball_uniform(rng, n, 100.0 * s)
    half = 500.0 * max(1.0, s)
    return Population("spheroid_2k", xyz, np.full(n, 8.41), np.full(n, 10.0), np.full(n, 0.4),
                      np.zeros(n, np.int32), np.full(3, -half), np.full(3, half),
                      A=1.25, h=30.0, dt=0.1, steps=100, meta={"seed": seed, "ball_radius": 100.0 * s})


def spheroid_1m(seed: int = 0, scale: float = 1.0) -> Population:
    rng = np.random.Generator(np.random.PCG64(seed))
    n = _scaled(1_000_000, scale)
    radius = 1100.0 * scale ** (1.0 / 3.0)
    xyz = ball_uniform(rng, n, radius)
    t, R, ccr, cca = three_types(rng, n)
    lo, hi = centred_domain(radius, 30.0)
    return Population("spheroid_1m", xyz, R, ccr, cca, t, lo, hi, A=1.25, h=30.0, dt=0.1,
                      steps=1000, meta={"seed": seed, "ball_radius": radius})


def clustered_20m(seed: int = 0, scale: float = 1.0) -> Population:
    rng = np.random.Generator(np.random.PCG64(seed))
    n_core = _scaled(16_000_000, scale)
    n_shell = _scaled(4_000_000, scale)
    s = scale ** (1.0 / 3.0)
    core = ball_uniform(rng, n_core, 2500.0 * s)
    shell = cube_uniform(rng, n_shell, 5000.0 * s)
    xyz = np.concatenate([core, shell])
    n = xyz.shape[0]
    half = 5000.0 * s
    return Population("clustered_20m", xyz, np.full(n, 8.41), np.full(n, 10.0), np.full(n, 0.4),
                      np.zeros(n, np.int32), np.full(3, -half), np.full(3, half), A=1.25, h=30.0,
                      dt=0.1, steps=200,
                      meta={"seed": seed, "core_radius": 2500.0 * s, "n_core": n_core, "n_shell": n_shell})


def _rep_spheroid(name, seed, r, n, rbar, typed, ccr_r=None, cca_r=None, h=30.0, steps=100):
    rng = np.random.Generator(np.random.PCG64(seed + r))
    radius = rbar * (n / PACKING) ** (1.0 / 3.0)
    xyz = ball_uniform(rng, n, radius)
    if typed:
        t, R, ccr, cca = three_types(rng, n)
    else:
        t = np.zeros(n, np.int32)
        R = np.full(n, 8.41)
        ccr = np.full(n, ccr_r)
        cca = np.full(n, cca_r)
    lo, hi = centred_domain(radius, h)
    return Population(f"{name}[{r}]", xyz, R, ccr, cca, t, lo, hi, A=1.25, h=h, dt=0.1, steps=steps,
                      meta={"seed": seed + r, "ball_radius": radius})


def ensemble_256(seed: int = 0, scale: float = 1.0, n_rep: int = 256) -> Ensemble:
    meta = np.random.Generator(np.random.PCG64(np.random.SeedSequence((seed, 1))))
    counts = np.exp(meta.uniform(math.log(1e3), math.log(2e5), size=n_rep))
    counts = np.maximum(1, np.round(counts * scale)).astype(np.int64)
    ccr = meta.uniform(5.0, 15.0, size=n_rep)
    cca = meta.uniform(0.1, 0.8, size=n_rep)
    reps = [_rep_spheroid("ensemble_256", seed, r, int(counts[r]), 8.41, False, ccr[r], cca[r], steps=100)
            for r in range(n_rep)]
    return Ensemble("ensemble_256", reps, steps=100, meta={"seed": seed, "scale": scale})


def ensemble_32_long(seed: int = 0, scale: float = 1.0, n_rep: int = 32) -> Ensemble:
    meta = np.random.Generator(np.random.PCG64(np.random.SeedSequence((seed, 1))))
    counts = np.exp(meta.uniform(math.log(5e5), math.log(5e6), size=n_rep))
    counts = np.maximum(1, np.round(counts * scale)).astype(np.int64)
    reps = [_rep_spheroid("ensemble_32_long", seed, r, int(counts[r]), 8.4, True, steps=10_000)
            for r in range(n_rep)]
    return Ensemble("ensemble_32_long", reps, steps=10_000, meta={"seed": seed, "scale": scale})


WORKLOADS = {
    "spheroid_2k": spheroid_2k,
    "spheroid_1m": spheroid_1m,
    "clustered_20m": clustered_20m,
    "ensemble_256": ensemble_256,
    "ensemble_32_long": ensemble_32_long,
}
