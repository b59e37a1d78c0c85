"""Autotuner for the mechanics step: internal voxel side, voxel-tile setting,
threads per voxel in dense tiles (one per target cell, or a warp of 32 per
voxel) and thread-per-cell block size.

For a handle (one population or a batch of replicates) it saves the exact
state, times a few steps of each candidate setting with the library's own
per-phase CUDA-event profiler, restores the saved state (so the run continues
bit-identically from where it was) and applies the fastest setting.  Results
are cached in a small JSON file keyed by the GPU, the cell count (power-of-two
bucket) and the mean cell density, so a later run of a similar workload skips
the search.

The voxel side is only a performance knob: any side >= 2 A max R finds every
interacting pair (the 27-voxel stencil covers the cutoff); a smaller voxel
means fewer candidates per cell but more voxels to scan and histogram.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

from . import mech

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "mech_autotune.json")


def _gpu_name() -> str:
    """Name and SM count of the current CUDA device (a runtime property query)."""
    try:
        import torch
        p = torch.cuda.get_device_properties(torch.cuda.current_device())
        return f"{p.name}/{p.multi_processor_count}sm"
    except Exception:
        return "unknown"


def workload_key(n_cells: int, cells_per_um3: float, mode: int) -> str:
    nb = int(round(math.log2(max(n_cells, 1))))
    db = int(round(math.log2(max(cells_per_um3, 1e-12) * 1e6)))  # cells per 100^3 um^3, log2 bucket
    return f"{_gpu_name()}|n2^{nb}|rho2^{db}|mode{mode}"


def candidates(min_voxel: float, user_voxel: float):
    """Settings tried: voxel sides from the smallest valid one up to the user's,
    three tile shapes (two density thresholds for two of them) and no tiles,
    the two dense-tile kernels (threads per voxel: one per target cell with
    the halo in shared memory, or 32) for the common tile settings, two block
    sizes."""
    up = lambda v: math.ceil(v * 1e4) / 1e4  # round up: never below the smallest valid side
    sides = sorted({up(min_voxel * f) for f in (1.0, 1.04, 1.1)} | {up(user_voxel)})
    sides = [s for s in sides if s <= max(up(user_voxel), up(min_voxel))]
    out = []
    for h in sides:
        for tile, dmin, kernels in (((4, 4, 4), 12, ("block_per_tile", "warp_per_voxel")),
                                    ((4, 4, 4), 24, ("block_per_tile",)),
                                    ((8, 4, 4), 16, ("block_per_tile", "warp_per_voxel")),
                                    ((4, 4, 8), 16, ("block_per_tile",)), ((4, 4, 8), 48, ("block_per_tile",)),
                                    (None, 0, ("block_per_tile",))):
            for kernel in kernels:
                for block in (128, 256):
                    out.append({"voxel": h, "tile": tile, "dense_min": dmin, "dense_kernel": kernel,
                                "block": block})
    return out


KEYS = ("voxel", "tile", "dense_min", "dense_kernel", "block")


def apply(m: "mech.Mech", cfg: dict) -> None:
    m.set_internal_voxel(cfg["voxel"])
    m.set_tiling(cfg["tile"], cfg["dense_min"] or 32)
    m.set_dense_kernel(cfg.get("dense_kernel", "block_per_tile"))
    m.set_launch(cfg["block"])


def time_steps(m: "mech.Mech", steps: int, warmup: int) -> float:
    """Device milliseconds per step (sum of the profiled phases)."""
    m.step(warmup)
    m.sync()
    m.set_profiling(True)
    m.step(steps)
    phases, n = m.read_profile()
    m.set_profiling(False)
    return sum(phases.values()) / max(n, 1)


def autotune(m: "mech.Mech", min_voxel: float, user_voxel: float, steps: int = 8, warmup: int = 3,
             cache_path: str | None = DEFAULT_CACHE, cells_per_um3: float | None = None,
             configs=None, verbose: bool = False) -> dict:
    """Pick and apply the fastest setting; the state is restored afterwards.
    Returns {"best": cfg, "ms_per_step": t, "trials": [...], "cached": bool}."""
    info = m.info()
    key = None
    if cache_path and cells_per_um3 is not None:
        key = workload_key(info["n_cells"], cells_per_um3, info["mode"])
        try:
            with open(cache_path) as f:
                cache = json.load(f)
            if key in cache:
                best = cache[key]["best"]
                apply(m, best)
                return {"best": best, "ms_per_step": cache[key]["ms_per_step"], "trials": [], "cached": True}
        except (OSError, ValueError):
            pass
    saved = m.read_state()
    trials = []
    cfgs = list(configs or candidates(min_voxel, user_voxel))
    # two passes in opposite orders; a setting's time is the smaller of its two
    for order in (cfgs, cfgs[::-1]):
        for cfg in order:
            t0 = time.perf_counter()
            apply(m, cfg)
            m.load_state(saved)
            ms = time_steps(m, steps, warmup)
            trials.append({**cfg, "ms_per_step": ms, "wall_s": time.perf_counter() - t0})
            if verbose:
                print(f"autotune {cfg} -> {ms:.3f} ms/step")
    best_of = {}
    for t in trials:
        k = json.dumps({c: t[c] for c in KEYS}, sort_keys=True)
        if k not in best_of or t["ms_per_step"] < best_of[k]["ms_per_step"]:
            best_of[k] = t
    best = min(best_of.values(), key=lambda t: t["ms_per_step"])
    best_cfg = {k: best[k] for k in KEYS}
    apply(m, best_cfg)
    m.load_state(saved)
    if key is not None:
        try:
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            try:
                with open(cache_path) as f:
                    cache = json.load(f)
            except (OSError, ValueError):
                cache = {}
            cache[key] = {"best": best_cfg, "ms_per_step": best["ms_per_step"]}
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return {"best": best_cfg, "ms_per_step": best["ms_per_step"], "trials": trials, "cached": False}


def population_density(xyz: np.ndarray, radius_quantile: float = 0.5) -> float:
    """Cells per um^3 inside the ball holding the given fraction of the cells
    around their centroid (a cheap density figure for the cache key)."""
    c = xyz.mean(axis=0)
    r = np.quantile(np.linalg.norm(xyz - c, axis=1), radius_quantile)
    return radius_quantile * xyz.shape[0] / (4.0 / 3.0 * math.pi * max(r, 1e-9) ** 3)
