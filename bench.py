#!/usr/bin/env python
"""Benchmark of the mechanics step (binning + neighbour-gather velocity + AB2).

Default workload: the 20M-cell clustered population (16M cells in a 2.5 mm
core + 4M uniform in a 10 mm cube, voxel 30 um), the configuration whose
memory roofline the project is measured against.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--mode kahan|mixed|fp64] [--scale S]

One step = one pass of the whole hot path (bin, force, AB2) over all cells.
`value` is device-timed (CUDA events on the library's stream, state resident
in HBM); `e2e` goes through the C ABI with the positions copied in from pinned
host memory and read back every step.  `roofline` is the force phase against
the measured HBM copy bandwidth with the fixed byte model (84 B/cell),
`step_roofline` the whole step (228 B/cell + 20 B/voxel).  On one GPU the
line also carries `second_arm` (the same workload in the other FP32 position
mode: FP64 positions next to compensated FP32 ones) and `batched_vs_plain`
(the 256-replicate ensemble advanced by one batched handle against the plain
handles looped over the replicates, with and without a CUDA graph per
handle).  Under torchrun every rank advances its own copy of the workload on
its own GPU (independent replicas; the method needs no exchange between
GPUs), and rank 0 reports the aggregate.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "mechanics cell-steps/s (bin+force+AB2), batched vs plain, at <=1e-3 um pos error"
UNIT = "cell-steps/s"
# Algorithmic bytes (compulsory HBM traffic) of the fixed byte model.
FORCE_BYTES_PER_CELL = 84      # read x 24 + params 12 + v_prev 12, write x 24 + v 12
STEP_BYTES_PER_CELL = 228      # key+hist 28, scatter 116, force+AB2 84
STEP_BYTES_PER_VOXEL = 20      # histogram zero/atomics 12, scan 8
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "force_traffic.json")
FORCE_SRC = os.path.join(ROOT, "paper_2306_11544_gb300", "csrc", "mech_force.cu")
DTYPES = {"kahan": "f32 (positions f32 + Kahan c)", "mixed": "f32 (positions f64)", "fp64": "f64"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="clustered_20m")
    p.add_argument("--scale", type=float, default=1.0)
    p.add_argument("--mode", default="kahan", choices=["kahan", "mixed", "fp64"])
    p.add_argument("--voxel", default="min",
                   help="internal voxel side: a number, 'min' (2 A max R, the smallest valid) or 'user' (the workload's)")
    p.add_argument("--block", type=int, default=0)
    p.add_argument("--graph", type=int, default=0)
    p.add_argument("--tile", default="4,4,4",
                   help="voxel tile for dense regions (4,4,4, 4,4,8 or 8,4,4), or 0 for none")
    p.add_argument("--dense-min", type=int, default=12)
    p.add_argument("--dense-kernel", default="block_per_tile", choices=["block_per_tile", "warp_per_voxel"],
                   help="kernel for the cells of dense tiles")
    p.add_argument("--e2e-steps", type=int, default=10)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-clocks", action="store_true")
    p.add_argument("--autotune", action="store_true", help="pick voxel/tile/block with the autotuner first")
    p.add_argument("--precision-study", action="store_true",
                   help="long-horizon study: batched Kahan and FP64-position runs of the 32-replicate ensemble "
                        "against an FP64 run of its smallest replicate; prints one JSON line")
    p.add_argument("--oracle-timing", action="store_true",
                   help="time the FP64 oracle on the host cores (all cores and one core) on bounded samples of "
                        "configs 1, 2, 3 and 5; prints one JSON line")
    p.add_argument("--plain-loop", action="store_true",
                   help="ensembles: also time the plain single-population path looped over replicates")
    p.add_argument("--no-ensemble", action="store_true",
                   help="single populations: skip the batched-vs-plain comparison on the 256-replicate ensemble")
    p.add_argument("--ensemble-scale", type=float, default=1.0)
    p.add_argument("--no-arm", action="store_true",
                   help="single populations: skip the second precision arm (FP64 positions next to Kahan)")
    p.add_argument("--turnover", type=float, default=0.0,
                   help="single populations: also time a loop in which this fraction of the cells dies every "
                        "--turnover-every steps and as many daughters are added next to random survivors")
    p.add_argument("--turnover-every", type=int, default=10)
    p.add_argument("--substrates", type=int, default=4,
                   help="--workload diffusion_75: substrates on the 75^3-voxel grid")
    return p.parse_args()


def reduce_max(x: float, pg, device) -> float:
    """Largest x over the ranks (the slowest rank sets the job's time); x
    itself without a process group."""
    if pg is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_throughput(cells_per_rank: int, world: int, steps: int, seconds: float) -> float:
    """Whole-job cell-steps/s: every rank advances its own replica by `steps`."""
    return cells_per_rank * world * steps / seconds


def dist_env():
    from paper_2306_11544_gb300 import shard
    return shard.dist_env()


def hbm_peak():
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def force_traffic():
    """DRAM bytes per force launch from the committed ncu summary, or None if
    the kernel source changed since the counters were taken."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
        with open(FORCE_SRC, "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()[:16]
        if t.get("source_sha256_16") != h:
            return None
        return t
    except Exception:
        return None


def issue_roofline(tr, args, n, t_tiles, sms, mhz):
    """The tile kernel against the instruction-issue ceiling that binds it:
    its warp instructions per launch (ncu, from the committed summary of the
    same source, scaled by the cell count) over its CUDA-event time t_tiles
    (s), against sms SMs x 4 schedulers x mhz.  Only for the configuration
    the count was taken on; None otherwise."""
    tk = (tr or {}).get("tile_kernel")
    if not tk or args.workload != "clustered_20m" or args.mode != "kahan" or args.tile != "4,4,4" \
            or args.dense_min != 12 or args.dense_kernel != "block_per_tile" or t_tiles <= 0:
        return None
    instr = tk["warp_instructions_per_launch"] * n / tk["cells"]
    peak = sms * 4 * mhz * 1e6
    return {"unit": "warp instructions/s", "achieved": instr / t_tiles, "peak": peak,
            "frac": instr / t_tiles / peak, "instructions_per_launch": instr,
            "source": tk["source"]}


def sm_max_mhz():
    """Maximum SM clock from the generated peaks file (2,070 MHz if absent)."""
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f).get("sm_max_mhz", 2070.0))
    except Exception:
        return 2070.0


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, enabled: bool = True):
        self.index = index
        self.enabled = enabled
        self.proc = None
        self.lines = []

    def __enter__(self):
        if self.enabled:
            try:
                self.proc = subprocess.Popen(
                    ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                     "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
                self._t = threading.Thread(target=self._read, daemon=True)
                self._t.start()
                time.sleep(0.3)
            except FileNotFoundError:
                self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.lines:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled"], "samples": 0}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        load = [s for s in sm if smax and s > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(name, scale):
    from paper_2306_11544_gb300 import synth
    fn = synth.WORKLOADS[name]
    return fn(seed=0, scale=scale)


def describe(pop_or_ens, name, args, n, V):
    from paper_2306_11544_gb300 import synth
    cfg = {"workload": name, "cells": n, "voxels": V, "mode": args.mode, "scale": args.scale,
           "tile": args.tile, "dense_min": args.dense_min, "dense_kernel": args.dense_kernel}
    if isinstance(pop_or_ens, synth.Population):
        p = pop_or_ens
        cfg.update({"voxel_um": p.h, "internal_voxel_um": getattr(args, "voxel_value", p.h), "dt_min": p.dt, "A": p.A,
                    "domain_um": [float(p.lo[0]), float(p.hi[0])]})
        if name == "clustered_20m":
            cfg["layout"] = "16M cells uniform in a 2.5 mm ball + 4M uniform in a 10 mm cube, R 8.41 um"
    else:
        cfg.update({"replicates": len(pop_or_ens.reps)})
    cfg["l2"] = "no flush: per-step working set (state + voxel arrays) is > 20x the 129 MB L2"
    return cfg


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, on a bounded sample
    (the same workload recipe at a reduced cell count), timed on host cores."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_2306_11544_gb300 import synth
    oracle.build()
    if args.workload == "diffusion_75":  # the diffusion oracle on the same field, one host core
        shape, dx, dt, D, lam, rho = diffusion_workload(max(1, args.substrates))
        steps = max(1, min(args.steps, 20))
        rho = oracle.diffusion_step(rho, D, lam, dx, dt, max(0, min(args.warmup, 3)))
        t0 = time.perf_counter()
        oracle.diffusion_step(rho, D, lam, dx, dt, steps)
        t = time.perf_counter() - t0
        nvals = int(np.prod(shape))
        value = nvals * steps / t
        line = {"impl": "reference", "metric": DIFF_METRIC, "value": value, "unit": DIFF_UNIT, "n_gpus": args.gpus,
                "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "diffusion_75", "grid": list(shape[1:]), "substrates": shape[0]},
                "cpu_baseline": {"value": value, "unit": DIFF_UNIT, "cores": 1, "kind": "oracle",
                                 "sample": f"{steps} oracle steps of the {shape[0]} x 75^3 field"},
                "e2e": {"value": value, "unit": DIFF_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    scale = args.scale * (1.0 / 64.0 if args.workload == "clustered_20m" else 0.05)
    pop = make_workload(args.workload, scale)
    reps = [pop] if isinstance(pop, synth.Population) else pop.reps
    states = []
    for p in reps:
        states.append([p, p.xyz.copy(), np.zeros_like(p.xyz), oracle.grid_dims(p.lo, p.hi, p.h)])
    n = sum(p.n for p in reps)

    def one_step():
        for st in states:
            p, x, vp, dims = st
            st[1], st[2], _ = oracle.run(x, p.R, p.ccr, p.cca, p.A, p.lo, p.h, dims, p.dt, 1, vprev=vp)

    for _ in range(args.warmup):
        one_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one_step()
    t = time.perf_counter() - t0
    value = n * args.steps / t
    sample = f"{args.workload} recipe at scale {scale:g} ({n} cells, same densities); one oracle step per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "cells": n, "mode": "fp64 oracle"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(pop):
    """The oracle on the host cores: one full step of the same workload."""
    import oracle
    from paper_2306_11544_gb300 import synth
    oracle.build()
    reps = [pop] if isinstance(pop, synth.Population) else pop.reps
    n = sum(p.n for p in reps)
    t0 = time.perf_counter()
    for p in reps:
        oracle.run(p.xyz, p.R, p.ccr, p.cca, p.A, p.lo, p.h, oracle.grid_dims(p.lo, p.hi, p.h), p.dt, 1)
    t = time.perf_counter() - t0
    return {"value": n / t, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"one full oracle step (bin+force+AB2, FP64) of all {n} cells, {t:.1f} s"}


DIFF_METRIC = "substrate diffusion voxel-updates/s (3 implicit line solves per step, FP64)"
DIFF_UNIT = "voxel-updates/s"


def diffusion_workload(S):
    """The paper's 75^3-voxel microenvironment (Sec. 5.2) with S substrates:
    20 um voxels, dt 0.01 min, diffusion coefficients from 1e5 um^2/min (an
    oxygen-like substrate) down by a factor 10 per substrate, decay 0.1/min,
    and a seeded field (a smooth bump on uniform noise)."""
    shape = (S, 75, 75, 75)
    D = 1e5 / 10.0 ** np.arange(S)
    lam = np.full(S, 0.1)
    rng = np.random.Generator(np.random.PCG64(0))
    z, y, x = np.meshgrid(*(np.arange(75),) * 3, indexing="ij")
    rho = rng.random(shape) + 5.0 * np.exp(-((x - 30) ** 2 + (y - 45) ** 2 + (z - 37) ** 2) / 50.0)[None]
    return shape, 20.0, 0.01, D, lam, rho


def run_diffusion(args):
    """Benchmark of the substrate diffusion solver (one JSON line, the same
    keys as the mechanics line)."""
    import torch
    from paper_2306_11544_gb300 import build as libbuild
    from paper_2306_11544_gb300 import mech
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    libbuild.build()
    mech.load_library()
    shape, dx, dt, D, lam, rho = diffusion_workload(max(1, args.substrates))
    S = shape[0]
    nv = int(np.prod(shape[1:]))
    stream = torch.cuda.Stream()
    with mech.Diffusion(shape[1:], dx, D, lam) as d:
        d.set_stream(stream.cuda_stream)
        d.write(rho)
        d.step(dt, args.warmup)
        d.sync()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with ClockSampler(local, enabled=not args.no_clocks) as clocks:
            ev0.record(stream)
            d.step(dt, args.steps)
            ev1.record(stream)
            ev1.synchronize()
        ms = ev0.elapsed_time(ev1)
        t = reduce_max(ms, None, "cuda")
        value = S * nv * args.steps / (t * 1e-3) * ws
        # end to end: densities in from pinned host memory, one step, densities out
        e2e = None
        if not args.no_e2e:
            host = torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
            host[...] = d.read()
            t0 = time.perf_counter()
            for _ in range(args.e2e_steps):
                d.write(host)
                d.step(dt, 1)
                host[...] = d.read()
            te = time.perf_counter() - t0
            e2e = {"value": S * nv * args.e2e_steps / te, "unit": DIFF_UNIT, "h2d_bytes_per_step": 8 * S * nv,
                   "d2h_bytes_per_step": 8 * S * nv, "steps": args.e2e_steps,
                   "path": "mech_diffusion_write -> mech_diffusion_step(1) -> mech_diffusion_read (pinned host)"}
    peak, peak_kind = hbm_peak()
    bytes_step = 3 * 16 * S * nv  # each of the three solves reads and writes every value once
    step_s = t * 1e-3 / args.steps
    line = {
        "metric": DIFF_METRIC, "value": value, "unit": DIFF_UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "diffusion_75", "grid": list(shape[1:]), "substrates": S, "voxel_um": dx,
                   "dt_min": dt, "D_um2_per_min": [float(v) for v in D], "decay_per_min": [float(v) for v in lam],
                   "l2": f"no flush: the {8 * S * nv / 1e6:.1f} MB of densities stay in the 129 MB L2, as they "
                         f"would between the solves of a simulation step"},
        "roofline": {"bound": "latency", "kernel": "k_diff_x_tiled + 2 x k_diff_yz per step",
                     "achieved": bytes_step / step_s / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": bytes_step / step_s / 1e9 / peak, "traffic": None,
                     "model": "48 B per voxel value per step (each solve reads and writes it once); the "
                              "recurrences along every grid line are sequential, so the kernels are bound by "
                              "the latency of their dependent steps, not by bandwidth",
                     "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"},
        "clocks": clocks.summary(),
        "e2e": e2e,
        "gpu_launches": 3 * args.steps,
    }
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        k = 2
        t0 = time.perf_counter()
        oracle.diffusion_step(rho, D, lam, dx, dt, k)
        tc = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": S * nv * k / tc, "unit": DIFF_UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{k} oracle steps of the same {S} x 75^3 field, {tc:.2f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def oracle_timing(args):
    """The FP64 oracle on the host cores, per workload, with every core and with
    one core: cell-steps/s over a bounded sample (stated per entry)."""
    import oracle
    from paper_2306_11544_gb300 import synth
    oracle.build()
    o = oracle._load()
    all_cores = o.num_threads()
    meta = np.random.Generator(np.random.PCG64(np.random.SeedSequence((0, 1))))
    counts = np.round(np.exp(meta.uniform(np.log(5e5), np.log(5e6), size=32))).astype(np.int64)
    r5 = int(np.argmin(counts))
    n5 = int(counts[r5])

    def rep5(f):
        return synth._rep_spheroid("ensemble_32_long", 0, r5, max(1, int(round(n5 * f))), 8.4, True, steps=10_000)

    # (name, recipe at a cell fraction, steps with all cores, fraction and steps with one core)
    cases = [("spheroid_2k", lambda f: synth.spheroid_2k(seed=0, scale=f), 100, 1.0, 100),
             ("spheroid_1m", lambda f: synth.spheroid_1m(seed=0, scale=f), 3, 1 / 16, 1),
             ("clustered_20m", lambda f: synth.clustered_20m(seed=0, scale=f), 1, 1 / 64, 1),
             ("ensemble_32_long smallest replicate", rep5, 5, 1 / 8, 1)]
    out = {"metric": "FP64 oracle cell-steps/s on the host cores", "unit": UNIT, "cores_all": all_cores,
           "cases": []}
    for name, make, steps_all, frac1, steps1 in cases:
        entry = {"workload": name}
        for cores, frac, steps in ((all_cores, 1.0, steps_all), (1, frac1, steps1)):
            p = make(frac)
            o.set_threads(cores)
            dims = oracle.grid_dims(p.lo, p.hi, p.h)
            t0 = time.perf_counter()
            oracle.run(p.xyz, p.R, p.ccr, p.cca, p.A, p.lo, p.h, dims, p.dt, steps)
            t = time.perf_counter() - t0
            entry[f"cores_{cores}"] = {"value": p.n * steps / t,
                                       "sample": f"{p.n} cells (recipe at {frac:g} of the cells) x {steps} steps, "
                                                 f"{t:.1f} s"}
        out["cases"].append(entry)
    o.set_threads(all_cores)
    print(json.dumps(out), flush=True)
    return 0


def turnover_events(pop, n_events, frac, seed=12345):
    """Precomputed death and division events that keep the cell count: each
    event's alive mask (caller order at that time) and as many daughters, half
    a radius from random survivors at their initial positions, with the
    parents' radius and coefficients."""
    rng = np.random.Generator(np.random.PCG64(seed))
    orig = np.arange(pop.n)  # initial index of each current cell
    events = []
    for _ in range(n_events):
        alive = rng.random(len(orig)) >= frac
        orig = orig[alive]
        r = int(len(alive) - alive.sum())
        parents = orig[rng.integers(0, len(orig), size=r)]
        u = rng.normal(size=(r, 3))
        u /= np.linalg.norm(u, axis=1)[:, None]
        xyz = pop.xyz[parents] + 0.5 * pop.R[parents][:, None] * u
        events.append((alive, xyz, pop.R[parents], pop.ccr[parents], pop.cca[parents]))
        orig = np.concatenate([orig, parents])
    return events


def time_turnover(m, pop, args, stream, torch, ms_per_step_plain):
    """The step loop with death and division every `turnover_every` steps
    (mech_remove_cells + mech_add_cells, host calls between steps), timed on
    the handle's stream like the main loop."""
    every = max(1, args.turnover_every)
    n_events = max(1, args.steps // every)

    def pinned(a):  # page-locked host copies, as a caller that moves data often would keep them
        out = torch.empty(a.shape, dtype=getattr(torch, a.dtype.name), pin_memory=True).numpy()
        out[...] = a
        return out

    events = [tuple(pinned(np.ascontiguousarray(x)) for x in (alive.astype(np.uint8), xyz, R, ccr, cca))
              for alive, xyz, R, ccr, cca in turnover_events(pop, n_events, args.turnover)]
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for alive, xyz, R, ccr, cca in events:
        m.step(every)
        m.remove_cells(alive)
        m.add_cells(xyz, R, ccr, cca)
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    steps = n_events * every
    return {"fraction": args.turnover, "every": every, "events": n_events,
            "cells_replaced_per_event": float(np.mean([len(e[1]) for e in events])),
            "value": pop.n * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
            "ms_per_event": (ms - steps * ms_per_step_plain) / n_events,
            "path": "mech_step(every) -> mech_remove_cells -> mech_add_cells (host calls between steps, "
                    "page-locked host arrays)"}


def time_plain_loop(ens, args, stream, torch, steps=None, warmup=None, graph=0):
    """The plain single-population API looped over the replicates: one handle
    per replicate, each advanced `steps` steps on the same stream, first with
    direct launches, then (graph > 0) with each handle replaying its own CUDA
    graph of `graph` steps.  Returns {"ungraphed": ..., "graphed": ...}."""
    from paper_2306_11544_gb300 import mech
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    mode = getattr(args, "ens_mode", args.mode)
    hs = []
    for p in ens.reps:
        h = mech.Mech.from_population(p, mode=mode)
        if args.voxel not in ("user", "0"):
            h.set_internal_voxel(2.0 * p.A * float(p.R.max()) * (1.0 + 1e-5) if args.voxel == "min"
                                 else float(args.voxel))
        tile = tuple(int(x) for x in args.tile.split(",")) if args.tile != "0" else None
        h.set_tiling(tile, args.dense_min)
        h.set_dense_kernel(args.dense_kernel)
        h.set_stream(stream)
        hs.append(h)
    n = sum(p.n for p in ens.reps)
    out = {}
    for kind, g in (("ungraphed", 0), ("graphed", graph)):
        if kind == "graphed" and not graph:
            continue
        for h in hs:
            h.set_graph(g)
            h.step(max(warmup, 2 * g if g else warmup))  # also captures the graphs
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for h in hs:
            h.step(steps)
        ev1.record(stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1)
        launches = sum(h.info()["launches_per_step"] for h in hs)
        out[kind] = {"value": n * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "handles": len(hs),
                     "launches_per_step": launches, "graph_steps": g}
    for h in hs:
        h.close()
    return out


def ensemble_comparison(args, stream, torch):
    """Batched versus plain on the 256-replicate ensemble (N_r log-uniform in
    [1e3, 2e5], FP32 force / FP64 position): the batched handle replays one
    graph holding all replicates; the plain arm loops the single-population
    handles, with and without a graph per handle.  Both give the same
    positions bit for bit (tests/test_gpu_parity.py), so the comparison is at
    equal error."""
    from paper_2306_11544_gb300 import mech, synth
    ens = synth.ensemble_256(seed=0, scale=args.ensemble_scale)
    steps = max(10, args.steps)
    graph = 10 if steps % 10 == 0 else 2
    m = mech.Mech.from_ensemble(ens, mode="mixed")
    if args.voxel not in ("user", "0"):
        m.set_internal_voxel(2.0 * ens.reps[0].A * max(float(p.R.max()) for p in ens.reps) * (1.0 + 1e-5))
    tile = tuple(int(x) for x in args.tile.split(",")) if args.tile != "0" else None
    m.set_tiling(tile, args.dense_min)
    m.set_dense_kernel(args.dense_kernel)
    m.set_stream(stream)
    m.set_graph(graph)
    m.step(max(args.warmup, 2 * graph))
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    m.step(steps)
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    info = m.info()
    m.close()
    n = ens.n_total
    batched = {"value": n * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "graph_steps": graph,
               "launches_per_step": info["launches_per_step"]}
    args.ens_mode = "mixed"
    plain = time_plain_loop(ens, args, stream, torch, steps=steps, warmup=args.warmup, graph=graph)
    return {"workload": "ensemble_256", "replicates": len(ens.reps), "cells": n, "mode": "mixed", "steps": steps,
            "scale": args.ensemble_scale, "batched": batched, "plain_graphed": plain["graphed"],
            "plain_ungraphed": plain["ungraphed"],
            "batched_over_plain_graphed": batched["value"] / plain["graphed"]["value"],
            "batched_over_plain_ungraphed": batched["value"] / plain["ungraphed"]["value"]}


def time_arm(wl, args, stream, torch, mode):
    """Device time of the single-population step in another precision mode,
    same launch configuration (the second arm of the 20M-cell configuration)."""
    from paper_2306_11544_gb300 import mech
    m = mech.Mech.from_population(wl, mode=mode)
    if args.voxel not in ("user", "0"):
        m.set_internal_voxel(args.voxel_value)
    tile = tuple(int(x) for x in args.tile.split(",")) if args.tile != "0" else None
    m.set_tiling(tile, args.dense_min)
    m.set_dense_kernel(args.dense_kernel)
    m.set_stream(stream)
    m.step(args.warmup)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    m.step(args.steps)
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    m.close()
    return {"mode": mode, "dtype": DTYPES[mode], "value": wl.n * args.steps / (ms * 1e-3), "unit": UNIT,
            "ms_per_step": ms / args.steps}


def precision_study(args):
    """Final-position error of the batched mixed modes after the workload's
    steps, on the smallest replicate, against the FP64 mode (whose every step
    reproduces the oracle's operations; its first step is checked against the
    oracle here on all cells of that replicate)."""
    import torch
    import oracle
    from paper_2306_11544_gb300 import build as libbuild
    from paper_2306_11544_gb300 import mech
    libbuild.build()
    oracle.build()
    ens = make_workload(args.workload if args.workload != "clustered_20m" else "ensemble_32_long", args.scale)
    steps = args.steps if args.steps != 200 else ens.steps
    small = min(range(len(ens.reps)), key=lambda r: ens.reps[r].n)
    p0 = ens.reps[small]
    off = sum(p.n for p in ens.reps[:small])
    out = {"metric": "final-position max error vs FP64, smallest replicate", "workload": ens.name,
           "replicates": len(ens.reps), "cells": ens.n_total, "steps": steps, "smallest_replicate_cells": p0.n}
    stream = torch.cuda.Stream()
    with mech.Mech.from_population(p0, mode="fp64") as ref:
        v0 = ref.compute_velocities()
        vr = oracle.velocities(p0.xyz, p0.R, p0.ccr, p0.cca, p0.A, p0.lo, p0.h, oracle.grid_dims(p0.lo, p0.hi, p0.h))
        out["fp64_first_step_bit_identical_to_oracle"] = bool(np.array_equal(v0, vr))
        ref.set_stream(stream)
        t0 = time.perf_counter()
        ref.step(steps)
        ref.sync()
        out["fp64_reference_s"] = time.perf_counter() - t0
        xref = ref.positions()
    for mode in ("kahan", "mixed"):
        with mech.Mech.from_ensemble(ens, mode=mode) as m:
            maxR = max(float(p.R.max()) for p in ens.reps)
            m.set_internal_voxel(2.0 * ens.reps[0].A * maxR * (1.0 + 1e-5))
            m.set_tiling((4, 4, 4), 16)
            m.set_stream(stream)
            m.set_graph(100 if steps % 100 == 0 else 0)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            m.step(steps)
            ev1.record(stream)
            ev1.synchronize()
            m.sync()
            ms = ev0.elapsed_time(ev1)
            x = m.positions()[off:off + p0.n]
        out[mode] = {"max_abs_err_um": float(np.abs(x - xref).max()), "ms_per_step": ms / steps,
                     "cell_steps_per_s": ens.n_total * steps / (ms * 1e-3)}
    print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.precision_study:
        return precision_study(args)
    if args.oracle_timing:
        return oracle_timing(args)
    if args.workload == "diffusion_75":
        return run_diffusion(args)
    ws, rank, local = dist_env()
    import torch
    from paper_2306_11544_gb300 import build as libbuild
    from paper_2306_11544_gb300 import mech, synth

    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    if rank == 0:
        libbuild.build()
    if pg:
        pg.barrier()
    mech.load_library()

    wl = make_workload(args.workload, args.scale)
    batched = not isinstance(wl, synth.Population)
    total_cells = None  # whole-job cells when the ranks share one ensemble
    sharding = None
    if batched and ws > 1:
        # the ensemble's replicates are split over the ranks (strong scaling):
        # each rank steps its own batch, with no data-path exchange
        from paper_2306_11544_gb300 import shard
        parts = shard.shard_replicates([p.n for p in wl.reps], ws)
        total_cells = wl.n_total
        sharding = {"replicates_per_rank": [len(x) for x in parts],
                    "cells_per_rank": [int(sum(wl.reps[i].n for i in x)) for x in parts]}
        wl, _ = shard.local_ensemble(wl, rank, ws)
    if not batched:
        m = mech.Mech.from_population(wl, mode=args.mode)
        n = wl.n
    else:
        m = mech.Mech.from_ensemble(wl, mode=args.mode)
        n = wl.n_total
        if not args.graph:
            args.graph = 100 if args.steps % 100 == 0 else 2 * max(1, args.steps // 20)
    if args.voxel not in ("user", "0"):
        maxR = max(float(p.R.max()) for p in ([wl] if isinstance(wl, synth.Population) else wl.reps))
        A = wl.A if isinstance(wl, synth.Population) else wl.reps[0].A
        vox = 2.0 * A * maxR * (1.0 + 1e-5) if args.voxel == "min" else float(args.voxel)
        m.set_internal_voxel(vox)
        args.voxel_value = vox
    if args.block:
        m.set_launch(args.block)
    tile = tuple(int(x) for x in args.tile.split(",")) if args.tile != "0" else None
    m.set_tiling(tile, args.dense_min)
    m.set_dense_kernel(args.dense_kernel)
    tuned = None
    if args.autotune:
        from paper_2306_11544_gb300 import autotune
        reps = [wl] if not batched else wl.reps
        maxR = max(float(p.R.max()) for p in reps)
        tuned = autotune.autotune(m, 2.0 * reps[0].A * maxR * (1.0 + 1e-5), reps[0].h, cache_path=None)
        args.voxel_value = tuned["best"]["voxel"]
    stream = torch.cuda.Stream()
    m.set_stream(stream)
    if args.graph:
        m.set_graph(args.graph)
    info = m.info()
    V = info["n_voxels"]

    # warm-up (also builds the first binning)
    m.step(args.warmup)
    m.sync()

    # timed region: K steps, events on the library's stream, phase events inside
    # (graphs replay without phase events; their phases come from a separate pass)
    profile = not args.graph
    if profile:
        m.set_profiling(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local, enabled=not args.no_clocks) as clocks:
        ev0.record(stream)
        m.step(args.steps)
        ev1.record(stream)
        ev1.synchronize()
    torch.cuda.synchronize()
    m.sync()
    ms = ev0.elapsed_time(ev1)
    phases, psteps = m.read_profile() if profile else ({}, 0)
    if profile:
        m.set_profiling(False)
    t_max = reduce_max(ms, pg, "cuda")
    if pg:
        pg.barrier()
    if total_cells is None:
        value = job_throughput(n, ws, args.steps, t_max * 1e-3)
    else:
        value = total_cells * args.steps / (t_max * 1e-3)
    if not profile:  # graph run: phases from a short profiled pass after the timed region
        m.set_profiling(True)
        m.step(max(2, min(20, args.steps)))
        phases, psteps = m.read_profile()
        m.set_profiling(False)
        profile = True

    plain = None
    if batched and args.plain_loop:
        plain = time_plain_loop(wl, args, stream, torch, graph=args.graph)
        for kind in list(plain):
            plain[kind]["batched_over_plain"] = n * args.steps / (t_max * 1e-3) / plain[kind]["value"]

    # end to end through the C ABI: pinned host positions in, step, positions out
    e2e = None
    if not args.no_e2e:
        xh = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
        m.positions(out=xh)
        for _ in range(2):
            m.write_positions(xh)
            m.step(1)
            m.positions(out=xh)
        if pg:
            pg.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            m.write_positions(xh)
            m.step(1)
            m.positions(out=xh)
        te = reduce_max(time.perf_counter() - t0, pg, "cuda")
        e2e = {"value": job_throughput(n, ws, args.e2e_steps, te), "unit": UNIT, "h2d_bytes_per_step": 24 * n,
               "d2h_bytes_per_step": 24 * n, "steps": args.e2e_steps,
               "path": "mech_write_positions (pinned host) -> mech_step(1) -> mech_read_positions (pinned host)"}
    stats = None
    if profile:
        # (neighbour tests, interacting pairs) of the final positions: on the
        # internal grid the step uses, then on the workload's own voxel grid
        tests_done, pairs = m.pair_stats()
        if args.voxel not in ("user", "0"):
            m.set_internal_voxel(0.0)
            tests_method, pairs_method = m.pair_stats()
            assert pairs_method == pairs  # the pair set does not depend on the grid
        else:
            tests_method = tests_done
        stats = (tests_method, tests_done, pairs)
    turnover = None
    if args.turnover > 0 and not batched:
        if args.voxel not in ("user", "0"):
            m.set_internal_voxel(args.voxel_value)  # the step's own grid again
        turnover = time_turnover(m, wl, args, stream, torch, t_max / args.steps)
    m.close()
    # the configuration's second precision arm and the batched-vs-plain
    # ensemble comparison (one GPU runs: extra lines of the same job)
    arm = None
    if not batched and ws == 1 and not args.no_arm and args.mode in ("kahan", "mixed"):
        arm = time_arm(wl, args, stream, torch, "mixed" if args.mode == "kahan" else "kahan")
    ens_cmp = None
    if not batched and ws == 1 and not args.no_ensemble:
        ens_cmp = ensemble_comparison(args, stream, torch)

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return 0

    peak, peak_kind = hbm_peak()
    roof = None
    if profile and psteps:
        # the force phase (velocity + AB2 kernels) is the dominant part of the
        # step; its algorithmic bytes are the fixed model's 84 B/cell
        t_force = (phases["classify"] + phases["tiles"] + phases["cells"]) / psteps * 1e-3
        cand, cand_done, pairs = stats
        tr = force_traffic()
        kern = ("k_force_fp64" if args.mode == "fp64"
                else "force phase: k_tile_classify + k_force_tile + k_sparse_list + k_force_cells")
        bytes_alg = FORCE_BYTES_PER_CELL * n
        roof = {"bound": "hbm", "kernel": kern,
                "achieved": bytes_alg / t_force / 1e9, "peak": peak, "unit": "GB/s",
                "frac": bytes_alg / t_force / 1e9 / peak,
                "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                "bytes_per_launch": bytes_alg,
                "bytes_model": f"{FORCE_BYTES_PER_CELL} B/cell (x 24, params 12, v_prev 12 in; x 24, v 12 out) x {n} cells",
                "launch_ms": 1e3 * t_force,
                "traffic": None if tr is None else tr.get("dram_bytes_per_cell", 0) * n,
                "traffic_source": None if tr is None else tr.get("source"),
                "work": {"neighbour_tests_performed": cand_done, "neighbour_tests_on_workload_grid": cand,
                         "interacting_pairs": pairs},
                "note": "not bound by HBM: instruction issue (ncu: profiles/force_tile_clustered_20m_x0.25.md)"}
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        issue = issue_roofline(tr, args, n, phases["tiles"] / psteps * 1e-3, sms, sm_max_mhz())
        if issue:
            roof["issue"] = issue
    # algorithmic model on the workload's own voxel grid (the internal grid the
    # autotuner may pick is a performance choice, not work of the problem)
    reps = [wl] if not batched else wl.reps
    V_user = int(sum(np.prod(np.maximum(1, np.ceil((p.hi - p.lo) / p.h))) for p in reps))
    step_bytes = STEP_BYTES_PER_CELL * n + STEP_BYTES_PER_VOXEL * V_user
    step_s = t_max * 1e-3 / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak" if sharding is None else "strong", "vs_baseline": None, "dtype": DTYPES[args.mode],
        "data": "synthetic",
        "config": describe(wl, args.workload, args, n, V),
        "roofline": roof,
        "step_roofline": {"bytes_per_step": step_bytes, "model": "228 B/cell + 20 B/voxel (workload voxel grid)",
                          "voxels_model": V_user, "voxels_internal": V,
                          "achieved": step_bytes / step_s / 1e9, "peak": peak, "unit": "GB/s",
                          "frac": step_bytes / step_s / 1e9 / peak},
        "phases_ms_per_step": {k: v / psteps for k, v in phases.items()} if psteps else None,
        "clocks": clocks.summary(),
        "e2e": e2e,
        "gpu_launches": info["launches_per_step"] * args.steps,
    }
    if arm is not None:
        line["second_arm"] = arm
    if ens_cmp is not None:
        line["batched_vs_plain"] = ens_cmp
    if turnover is not None:
        line["turnover"] = turnover
    if sharding is not None:
        line["sharding"] = sharding
    if batched:
        line["batched"] = {"replicates": len(wl.reps), "graph_steps": args.graph,
                           "launches_per_step": info["launches_per_step"]}
        if plain is not None:
            line["plain_looped"] = plain
    if tuned is not None:
        line["autotune"] = {"best": tuned["best"], "trials": [
            {k: t[k] for k in (*autotune.KEYS, "ms_per_step")} for t in tuned["trials"]]}
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(wl)
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
