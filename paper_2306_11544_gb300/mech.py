"""Python binding of libmech (the C ABI in ``include/mech.h``).

Argument marshalling only: every function here converts numpy arrays to
pointers and calls the C function of the same name; all computation runs in
the library's CUDA kernels.  There is no fallback: if ``libmech.so`` is not
built or fails to load, every call raises.

PyTorch is optional and used only as plumbing: a ``torch.cuda.Stream`` can be
handed to ``mech_set_stream`` and pinned host tensors (``.numpy()`` views) can
be passed wherever a host array is expected.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmech.so")

MECH_OK = 0
MECH_E_ARG = -1
MECH_E_NONFINITE = -2
MECH_E_VOXEL_TOO_SMALL = -3
MECH_E_OOM = -4
MECH_E_CUDA = -5
MECH_E_TIMEOUT = -6
MECH_E_DEVICE_FLAG = -7
MECH_E_STATE = -8

MECH_FP64 = 0
MECH_MIXED_FP64POS = 1
MECH_MIXED_KAHAN = 2

MECH_DENSE_WARP_PER_VOXEL = 0
MECH_DENSE_BLOCK_PER_TILE = 1
DENSE_KERNELS = {"warp_per_voxel": MECH_DENSE_WARP_PER_VOXEL, "block_per_tile": MECH_DENSE_BLOCK_PER_TILE}
MODES = {"fp64": MECH_FP64, "mixed": MECH_MIXED_FP64POS, "fp64pos": MECH_MIXED_FP64POS,
         "kahan": MECH_MIXED_KAHAN}

# Every symbol include/mech.h declares, in declaration order.
EXPORTS = [
    "mech_last_error", "mech_version", "mech_create", "mech_create_batch", "mech_set_params",
    "mech_set_domain", "mech_set_precision", "mech_set_internal_voxel", "mech_set_launch",
    "mech_set_tiling", "mech_set_dense_kernel", "mech_set_affinity", "mech_set_walls", "mech_set_stream", "mech_set_graph", "mech_step", "mech_compute_velocities", "mech_set_profiling",
    "mech_read_profile", "mech_sync",
    "mech_read_positions", "mech_read_velocities", "mech_write_positions", "mech_read_state",
    "mech_load_state", "mech_remove_cells", "mech_add_cells", "mech_add_cells_batch", "mech_debug_bins",
    "mech_pair_stats", "mech_bin_noalloc",
    "mech_debug_inject", "mech_info", "mech_grid", "mech_destroy",
    "mech_diffusion_create", "mech_diffusion_destroy", "mech_diffusion_set_stream", "mech_diffusion_write",
    "mech_diffusion_read", "mech_diffusion_step", "mech_diffusion_gradient", "mech_diffusion_sync",
]


class MechError(RuntimeError):
    def __init__(self, code: int, func: str, msg: str):
        super().__init__(f"{func} failed ({code}): {msg}")
        self.code = code


class MechInfo(ctypes.Structure):
    _fields_ = [
        ("n_cells", ctypes.c_int64),
        ("n_rep", ctypes.c_int32),
        ("mode", ctypes.c_int32),
        ("n_voxels", ctypes.c_int64),
        ("dims", ctypes.c_int32 * 3),
        ("voxel", ctypes.c_double),
        ("step", ctypes.c_int64),
        ("launches_per_step", ctypes.c_int32),
        ("graph_steps", ctypes.c_int32),
        ("device_bytes", ctypes.c_int64),
    ]


_lib = None
_lock = threading.Lock()
_P = ctypes.c_void_p


def load_library(path: str = LIB_PATH):
    """Load libmech.so (once).  Raises if it is missing: the library has no
    CPU fallback."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is not built; run `python -m paper_2306_11544_gb300.build`")
        lib = ctypes.CDLL(path)
        sig = {
            "mech_last_error": ([], ctypes.c_char_p),
            "mech_version": ([], ctypes.c_int),
            "mech_create": ([_P, ctypes.c_int64, _P, _P, _P, _P, _P], ctypes.c_int),
            "mech_create_batch": ([_P, ctypes.c_int32, _P, _P, _P, _P, _P, _P], ctypes.c_int),
            "mech_set_params": ([_P, ctypes.c_double, ctypes.c_double, ctypes.c_double], ctypes.c_int),
            "mech_set_domain": ([_P, ctypes.c_int32, _P, _P], ctypes.c_int),
            "mech_set_precision": ([_P, ctypes.c_int], ctypes.c_int),
            "mech_set_internal_voxel": ([_P, ctypes.c_double], ctypes.c_int),
            "mech_set_launch": ([_P, ctypes.c_int32], ctypes.c_int),
            "mech_set_tiling": ([_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
            "mech_set_dense_kernel": ([_P, ctypes.c_int32], ctypes.c_int),
            "mech_set_affinity": ([_P, ctypes.c_int32, _P], ctypes.c_int),
            "mech_set_walls": ([_P, ctypes.c_int32, ctypes.c_double], ctypes.c_int),
            "mech_set_stream": ([_P, _P], ctypes.c_int),
            "mech_set_graph": ([_P, ctypes.c_int32], ctypes.c_int),
            "mech_step": ([_P, ctypes.c_int64], ctypes.c_int),
            "mech_compute_velocities": ([_P, _P], ctypes.c_int),
            "mech_set_profiling": ([_P, ctypes.c_int32], ctypes.c_int),
            "mech_read_profile": ([_P, _P, _P], ctypes.c_int),
            "mech_sync": ([_P], ctypes.c_int),
            "mech_read_positions": ([_P, _P], ctypes.c_int),
            "mech_read_velocities": ([_P, _P], ctypes.c_int),
            "mech_write_positions": ([_P, _P], ctypes.c_int),
            "mech_read_state": ([_P, _P, _P, _P, _P], ctypes.c_int),
            "mech_load_state": ([_P, _P, _P, _P, ctypes.c_int64], ctypes.c_int),
            "mech_remove_cells": ([_P, _P], ctypes.c_int),
            "mech_add_cells": ([_P, ctypes.c_int64, _P, _P, _P, _P, _P], ctypes.c_int),
            "mech_add_cells_batch": ([_P, _P, _P, _P, _P, _P, _P], ctypes.c_int),
            "mech_debug_bins": ([_P, _P, _P, _P, _P], ctypes.c_int),
            "mech_pair_stats": ([_P, _P, _P], ctypes.c_int),
            "mech_bin_noalloc": ([ctypes.c_int64, _P, _P, ctypes.c_double, _P, _P, _P, _P, _P], ctypes.c_int),
            "mech_debug_inject": ([_P, ctypes.c_int32], ctypes.c_int),
            "mech_info": ([_P, _P], ctypes.c_int),
            "mech_grid": ([_P, ctypes.c_int32, _P, _P, _P], ctypes.c_int),
            "mech_destroy": ([_P], ctypes.c_int),
            "mech_diffusion_create": ([_P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_double, _P, _P], ctypes.c_int),
            "mech_diffusion_destroy": ([_P], ctypes.c_int),
            "mech_diffusion_set_stream": ([_P, _P], ctypes.c_int),
            "mech_diffusion_write": ([_P, _P], ctypes.c_int),
            "mech_diffusion_read": ([_P, _P], ctypes.c_int),
            "mech_diffusion_step": ([_P, ctypes.c_double, ctypes.c_int64], ctypes.c_int),
            "mech_diffusion_gradient": ([_P, _P], ctypes.c_int),
            "mech_diffusion_sync": ([_P], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def _check(rc: int, func: str):
    if rc != MECH_OK:
        msg = load_library().mech_last_error().decode(errors="replace")
        raise MechError(rc, func, msg)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(int(stream.cuda_stream))  # torch.cuda.Stream


# ---- C-named functions (marshalling only) ----

def mech_version() -> int:
    return load_library().mech_version()


def mech_create(n, xyz, R, ccr, cca, ctype=None):
    lib = load_library()
    h = ctypes.c_void_p()
    xyz = _f64(xyz, 3 * n)
    R, ccr, cca = _f64(R, n), _f64(ccr, n), _f64(cca, n)
    t = None if ctype is None else np.ascontiguousarray(ctype, dtype=np.int32)
    _check(lib.mech_create(ctypes.byref(h), int(n), _ptr(xyz), _ptr(R), _ptr(ccr), _ptr(cca), _ptr(t)),
           "mech_create")
    return h


def mech_remove_cells(h, n, alive):
    """Remove the cells whose alive flag is false (n flags, caller order);
    returns the new cell count."""
    a = np.ascontiguousarray(alive, dtype=np.uint8).reshape(-1)
    if a.size != n:
        raise ValueError(f"expected {n} flags, got {a.size}")
    _check(load_library().mech_remove_cells(h, _ptr(a)), "mech_remove_cells")
    return int(mech_info(h)["n_cells"])


def mech_add_cells(h, xyz, R, ccr, cca, ctype=None, counts=None):
    """Append cells; returns m.  counts (batch handles): new cells per
    replicate, the arrays holding them in replicate order."""
    xyz = _f64(xyz).reshape(-1)
    m = xyz.size // 3
    if xyz.size != 3 * m:
        raise ValueError("xyz must hold 3 values per cell")
    R, ccr, cca = _f64(R, m), _f64(ccr, m), _f64(cca, m)
    t = None if ctype is None else np.ascontiguousarray(ctype, dtype=np.int32)
    if counts is None:
        _check(load_library().mech_add_cells(h, int(m), _ptr(xyz), _ptr(R), _ptr(ccr), _ptr(cca), _ptr(t)),
               "mech_add_cells")
    else:
        c = np.ascontiguousarray(counts, dtype=np.int64)
        if int(c.sum()) != m:  # the library reads sum(counts) cells from the arrays
            raise ValueError(f"counts add up to {int(c.sum())}, the arrays hold {m} cells")
        _check(load_library().mech_add_cells_batch(h, _ptr(c), _ptr(xyz), _ptr(R), _ptr(ccr), _ptr(cca), _ptr(t)),
               "mech_add_cells_batch")
    return m


def mech_create_batch(counts, xyz, R, ccr, cca, ctype=None):
    lib = load_library()
    h = ctypes.c_void_p()
    counts = np.ascontiguousarray(counts, dtype=np.int64)
    n = int(counts.sum())
    xyz = _f64(xyz, 3 * n)
    R, ccr, cca = _f64(R, n), _f64(ccr, n), _f64(cca, n)
    t = None if ctype is None else np.ascontiguousarray(ctype, dtype=np.int32)
    _check(lib.mech_create_batch(ctypes.byref(h), counts.size, _ptr(counts), _ptr(xyz), _ptr(R), _ptr(ccr),
                                 _ptr(cca), _ptr(t)), "mech_create_batch")
    return h


def mech_set_params(h, A, voxel_size, dt):
    _check(load_library().mech_set_params(h, float(A), float(voxel_size), float(dt)), "mech_set_params")


def mech_set_domain(h, rep, lo, hi):
    lo, hi = _f64(lo, 3), _f64(hi, 3)
    _check(load_library().mech_set_domain(h, int(rep), _ptr(lo), _ptr(hi)), "mech_set_domain")


def mech_set_precision(h, mode):
    mode = MODES[mode] if isinstance(mode, str) else int(mode)
    _check(load_library().mech_set_precision(h, mode), "mech_set_precision")


def mech_set_internal_voxel(h, voxel):
    _check(load_library().mech_set_internal_voxel(h, float(voxel)), "mech_set_internal_voxel")


def mech_set_launch(h, force_block):
    _check(load_library().mech_set_launch(h, int(force_block)), "mech_set_launch")


def mech_set_tiling(h, tile=(4, 4, 4), dense_min=12):
    tx, ty, tz = (0, 0, 0) if tile is None else tile
    _check(load_library().mech_set_tiling(h, int(tx), int(ty), int(tz), int(dense_min)), "mech_set_tiling")


def mech_set_dense_kernel(h, kernel):
    k = DENSE_KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    _check(load_library().mech_set_dense_kernel(h, k), "mech_set_dense_kernel")


def mech_set_affinity(h, aff):
    """aff: an ntypes x ntypes symmetric matrix, or None to switch the affinity off."""
    if aff is None:
        _check(load_library().mech_set_affinity(h, 0, None), "mech_set_affinity")
        return
    a = np.ascontiguousarray(aff, dtype=np.float64)
    if a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise ValueError("affinity must be a square matrix")
    _check(load_library().mech_set_affinity(h, int(a.shape[0]), a.ctypes.data_as(ctypes.c_void_p)),
           "mech_set_affinity")


def mech_set_walls(h, face_mask, c_wall):
    _check(load_library().mech_set_walls(h, int(face_mask), float(c_wall)), "mech_set_walls")


def mech_set_stream(h, stream):
    _check(load_library().mech_set_stream(h, _stream_handle(stream)), "mech_set_stream")


def mech_set_graph(h, steps_per_graph):
    _check(load_library().mech_set_graph(h, int(steps_per_graph)), "mech_set_graph")


def mech_step(h, n_steps):
    _check(load_library().mech_step(h, int(n_steps)), "mech_step")


def mech_set_profiling(h, enable):
    _check(load_library().mech_set_profiling(h, int(bool(enable))), "mech_set_profiling")


PHASES = ("scan", "scatter", "canon", "classify", "tiles", "cells")


def mech_read_profile(h):
    """Summed device ms per phase since the last read, and the step count."""
    ms = np.zeros(len(PHASES))
    steps = ctypes.c_int64()
    _check(load_library().mech_read_profile(h, _ptr(ms), ctypes.byref(steps)), "mech_read_profile")
    return dict(zip(PHASES, ms.tolist())), int(steps.value)


def mech_sync(h):
    _check(load_library().mech_sync(h), "mech_sync")


def mech_compute_velocities(h, n, out=None):
    out = np.empty((n, 3), dtype=np.float64) if out is None else out
    _check(load_library().mech_compute_velocities(h, _ptr(out)), "mech_compute_velocities")
    return out


def mech_read_positions(h, n, out=None):
    out = np.empty((n, 3), dtype=np.float64) if out is None else out
    _check(load_library().mech_read_positions(h, _ptr(out)), "mech_read_positions")
    return out


def mech_read_velocities(h, n, out=None):
    out = np.empty((n, 3), dtype=np.float64) if out is None else out
    _check(load_library().mech_read_velocities(h, _ptr(out)), "mech_read_velocities")
    return out


def mech_write_positions(h, n, xyz):
    xyz = xyz if (isinstance(xyz, np.ndarray) and xyz.dtype == np.float64 and xyz.flags.c_contiguous) \
        else _f64(xyz)
    if xyz.size != 3 * n:
        raise ValueError("positions must hold 3n values")
    _check(load_library().mech_write_positions(h, _ptr(xyz)), "mech_write_positions")


def mech_read_state(h, n):
    xyz = np.empty((n, 3)); vprev = np.empty((n, 3)); comp = np.empty((n, 3))
    step = ctypes.c_int64()
    _check(load_library().mech_read_state(h, _ptr(xyz), _ptr(vprev), _ptr(comp), ctypes.byref(step)),
           "mech_read_state")
    return {"xyz": xyz, "vprev": vprev, "comp": comp, "step": int(step.value)}


def mech_load_state(h, n, state):
    xyz = _f64(state["xyz"], 3 * n)
    vprev = _f64(state["vprev"], 3 * n)
    comp = None if state.get("comp") is None else _f64(state["comp"], 3 * n)
    _check(load_library().mech_load_state(h, _ptr(xyz), _ptr(vprev), _ptr(comp), int(state.get("step", 0))),
           "mech_load_state")


def mech_info(h) -> dict:
    info = MechInfo()
    _check(load_library().mech_info(h, ctypes.byref(info)), "mech_info")
    return {"n_cells": info.n_cells, "n_rep": info.n_rep, "mode": info.mode, "n_voxels": info.n_voxels,
            "dims": tuple(info.dims), "voxel": info.voxel, "step": info.step,
            "launches_per_step": info.launches_per_step, "graph_steps": info.graph_steps,
            "device_bytes": info.device_bytes}


def mech_grid(h, rep):
    lo = np.empty(3); dims = np.empty(3, dtype=np.int32); vb = ctypes.c_int64()
    _check(load_library().mech_grid(h, int(rep), _ptr(lo), _ptr(dims), ctypes.byref(vb)), "mech_grid")
    return lo, dims, int(vb.value)


def mech_pair_stats(h):
    """(candidates, interacting pairs) of the current positions."""
    c = ctypes.c_int64(0)
    p = ctypes.c_int64(0)
    _check(load_library().mech_pair_stats(h, ctypes.byref(c), ctypes.byref(p)), "mech_pair_stats")
    return int(c.value), int(p.value)


def mech_debug_bins(h, n):
    V = mech_info(h)["n_voxels"]
    key = np.empty(n, dtype=np.uint32)
    count = np.empty(V, dtype=np.uint32)
    start = np.empty(V + 1, dtype=np.uint32)
    order = np.empty(n, dtype=np.int64)
    _check(load_library().mech_debug_bins(h, _ptr(key), _ptr(count), _ptr(start), _ptr(order)), "mech_debug_bins")
    return key, count, start, order


def mech_bin_noalloc(n, xyz_dev, lo, voxel, dims, key_dev, start_dev, order_dev, stream=None):
    """Binning into caller-owned device buffers (raw device addresses as ints)
    with no device allocation by the library: for callers that cannot
    allocate device memory at the point of the call (see include/mech.h)."""
    lo = _f64(lo, 3)
    dims = np.ascontiguousarray(dims, dtype=np.int32)
    _check(load_library().mech_bin_noalloc(int(n), ctypes.c_void_p(int(xyz_dev)), _ptr(lo), float(voxel), _ptr(dims),
                                           ctypes.c_void_p(int(key_dev)), ctypes.c_void_p(int(start_dev)),
                                           ctypes.c_void_p(int(order_dev)), _stream_handle(stream)),
           "mech_bin_noalloc")


MECH_FAULT_NONE = 0
MECH_FAULT_TILE_WAIT = 1
MECH_FAULT_ALLOC = 2


def mech_debug_inject(h, fault):
    _check(load_library().mech_debug_inject(h, int(fault)), "mech_debug_inject")


def mech_destroy(h):
    if h is not None:
        _check(load_library().mech_destroy(h), "mech_destroy")


# ---- convenience wrapper ----

class Mech:
    """One libmech handle (a population, or a batch of replicates)."""

    def __init__(self, xyz, R, ccr, cca, ctype=None, counts=None):
        xyz = _f64(xyz).reshape(-1, 3)
        self.n = xyz.shape[0]
        if counts is None:
            self.h = mech_create(self.n, xyz, R, ccr, cca, ctype)
            self.counts = np.array([self.n], dtype=np.int64)
        else:
            self.counts = np.asarray(counts, dtype=np.int64)
            self.h = mech_create_batch(self.counts, xyz, R, ccr, cca, ctype)

    @classmethod
    def from_population(cls, pop, mode="mixed", domain=True):
        m = cls(pop.xyz, pop.R, pop.ccr, pop.cca, pop.ctype)
        m.set_params(pop.A, pop.h, pop.dt)
        if domain:
            m.set_domain(-1, pop.lo, pop.hi)
        m.set_precision(mode)
        return m

    @classmethod
    def from_ensemble(cls, ens, mode="mixed"):
        reps = ens.reps
        xyz = np.concatenate([p.xyz for p in reps])
        cat = lambda f: np.concatenate([getattr(p, f) for p in reps])
        m = cls(xyz, cat("R"), cat("ccr"), cat("cca"), cat("ctype"), counts=[p.n for p in reps])
        p0 = reps[0]
        m.set_params(p0.A, p0.h, p0.dt)
        for r, p in enumerate(reps):
            m.set_domain(r, p.lo, p.hi)
        m.set_precision(mode)
        return m

    def set_params(self, A, voxel, dt):
        mech_set_params(self.h, A, voxel, dt)

    def set_domain(self, rep, lo, hi):
        mech_set_domain(self.h, rep, lo, hi)

    def set_precision(self, mode):
        mech_set_precision(self.h, mode)

    def set_internal_voxel(self, v):
        mech_set_internal_voxel(self.h, v)

    def set_launch(self, block):
        mech_set_launch(self.h, block)

    def set_tiling(self, tile=(4, 4, 4), dense_min=12):
        mech_set_tiling(self.h, tile, dense_min)

    def set_dense_kernel(self, kernel):
        mech_set_dense_kernel(self.h, kernel)

    def set_affinity(self, aff):
        mech_set_affinity(self.h, aff)

    def set_walls(self, face_mask, c_wall):
        mech_set_walls(self.h, face_mask, c_wall)

    def set_stream(self, stream):
        mech_set_stream(self.h, stream)

    def set_graph(self, steps):
        mech_set_graph(self.h, steps)

    def step(self, n=1):
        mech_step(self.h, n)

    def sync(self):
        mech_sync(self.h)

    def set_profiling(self, enable=True):
        mech_set_profiling(self.h, enable)

    def read_profile(self):
        return mech_read_profile(self.h)

    def positions(self, out=None):
        return mech_read_positions(self.h, self.n, out)

    def velocities(self, out=None):
        return mech_read_velocities(self.h, self.n, out)

    def compute_velocities(self, out=None):
        return mech_compute_velocities(self.h, self.n, out)

    def write_positions(self, xyz):
        mech_write_positions(self.h, self.n, xyz)

    def read_state(self):
        return mech_read_state(self.h, self.n)

    def load_state(self, state):
        mech_load_state(self.h, self.n, state)

    def remove_cells(self, alive):
        """Keep the cells whose flag is true; survivors are renumbered in order."""
        alive = np.asarray(alive).reshape(-1)
        self.n = mech_remove_cells(self.h, self.n, alive)
        if len(self.counts) == 1:
            self.counts = np.array([self.n], dtype=np.int64)
        else:  # survivors per replicate
            edges = np.concatenate([[0], np.cumsum(self.counts)])
            self.counts = np.array([np.count_nonzero(alive[a:b]) for a, b in zip(edges[:-1], edges[1:])],
                                   dtype=np.int64)

    def add_cells(self, xyz, R, ccr, cca, ctype=None, counts=None):
        """Append cells after the current ones (zero previous velocity); a
        batch takes counts, the new cells per replicate in replicate order."""
        self.n += mech_add_cells(self.h, xyz, R, ccr, cca, ctype, counts)
        self.counts = (np.array([self.n], dtype=np.int64) if counts is None
                       else self.counts + np.asarray(counts, dtype=np.int64))

    def bins(self):
        return mech_debug_bins(self.h, self.n)

    def pair_stats(self):
        """(candidate pairs tested by one step, interacting pairs) of the current positions."""
        return mech_pair_stats(self.h)

    def info(self):
        return mech_info(self.h)

    def grid(self, rep=0):
        return mech_grid(self.h, rep)

    def close(self):
        if getattr(self, "h", None) is not None:
            mech_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Diffusion:
    """One substrate-diffusion handle: S densities on an nx x ny x nz voxel
    grid (arrays shaped (S, nz, ny, nx)), no-flux faces."""

    def __init__(self, shape, dx, D, lam):
        nz, ny, nx = (int(v) for v in shape)
        D = _f64(D).reshape(-1)
        lam = _f64(lam, D.size)
        self.shape = (D.size, nz, ny, nx)
        self.h = ctypes.c_void_p()
        _check(load_library().mech_diffusion_create(ctypes.byref(self.h), nx, ny, nz, int(D.size), float(dx),
                                                    _ptr(D), _ptr(lam)), "mech_diffusion_create")

    def write(self, rho):
        rho = _f64(rho, int(np.prod(self.shape)))
        _check(load_library().mech_diffusion_write(self.h, _ptr(rho)), "mech_diffusion_write")

    def read(self):
        out = np.empty(self.shape)
        _check(load_library().mech_diffusion_read(self.h, _ptr(out)), "mech_diffusion_read")
        return out

    def step(self, dt, n=1):
        _check(load_library().mech_diffusion_step(self.h, float(dt), int(n)), "mech_diffusion_step")

    def gradient(self):
        S, nz, ny, nx = self.shape
        out = np.empty((S, 3, nz, ny, nx))
        _check(load_library().mech_diffusion_gradient(self.h, _ptr(out)), "mech_diffusion_gradient")
        return out

    def set_stream(self, stream):
        _check(load_library().mech_diffusion_set_stream(self.h, ctypes.c_void_p(stream)), "mech_diffusion_set_stream")

    def sync(self):
        _check(load_library().mech_diffusion_sync(self.h), "mech_diffusion_sync")

    def close(self):
        if self.h:
            load_library().mech_diffusion_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
