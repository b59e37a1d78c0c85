"""Oracles: plain FP64 CPU code for the cell-mechanics step (``mech_oracle.c``)
and for the substrate diffusion step and its gradients (``diffusion_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library (``paper_2306_11544_gb300``) never imports it and
shares no code with it.

The C file holds the definition (binning by stable counting sort, the
neighbour-gather repulsion/adhesion velocity of the paper's "update velocity"
region, Sec. 5.4, and two-step Adams-Bashforth integration, with the per-type
adhesion affinity and domain-wall variants of that region); the second the
diffusion-decay step (three one-dimensional implicit solves, no-flux faces)
and the gradients of the microenvironment regions of Sec. 5.1-5.2.  This module
only compiles them and marshals numpy arrays; it adds no arithmetic of its own.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mech_oracle.c")
_SRC_DIFF = os.path.join(_HERE, "diffusion_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]


def build_command():
    return ["gcc", *CFLAGS, _SRC, _SRC_DIFF, "-o", _LIB, "-lm"]


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC),
                                                                          os.path.getmtime(_SRC_DIFF)):
        subprocess.run(build_command(), check=True)
    return _LIB


_I64 = ctypes.c_int64
_P = ctypes.c_void_p
_D = ctypes.c_double


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None:
        assert a.size == n, (a.size, n)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _grid(lo, dims):
    lo = np.ascontiguousarray(lo, dtype=np.float64).reshape(3)
    dims = np.ascontiguousarray(dims, dtype=np.int32).reshape(3)
    return lo, dims


class OracleLib:
    """numpy front end of one compiled copy of mech_oracle.c."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_keys.argtypes = [_I64, _P, _P, _D, _P, _P]
        lib.oracle_keys_f32.argtypes = [_I64, _P, _P, _D, _P, _P]
        lib.oracle_counting_sort.argtypes = [_I64, _P, _I64, _P, _P, _P]
        lib.oracle_velocities.argtypes = [_I64, _P, _P, _P, _P, _D, _P, _D, _P, _P]
        lib.oracle_velocities.restype = ctypes.c_int
        lib.oracle_velocities_subset.argtypes = [_I64, _P, _P, _P, _P, _D, _P, _D, _P, _I64, _P, _P]
        lib.oracle_velocities_subset.restype = ctypes.c_int
        lib.oracle_velocities_allpairs.argtypes = [_I64, _P, _P, _P, _P, _D, _P]
        lib.oracle_pairs.argtypes = [_I64, _P, _P, _D, _P, _D, _P, _I64, _P]
        lib.oracle_pairs.restype = _I64
        lib.oracle_pairs_allpairs.argtypes = [_I64, _P, _P, _D, _I64, _P]
        lib.oracle_pairs_allpairs.restype = _I64
        lib.oracle_ab2.argtypes = [_I64, _P, _P, _P, _D]
        lib.oracle_run.argtypes = [_I64, _P, _P, _P, _P, _P, _D, _P, _D, _P, _D, _I64, _P]
        lib.oracle_run.restype = ctypes.c_int
        lib.oracle_velocities_ext.argtypes = [_I64, _P, _P, _P, _P, _D, _P, _D, _P, ctypes.c_int32, _P, _P,
                                              ctypes.c_int32, _P, _P, _D, _P]
        lib.oracle_velocities_ext.restype = ctypes.c_int
        lib.oracle_velocities_allpairs_ext.argtypes = [_I64, _P, _P, _P, _P, _D, ctypes.c_int32, _P, _P,
                                                       ctypes.c_int32, _P, _P, _D, _P]
        lib.oracle_run_ext.argtypes = [_I64, _P, _P, _P, _P, _P, _D, _P, _D, _P, ctypes.c_int32, _P, _P,
                                       ctypes.c_int32, _P, _P, _D, _D, _I64, _P]
        lib.oracle_run_ext.restype = ctypes.c_int
        if hasattr(lib, "oracle_diffusion_step"):  # absent from single-file test variants
            lib.oracle_diffusion_step.argtypes = [_I64, _I64, _I64, ctypes.c_int32, _P, _P, _P, _D, _D, _I64]
            lib.oracle_diffusion_step.restype = ctypes.c_int
            lib.oracle_diffusion_gradient.argtypes = [_I64, _I64, _I64, ctypes.c_int32, _P, _D, _P]
        self.lib = lib
        self.path = path

    def num_threads(self) -> int:
        return self.lib.oracle_num_threads()

    def set_threads(self, t: int) -> None:
        self.lib.oracle_set_threads(int(t))

    def keys(self, xyz, lo, h, dims):
        """Voxel key of every cell from FP64 positions (xyz: (n,3))."""
        xyz = _f64(xyz).reshape(-1, 3)
        n = xyz.shape[0]
        lo, dims = _grid(lo, dims)
        out = np.empty(n, dtype=np.uint32)
        self.lib.oracle_keys(n, _ptr(xyz), _ptr(lo), float(h), _ptr(dims), _ptr(out))
        return out

    def keys_f32(self, xyz32, lo, h, dims):
        """Voxel key from FP32 positions, decided in FP32 arithmetic."""
        xyz32 = np.ascontiguousarray(xyz32, dtype=np.float32).reshape(-1, 3)
        n = xyz32.shape[0]
        lo, dims = _grid(lo, dims)
        out = np.empty(n, dtype=np.uint32)
        self.lib.oracle_keys_f32(n, _ptr(xyz32), _ptr(lo), float(h), _ptr(dims), _ptr(out))
        return out

    def counting_sort(self, key, V):
        """Stable counting sort: returns (count[V], start[V+1], order[n])."""
        key = np.ascontiguousarray(key, dtype=np.uint32)
        n = key.size
        count = np.empty(V, dtype=np.uint32)
        start = np.empty(V + 1, dtype=np.uint32)
        order = np.empty(n, dtype=np.int64)
        self.lib.oracle_counting_sort(n, _ptr(key), int(V), _ptr(count), _ptr(start), _ptr(order))
        return count, start, order

    def velocities(self, xyz, R, ccr, cca, A, lo, h, dims):
        xyz = _f64(xyz).reshape(-1, 3)
        n = xyz.shape[0]
        R, ccr, cca = _f64(R, n), _f64(ccr, n), _f64(cca, n)
        lo, dims = _grid(lo, dims)
        v = np.empty((n, 3), dtype=np.float64)
        if self.lib.oracle_velocities(n, _ptr(xyz), _ptr(R), _ptr(ccr), _ptr(cca), float(A), _ptr(lo),
                                      float(h), _ptr(dims), _ptr(v)) != 0:
            raise MemoryError("oracle_velocities: allocation failed")
        return v

    def velocities_subset(self, xyz, R, ccr, cca, A, lo, h, dims, idx):
        xyz = _f64(xyz).reshape(-1, 3)
        n = xyz.shape[0]
        R, ccr, cca = _f64(R, n), _f64(ccr, n), _f64(cca, n)
        lo, dims = _grid(lo, dims)
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        v = np.empty((idx.size, 3), dtype=np.float64)
        if self.lib.oracle_velocities_subset(n, _ptr(xyz), _ptr(R), _ptr(ccr), _ptr(cca), float(A),
                                             _ptr(lo), float(h), _ptr(dims), idx.size, _ptr(idx),
                                             _ptr(v)) != 0:
            raise MemoryError("oracle_velocities_subset: allocation failed")
        return v

    def velocities_allpairs(self, xyz, R, ccr, cca, A):
        xyz = _f64(xyz).reshape(-1, 3)
        n = xyz.shape[0]
        R, ccr, cca = _f64(R, n), _f64(ccr, n), _f64(cca, n)
        v = np.empty((n, 3), dtype=np.float64)
        self.lib.oracle_velocities_allpairs(n, _ptr(xyz), _ptr(R), _ptr(ccr), _ptr(cca), float(A), _ptr(v))
        return v

    @staticmethod
    def _pairs(fn, *args):
        cap = 1024
        while True:
            buf = np.empty((cap, 2), dtype=np.int64)
            cnt = fn(*args, cap, _ptr(buf))
            if cnt < 0:
                raise MemoryError("oracle pair search failed")
            if cnt <= cap:
                return buf[:cnt].copy()
            cap = int(cnt)

    def pairs(self, xyz, R, A, lo, h, dims):
        """Interacting pairs (i<j) found through the voxel bins, as an (m,2) array."""
        xyz = _f64(xyz).reshape(-1, 3)
        n = xyz.shape[0]
        R = _f64(R, n)
        lo, dims = _grid(lo, dims)
        return self._pairs(self.lib.oracle_pairs, n, _ptr(xyz), _ptr(R), float(A), _ptr(lo), float(h),
                           _ptr(dims))

    def pairs_allpairs(self, xyz, R, A):
        xyz = _f64(xyz).reshape(-1, 3)
        n = xyz.shape[0]
        R = _f64(R, n)
        return self._pairs(self.lib.oracle_pairs_allpairs, n, _ptr(xyz), _ptr(R), float(A))

    def ab2(self, xyz, v, vprev, dt):
        """One Adams-Bashforth-2 update; returns (new xyz, new vprev)."""
        xyz = _f64(xyz).reshape(-1, 3).copy()
        v = _f64(v).reshape(-1, 3)
        vprev = _f64(vprev).reshape(-1, 3).copy()
        self.lib.oracle_ab2(xyz.shape[0], _ptr(xyz), _ptr(v), _ptr(vprev), float(dt))
        return xyz, vprev

    def run(self, xyz, R, ccr, cca, A, lo, h, dims, dt, steps, vprev=None):
        """Advance `steps` full steps.  Returns (xyz, vprev, v_last)."""
        xyz = _f64(xyz).reshape(-1, 3).copy()
        n = xyz.shape[0]
        R, ccr, cca = _f64(R, n), _f64(ccr, n), _f64(cca, n)
        vprev = np.zeros((n, 3)) if vprev is None else _f64(vprev).reshape(-1, 3).copy()
        v = np.zeros((n, 3), dtype=np.float64)
        lo, dims = _grid(lo, dims)
        if self.lib.oracle_run(n, _ptr(xyz), _ptr(vprev), _ptr(R), _ptr(ccr), _ptr(cca), float(A),
                               _ptr(lo), float(h), _ptr(dims), float(dt), int(steps), _ptr(v)) != 0:
            raise MemoryError("oracle_run: allocation failed")
        return xyz, vprev, v


    @staticmethod
    def _variant(n, types, aff, walls):
        """Marshal the variant arguments: types (n ints in [0, T)), aff (T x T,
        None = no affinity: T = 1, all ones), walls (None or (wlo, whi, mask,
        c_w))."""
        if aff is None:
            aff = np.ones((1, 1))
            types = np.zeros(n, dtype=np.int32)
        aff = _f64(aff).reshape(aff.shape[0] if hasattr(aff, "shape") else len(aff), -1)
        T = aff.shape[0]
        types = np.ascontiguousarray(types, dtype=np.int32).reshape(n)
        if n and (types.min() < 0 or types.max() >= T):
            raise ValueError("cell types outside [0, T)")
        if walls is None:
            wlo, whi, mask, cw = np.zeros(3), np.zeros(3), 0, 0.0
        else:
            wlo, whi, mask, cw = walls
        wlo = _f64(wlo, 3)
        whi = _f64(whi, 3)
        return T, types, np.ascontiguousarray(aff), wlo, whi, int(mask), float(cw)

    def velocities_ext(self, xyz, R, ccr, cca, A, lo, h, dims, types=None, aff=None, walls=None):
        xyz = _f64(xyz).reshape(-1, 3)
        n = xyz.shape[0]
        R, ccr, cca = _f64(R, n), _f64(ccr, n), _f64(cca, n)
        lo, dims = _grid(lo, dims)
        T, types, aff, wlo, whi, mask, cw = self._variant(n, types, aff, walls)
        v = np.empty((n, 3), dtype=np.float64)
        if self.lib.oracle_velocities_ext(n, _ptr(xyz), _ptr(R), _ptr(ccr), _ptr(cca), float(A), _ptr(lo),
                                          float(h), _ptr(dims), T, _ptr(types), _ptr(aff), mask, _ptr(wlo),
                                          _ptr(whi), cw, _ptr(v)) != 0:
            raise MemoryError("oracle_velocities_ext: allocation failed")
        return v

    def velocities_allpairs_ext(self, xyz, R, ccr, cca, A, types=None, aff=None, walls=None):
        xyz = _f64(xyz).reshape(-1, 3)
        n = xyz.shape[0]
        R, ccr, cca = _f64(R, n), _f64(ccr, n), _f64(cca, n)
        T, types, aff, wlo, whi, mask, cw = self._variant(n, types, aff, walls)
        v = np.empty((n, 3), dtype=np.float64)
        self.lib.oracle_velocities_allpairs_ext(n, _ptr(xyz), _ptr(R), _ptr(ccr), _ptr(cca), float(A), T,
                                                _ptr(types), _ptr(aff), mask, _ptr(wlo), _ptr(whi), cw, _ptr(v))
        return v

    def run_ext(self, xyz, R, ccr, cca, A, lo, h, dims, dt, steps, types=None, aff=None, walls=None,
                vprev=None):
        """Advance `steps` steps with the variants.  Returns (xyz, vprev, v_last)."""
        xyz = _f64(xyz).reshape(-1, 3).copy()
        n = xyz.shape[0]
        R, ccr, cca = _f64(R, n), _f64(ccr, n), _f64(cca, n)
        vprev = np.zeros((n, 3)) if vprev is None else _f64(vprev).reshape(-1, 3).copy()
        v = np.zeros((n, 3), dtype=np.float64)
        lo, dims = _grid(lo, dims)
        T, types, aff, wlo, whi, mask, cw = self._variant(n, types, aff, walls)
        if self.lib.oracle_run_ext(n, _ptr(xyz), _ptr(vprev), _ptr(R), _ptr(ccr), _ptr(cca), float(A), _ptr(lo),
                                   float(h), _ptr(dims), T, _ptr(types), _ptr(aff), mask, _ptr(wlo), _ptr(whi),
                                   cw, float(dt), int(steps), _ptr(v)) != 0:
            raise MemoryError("oracle_run_ext: allocation failed")
        return xyz, vprev, v

    def diffusion_step(self, rho, D, lam, dx, dt, steps):
        """rho: (S, nz, ny, nx) densities, advanced `steps` steps (a copy is returned)."""
        rho = _f64(rho).copy()
        S, nz, ny, nx = rho.shape
        D, lam = _f64(D, S), _f64(lam, S)
        if self.lib.oracle_diffusion_step(nx, ny, nz, S, _ptr(rho), _ptr(D), _ptr(lam), float(dx), float(dt),
                                          int(steps)) != 0:
            raise MemoryError("oracle_diffusion_step: allocation failed")
        return rho

    def diffusion_gradient(self, rho, dx):
        """Gradients (S, 3, nz, ny, nx) of rho (S, nz, ny, nx)."""
        rho = _f64(rho)
        S, nz, ny, nx = rho.shape
        out = np.empty((S, 3, nz, ny, nx))
        self.lib.oracle_diffusion_gradient(nx, ny, nz, S, _ptr(rho), float(dx), _ptr(out))
        return out


def _load() -> OracleLib:
    global _lib
    with _lock:
        if _lib is None:
            _lib = OracleLib(build())
    return _lib


def compile_variant(src_text: str, out_path: str) -> OracleLib:
    """Compile a (test-modified) copy of the oracle source and load it."""
    src_path = out_path[:-3] + ".c"
    with open(src_path, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", *CFLAGS, src_path, "-o", out_path, "-lm"], check=True)
    return OracleLib(out_path)


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def num_threads() -> int:
    return _load().num_threads()


def set_threads(t: int) -> None:
    _load().set_threads(t)


def keys(xyz, lo, h, dims):
    return _load().keys(xyz, lo, h, dims)


def keys_f32(xyz32, lo, h, dims):
    return _load().keys_f32(xyz32, lo, h, dims)


def counting_sort(key, V):
    return _load().counting_sort(key, V)


def velocities(xyz, R, ccr, cca, A, lo, h, dims):
    return _load().velocities(xyz, R, ccr, cca, A, lo, h, dims)


def velocities_subset(xyz, R, ccr, cca, A, lo, h, dims, idx):
    return _load().velocities_subset(xyz, R, ccr, cca, A, lo, h, dims, idx)


def velocities_allpairs(xyz, R, ccr, cca, A):
    return _load().velocities_allpairs(xyz, R, ccr, cca, A)


def pairs(xyz, R, A, lo, h, dims):
    return _load().pairs(xyz, R, A, lo, h, dims)


def pairs_allpairs(xyz, R, A):
    return _load().pairs_allpairs(xyz, R, A)


def ab2(xyz, v, vprev, dt):
    return _load().ab2(xyz, v, vprev, dt)


def run(xyz, R, ccr, cca, A, lo, h, dims, dt, steps, vprev=None):
    return _load().run(xyz, R, ccr, cca, A, lo, h, dims, dt, steps, vprev)


def velocities_ext(xyz, R, ccr, cca, A, lo, h, dims, types=None, aff=None, walls=None):
    return _load().velocities_ext(xyz, R, ccr, cca, A, lo, h, dims, types, aff, walls)


def velocities_allpairs_ext(xyz, R, ccr, cca, A, types=None, aff=None, walls=None):
    return _load().velocities_allpairs_ext(xyz, R, ccr, cca, A, types, aff, walls)


def run_ext(xyz, R, ccr, cca, A, lo, h, dims, dt, steps, types=None, aff=None, walls=None, vprev=None):
    return _load().run_ext(xyz, R, ccr, cca, A, lo, h, dims, dt, steps, types, aff, walls, vprev)


def diffusion_step(rho, D, lam, dx, dt, steps):
    return _load().diffusion_step(rho, D, lam, dx, dt, steps)


def diffusion_gradient(rho, dx):
    return _load().diffusion_gradient(rho, dx)


def grid_dims(lo, hi, h):
    """n_d = ceil((hi_d - lo_d) / h), at least 1 (the oracle's own copy of the
    grid-size rule; the library computes it independently)."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return np.maximum(1, np.ceil((hi - lo) / float(h))).astype(np.int32)
