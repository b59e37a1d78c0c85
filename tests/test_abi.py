"""The C-ABI library loads and exports every symbol include/mech.h declares,
and its host-side argument checks answer without a GPU (CPU only: no call
here reaches a kernel)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2306_11544_gb300 import build, mech
    build.build()
    return mech.load_library()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "mech.h")).read()
    return re.findall(r"MECH_API\s+[\w\s\*]+?\b(mech_\w+)\s*\(", text)


def test_header_declares_the_binding_list():
    from paper_2306_11544_gb300 import mech
    assert declared_symbols() == mech.EXPORTS


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name


def test_version_and_error_string(lib):
    assert lib.mech_version() == 100
    assert isinstance(lib.mech_last_error(), bytes)


def test_host_validation_needs_no_gpu(lib):
    from paper_2306_11544_gb300 import mech
    h = ctypes.c_void_p()
    # null handles
    assert lib.mech_step(None, 1) == mech.MECH_E_ARG
    assert lib.mech_set_params(None, 1.25, 30.0, 0.1) == mech.MECH_E_ARG
    assert lib.mech_destroy(None) == mech.MECH_OK
    # bad counts / arrays are rejected before any device call
    assert lib.mech_create(ctypes.byref(h), -1, None, None, None, None, None) == mech.MECH_E_ARG
    assert lib.mech_create(ctypes.byref(h), 2, None, None, None, None, None) == mech.MECH_E_ARG
    xyz = np.zeros(6)
    xyz[4] = np.nan
    R = np.full(2, 8.0)
    c = np.ones(2)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    assert lib.mech_create(ctypes.byref(h), 2, p(xyz), p(R), p(c), p(c), None) == mech.MECH_E_NONFINITE
    xyz[4] = 0.0
    Rbad = np.array([8.0, 0.0])
    assert lib.mech_create(ctypes.byref(h), 2, p(xyz), p(Rbad), p(c), p(c), None) == mech.MECH_E_ARG
    neg = np.array([1.0, -0.5])
    assert lib.mech_create(ctypes.byref(h), 2, p(xyz), p(R), p(c), p(neg), None) == mech.MECH_E_ARG
    counts = np.array([1, -1], dtype=np.int64)
    assert lib.mech_create_batch(ctypes.byref(h), 2, p(counts), p(xyz), p(R), p(c), p(c), None) == mech.MECH_E_ARG
    assert lib.mech_create_batch(ctypes.byref(h), 0, p(counts), p(xyz), p(R), p(c), p(c), None) == mech.MECH_E_ARG
    assert b"replicate" in lib.mech_last_error() or b"n_rep" in lib.mech_last_error()
    # cell types travel in 4 bits of the force record: outside [0, 16) is refused
    for bad in ([0, 16], [-1, 2]):
        t = np.array(bad, dtype=np.int32)
        assert lib.mech_create(ctypes.byref(h), 2, p(xyz), p(R), p(c), p(c), p(t)) == mech.MECH_E_ARG
        assert b"types" in lib.mech_last_error()
    # variant setters refuse a null handle
    assert lib.mech_set_affinity(None, 1, p(np.ones(1))) == mech.MECH_E_ARG
    assert lib.mech_set_walls(None, 1, 1.0) == mech.MECH_E_ARG


def test_binding_raises_without_library(tmp_path):
    from paper_2306_11544_gb300 import mech
    saved = mech._lib
    try:
        mech._lib = None
        with pytest.raises(RuntimeError):
            mech.load_library(str(tmp_path / "missing.so"))
    finally:
        mech._lib = saved


def test_fault_injection_arming_is_host_only(lib):
    """Arming and disarming the allocation fault needs no GPU; an unknown
    fault or a missing handle for a handle-scoped fault is an argument error."""
    from paper_2306_11544_gb300 import mech
    assert lib.mech_debug_inject(None, mech.MECH_FAULT_ALLOC) == mech.MECH_OK
    assert lib.mech_debug_inject(None, mech.MECH_FAULT_NONE) == mech.MECH_OK
    assert lib.mech_debug_inject(None, mech.MECH_FAULT_TILE_WAIT) == mech.MECH_E_ARG
    assert lib.mech_debug_inject(None, 99) == mech.MECH_E_ARG
