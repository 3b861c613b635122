"""Host-only checks of the C ABI library: it builds for sm_103a, loads, and
exports every function include/swe.h declares.  No CUDA device calls."""
import ctypes

import pytest

from paper_2103_15196_gb300 import build, swe


def test_library_builds_and_exports_header_symbols():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = swe.header_functions()
    assert {"swe_create", "swe_set_state", "swe_step", "swe_advance", "swe_get_state", "swe_destroy"} <= set(names)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_header_function():
    """The ctypes binding gives every function of include/swe.h its argument
    and return types (none is left to ctypes' default int conversion)."""
    L = swe.load_library()
    missing = [n for n in swe.header_functions() if n not in L.swe_signatures]
    assert not missing, missing


def test_params_default_host_only():
    L = swe.load_library()
    p = swe.Params()
    assert L.swe_params_default(ctypes.byref(p), 64, 32, 2.0) == swe.SWE_OK
    assert (p.nx, p.ny, p.dx) == (64, 32, 2.0)
    assert p.g == 9.81 and p.cfl_K == 0.4 and p.psi == 0.4 and p.A_J == 0.001 and p.C_J == 2.0
    assert p.precision == swe.SWE_FP32 and p.hgs_skip == 1
    assert L.swe_params_default(None, 1, 1, 1.0) == swe.SWE_EINVAL


def test_create_rejects_bad_params_before_touching_the_device():
    L = swe.load_library()
    p = swe.Params()
    L.swe_params_default(ctypes.byref(p), 8, 8, 1.0)
    h = ctypes.c_void_p()
    for field, bad in [("nx", 0), ("dx", -1.0), ("cfl_K", 1.0), ("psi", 1.0), ("d50", 0.0), ("precision", 7)]:
        q = swe.Params.from_buffer_copy(p)
        setattr(q, field, bad)
        assert L.swe_create(ctypes.byref(q), None, ctypes.byref(h)) == swe.SWE_EINVAL, field
    for side in range(4):
        q = swe.Params.from_buffer_copy(p)
        q.bc[side] = 2                      # neither a wall nor an open side
        assert L.swe_create(ctypes.byref(q), None, ctypes.byref(h)) == swe.SWE_EINVAL, side


def test_ensemble_create_rejects_counts_outside_its_table_before_touching_the_device():
    """An ensemble holds 1 .. SWE_ENSEMBLE_MAX (64) scenarios: its scenario
    table travels in the persistent launch's parameters."""
    L = swe.load_library()
    p = swe.Params()
    L.swe_params_default(ctypes.byref(p), 8, 8, 1.0)
    arr = (swe.Params * 65)(*([p] * 65))
    e = ctypes.c_void_p()
    for n in (0, 65):
        assert L.swe_ensemble_create(n, arr, None, ctypes.byref(e)) == swe.SWE_EINVAL, n


def test_boundary_kinds_default_to_walls_and_map_by_side():
    L = swe.load_library()
    p = swe.Params()
    L.swe_params_default(ctypes.byref(p), 8, 8, 1.0)
    assert list(p.bc) == [swe.SWE_BC_WALL] * 4
    for k, side in enumerate(("bc_w", "bc_e", "bc_s", "bc_n")):
        q = swe.Params.from_buffer_copy(p)
        swe._set_param(q, side, swe.SWE_BC_OPEN)
        assert [q.bc[i] for i in range(4)] == [int(i == k) for i in range(4)]
