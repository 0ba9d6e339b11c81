"""C ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports every function include/ace.h declares; host-side validation returns
the documented error codes before any device work."""
import ctypes
import math
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ace.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ace_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1601_07159_gb300 import build_lib
    if not os.path.exists(build_lib.LIB):
        if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
            pytest.skip("nvcc not available")
        build_lib.build()
    return ctypes.CDLL(build_lib.LIB)


def test_header_declares_the_entry_points():
    names = _declared_functions()
    for want in ("ace_exchange_apply", "ace_build", "ace_apply", "ace_exchange_energy_grad",
                 "ace_plan_create", "ace_plan_destroy", "ace_workspace_size", "ace_status_sync",
                 "ace_last_error", "ace_supported_edge"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_validation_without_gpu(lib):
    from paper_1601_07159_gb300.ace import Desc, ACE_ERR_ARG, ACE_ERR_UNSUPPORTED
    lib.ace_plan_create.restype = ctypes.c_int
    lib.ace_last_error.restype = ctypes.c_char_p
    lib.ace_supported_edge.restype = ctypes.c_int
    lib.ace_workspace_size.restype = ctypes.c_size_t
    lib.ace_workspace_size.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]

    def make(**kw):
        d = Desc()
        d.n_occ, d.dtype, d.kernel = 8, 2, 0
        d.n[0] = d.n[1] = d.n[2] = 24
        d.L[0] = d.L[1] = d.L[2] = 10.0
        d.omega, d.g0_value, d.alpha, d.max_pairs, d.tile = 0.0, math.nan, 1.0, 0, 0
        for k, v in kw.items():
            if k == "n":
                v = (v,) * 3 if isinstance(v, int) else v
                d.n[0], d.n[1], d.n[2] = v
            else:
                setattr(d, k, v)
        return d

    h = ctypes.c_void_p()
    assert lib.ace_plan_create(None, ctypes.byref(h)) == ACE_ERR_ARG
    assert lib.ace_plan_create(ctypes.byref(make(n_occ=0)), ctypes.byref(h)) == ACE_ERR_ARG
    assert h.value is None
    assert lib.ace_plan_create(ctypes.byref(make(dtype=7)), ctypes.byref(h)) == ACE_ERR_ARG
    assert lib.ace_plan_create(ctypes.byref(make(kernel=1, omega=0.0)), ctypes.byref(h)) == ACE_ERR_ARG
    assert lib.ace_plan_create(ctypes.byref(make(tile=9)), ctypes.byref(h)) == ACE_ERR_ARG
    assert lib.ace_plan_create(ctypes.byref(make(n=50)), ctypes.byref(h)) == ACE_ERR_UNSUPPORTED
    assert b"50" in lib.ace_last_error()
    assert lib.ace_plan_create(ctypes.byref(make(n=(24, 24, 0))), ctypes.byref(h)) == ACE_ERR_ARG
    assert lib.ace_plan_create(ctypes.byref(make(ld=24 ** 3 - 2)), ctypes.byref(h)) == ACE_ERR_ARG
    assert lib.ace_plan_create(ctypes.byref(make(ld=24 ** 3 + 1)), ctypes.byref(h)) == ACE_ERR_ARG
    assert lib.ace_plan_create(ctypes.byref(make(prec=9)), ctypes.byref(h)) == ACE_ERR_ARG
    assert lib.ace_plan_create(ctypes.byref(make(dtype=1, prec=3)), ctypes.byref(h)) == ACE_ERR_UNSUPPORTED
    assert h.value is None
    assert lib.ace_supported_edge(48, 2) == 1 and lib.ace_supported_edge(64, 2) == 1
    assert lib.ace_supported_edge(7, 2) == 0 and lib.ace_supported_edge(50, 1) == 0
    assert lib.ace_supported_edge(64, 1) == 1 and lib.ace_supported_edge(96, 0) == 1
    assert lib.ace_workspace_size(None, 0, 4) == 0
    grid = ctypes.c_int * 3
    lib.ace_supported_grid.restype = ctypes.c_int
    lib.ace_supported_grid.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.c_int]
    for n3 in ((12, 16, 20), (48, 40, 36), (16, 16, 64), (96, 96, 8), (40, 48, 96)):
        for dt in (0, 1, 2):
            assert lib.ace_supported_grid(grid(*n3), dt) == 1, (n3, dt)
    for n3 in ((12, 20, 16), (50, 50, 50), (48, 48, 50), (7, 7, 7)):
        assert lib.ace_supported_grid(grid(*n3), 2) == 0, n3
    assert lib.ace_plan_create(ctypes.byref(make(n=(12, 20, 16))), ctypes.byref(h)) == ACE_ERR_UNSUPPORTED


def test_batched_and_autotune_validation_without_gpu(lib):
    """The batched build and the autotuner reject bad arguments on the host,
    before any device call; an empty batch is a no-op."""
    from paper_1601_07159_gb300.ace import ACE_OK, ACE_ERR_ARG
    vp = ctypes.c_void_p
    lib.ace_build_batched.restype = ctypes.c_int
    lib.ace_build_batched.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), vp,
                                      ctypes.c_int, ctypes.c_int, vp, ctypes.c_size_t, vp]
    lib.ace_workspace_size_batched.restype = ctypes.c_size_t
    lib.ace_workspace_size_batched.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
    lib.ace_autotune.restype = ctypes.c_int
    lib.ace_autotune.argtypes = [vp, ctypes.c_int, vp, vp]
    assert lib.ace_build_batched(None, None, None, None, 0, 0, None, 0, None) == ACE_OK
    assert lib.ace_build_batched(None, None, None, None, -1, 0, None, 0, None) == ACE_ERR_ARG
    assert lib.ace_build_batched(None, None, None, None, 2, 0, None, 0, None) == ACE_ERR_ARG
    assert lib.ace_build_batched(None, None, None, None, 1, -2, None, 0, None) == ACE_ERR_ARG
    assert lib.ace_workspace_size_batched(None, 3) == 0
    assert lib.ace_autotune(None, 3, None, None) == ACE_ERR_ARG


def test_allocation_failure_hook_without_gpu(lib):
    """ace_debug_fail_alloc makes the library's k-th device allocation fail as
    if the device were out of memory: plan creation then returns ACE_ERR_CUDA
    with that reason (here before any device is touched), leaves no plan, and
    the hook reports how many allocations it counted. NULL plans are refused
    by ace_debug_engine_wait."""
    from paper_1601_07159_gb300.ace import Desc, ACE_ERR_ARG, ACE_ERR_CUDA
    lib.ace_plan_create.restype = ctypes.c_int
    lib.ace_last_error.restype = ctypes.c_char_p
    lib.ace_debug_fail_alloc.restype = ctypes.c_longlong
    lib.ace_debug_fail_alloc.argtypes = [ctypes.c_longlong]
    lib.ace_debug_engine_wait.restype = ctypes.c_int
    lib.ace_debug_engine_wait.argtypes = [ctypes.c_void_p, ctypes.c_uint, ctypes.c_int]
    d = Desc()
    d.n_occ, d.dtype, d.kernel = 4, 2, 0
    d.n[0] = d.n[1] = d.n[2] = 16
    d.L[0] = d.L[1] = d.L[2] = 8.0
    d.omega, d.g0_value, d.alpha = 0.0, math.nan, 1.0
    h = ctypes.c_void_p()
    lib.ace_debug_fail_alloc(1)
    try:
        assert lib.ace_plan_create(ctypes.byref(d), ctypes.byref(h)) == ACE_ERR_CUDA
        assert h.value is None
        assert b"out of memory" in lib.ace_last_error()
    finally:
        assert lib.ace_debug_fail_alloc(0) == 1
    assert lib.ace_debug_engine_wait(None, 0, 0) == ACE_ERR_ARG
