"""The C-ABI library builds, loads without a GPU, exports every symbol that
include/cs_omp.h declares, and rejects bad arguments on the host before any
CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2501_11592_gb300 import build
    path = build.build()
    L = ctypes.CDLL(path)
    L.cs_last_error.restype = ctypes.c_char_p
    return L


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cs_omp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:cs_status|const char\s*\*)\s*(\w+)\s*\(", src, flags=re.M)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 13, names
    for fn in names:
        assert hasattr(lib, fn), f"{fn} declared in cs_omp.h but not exported"


def test_plan_argument_checks_without_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.cs_plan_create(ctypes.byref(h), 0, 10, 10, 4) == -1
    assert b"sizes" in lib.cs_last_error()
    assert lib.cs_plan_create(ctypes.byref(h), 64, 256, 10, 4097) == -5
    assert lib.cs_plan_create(ctypes.byref(h), 32769, 256, 10, 8) == -5
    assert lib.cs_plan_create(None, 64, 256, 10, 8) == -1
    assert lib.cs_plan_destroy(None) == 0


def test_solve_argument_checks_without_gpu(lib):
    from paper_2501_11592_gb300 import OmpParams
    p = OmpParams(4, 0.0, 0, 0, 0)
    vp = ctypes.c_void_p
    null = vp(0)
    rc = lib.omp_solve_batched(null, null, 16, 40, 16, null, 16, 3, null, null, null, null, null,
                               ctypes.byref(p), null)
    assert rc == -1 and b"plan" in lib.cs_last_error()
    lib.clfit_forward.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, vp, vp,
                                  ctypes.c_int32, ctypes.c_int32, vp, ctypes.c_int32, ctypes.c_int32,
                                  vp, ctypes.c_int32, vp, vp]
    assert lib.clfit_forward(null, 16, 40, 8, null, null, 2, 2, null, 16, 1, null, 16, null, null) == -1
    assert b"leading" in lib.cs_last_error()
    assert lib.clfit_adam_step(null, 16, 40, 16, null, null, 2, 2, null, 16, 1, null, null, 0,
                               ctypes.c_float(0.01), ctypes.c_float(0.9), ctypes.c_float(0.999),
                               ctypes.c_float(1e-8), null, null) == -1


def test_plan_setters_reject_a_null_plan(lib):
    lib.cs_plan_set_A_generation.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    assert lib.cs_plan_set_A_generation(None, 1) == -1
    assert b"plan" in lib.cs_last_error()
    assert lib.cs_plan_set_profiling(None, 1) == -1
    assert lib.cs_plan_set_option(None, 0, 1) == -1
