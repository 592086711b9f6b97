"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every function that include/pr_sed.h declares, and rejects bad arguments
before touching the GPU."""
import ctypes as C
import os
import re

import pytest

from paper_2108_01814_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pr_sed.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(prs_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    return B.load()


def test_header_and_binding_agree():
    assert _declared() == sorted(B.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_bad_grid_arguments_rejected_without_gpu(lib):
    out = C.c_void_p()
    per = (C.c_int * 3)(1, 1, 1)
    st = lib.prs_create_grid(0, 8, 8, 1.0, C.cast(per, C.c_void_p), None, B.PRS_FP64, None,
                             None, C.byref(out))
    assert st == -1 and not out.value
    assert b"positive" in lib.prs_last_error_string()
    st = lib.prs_create_grid(8, 8, 8, -1.0, C.cast(per, C.c_void_p), None, B.PRS_FP64, None,
                             None, C.byref(out))
    assert st == -1
    st = lib.prs_create_grid(8, 8, 8, 1.0, C.cast(per, C.c_void_p), None, 7, None, None,
                             C.byref(out))
    assert st == -1 and b"precision" in lib.prs_last_error_string()
    off = (C.c_double * 9)(*([0.5] * 8 + [1.5]))
    st = lib.prs_create_grid(8, 8, 8, 1.0, C.cast(per, C.c_void_p), C.cast(off, C.c_void_p),
                             B.PRS_FP64, None, None, C.byref(out))
    assert st == -1 and b"offsets" in lib.prs_last_error_string()


def test_null_context_rejected(lib):
    assert lib.prs_create_particles(None, 10, 1.0, 2.0, 1.0, 0) == -1
    assert lib.prs_sync(None) == -1
    assert lib.prs_dem_step(None, 1e-3, 1, None) == -4
    assert lib.prs_set_graphs(None, 1) == -1
    assert lib.prs_set_profiling(None, 1) == -1
    lib.prs_destroy(None)  # no-op


def test_library_is_sm103a_only():
    # one -gencode, for sm_103a, in the build recipe
    from paper_2108_01814_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
