"""Host-side checks of the C ABI library (no GPU needed): it loads and exports every
function that include/kifmm.h declares, and the Python binding marshals arguments only."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "kifmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kifmm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__  # noqa: F401
    from paper_1605_01715_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_library_exports_every_declared_symbol(lib):
    names = declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_declared_symbols():
    from paper_1605_01715_gb300 import capi
    assert sorted(capi.exported_symbols()) == declared()


def test_version_and_error_string(lib):
    lib.kifmm_version.restype = ctypes.c_char_p
    lib.kifmm_last_error.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.kifmm_version()
    assert isinstance(lib.kifmm_last_error(), bytes)


def test_null_arguments_rejected_without_a_gpu(lib):
    """Argument checks run on the host before any CUDA call."""
    out = ctypes.c_void_p()
    lib.kifmm_tree_build.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    assert lib.kifmm_tree_build(None, 10, None, 0, 8, None, ctypes.byref(out)) == -1
    assert not out.value
    lib.kifmm_fmm_matvec.argtypes = [ctypes.c_void_p] * 4
    assert lib.kifmm_fmm_matvec(None, None, None, None) == -1
    lib.kifmm_tree_destroy.argtypes = [ctypes.c_void_p]
    assert lib.kifmm_tree_destroy(None) == 0


def test_forest_arguments_rejected_without_a_gpu(lib):
    """kifmm_forest_build checks sizes and offsets on the host before any CUDA call."""
    import numpy as np
    out = ctypes.c_void_p()
    f = lib.kifmm_forest_build
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                  ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    fake = ctypes.c_void_p(0x1000)             # never dereferenced: the checks fail first
    for off, n in (([1, 10], 10), ([0, 5, 5, 10], 10), ([0, 4, 9], 10), ([0, 10], 11)):
        a = np.asarray(off, dtype=np.int64)
        assert f(fake, n, a.ctypes.data, len(off) - 1, 16, None, ctypes.byref(out)) == -1
        assert not out.value
    a = np.zeros(2, dtype=np.int64)
    assert f(fake, 10, a.ctypes.data, 0, 16, None, ctypes.byref(out)) == -1        # no instances
    assert f(None, 10, a.ctypes.data, 1, 16, None, ctypes.byref(out)) == -1        # NULL points
