"""CPU-side checks of the C ABI: the shared library builds, loads without a
GPU and exports every function that include/simdsearch.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "simdsearch.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+(ss_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built():
    from paper_2112_03229_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("ss_search_1d", "ss_search_interp_2d", "ss_sync_status", "ss_last_error", "ss_version"):
        assert want in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    for name in declared_functions():
        assert hasattr(lib, name), name
    lib.ss_version.restype = ctypes.c_int32
    assert lib.ss_version() >= 10000


def test_argument_errors_without_gpu(built):
    # argument checks run before any CUDA call, so they work on a CPU-only host
    import paper_2112_03229_gb300 as ss
    L = ss.lib()
    assert L.ss_search_1d(None, 64, None, 10, None, 0, 0, None, None) == 1          # null pointers
    assert b"null" in L.ss_last_error()
    buf = ctypes.create_string_buffer(64)
    p = ctypes.addressof(buf)
    assert L.ss_search_1d(p, 1, p, 1, p, 0, 0, None, None) == 1                      # n < 2
    assert L.ss_search_1d(p, 4, p, -1, p, 0, 0, None, None) == 1                     # m < 0
    assert L.ss_search_1d(p, 4, p + 1, 1, p, 0, 0, None, None) == 1                  # misaligned
    assert L.ss_search_1d(p, 4, p, 1, p, 7, 0, None, None) == 1                      # bad side
    assert L.ss_search_1d(p, 4, p, 0, p, 0, 0, None, None) == 0                      # m == 0: nothing to do
    assert L.ss_search_interp_2d(p, 1, p, 4, p, p, 1, p, p, 0, None, None) == 1      # axis < 2
