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
    # directory budgets above SS_MAX_DIR_CAP (65536) are refused
    assert L.ss_search_1d_tuned(p, 4, p, 1, p, 0, 2, 65537, 0, None, None) == 1
    assert L.ss_search_1d_tuned(p, 4, p, 1, p, 0, 2, -1, 0, None, None) == 1
    for kind in (1, 2):
        o = ss.plan_opts(dir_cap=65537)
        h = ctypes.c_void_p()
        off = (ctypes.c_int64 * 2)(0, 4)
        if kind == 1:
            st = L.ss_plan_create_1d(ctypes.byref(h), 1, off, p, ctypes.byref(o), None)
        else:
            st = L.ss_plan_create_2d(ctypes.byref(h), 1, off, p, off, p, off, p, ctypes.byref(o), None)
        assert st == 1 and b"dir_cap" in L.ss_last_error() and not h.value
    # the other option checks of plan creation, also before any CUDA call
    off = (ctypes.c_int64 * 2)(0, 4)
    h = ctypes.c_void_p()
    for kind, kw, msg in ((1, dict(tile=-1), b"negative"), (1, dict(model="hunt", algo="binary"), b"bucket search"),
                          (1, dict(side=5), b"side"), (2, dict(side=1), b"SS_SIDE_LT"),
                          (2, dict(algo="ballot"), b"auto, binary or bucket"), (1, dict(mlp_lr=float("nan")), b"mlp_lr")):
        o = ss.plan_opts(**kw)
        if kind == 1:
            st = L.ss_plan_create_1d(ctypes.byref(h), 1, off, p, ctypes.byref(o), None)
        else:
            st = L.ss_plan_create_2d(ctypes.byref(h), 1, off, p, off, p, off, p, ctypes.byref(o), None)
        assert st == 1 and msg in L.ss_last_error(), (kw, L.ss_last_error())
    # host-array 2D lookup: axes above SS_MAX_AXIS_2D (4096) are refused before any allocation
    H = ss._host_lib()                   # declares the host-array signatures
    assert H.ss_search_interp_2d_host(p, 4097, p, 4, p, p, 1, p, p, 0) == 6
    assert b"SS_MAX_AXIS_2D" in L.ss_last_error()
    o = ss.plan_opts()
    o.extrap = 2
    assert L.ss_plan_create_2d(ctypes.byref(h), 1, off, p, off, p, off, p, ctypes.byref(o), None) == 1
    assert b"extrap" in L.ss_last_error() and not h.value


def test_static_batched_offset_messages_without_gpu(built):
    # the no-allocation batched search checks its host offsets before any
    # CUDA call, each bad offset with its own message naming the table
    import paper_2112_03229_gb300 as ss
    L = ss.lib()
    L.ss_search_1d_batched_static.restype = ctypes.c_int32
    buf = ctypes.create_string_buffer(64)
    p = ctypes.c_void_p(ctypes.addressof(buf))

    def call(xo, yo, side=0):
        n = len(xo) - 1
        st = L.ss_search_1d_batched_static(ctypes.c_int32(n), (ctypes.c_int64 * len(xo))(*xo), p,
                                           (ctypes.c_int64 * len(yo))(*yo), p, p, ctypes.c_int32(side), None, None)
        return st, L.ss_last_error()

    for xo, yo, msg in (([0, 4, 5], [0, 1, 2], b"table 1 has 1 entries"),
                        ([-2, 4, 8], [0, 1, 2], b"negative table offset"),
                        ([0, 4, 2], [0, 1, 2], b"table offsets decrease"),
                        ([0, 4, 8], [-1, 1, 2], b"negative target offset"),
                        ([0, 4, 8], [0, 3, 2], b"target offsets decrease")):
        st, err = call(xo, yo)
        assert st == 1 and msg in err, (xo, yo, err)
    assert call([0, 4, 8], [0, 1, 2], side=3)[0] == 1


def test_checked_entry_points_in_the_ordinary_build(built):
    # the bounds-checked build's counters exist only with -DSS_CHECKED
    import paper_2112_03229_gb300 as ss
    L = ss.lib()
    v = ctypes.c_uint64(7)
    assert L.ss_checked_hits(ctypes.byref(v), 0) == 6 and v.value == 7
    assert b"SS_CHECKED" in L.ss_last_error()
    assert L.ss_checked_selftest() == 6


def plan_file_version():
    src = open(os.path.join(ROOT, "paper_2112_03229_gb300", "csrc", "plan_io.cu")).read()
    return int(re.search(r"kVersion = (\d+);", src).group(1))


def test_plan_load_checks_without_gpu(built, tmp_path):
    # a plan file is checked on the host before anything reaches the device:
    # unreadable, foreign, truncated and inconsistent files are refused
    import struct
    import paper_2112_03229_gb300 as ss
    L = ss.lib()
    h = ctypes.c_void_p()

    def load(data):
        path = tmp_path / "p.bin"
        path.write_bytes(data)
        return L.ss_plan_load(ctypes.byref(h), str(path).encode(), None)

    assert L.ss_plan_load(ctypes.byref(h), str(tmp_path / "missing.bin").encode(), None) == 1
    magic = b"SSPLAN\x00\x01"
    head = magic + struct.pack("<iii", plan_file_version(), 1, 1)
    assert load(b"not a plan") == 1
    assert load(magic + struct.pack("<iii", plan_file_version() + 1, 1, 1)) == 1
    assert b"version" in L.ss_last_error()
    assert load(head) == 1                                          # truncated after the header

    def vec(fmt, vals):
        return struct.pack("<q", len(vals)) + struct.pack("<%d%s" % (len(vals), fmt), *vals)

    def one_table(opts, blob_bytes, dir_cap=256):
        body = bytes(opts) + vec("i", [64]) + vec("i", []) + vec("q", [0, 64]) + vec("i", [dir_cap]) + vec("i", [0])
        body += vec("q", [0]) + vec("q", [])
        body += struct.pack("<8i", *[0] * 8) + struct.pack("<8f", *[1.0] * 8) + struct.pack("<8i", 1, *[0] * 7)
        body += struct.pack("<i", 0) + struct.pack("<q", blob_bytes)
        return head + body + bytes(blob_bytes)

    assert load(one_table(ss.plan_opts(dir_cap=65537), 4096)) == 1   # options out of range
    assert b"dir_cap" in L.ss_last_error()
    assert load(one_table(ss.plan_opts(), 256)) == 1                  # blob bytes off the layout
    assert b"corrupt plan file" in L.ss_last_error()
    assert load(one_table(ss.plan_opts(), 4096, dir_cap=0)) == 1      # no directory budget
    assert not h.value
