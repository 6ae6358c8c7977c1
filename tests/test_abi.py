"""The C ABI library builds, loads and exports every symbol include/tj.h
declares; host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_2602_21237_gb300 import api
from paper_2602_21237_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(tj_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    path = build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "tj_join_inner" in names and "tj_sort" in names and "tj_join_batch" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_status_strings(lib):
    lib.tj_status_str.restype = ctypes.c_char_p
    lib.tj_status_str.argtypes = [ctypes.c_int]
    assert lib.tj_status_str(0) == b"TJ_OK"
    assert lib.tj_status_str(3) == b"TJ_ERR_CAPACITY"
    assert lib.tj_status_str(99) == b"TJ_ERR_UNKNOWN"


def test_host_side_argument_checks(lib):
    l = api._load()
    cnt = ctypes.c_int64(-1)
    # null out_count
    assert l.tj_join_inner(1, 0, 0, 0, 0, 0, 0, 0, 0, 0, None, 0) == api.TJ_ERR_INVALID
    # negative size
    assert l.tj_join_inner(1, 0, 0, -1, 0, 0, 0, 0, 0, 0, ctypes.byref(cnt), 0) == api.TJ_ERR_INVALID
    # null pointers with n > 0
    assert l.tj_join_inner(1, 0, 0, 5, 0, 0, 5, 0, 0, 0, ctypes.byref(cnt), 0) == api.TJ_ERR_INVALID
    # too many rows
    assert l.tj_sort(1, 8, 8, 1 << 30, 0) == api.TJ_ERR_INVALID
    # unknown dtype
    assert l.tj_join_inner(7, 8, 8, 1, 8, 8, 1, 0, 8, 1, ctypes.byref(cnt), 0) == api.TJ_ERR_INVALID
    assert b"dtype" in l.tj_last_error()
    # empty inputs need no device work
    assert l.tj_join_inner(1, 0, 0, 0, 0, 0, 0, 0, 0, 0, ctypes.byref(cnt), 0) == api.TJ_OK
    assert cnt.value == 0
    assert l.tj_sort(0, 0, 0, 0, 0) == api.TJ_OK
    # batch: decreasing offsets
    ro = (ctypes.c_int64 * 3)(0, 5, 3)
    so = (ctypes.c_int64 * 3)(0, 1, 2)
    assert l.tj_join_batch(0, 2, ro, so, 8, 8, 8, 8, 8, 10, 8, ctypes.byref(cnt), 0) == \
        api.TJ_ERR_INVALID
    assert l.tj_join_batch(0, 0, None, None, 0, 0, 0, 0, 0, 0, None, ctypes.byref(cnt), 0) == \
        api.TJ_OK


def test_gather_and_multi_sort_argument_checks(lib):
    l = api._load()
    col = api._Column(8, 16, 0, 8)
    # negative size, unknown dtype, bad element width or side, null column
    assert l.tj_gather_pairs(1, 16, -1, 4, 4, ctypes.byref(col), 1, 0) == api.TJ_ERR_INVALID
    assert l.tj_gather_pairs(5, 16, 1, 4, 4, ctypes.byref(col), 1, 0) == api.TJ_ERR_INVALID
    assert l.tj_gather_pairs(1, 16, 1, 4, 4, ctypes.byref(api._Column(8, 16, 0, 3)), 1, 0) == \
        api.TJ_ERR_INVALID
    assert l.tj_gather_pairs(1, 16, 1, 4, 4, ctypes.byref(api._Column(8, 16, 2, 8)), 1, 0) == \
        api.TJ_ERR_INVALID
    assert l.tj_gather_pairs(1, 16, 1, 4, 4, ctypes.byref(api._Column(0, 16, 0, 8)), 1, 0) == \
        api.TJ_ERR_INVALID
    # pairs off the pair grid (int64 ids: 16-byte pairs)
    assert l.tj_gather_pairs(1, 8, 1, 4, 4, ctypes.byref(col), 1, 0) == api.TJ_ERR_INVALID
    # nothing to gather needs no device work
    assert l.tj_gather_pairs(1, 0, 0, 4, 4, ctypes.byref(col), 1, 0) == api.TJ_OK
    assert l.tj_gather_pairs(1, 16, 3, 4, 4, None, 0, 0) == api.TJ_OK
    ptrs = (ctypes.c_void_p * 1)(None)
    assert l.tj_sort_multi(1, ptrs, -1, None, 4, 0, 0) == api.TJ_ERR_INVALID
    assert l.tj_sort_multi(1, None, 1, None, 4, 0, 0) == api.TJ_ERR_INVALID
    assert l.tj_sort_multi(1, ptrs, 1, None, 4, 0, 0) == api.TJ_ERR_INVALID  # NULL column
    assert l.tj_sort_multi(1, ptrs, 1, None, 1, 0, 0) == api.TJ_ERR_INVALID
    assert l.tj_sort_multi(1, ptrs, 0, None, 4, 3, 0) == api.TJ_ERR_INVALID  # unknown path
    assert l.tj_sort_multi(1, ptrs, 0, None, 4, 0, 0) == api.TJ_OK


def test_trace_table_is_empty_without_calls(lib):
    api.trace_reset()
    assert api.trace_table() == {}
