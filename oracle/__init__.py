"""CPU oracle for the tensor-path join and sort -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline``
and ``--impl reference`` legs may import this package.  It shares no code with
the CUDA library in ``paper_2602_21237_gb300`` and neither imports the other.

``join_inner`` / ``sort`` / ``join_batch`` wrap ``tj_oracle.c`` (plain C, built
with gcc on first use).  ``learned`` holds the fp64 oracle of the learned
partitioner (numpy).

Every function here follows a definition in the paper:
  * join: Sec. 4.1 (align both relations on the common key axis and combine);
    the result must not depend on the path chosen (Sec. 3.3, Sec. 5.1).
  * sort: Sec. 4.2 (relocation along the sort-key axis), read as a stable sort.
The output order of the join (key, then S input position, then R input
position) is this library's convention; the paper fixes none.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tj_oracle.c")
_LIB = os.path.join(_HERE, "libtj_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile tj_oracle.c into libtj_oracle.so with gcc (portable flags only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, vp, ci = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
            lib.oracle_join_inner.argtypes = [ci, vp, vp, i64, vp, vp, i64, vp, i64]
            lib.oracle_join_inner.restype = i64
            lib.oracle_sort.argtypes = [ci, vp, vp, i64]
            lib.oracle_sort.restype = ci
            lib.oracle_join_batch.argtypes = [ci, i64, vp, vp, vp, vp, vp, vp, vp, i64, vp]
            lib.oracle_join_batch.restype = i64
            _lib = lib
    return _lib


def _dt(a: np.ndarray) -> int:
    if a.dtype == np.int32:
        return 0
    if a.dtype == np.int64:
        return 1
    raise TypeError(f"keys/ids must be int32 or int64, got {a.dtype}")


def _c(a: np.ndarray, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def join_inner(keys_r, ids_r, keys_s, ids_s, count_only: bool = False):
    """Inner equi-join (Sec. 4.1).  Returns an (|J|, 2) array of (r_id, s_id),
    ordered by key, then S position, then R position; or |J| if count_only."""
    kr = np.asarray(keys_r)
    dt = _dt(kr)
    ty = kr.dtype
    kr, ir = _c(kr, ty), _c(ids_r, ty)
    ks, is_ = _c(keys_s, ty), _c(ids_s, ty)
    assert kr.shape == ir.shape and ks.shape == is_.shape
    lib = _load()
    args = (dt, kr.ctypes.data, ir.ctypes.data, kr.size, ks.ctypes.data, is_.ctypes.data, ks.size)
    total = lib.oracle_join_inner(*args, None, 0)
    if total < 0:
        raise MemoryError("oracle: host allocation failed")
    if count_only:
        return int(total)
    out = np.empty((total, 2), dtype=ty)
    got = lib.oracle_join_inner(*args, out.ctypes.data if total else None, total)
    assert got == total
    return out


def sort(keys, ids):
    """Stable ORDER BY key (Sec. 4.2).  Returns sorted copies (keys, ids)."""
    k = np.array(keys, copy=True)
    dt = _dt(k)
    i = np.array(ids, dtype=k.dtype, copy=True)
    k, i = np.ascontiguousarray(k), np.ascontiguousarray(i)
    if _load().oracle_sort(dt, k.ctypes.data, i.ctypes.data, k.size) != 0:
        raise MemoryError("oracle: host allocation failed")
    return k, i


def join_batch(r_off, s_off, keys_r, ids_r, keys_s, ids_s):
    """Many independent joins stored back to back.  Returns (pairs, out_off)
    with out_off[j] the first output row of job j (n_jobs + 1 entries)."""
    kr = np.asarray(keys_r)
    dt = _dt(kr)
    ty = kr.dtype
    kr, ir, ks, is_ = _c(kr, ty), _c(ids_r, ty), _c(keys_s, ty), _c(ids_s, ty)
    ro = _c(r_off, np.int64)
    so = _c(s_off, np.int64)
    nj = ro.size - 1
    off = np.zeros(nj + 1, dtype=np.int64)
    lib = _load()
    args = (dt, nj, ro.ctypes.data, so.ctypes.data, kr.ctypes.data, ir.ctypes.data,
            ks.ctypes.data, is_.ctypes.data)
    total = lib.oracle_join_batch(*args, None, 0, off.ctypes.data)
    if total < 0:
        raise MemoryError("oracle: host allocation failed")
    out = np.empty((total, 2), dtype=ty)
    got = lib.oracle_join_batch(*args, out.ctypes.data if total else None, total,
                                off.ctypes.data)
    assert got == total
    return out, off


def gather_pairs(pairs, r_cols=(), s_cols=()):
    """Late materialisation (Sec. 3.1; the multi-attribute join of Sec. 3.2,
    R(A, B, C) with S(B, D, E) on B): row i of every output column is the R
    column at r_id = pairs[i, 0], or the S column at s_id = pairs[i, 1].  Ids
    are row positions; one outside its relation raises ValueError.  Returns
    (R outputs, S outputs) as lists of numpy arrays."""
    p = np.asarray(pairs).reshape(-1, 2)
    outs = []
    for side, cols in ((0, r_cols), (1, s_cols)):
        res = []
        for c in cols:
            c = np.asarray(c)
            ids = p[:, side]
            if ids.size and (ids.min() < 0 or ids.max() >= c.size):
                raise ValueError("oracle: an id is not a row of its relation")
            res.append(c[ids])
        outs.append(res)
    return outs[0], outs[1]


def sort_multi(cols, ids=None):
    """ORDER BY several key columns, cols[0] first (Sec. 3.2's multi-attribute
    sort key; Sec. 4.2), stable: rows equal in every key keep their input
    order.  Returns (sorted copies of the columns, ids permuted along)."""
    cols = [np.asarray(c) for c in cols]
    n = cols[0].size if cols else (0 if ids is None else np.asarray(ids).size)
    if not cols or n <= 1:
        return [c.copy() for c in cols], None if ids is None else np.array(ids, copy=True)
    # np.lexsort: the last key given is the primary one; the sort is stable
    perm = np.lexsort(tuple(reversed(cols)))
    return [c[perm] for c in cols], None if ids is None else np.asarray(ids)[perm]
