"""ctypes binding of libtj.so (include/tj.h): argument marshalling only.

Every function takes torch CUDA tensors, passes their device pointers, sizes and
the current CUDA stream to the C ABI, and raises TjError on a non-OK status.
No step of the join or sort runs here; there is no CPU fallback.  If libtj.so
is missing the first call raises -- build it with ``__graft_entry__.build()``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libtj.so")
_lock = threading.Lock()
_lib = None

TJ_OK, TJ_ERR_INVALID, TJ_ERR_BUDGET, TJ_ERR_CAPACITY, TJ_ERR_CUDA, TJ_ERR_TIMEOUT, \
    TJ_ERR_INTERNAL = range(7)
TJ_I32, TJ_I64 = 0, 1


class TjError(RuntimeError):
    def __init__(self, status: int, name: str, detail: str):
        super().__init__(f"{name}: {detail}")
        self.status = status
        self.name = name
        self.detail = detail


class _Stats(ctypes.Structure):
    _fields_ = [("key_bits", ctypes.c_int32), ("radix_passes", ctypes.c_int32),
                ("digit_bits", ctypes.c_int32), ("groups", ctypes.c_int32),
                ("scratch_peak", ctypes.c_int64), ("staging_bytes", ctypes.c_int64),
                ("out_count", ctypes.c_int64), ("used_hbm_table", ctypes.c_int32),
                ("learned", ctypes.c_int32)]


def lib_path() -> str:
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"libtj.so not built ({_LIB_PATH}); run __graft_entry__.build()")
        lib = ctypes.CDLL(_LIB_PATH)
        i64, vp, ci, sz = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        p64 = ctypes.POINTER(ctypes.c_int64)
        lib.tj_join_inner.argtypes = [ci, vp, vp, i64, vp, vp, i64, sz, vp, i64, p64, vp]
        lib.tj_join_inner.restype = ci
        lib.tj_sort.argtypes = [ci, vp, vp, i64, vp]
        lib.tj_sort.restype = ci
        lib.tj_join_batch.argtypes = [ci, i64, p64, p64, vp, vp, vp, vp, vp, i64, vp, p64, vp]
        lib.tj_join_batch.restype = ci
        lib.tj_status_str.argtypes = [ci]
        lib.tj_status_str.restype = ctypes.c_char_p
        lib.tj_last_error.argtypes = []
        lib.tj_last_error.restype = ctypes.c_char_p
        lib.tj_get_stats.argtypes = [ctypes.POINTER(_Stats)]
        lib.tj_get_stats.restype = ci
        lib.tj_version.argtypes = []
        lib.tj_version.restype = ctypes.c_char_p
        lib.tj_trace_enable.argtypes = [ci]
        lib.tj_trace_enable.restype = None
        lib.tj_trace_reset.argtypes = []
        lib.tj_trace_reset.restype = None
        lib.tj_trace_count.argtypes = []
        lib.tj_trace_count.restype = ci
        lib.tj_trace_get.argtypes = [ci, ctypes.c_char_p, ci, p64,
                                     ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]
        lib.tj_trace_get.restype = ci
        _lib = lib
        return lib


def _check(lib, st: int):
    if st != TJ_OK:
        raise TjError(st, lib.tj_status_str(st).decode(), lib.tj_last_error().decode())


def _dt(t: torch.Tensor) -> int:
    if t.dtype == torch.int32:
        return TJ_I32
    if t.dtype == torch.int64:
        return TJ_I64
    raise TypeError(f"keys/ids must be int32 or int64, got {t.dtype}")


def _need(t: torch.Tensor, dtype, device, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or t.device != device:
        raise TypeError(f"{name}: expected {dtype} on {device}, got {t.dtype} on {t.device}")
    if t.dim() != 1 or not t.is_contiguous():
        raise ValueError(f"{name} must be 1-D and contiguous")


def _stream(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def stats() -> dict:
    """Counters of this thread's last successful call."""
    lib = _load()
    s = _Stats()
    lib.tj_get_stats(ctypes.byref(s))
    return {f: getattr(s, f) for f, _ in _Stats._fields_}


def trace_enable(on: bool = True):
    """Bracket every library kernel with CUDA events (see tj_trace_enable)."""
    _load().tj_trace_enable(1 if on else 0)


def trace_reset():
    _load().tj_trace_reset()


def trace_table() -> dict:
    """{kernel: {"launches", "ms", "bytes"}} accumulated since the last reset."""
    lib = _load()
    out = {}
    for i in range(lib.tj_trace_count()):
        name = ctypes.create_string_buffer(64)
        n = ctypes.c_int64(0)
        ms = ctypes.c_double(0)
        by = ctypes.c_double(0)
        if lib.tj_trace_get(i, name, 64, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)) == 0:
            out[name.value.decode()] = {"launches": n.value, "ms": ms.value, "bytes": by.value}
    return out


def version() -> str:
    return _load().tj_version().decode()


def join_inner(keys_r, ids_r, keys_s, ids_s, mem_budget_bytes: int = 0, out=None,
               stream=None):
    """Inner equi-join (paper Sec. 4.1) -> (count, 2) tensor of (r_id, s_id)
    ordered by key, then S position, then R position.

    `out`, if given, is a (capacity, 2) tensor of the id dtype that receives the
    pairs; otherwise one of n_s rows is tried first and, if the result is
    larger, the join is run again into a buffer of the exact size."""
    lib = _load()
    dev = keys_r.device
    dt = _dt(keys_r)
    for t, n in ((keys_r, "keys_r"), (ids_r, "ids_r"), (keys_s, "keys_s"), (ids_s, "ids_s")):
        _need(t, keys_r.dtype, dev, n)
    if ids_r.numel() != keys_r.numel() or ids_s.numel() != keys_s.numel():
        raise ValueError("keys and ids must have the same length")
    cnt = ctypes.c_int64(0)
    with torch.cuda.device(dev):
        sp = _stream(stream)

        def run(buf):
            cap = 0 if buf is None else buf.shape[0]
            return lib.tj_join_inner(dt, keys_r.data_ptr(), ids_r.data_ptr(), keys_r.numel(),
                                     keys_s.data_ptr(), ids_s.data_ptr(), keys_s.numel(),
                                     int(mem_budget_bytes), 0 if buf is None else buf.data_ptr(),
                                     cap, ctypes.byref(cnt), sp)

        if out is not None:
            if out.dim() != 2 or out.shape[1] != 2 or out.dtype != keys_r.dtype or \
                    not out.is_contiguous() or out.device != dev:
                raise ValueError("out must be a contiguous (capacity, 2) tensor of the id dtype")
            _check(lib, run(out))
            return out[: cnt.value]
        buf = torch.empty((max(1, keys_s.numel()), 2), dtype=keys_r.dtype, device=dev)
        st = run(buf)
        if st == TJ_ERR_CAPACITY:
            buf = torch.empty((cnt.value, 2), dtype=keys_r.dtype, device=dev)
            st = run(buf)
        _check(lib, st)
        return buf[: cnt.value]


def sort(keys, ids, stream=None):
    """Stable ORDER BY key (paper Sec. 4.2), in place.  Returns (keys, ids)."""
    lib = _load()
    dt = _dt(keys)
    _need(keys, keys.dtype, keys.device, "keys")
    _need(ids, keys.dtype, keys.device, "ids")
    if ids.numel() != keys.numel():
        raise ValueError("keys and ids must have the same length")
    with torch.cuda.device(keys.device):
        _check(lib, lib.tj_sort(dt, keys.data_ptr(), ids.data_ptr(), keys.numel(),
                                _stream(stream)))
    return keys, ids


def join_batch(r_off, s_off, keys_r, ids_r, keys_s, ids_s, out=None, stream=None):
    """Many independent joins stored back to back (job j: R rows
    [r_off[j], r_off[j+1]), S rows [s_off[j], s_off[j+1])).  Returns
    (pairs, out_off) with out_off a device int64 tensor of n_jobs + 1 entries."""
    lib = _load()
    dev = keys_r.device
    dt = _dt(keys_r)
    for t, n in ((keys_r, "keys_r"), (ids_r, "ids_r"), (keys_s, "keys_s"), (ids_s, "ids_s")):
        _need(t, keys_r.dtype, dev, n)
    ro = (ctypes.c_int64 * len(r_off))(*[int(x) for x in r_off])
    so = (ctypes.c_int64 * len(s_off))(*[int(x) for x in s_off])
    nj = len(r_off) - 1
    if len(s_off) != nj + 1:
        raise ValueError("r_off and s_off must have the same length")
    if r_off[-1] != keys_r.numel() or s_off[-1] != keys_s.numel():
        raise ValueError("offsets must end at the column lengths")
    cnt = ctypes.c_int64(0)
    with torch.cuda.device(dev):
        out_off = torch.zeros(nj + 1, dtype=torch.int64, device=dev)
        sp = _stream(stream)

        def run(buf):
            return lib.tj_join_batch(dt, nj, ro, so, keys_r.data_ptr(), ids_r.data_ptr(),
                                     keys_s.data_ptr(), ids_s.data_ptr(),
                                     0 if buf is None else buf.data_ptr(),
                                     0 if buf is None else buf.shape[0], out_off.data_ptr(),
                                     ctypes.byref(cnt), sp)

        if out is not None:
            _check(lib, run(out))
            return out[: cnt.value], out_off
        buf = torch.empty((max(1, keys_s.numel()), 2), dtype=keys_r.dtype, device=dev)
        st = run(buf)
        if st == TJ_ERR_CAPACITY:
            buf = torch.empty((cnt.value, 2), dtype=keys_r.dtype, device=dev)
            st = run(buf)
        _check(lib, st)
        return buf[: cnt.value], out_off
