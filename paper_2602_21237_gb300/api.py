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
TJ_JOIN_NO_FUSED = 1


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
                ("out_count", ctypes.c_int64), ("route_regions", ctypes.c_int32),
                ("learned", ctypes.c_int32), ("partitions", ctypes.c_int32),
                ("heavy_keys", ctypes.c_int32), ("max_partition", ctypes.c_int64),
                ("balance", ctypes.c_double), ("radix_balance", ctypes.c_double),
                ("tile_rows", ctypes.c_int32), ("digit_cap", ctypes.c_int32),
                ("lanes", ctypes.c_int32), ("packed_keys", ctypes.c_int32),
                ("learned_balance", ctypes.c_double), ("fused_batches", ctypes.c_int32),
                ("mlp_steps", ctypes.c_int32)]


class _Opts(ctypes.Structure):
    _fields_ = [("router", ctypes.c_int32), ("partitions", ctypes.c_int32),
                ("sample_stride", ctypes.c_int32), ("pla_segments", ctypes.c_int32),
                ("mlp_steps", ctypes.c_int32), ("mlp_batch", ctypes.c_int32),
                ("mlp_lr", ctypes.c_float), ("seed", ctypes.c_uint64),
                ("radix_judge", ctypes.c_float), ("flags", ctypes.c_int32)]


class _Column(ctypes.Structure):
    _fields_ = [("src", ctypes.c_void_p), ("dst", ctypes.c_void_p), ("side", ctypes.c_int32),
                ("elem_bytes", ctypes.c_int32)]


ROUTERS = {"auto": 0, "single": 1, "radix": 2, "pla": 3, "mlp": 4}


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
        lib.tj_join_inner_ex.argtypes = [ci, vp, vp, i64, vp, vp, i64, sz,
                                         ctypes.POINTER(_Opts), vp, i64, p64, vp]
        lib.tj_join_inner_ex.restype = ci
        lib.tj_sort.argtypes = [ci, vp, vp, i64, vp]
        lib.tj_gather_pairs.argtypes = [ci, vp, i64, i64, i64, ctypes.POINTER(_Column),
                                        ctypes.c_int32, vp]
        lib.tj_gather_pairs.restype = ci
        lib.tj_sort_multi.argtypes = [ci, ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, vp,
                                      i64, ctypes.c_int32, vp]
        lib.tj_sort_multi.restype = ci
        lib.tj_sort.restype = ci
        lib.tj_sort_noalloc.argtypes = [ci, vp, vp, i64, vp]
        lib.tj_sort_noalloc.restype = ci
        lib.tj_join_batch.argtypes = [ci, i64, p64, p64, vp, vp, vp, vp, vp, i64, vp, p64, vp]
        lib.tj_join_batch.restype = ci
        lib.tj_autotune_batch.argtypes = [ci, i64, p64, p64, vp, vp, vp, vp, vp, i64, vp, p64, vp]
        lib.tj_autotune_batch.restype = ci
        lib.tj_status_str.argtypes = [ci]
        lib.tj_status_str.restype = ctypes.c_char_p
        lib.tj_last_error.argtypes = []
        lib.tj_last_error.restype = ctypes.c_char_p
        lib.tj_get_stats.argtypes = [ctypes.POINTER(_Stats)]
        lib.tj_get_stats.restype = ci
        lib.tj_version.argtypes = []
        lib.tj_version.restype = ctypes.c_char_p
        lib.tj_mlp_grad.argtypes = [vp, vp, vp, ci, vp, vp]
        lib.tj_mlp_grad.restype = ci
        lib.tj_mlp_adam.argtypes = [vp, vp, vp, vp, ci, ci, ctypes.c_float, vp]
        lib.tj_mlp_adam.restype = ci
        lib.tj_mlp_table.argtypes = [vp, ci, vp, ci, ci, vp, i64, vp, vp]
        lib.tj_mlp_table.restype = ci
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


def mlp_grad(theta, x, y, stream=None):
    """Gradient (1153 fp32) of the learned partitioner's network on a batch
    (tj_mlp_grad); theta, x, y are CUDA float32 tensors."""
    lib = _load()
    for t in (theta, x, y):
        if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
            raise TypeError("theta, x, y must be contiguous CUDA float32 tensors")
    g = torch.empty_like(theta)
    with torch.cuda.device(theta.device):
        _check(lib, lib.tj_mlp_grad(theta.data_ptr(), x.data_ptr(), y.data_ptr(), x.numel(),
                                    g.data_ptr(), _stream(stream)))
    return g


def mlp_adam(theta, m, v, g, t: int, lr: float, stream=None):
    """One Adam step in place on CUDA float32 tensors (tj_mlp_adam)."""
    lib = _load()
    with torch.cuda.device(theta.device):
        _check(lib, lib.tj_mlp_adam(theta.data_ptr(), m.data_ptr(), v.data_ptr(), g.data_ptr(),
                                    theta.numel(), int(t), float(lr), _stream(stream)))
    return theta, m, v


def mlp_table(theta, T: int, parts: int, sorted_sample, stream=None):
    """Monotone tabulation of the network on T + 1 grid points and the
    parts - 1 batch boundaries it gives over a sorted sample (tj_mlp_table).
    Returns (table fp32 of T + 1, boundaries of the sample's dtype)."""
    lib = _load()
    if not theta.is_cuda or theta.dtype != torch.float32 or not theta.is_contiguous():
        raise TypeError("theta must be a contiguous CUDA float32 tensor")
    _need(sorted_sample, sorted_sample.dtype, theta.device, "sorted_sample")
    table = torch.empty(T + 1, dtype=torch.float32, device=theta.device)
    bounds = torch.empty(parts - 1, dtype=sorted_sample.dtype, device=theta.device)
    with torch.cuda.device(theta.device):
        _check(lib, lib.tj_mlp_table(theta.data_ptr(), int(T), table.data_ptr(), int(parts),
                                     _dt(sorted_sample), sorted_sample.data_ptr(),
                                     sorted_sample.numel(), bounds.data_ptr(), _stream(stream)))
    return table, bounds


def version() -> str:
    return _load().tj_version().decode()


def join_inner(keys_r, ids_r, keys_s, ids_s, mem_budget_bytes: int = 0, out=None,
               stream=None, router: str | None = None, partitions: int = 0,
               sample_stride: int = 0, pla_segments: int = 0, mlp_steps: int = 0,
               mlp_batch: int = 0, mlp_lr: float = 0.0, seed: int = 0,
               radix_judge: float = 0.0, fused: bool = True):
    """Inner equi-join (paper Sec. 4.1) -> (count, 2) tensor of (r_id, s_id)
    ordered by key, then S position, then R position.

    `out`, if given, is a (capacity, 2) tensor of the id dtype that receives the
    pairs; otherwise one of n_s rows is tried first and, if the result is
    larger, the join is run again into a buffer of the exact size.  `router`
    ('auto', 'single', 'radix', 'pla', 'mlp') and the other keywords fill
    tj_join_opts (0 = library default; radix_judge < 0 keeps a learned model
    whatever the radix judge finds; fused=False sorts every batch by LSD
    passes instead of the partition-resident phase)."""
    opts = None
    if router is not None or partitions or sample_stride or pla_segments or mlp_steps or \
            mlp_batch or mlp_lr or seed or radix_judge or not fused:
        opts = _Opts(ROUTERS[router or "auto"], int(partitions), int(sample_stride),
                     int(pla_segments), int(mlp_steps), int(mlp_batch), float(mlp_lr), int(seed),
                     float(radix_judge), 0 if fused else TJ_JOIN_NO_FUSED)
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
            return lib.tj_join_inner_ex(dt, keys_r.data_ptr(), ids_r.data_ptr(), keys_r.numel(),
                                        keys_s.data_ptr(), ids_s.data_ptr(), keys_s.numel(),
                                        int(mem_budget_bytes),
                                        ctypes.byref(opts) if opts is not None else None,
                                        0 if buf is None else buf.data_ptr(),
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


SORT_PATHS = {"auto": 0, "per_column": 1, "packed": 2}


def sort_multi(cols, ids=None, stream=None, path: str = "auto"):
    """ORDER BY several key columns, cols[0] first (paper Sec. 3.2's
    multi-attribute sort key, Sec. 4.2), stable, in place.  `path`: 'auto'
    (chosen from the columns' key statistics, Sec. 3.3), 'per_column' (one
    radix sort per column carrying the row permutation) or 'packed' (the
    columns folded into one key; TjError if their bits do not fit).  Columns
    and ids: 1-D contiguous CUDA tensors of one int dtype, same length.
    Returns (cols, ids)."""
    lib = _load()
    cols = list(cols)
    if not cols:
        return cols, ids
    dt = _dt(cols[0])
    n = cols[0].numel()
    for i, c in enumerate(cols):
        _need(c, cols[0].dtype, cols[0].device, f"cols[{i}]")
        if c.numel() != n:
            raise ValueError("key columns must have the same length")
    if ids is not None:
        _need(ids, cols[0].dtype, cols[0].device, "ids")
        if ids.numel() != n:
            raise ValueError("ids must have the columns' length")
    ptrs = (ctypes.c_void_p * len(cols))(*[c.data_ptr() for c in cols])
    with torch.cuda.device(cols[0].device):
        _check(lib, lib.tj_sort_multi(dt, ptrs, len(cols), None if ids is None else ids.data_ptr(),
                                      n, SORT_PATHS[path], _stream(stream)))
    return cols, ids


def gather_pairs(pairs, r_cols=(), s_cols=(), n_r=None, n_s=None, stream=None):
    """Late materialisation (paper Sec. 3.1, Sec. 3.2): for a (n, 2) tensor of
    (r_id, s_id) pairs, as join_inner returns them, gather every column of R
    at r_id and of S at s_id.  Columns are 1-D contiguous CUDA tensors of a
    4- or 8-byte dtype, all of R's n_r rows long and all of S's n_s (n_r and
    n_s default to the columns' length).  Returns (R outputs, S outputs), lists
    of n-element tensors of the columns' dtypes."""
    lib = _load()
    if pairs.dim() != 2 or pairs.shape[1] != 2 or not pairs.is_contiguous() or not pairs.is_cuda:
        raise ValueError("pairs must be a contiguous (n, 2) CUDA tensor")
    dt = _dt(pairs)
    dev = pairs.device
    n = pairs.shape[0]
    r_cols, s_cols = list(r_cols), list(s_cols)
    sizes = {}
    for side, cols, given in ((0, r_cols, n_r), (1, s_cols, n_s)):
        rows = given if given is not None else (cols[0].numel() if cols else 0)
        for c in cols:
            if not isinstance(c, torch.Tensor) or not c.is_cuda or c.device != dev:
                raise TypeError("columns must be CUDA tensors on the pairs' device")
            if c.dim() != 1 or not c.is_contiguous() or c.numel() != rows:
                raise ValueError("columns of a side must be 1-D, contiguous and of its length")
            if c.element_size() not in (4, 8):
                raise TypeError("columns must have 4- or 8-byte elements")
        sizes[side] = rows
    outs = [torch.empty(n, dtype=c.dtype, device=dev) for c in r_cols + s_cols]
    desc = (_Column * max(1, len(outs)))()
    for i, (c, o) in enumerate(zip(r_cols + s_cols, outs)):
        desc[i] = _Column(c.data_ptr(), o.data_ptr(), 0 if i < len(r_cols) else 1,
                          c.element_size())
    with torch.cuda.device(dev):
        _check(lib, lib.tj_gather_pairs(dt, pairs.data_ptr(), n, sizes[0], sizes[1], desc,
                                        len(outs), _stream(stream)))
    return outs[:len(r_cols)], outs[len(r_cols):]


def join_batch(r_off, s_off, keys_r, ids_r, keys_s, ids_s, out=None, stream=None,
               autotune: bool = False):
    """Many independent joins stored back to back (job j: R rows
    [r_off[j], r_off[j+1]), S rows [s_off[j], s_off[j+1])).  Returns
    (pairs, out_off) with out_off a device int64 tensor of n_jobs + 1 entries.
    autotune=True runs tj_autotune_batch (times the candidate digit widths and
    tiles on this batch and caches the fastest)."""
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

        fn = lib.tj_autotune_batch if autotune else lib.tj_join_batch

        def run(buf):
            return fn(dt, nj, ro, so, keys_r.data_ptr(), ids_r.data_ptr(),
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


# ---------------------------------------------------------------------------
# serving loop (tj_server_*)
# ---------------------------------------------------------------------------
class _Req(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("dt", ctypes.c_int32), ("keys_r", ctypes.c_void_p),
                ("ids_r", ctypes.c_void_p), ("n_r", ctypes.c_int64),
                ("keys_s", ctypes.c_void_p), ("ids_s", ctypes.c_void_p),
                ("n_s", ctypes.c_int64), ("out_pairs", ctypes.c_void_p),
                ("out_capacity", ctypes.c_int64)]


class _Res(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("out_count", ctypes.c_int64),
                ("latency_ms", ctypes.c_double)]


class _SStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("tuples", ctypes.c_int64),
                ("makespan_s", ctypes.c_double), ("peak_reserved", ctypes.c_int64),
                ("peak_inflight", ctypes.c_int32), ("bypasses", ctypes.c_int64)]


def _server_lib():
    lib = _load()
    if not getattr(lib, "_srv_ready", False):
        vp, i64, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        p64 = ctypes.POINTER(ctypes.c_int64)
        lib.tj_server_create.argtypes = [ctypes.c_size_t, ci, ctypes.POINTER(vp)]
        lib.tj_server_create.restype = ci
        lib.tj_server_submit.argtypes = [vp, ctypes.POINTER(_Req), p64]
        lib.tj_server_submit.restype = ci
        lib.tj_server_replay.argtypes = [vp, ctypes.POINTER(_Req),
                                         ctypes.POINTER(ctypes.c_double), i64, p64]
        lib.tj_server_replay.restype = ci
        lib.tj_server_wait.argtypes = [vp, i64, ctypes.POINTER(_Res)]
        lib.tj_server_wait.restype = ci
        lib.tj_server_drain.argtypes = [vp]
        lib.tj_server_drain.restype = ci
        lib.tj_server_report.argtypes = [vp, ctypes.POINTER(_SStats)]
        lib.tj_server_report.restype = ci
        lib.tj_server_reset_stats.argtypes = [vp]
        lib.tj_server_reset_stats.restype = ci
        lib.tj_server_destroy.argtypes = [vp]
        lib.tj_server_destroy.restype = None
        lib._srv_ready = True
    return lib


class Server:
    """Continuous-batching server over the C ABI (tj_server_*): requests are
    admitted FIFO as workers and device memory (mem_budget_bytes) free up and
    run concurrently on the workers' streams."""

    def __init__(self, mem_budget_bytes: int, workers: int = 4):
        self._lib = _server_lib()
        h = ctypes.c_void_p()
        _check(self._lib, self._lib.tj_server_create(int(mem_budget_bytes), int(workers),
                                                     ctypes.byref(h)))
        self._h = h
        self._keep = {}

    @staticmethod
    def join_request(keys_r, ids_r, keys_s, ids_s, out=None, capacity: int = 0):
        """out=None: the server allocates `capacity` pairs (default n_s) for the
        request's output inside its reservation, counts them and releases them."""
        cap = out.shape[0] if out is not None else int(capacity or keys_s.numel())
        r = _Req(0, _dt(keys_r), keys_r.data_ptr(), ids_r.data_ptr(), keys_r.numel(),
                 keys_s.data_ptr(), ids_s.data_ptr(), keys_s.numel(),
                 out.data_ptr() if out is not None else None, cap)
        r._tensors = (keys_r, ids_r, keys_s, ids_s, out)
        return r

    @staticmethod
    def sort_request(keys, ids):
        r = _Req(1, _dt(keys), keys.data_ptr(), ids.data_ptr(), keys.numel(), None, None, 0,
                 None, 0)
        r._tensors = (keys, ids)
        return r

    def submit(self, req) -> int:
        t = ctypes.c_int64(0)
        _check(self._lib, self._lib.tj_server_submit(self._h, ctypes.byref(req), ctypes.byref(t)))
        self._keep[t.value] = req
        return t.value

    def replay(self, reqs, arrival_s):
        n = len(reqs)
        arr = (_Req * n)(*reqs)
        ts = (ctypes.c_double * n)(*[float(x) for x in arrival_s])
        tk = (ctypes.c_int64 * n)()
        _check(self._lib, self._lib.tj_server_replay(self._h, arr, ts, n, tk))
        out = list(tk)
        for t, r in zip(out, reqs):
            self._keep[t] = r
        return out

    def wait(self, ticket: int) -> dict:
        r = _Res()
        _check(self._lib, self._lib.tj_server_wait(self._h, int(ticket), ctypes.byref(r)))
        self._keep.pop(ticket, None)
        return {"status": r.status, "out_count": r.out_count, "latency_ms": r.latency_ms}

    def drain(self):
        _check(self._lib, self._lib.tj_server_drain(self._h))

    def report(self) -> dict:
        s = _SStats()
        _check(self._lib, self._lib.tj_server_report(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in _SStats._fields_}

    def reset_stats(self):
        _check(self._lib, self._lib.tj_server_reset_stats(self._h))

    def close(self):
        if self._h:
            self._lib.tj_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
