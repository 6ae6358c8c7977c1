"""tj_sort_noalloc: the sort for callers that cannot allocate device memory
(an outer framework owns the pool, allocation-free real-time paths, processes
that must not grow device memory after start-up).  Its output must equal the
regular tj_sort's on two calls in a row (the shared scratch array keeps the
previous call's contents), through the C ABI.  This file is collected last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2602_21237_gb300 import api

pytestmark = pytest.mark.gpu


def _c_sort(fn, dt, keys, ids):
    lib = api._load()
    st = getattr(lib, fn)(dt, keys.data_ptr(), ids.data_ptr(), keys.numel(),
                          torch.cuda.current_stream().cuda_stream)
    assert st == 0, lib.tj_last_error().decode()


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64])
def test_noalloc_sort_equals_tj_sort_twice(dtype):
    dev = torch.device("cuda:0")
    dt = 0 if dtype == torch.int32 else 1
    info = torch.iinfo(dtype)
    g = torch.Generator().manual_seed(2026)
    for n in (1 << 20, 123_457):  # two calls in a row, the second smaller
        keys = torch.randint(info.min, info.max, (n,), generator=g, dtype=torch.int64).to(dtype)
        keys[: n // 4] = keys[0]  # duplicates: checks stability too
        ids = torch.arange(n, dtype=dtype)
        k1, i1 = keys.to(dev), ids.to(dev)
        k2, i2 = keys.to(dev), ids.to(dev)
        _c_sort("tj_sort", dt, k1, i1)
        _c_sort("tj_sort_noalloc", dt, k2, i2)
        torch.cuda.synchronize()
        assert torch.equal(k1, k2) and torch.equal(i1, i2)


def test_noalloc_rejects_oversized_input():
    lib = api._load()
    keys = torch.zeros((1 << 20) + 1, dtype=torch.int64, device="cuda:0")
    st = lib.tj_sort_noalloc(1, keys.data_ptr(), keys.data_ptr(), keys.numel(), None)
    assert st == api.TJ_ERR_INVALID
    assert b"at most" in lib.tj_last_error()
