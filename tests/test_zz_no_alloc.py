"""tj_sort_noalloc: the sort for callers that cannot allocate memory when they
sort (an outer framework owns the device's memory pool, allocation-free
real-time paths, processes that must not grow device memory after start-up).
Its output must equal the regular tj_sort's, and the CPU oracle's, on two
calls in a row (the shared scratch array keeps the previous call's contents),
through the C ABI; a warmed-up call must leave the device's free memory
unchanged.  This file is collected last."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
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
        st = api.stats()
        assert st["scratch_peak"] == 0 and st["radix_passes"] >= 2
        ek, ei = oracle.sort(keys.numpy(), ids.numpy())
        assert np.array_equal(k2.cpu().numpy(), ek) and np.array_equal(i2.cpu().numpy(), ei)


def test_noalloc_call_leaves_free_device_memory_unchanged():
    dev = torch.device("cuda:0")
    g = torch.Generator().manual_seed(7)
    keys = torch.randint(-(1 << 40), 1 << 40, (300_001,), generator=g).to(dev)
    ids = torch.arange(300_001, device=dev)
    k, i = keys.clone(), ids.clone()
    _c_sort("tj_sort_noalloc", 1, k, i)  # warm-up: module and array loaded
    torch.cuda.synchronize()
    k.copy_(keys)
    i.copy_(ids)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    _c_sort("tj_sort_noalloc", 1, k, i)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert free1 == free0
    ek, ei = oracle.sort(keys.cpu().numpy(), ids.cpu().numpy())
    assert np.array_equal(k.cpu().numpy(), ek) and np.array_equal(i.cpu().numpy(), ei)


def test_noalloc_rejects_oversized_input():
    lib = api._load()
    keys = torch.zeros((1 << 20) + 1, dtype=torch.int64, device="cuda:0")
    st = lib.tj_sort_noalloc(1, keys.data_ptr(), keys.data_ptr(), keys.numel(), None)
    assert st == api.TJ_ERR_INVALID
    assert b"at most" in lib.tj_last_error()
