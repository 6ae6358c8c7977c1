"""GPU parity of tj_sort (stable ORDER BY key, in place) against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_21237_gb300 import api
from gpu_util import DEV, np_of

pytestmark = pytest.mark.gpu


def check(keys, ids):
    k, i = keys.to(DEV), ids.to(DEV)
    api.sort(k, i)
    ek, ei = oracle.sort(keys.numpy(), ids.numpy())
    assert np.array_equal(np_of(k), ek)
    assert np.array_equal(np_of(i), ei)


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64])
@pytest.mark.parametrize("n", [1, 2, 3071, 3072, 3073, 3839, 3840, 3841, 4095, 4096, 4097, 6145,
                               7681, 100003, 1_000_000])
@pytest.mark.parametrize("dist", ["full", "narrow", "dups"])
def test_sort_matches_oracle(dtype, n, dist):
    info = torch.iinfo(dtype)
    g = torch.Generator().manual_seed(n)
    if dist == "full":
        keys = torch.randint(info.min, info.max, (n,), generator=g, dtype=torch.int64)
    elif dist == "narrow":
        keys = torch.randint(-(1 << 20), 1 << 20, (n,), generator=g, dtype=torch.int64)
    else:
        keys = torch.randint(0, 7, (n,), generator=g, dtype=torch.int64)
    keys = keys.to(dtype)
    ids = torch.arange(n, dtype=dtype)
    check(keys, ids)


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64])
def test_sort_edge_keys(dtype):
    info = torch.iinfo(dtype)
    keys = torch.tensor([info.max, info.min, 0, -1, 1, info.min, info.max] * 1000, dtype=dtype)
    ids = torch.arange(keys.numel(), dtype=dtype) * -3
    check(keys, ids)


def test_sort_all_equal_and_empty():
    keys = torch.full((10000,), 42, dtype=torch.int64)
    ids = torch.arange(10000, dtype=torch.int64).flip(0)
    check(keys, ids)
    assert api.stats()["radix_passes"] == 0
    e = torch.zeros(0, dtype=torch.int32, device=DEV)
    api.sort(e, e)


def test_sort_even_pass_count_lands_in_place():
    keys = torch.randint(0, 1 << 27, (300000,), dtype=torch.int64)
    ids = torch.arange(300000, dtype=torch.int64)
    check(keys, ids)
    st = api.stats()
    assert st["radix_passes"] % 2 == 0 and st["key_bits"] == 27


@pytest.mark.parametrize("dtype,bits,digit", [(torch.int32, 20, 10), (torch.int32, 18, 9),
                                              (torch.int32, 16, 8), (torch.int64, 18, 9),
                                              (torch.int64, 16, 8), (torch.int64, 14, 7)])
def test_sort_digit_widths_with_colliding_digits(dtype, bits, digit):
    """Every digit width of the warp ranking (7 bits through its lane-mask table,
    wider ones with a ballot per higher bit), on keys from 40 values so that
    many lanes of a warp share a digit, ids in reverse order so that a wrong
    tie order shows."""
    n = 50_000
    g = torch.Generator().manual_seed(bits * 10 + digit)
    vals = torch.randint(0, 1 << bits, (40,), generator=g, dtype=torch.int64)
    vals[0] = (1 << bits) - 1
    vals[1] = 0
    keys = vals[torch.randint(0, 40, (n,), generator=g)].to(dtype)
    ids = torch.arange(n, dtype=dtype).flip(0)
    check(keys, ids)
    st = api.stats()
    assert st["key_bits"] == bits and st["digit_bits"] == digit
