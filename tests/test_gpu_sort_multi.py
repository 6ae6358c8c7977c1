"""GPU parity of ORDER BY several key columns (paper Sec. 3.2's
multi-attribute sort key, Sec. 4.2): per-column stable radix sorts carrying
the row permutation must give exactly the oracle's stable lexicographic
order, for every column and the ids."""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_21237_gb300 import api
from gpu_util import DEV

pytestmark = pytest.mark.gpu


def _run(cols, ids, path="auto"):
    d = [c.to(DEV) for c in cols]
    di = None if ids is None else ids.to(DEV)
    api.sort_multi(d, di, path=path)
    st = api.stats()
    exp, eids = oracle.sort_multi([c.numpy() for c in cols], None if ids is None else ids.numpy())
    for g, e in zip(d, exp):
        assert np.array_equal(g.cpu().numpy(), e)
    if ids is not None:
        assert np.array_equal(di.cpu().numpy(), eids)
    return st


def _stats_packed():
    return api.stats()["packed_keys"]


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64])
@pytest.mark.parametrize("n", [2, 1000, 3841, 100_003])
def test_two_and_three_columns_with_ties(dtype, n):
    g = torch.Generator().manual_seed(n)
    lim = 1 << 30 if dtype == torch.int32 else 1 << 62
    cols = [torch.randint(-5, 5, (n,), generator=g, dtype=dtype),
            torch.randint(-lim, lim, (n,), generator=g, dtype=dtype),
            torch.randint(0, 3, (n,), generator=g, dtype=dtype)]
    ids = torch.randint(0, 1 << 20, (n,), generator=g, dtype=dtype)
    # a (nearly) full-range column: the bits do not fit one key, one sort per
    # column (a handful of rows may span fewer bits)
    wide = n >= 1000
    assert _run(cols[:2], ids)["packed_keys"] == (0 if wide else _stats_packed())
    assert _run(cols, ids)["packed_keys"] == (0 if wide else _stats_packed())
    # narrow columns: folded into one key, or forced per column
    assert _run([cols[2], cols[0]], None)["packed_keys"] == 1
    assert _run([cols[2], cols[0]], ids, path="per_column")["packed_keys"] == 0
    assert _run([cols[0], cols[2]], ids, path="packed")["packed_keys"] == 1
    if wide:
        with pytest.raises(api.TjError):
            api.sort_multi([c.to(DEV) for c in cols[:2]], None, path="packed")


def test_one_column_is_tj_sort_and_no_columns_is_a_no_op():
    g = torch.Generator().manual_seed(3)
    k = torch.randint(-100, 100, (50_001,), generator=g, dtype=torch.int64)
    i = torch.arange(50_001, dtype=torch.int64)
    a_k, a_i = k.to(DEV), i.to(DEV)
    api.sort_multi([a_k], a_i)
    b_k, b_i = api.sort(k.to(DEV), i.to(DEV))
    assert torch.equal(a_k, b_k) and torch.equal(a_i, b_i)
    assert api.sort_multi([], None) == ([], None)
