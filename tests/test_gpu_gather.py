"""GPU parity of the late materialisation of payload columns (paper Sec. 3.1,
Sec. 3.2): after a join on B of R(A, B, C) and S(B, D, E), the other columns
are gathered through the (r_id, s_id) pairs; every output must equal the
oracle's byte for byte."""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_21237_gb300 import api, datagen
from gpu_util import DEV

pytestmark = pytest.mark.gpu


def _cols(n, seed):
    g = torch.Generator().manual_seed(seed)
    return [torch.randint(-(1 << 62), 1 << 62, (n,), generator=g, dtype=torch.int64),
            torch.randint(-(1 << 30), 1 << 30, (n,), generator=g, dtype=torch.int32),
            torch.randn(n, generator=g, dtype=torch.float32),
            torch.randn(n, generator=g, dtype=torch.float64)]


def _check(pairs, rc, sc):
    got_r, got_s = api.gather_pairs(pairs, [c.to(DEV) for c in rc], [c.to(DEV) for c in sc])
    p = pairs.cpu().numpy()
    exp_r, exp_s = oracle.gather_pairs(p, [c.numpy() for c in rc], [c.numpy() for c in sc])
    for g, e in zip(got_r + got_s, exp_r + exp_s):
        assert g.dtype == torch.from_numpy(e).dtype
        assert np.array_equal(g.cpu().numpy().view(np.uint8), e.view(np.uint8))


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64])
def test_payload_of_fk_join(dtype):
    n_r, n_s = 50_000, 200_003
    kr, ir, ks, is_ = datagen.fk_zipf(n_r, n_s, 0.8, 61, dtype=dtype)
    pairs = api.join_inner(kr.to(DEV), ir.to(DEV), ks.to(DEV), is_.to(DEV))
    assert pairs.shape[0] == n_s
    _check(pairs, _cols(n_r, 1), _cols(n_s, 2))


def test_many_to_many_and_more_columns_than_one_launch_takes():
    g = torch.Generator().manual_seed(5)
    kr = torch.randint(0, 300, (3000,), generator=g, dtype=torch.int64)
    ks = torch.randint(0, 300, (2000,), generator=g, dtype=torch.int64)
    pairs = api.join_inner(kr.to(DEV), torch.arange(3000, device=DEV),
                           ks.to(DEV), torch.arange(2000, device=DEV))
    rc = [c for s in range(3) for c in _cols(3000, 10 + s)]  # 12 R columns
    sc = [c for s in range(2) for c in _cols(2000, 20 + s)]  # 8 S columns
    _check(pairs, rc, sc)


def test_empty_pairs_and_no_columns():
    pairs = torch.empty((0, 2), dtype=torch.int64, device=DEV)
    r, s = api.gather_pairs(pairs, [torch.arange(4, device=DEV)], [])
    assert r[0].numel() == 0 and s == []
    pairs = torch.tensor([[1, 2]], dtype=torch.int64, device=DEV)
    assert api.gather_pairs(pairs, [], []) == ([], [])


def test_out_of_range_and_misaligned_are_rejected():
    col = torch.arange(10, dtype=torch.int64, device=DEV)
    for bad in ([[10, 0]], [[0, -1]]):
        with pytest.raises(api.TjError) as ei:
            api.gather_pairs(torch.tensor(bad, dtype=torch.int64, device=DEV), [col], [col])
        assert ei.value.status == api.TJ_ERR_INVALID
    flat = torch.zeros(9, dtype=torch.int64, device=DEV)
    with pytest.raises(api.TjError) as ei:
        api.gather_pairs(flat[1:].view(4, 2), [col], [])  # pairs off their 16-byte grid
    assert ei.value.status == api.TJ_ERR_INVALID
