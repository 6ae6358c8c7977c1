"""GPU parity of tj_join_batch (many joins in one graph) against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_21237_gb300 import api, datagen
from gpu_util import DEV, assert_pairs_equal, np_of

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_jobs,lo,hi", [(1, 10, 10), (37, 10, 5000), (300, 1000, 20000)])
def test_batch_matches_oracle(n_jobs, lo, hi):
    r_off, s_off, kr, ir, ks, is_ = datagen.batch_jobs(n_jobs, lo, hi, datagen.BASE_SEED + 3)
    pairs, off = api.join_batch(r_off, s_off, kr.to(DEV), ir.to(DEV), ks.to(DEV), is_.to(DEV))
    exp, eoff = oracle.join_batch(np.array(r_off), np.array(s_off), kr.numpy(), ir.numpy(),
                                  ks.numpy(), is_.numpy())
    assert np.array_equal(np_of(off), eoff)
    assert_pairs_equal(pairs, exp)


def test_batch_edge_jobs():
    # jobs with empty R, empty S, disjoint ranges, all-equal keys, one row
    parts_r = [np.array([], np.int32), np.arange(5, dtype=np.int32), np.arange(100, 200, dtype=np.int32),
               np.full(30, 9, np.int32), np.array([3], np.int32), np.arange(7000, dtype=np.int32) % 50]
    parts_s = [np.arange(4, dtype=np.int32), np.array([], np.int32), np.arange(300, 400, dtype=np.int32),
               np.full(20, 9, np.int32), np.array([3], np.int32), np.arange(9000, dtype=np.int32) % 77]
    r_off = np.concatenate([[0], np.cumsum([len(p) for p in parts_r])])
    s_off = np.concatenate([[0], np.cumsum([len(p) for p in parts_s])])
    kr = np.concatenate(parts_r).astype(np.int32)
    ks = np.concatenate(parts_s).astype(np.int32)
    ir = np.concatenate([np.arange(len(p)) for p in parts_r]).astype(np.int32)
    is_ = np.concatenate([np.arange(len(p)) * 10 for p in parts_s]).astype(np.int32)
    pairs, off = api.join_batch(r_off.tolist(), s_off.tolist(), torch.from_numpy(kr).to(DEV),
                                torch.from_numpy(ir).to(DEV), torch.from_numpy(ks).to(DEV),
                                torch.from_numpy(is_).to(DEV))
    exp, eoff = oracle.join_batch(r_off, s_off, kr, ir, ks, is_)
    assert np.array_equal(np_of(off), eoff)
    assert_pairs_equal(pairs, exp)


def test_batch_equals_one_at_a_time():
    r_off, s_off, kr, ir, ks, is_ = datagen.batch_jobs(20, 100, 30000, 77)
    d = [x.to(DEV) for x in (kr, ir, ks, is_)]
    pairs, off = api.join_batch(r_off, s_off, *d)
    off = np_of(off)
    for j in range(20):
        one = api.join_inner(d[0][r_off[j]:r_off[j + 1]], d[1][r_off[j]:r_off[j + 1]],
                             d[2][s_off[j]:s_off[j + 1]], d[3][s_off[j]:s_off[j + 1]])
        assert torch.equal(one, pairs[off[j]:off[j + 1]])


def test_autotune_keeps_results_and_caches_choice():
    r_off, s_off, kr, ir, ks, is_ = datagen.batch_jobs(64, 1000, 20000, 91)
    d = [x.to(DEV) for x in (kr, ir, ks, is_)]
    exp, eoff = oracle.join_batch(np.array(r_off), np.array(s_off), kr.numpy(), ir.numpy(),
                                  ks.numpy(), is_.numpy())
    pairs, off = api.join_batch(r_off, s_off, *d, autotune=True)
    assert_pairs_equal(pairs, exp)
    tuned = (api.stats()["tile_rows"], api.stats()["digit_cap"])
    # 4 or 8 rows per thread of a 384-thread onesweep CTA
    assert tuned[0] in (1536, 3072) and 6 <= tuned[1] <= 10
    pairs2, off2 = api.join_batch(r_off, s_off, *d)  # uses the cached choice
    assert (api.stats()["tile_rows"], api.stats()["digit_cap"]) == tuned
    assert torch.equal(pairs2, pairs) and np.array_equal(np_of(off2), eoff)
