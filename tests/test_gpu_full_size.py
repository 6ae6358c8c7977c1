"""GPU parity at the benchmark's full sizes, in the configuration it times.

The oracle cannot join 5x10^8 rows within a test, so each full-size result is
checked two ways.  Exactly, against the oracle, on sampled key ranges: the
output is ordered by key, so the rows of both relations inside a range [a, b)
join to one contiguous block of it.  And everywhere, by properties that fix
the whole output: every pair's keys are equal, keys never decrease, equal
keys are ordered by S position and then R position (so no pair repeats), and
each S row appears as many times as R holds its key.  Ids are row positions
in these workloads, so a pair's keys are looked up through its ids.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_21237_gb300 import api, datagen
from gpu_util import DEV, assert_pairs_equal, np_of

pytestmark = pytest.mark.gpu

N_R, N_S, N_SORT = 10**8, 4 * 10**8, 10**8
BUDGET = 256 << 20


def check_properties(kr, ks, got):
    """The properties that fix an inner join ordered by (key, S position,
    R position), for ids that are row positions."""
    r, s = got[:, 0], got[:, 1]
    k = kr[r]
    assert torch.equal(k, ks[s]), "a pair joins rows with different keys"
    assert bool((k[1:] >= k[:-1]).all()), "keys decrease"
    tie = k[1:] == k[:-1]
    after = (s[1:] > s[:-1]) | ((s[1:] == s[:-1]) & (r[1:] > r[:-1]))
    assert bool((after | ~tie).all()), "equal keys out of (S, R) position order"
    # each S row appears once per R row with its key
    uk, cnt = torch.unique(kr, return_counts=True)
    pos = torch.searchsorted(uk, ks).clamp_(max=uk.numel() - 1)
    want = torch.where(uk[pos] == ks, cnt[pos], torch.zeros_like(cnt[pos]))
    have = torch.bincount(s, minlength=ks.numel())
    assert torch.equal(have, want), "an S row has the wrong number of pairs"
    return k


def check_slices(kr, ir, ks, is_, got, k, starts, width):
    """Exact comparison with the oracle on the key ranges [a, a + width)."""
    checked = 0
    for a in starts:
        b = a + width
        mr = (kr >= a) & (kr < b)
        ms = (ks >= a) & (ks < b)
        if int(ms.sum()) > 5_000_000:
            continue  # a hot key: its block is left to the properties
        exp = oracle.join_inner(np_of(kr[mr]), np_of(ir[mr]), np_of(ks[ms]), np_of(is_[ms]))
        lo = int(torch.searchsorted(k, torch.tensor([a], device=k.device, dtype=k.dtype)))
        hi = int(torch.searchsorted(k, torch.tensor([b], device=k.device, dtype=k.dtype)))
        assert_pairs_equal(got[lo:hi], exp)
        checked += 1
    assert checked >= len(starts) // 2


@pytest.mark.parametrize("s", [0.0, 0.8, 1.2])
def test_fk_join_1e8x4e8_budgeted(s):
    """The benchmark's join: R = 10^8 unique int64 keys, S = 4x10^8 foreign
    keys of Zipf skew s, a 256 MiB budget (route pass, groups on two lanes)."""
    kr, ir, ks, is_ = datagen.fk_zipf(N_R, N_S, s, datagen.BASE_SEED + 1, device=DEV)
    out = torch.empty((N_S, 2), dtype=torch.int64, device=DEV)
    got = api.join_inner(kr, ir, ks, is_, mem_budget_bytes=BUDGET, out=out)
    st = api.stats()
    assert got.shape[0] == N_S  # every S key is in R once
    assert st["scratch_peak"] <= BUDGET and st["groups"] > 1 and st["lanes"] == 2
    k = check_properties(kr, ks, got)
    g = torch.Generator().manual_seed(11)
    starts = torch.randint(0, N_R - (1 << 16), (8,), generator=g).tolist()
    check_slices(kr, ir, ks, is_, got, k, starts, 1 << 16)


def test_sort_1e8_int64():
    """The benchmark's sort: 10^8 int64 keys (a permutation of 27-bit values),
    ids are positions; then the same keys with every value 16 times.  Keys in
    order, each key where its id says, ids a permutation and stable: that is
    the stable sort; key ranges are compared with the oracle as well."""
    kr, ir, _, _ = datagen.fk_zipf(N_SORT, 1000, 0.0, datagen.BASE_SEED + 1, device=DEV)
    for src in (kr, kr // 16):
        keys = src.clone()
        ids = ir.clone()
        api.sort(keys, ids)
        assert bool((keys[1:] >= keys[:-1]).all())
        assert torch.equal(keys, src[ids])
        tie = keys[1:] == keys[:-1]
        assert bool(((ids[1:] > ids[:-1]) | ~tie).all()), "not stable"
        assert torch.equal(torch.bincount(ids, minlength=N_SORT),
                           torch.ones(N_SORT, dtype=torch.int64, device=DEV))
        # the oracle on key ranges: their rows form one block of the output
        g = torch.Generator().manual_seed(3)
        for a in torch.randint(0, int(src.max()) - 4096, (8,), generator=g).tolist():
            m = (src >= a) & (src < a + 4096)
            ek, ei = oracle.sort(np_of(src[m]), np_of(ir[m]))
            t = torch.tensor([a, a + 4096], device=DEV, dtype=keys.dtype)
            lo, hi = torch.searchsorted(keys, t).tolist()
            assert np.array_equal(np_of(keys[lo:hi]), ek)
            assert np.array_equal(np_of(ids[lo:hi]), ei)


def test_lognormal_2e28_pla_under_1gb():
    """The learned-partitioner workload: 2^28 int64 keys per side from a
    log-normal mixture (many-to-many), PLA router, 1024 batches, 1 GB budget."""
    n = 1 << 28
    kr, ir = datagen.lognormal_mix(n, 20260223, device=DEV)
    ks, is_ = datagen.lognormal_mix(n, 20260233, device=DEV)
    out = torch.empty((2 * n, 2), dtype=torch.int64, device=DEV)
    got = api.join_inner(kr, ir, ks, is_, mem_budget_bytes=1 << 30, out=out, router="pla",
                         partitions=1024)
    st = api.stats()
    assert st["scratch_peak"] <= 1 << 30 and st["groups"] > 1
    k = check_properties(kr, ks, got)
    g = torch.Generator().manual_seed(5)
    pick = torch.randint(0, got.shape[0], (8,), generator=g).to(DEV)
    starts = k[pick].tolist()
    check_slices(kr, ir, ks, is_, got, k, starts, 1 << 10)


def batch_as_one_join(r_off, s_off, kr, ks, got, out_off):
    """A batch of joins seen as one join: each row's key becomes (job, key)
    and each id a global row position, so check_properties applies."""
    nj = len(r_off) - 1
    dev = kr.device
    jobs = torch.arange(nj, device=dev, dtype=torch.int64)
    nr = torch.tensor(r_off, device=dev).diff()
    ns = torch.tensor(s_off, device=dev).diff()
    kr64 = (jobs.repeat_interleave(nr) << 32) | kr.to(torch.int64)
    ks64 = (jobs.repeat_interleave(ns) << 32) | ks.to(torch.int64)
    pj = jobs.repeat_interleave(out_off.diff())  # job of each pair
    r0 = torch.tensor(r_off[:-1], device=dev)[pj]
    s0 = torch.tensor(s_off[:-1], device=dev)[pj]
    glob = torch.stack([r0 + got[:, 0].to(torch.int64), s0 + got[:, 1].to(torch.int64)], 1)
    return kr64, ks64, glob


def test_batched_4096_joins_full_size():
    """The batched workload: 4096 int32 joins, |R| and |S| log-uniform in
    [10^3, 10^6], keys uniform over [0, 2|R|), one batched call.  The whole
    batch is checked by the join properties (keys made (job, key)), eight
    sampled jobs byte for byte against the oracle."""
    r_off, s_off, kr, ir, ks, is_ = datagen.batch_jobs(4096, 1e3, 1e6, 20260224, device=DEV)
    out = torch.empty((s_off[-1] * 2, 2), dtype=torch.int32, device=DEV)
    got, out_off = api.join_batch(r_off, s_off, kr, ir, ks, is_, out=out)
    assert int(out_off[-1]) == got.shape[0]
    kr64, ks64, glob = batch_as_one_join(r_off, s_off, kr, ks, got, out_off)
    check_properties(kr64, ks64, glob)
    oo = out_off.tolist()
    g = torch.Generator().manual_seed(17)
    for j in torch.randint(0, 4096, (8,), generator=g).tolist():
        a, b, c, d = r_off[j], r_off[j + 1], s_off[j], s_off[j + 1]
        exp = oracle.join_inner(np_of(kr[a:b]), np_of(ir[a:b]), np_of(ks[c:d]), np_of(is_[c:d]))
        assert_pairs_equal(got[oo[j]:oo[j + 1]], exp)
