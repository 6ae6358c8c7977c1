"""GPU parity of the partition-resident phase of the partitioned join: batches
whose key range spans 10 to 20 bits are cut by one MSD pass into sub-batches
of 1024 key values, each sorted and aligned on chip (one CTA per tile of at
most 4608 S rows; larger sub-batches are split into tiles that share per-key
counts).  The result must equal the oracle's byte for byte, and the LSD path
(fused=False) must give the same bytes."""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_21237_gb300 import api, datagen
from gpu_util import DEV, assert_pairs_equal

pytestmark = pytest.mark.gpu


def run(kr, ir, ks, is_, **kw):
    d = [t.to(DEV) for t in (kr, ir, ks, is_)]
    got = api.join_inner(*d, **kw)
    return got, api.stats()


def check(kr, ir, ks, is_, **kw):
    got, st = run(kr, ir, ks, is_, **kw)
    exp = oracle.join_inner(kr.numpy(), ir.numpy(), ks.numpy(), is_.numpy())
    assert_pairs_equal(got, exp)
    return st


@pytest.mark.parametrize("s", [0.0, 0.8, 1.2])
def test_fk_zipf_under_budget(s):
    # 2^21 R keys (range 21 bits -> 128 batches of 14 bits: 4 MSD bits,
    # sub-batches of 1024 keys); Zipf 1.2 puts many S rows on a few keys, so
    # their sub-batches span many tiles
    kr, ir, ks, is_ = datagen.fk_zipf(1 << 21, 1 << 23, s, 71)
    st = check(kr, ir, ks, is_, mem_budget_bytes=48 << 20, router="radix")
    assert st["fused_batches"] > 0 and st["groups"] > 1
    assert st["scratch_peak"] <= 48 << 20
    st2 = check(kr, ir, ks, is_, mem_budget_bytes=48 << 20, router="radix", fused=False)
    assert st2["fused_batches"] == 0


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64])
def test_many_to_many_on_chip(dtype):
    # about 1.5 R rows and 3 S rows per key value: R sub-batches of ~1500 rows
    # fit on chip, every S row has one or more partners, some none
    g = torch.Generator().manual_seed(5)
    nk = 1 << 18
    kr = torch.randint(-nk, nk, (int(1.5 * 2 * nk),), generator=g).to(dtype)
    ks = torch.randint(-nk, nk, (3 * 2 * nk,), generator=g).to(dtype)
    ir = torch.arange(kr.numel(), dtype=dtype) * 3
    is_ = torch.arange(ks.numel(), dtype=dtype) - 7
    st = check(kr, ir, ks, is_, router="radix", partitions=64)
    assert st["fused_batches"] > 0


def test_r_sub_batch_too_large_falls_back_to_lsd():
    # every R key 4 times: a sub-batch of 1024 key values holds ~4096 R rows,
    # more than the 2048 kept on chip, so the batches take the LSD path
    g = torch.Generator().manual_seed(6)
    base = torch.randperm(1 << 17, generator=g).to(torch.int64)
    kr = base.repeat(4)[torch.randperm(4 << 17, generator=g)]
    ks = torch.randint(0, 1 << 17, (1 << 19,), generator=g, dtype=torch.int64)
    ir = torch.arange(kr.numel(), dtype=torch.int64)
    is_ = torch.arange(ks.numel(), dtype=torch.int64)
    st = check(kr, ir, ks, is_, router="radix", partitions=32)
    assert st["fused_batches"] == 0 and st["partitions"] == 32


def test_sub_batches_at_tile_boundaries():
    # one key value per sub-batch holds exactly 4608, 4609 and 9217 S rows
    # (one tile, two tiles with one row in the second, three tiles); the
    # other sub-batches are small, some empty on one side
    g = torch.Generator().manual_seed(7)
    kr = torch.randperm(1 << 16, generator=g).to(torch.int64) * 3  # range 18 bits
    ks = kr[torch.randint(0, kr.numel(), (50_000,), generator=g)]
    tile = 4608
    hot = torch.cat([torch.full((tile - 40,), 3 * 1000), torch.full((tile + 1,), 3 * 30_000),
                     torch.full((2 * tile + 1,), 3 * 60_000)]).to(torch.int64)
    ks = torch.cat([ks, hot])[torch.randperm(ks.numel() + hot.numel(), generator=g)]
    ks = torch.cat([ks, torch.tensor([1, 3 * 5000 + 1, 3 * (1 << 16) - 1])])  # no partners
    ir = torch.arange(kr.numel(), dtype=torch.int64)
    is_ = torch.arange(ks.numel(), dtype=torch.int64)
    st = check(kr, ir, ks, is_, router="radix", partitions=16)
    assert st["partitions"] == 16


def test_fused_and_lsd_paths_agree_on_the_learned_route():
    kr, ir, ks, is_ = datagen.fk_zipf(600_000, 2_400_000, 0.8, 73)
    a, sa = run(kr, ir, ks, is_, mem_budget_bytes=16 << 20, router="pla", radix_judge=-1)
    b, sb = run(kr, ir, ks, is_, mem_budget_bytes=16 << 20, router="pla", radix_judge=-1,
                fused=False)
    assert sa["fused_batches"] > 0 and sb["fused_batches"] == 0
    assert torch.equal(a, b)
    exp = oracle.join_inner(kr.numpy(), ir.numpy(), ks.numpy(), is_.numpy())
    assert_pairs_equal(a, exp)


def test_capacity_error_with_multi_tile_sub_batches():
    kr, ir, ks, is_ = datagen.fk_zipf(1 << 18, 1 << 21, 1.2, 75)
    d = [t.to(DEV) for t in (kr, ir, ks, is_)]
    out = torch.empty((ks.numel() - 1, 2), dtype=torch.int64, device=DEV)
    with pytest.raises(api.TjError) as ei:
        api.join_inner(*d, out=out, router="radix", partitions=64)
    assert ei.value.status == api.TJ_ERR_CAPACITY


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64])
def test_single_key_batches_are_streamed(dtype):
    # two heavy S keys the PLA cuts isolate: key 777 has four R rows (pairs
    # in S position, then R position order), key 5000 one; their batches'
    # pairs are streamed by k_cross, the rest go through the other paths
    g = torch.Generator().manual_seed(8)
    kr = torch.cat([torch.randperm(1 << 17, generator=g), torch.full((3,), 777)])
    kr = kr[torch.randperm(kr.numel(), generator=g)]
    ks = torch.cat([torch.randint(0, 1 << 17, (400_000,), generator=g),
                    torch.full((200_000,), 777), torch.full((300_001,), 5000)])
    ks = ks[torch.randperm(ks.numel(), generator=g)]
    kr, ks = kr.to(dtype), ks.to(dtype)
    ir = torch.arange(kr.numel(), dtype=dtype) * 5
    is_ = torch.arange(ks.numel(), dtype=dtype) + 11
    api.trace_reset()
    api.trace_enable(True)
    try:
        st = check(kr, ir, ks, is_, router="pla", partitions=64, radix_judge=-1)
    finally:
        api.trace_enable(False)
    assert st["heavy_keys"] >= 2
    assert api.trace_table()["cross"]["launches"] >= 1
    a, _ = run(kr, ir, ks, is_, router="pla", partitions=64, radix_judge=-1)
    b, _ = run(kr, ir, ks, is_, router="pla", partitions=64, radix_judge=-1, fused=False)
    assert torch.equal(a, b)
    # a capacity one pair short: nothing is written past it, the count is reported
    d = [t.to(DEV) for t in (kr, ir, ks, is_)]
    out = torch.empty((a.shape[0] - 1, 2), dtype=dtype, device=DEV)
    with pytest.raises(api.TjError) as ei:
        api.join_inner(*d, out=out, router="pla", partitions=64, radix_judge=-1)
    assert ei.value.status == api.TJ_ERR_CAPACITY


def test_ten_bit_msd_pass():
    # 2^22 R keys in 4 equal-width batches of 20 bits, about 2M rows each
    # (2048 per sub-batch): one 10-bit MSD pass each
    kr, ir, ks, is_ = datagen.fk_zipf(1 << 22, 1 << 22, 0.5, 77)
    st = check(kr, ir, ks, is_, router="radix", partitions=4)
    assert st["partitions"] == 4 and st["fused_batches"] == 4
    assert st["digit_bits"] == 10
