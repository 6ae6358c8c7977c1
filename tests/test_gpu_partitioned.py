"""GPU parity of the partitioned (multi-pass) join: key-range batches from
equal-width ranges (radix) or sample quantiles (PLA), grouped under a device
memory budget.  Whatever the router and the budget, the result must equal the
oracle's byte for byte; the working set must stay within the budget."""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_21237_gb300 import api, datagen
from gpu_util import DEV, assert_pairs_equal

pytestmark = pytest.mark.gpu


def check(kr, ir, ks, is_, **kw):
    got = api.join_inner(kr.to(DEV), ir.to(DEV), ks.to(DEV), is_.to(DEV), **kw)
    exp = oracle.join_inner(kr.numpy(), ir.numpy(), ks.numpy(), is_.numpy())
    assert_pairs_equal(got, exp)
    return api.stats()


@pytest.mark.parametrize("router", ["radix", "pla"])
@pytest.mark.parametrize("dtype", [torch.int32, torch.int64])
def test_router_unbounded(router, dtype):
    kr, ir, ks, is_ = datagen.uniform_pair(200_000, 300_003, -50_000, 150_000, 31, dtype)
    st = check(kr, ir, ks, is_, router=router)
    assert st["partitions"] > 1 and st["groups"] == 1
    # uniform keys: the radix judge replaces the piecewise-linear model
    assert st["learned"] == (api.ROUTERS["pla"] + 100 if router == "pla" else api.ROUTERS["radix"])
    st = check(kr, ir, ks, is_, router=router, radix_judge=-1)  # the cut table routes
    assert st["learned"] == api.ROUTERS[router]


def test_radix_judge_replaces_a_model_no_better_than_equal_ranges():
    # uniform keys: equal-width ranges are within the judge's factor of
    # perfect balance, so no model is fitted (learned_balance 0) and both
    # routers fall back to radix (+100); the result is the same.
    kr, ir, ks, is_ = datagen.uniform_pair(150_000, 250_007, -(1 << 40), 1 << 40, 37, torch.int64)
    m = (150_000 + 250_007) // 100  # the 1% sample; 128 ranges, 3-sigma allowance
    noise = 3 / np.sqrt(m / 128)
    for router in ("pla", "mlp"):
        st = check(kr, ir, ks, is_, router=router, partitions=128)
        assert st["learned"] == api.ROUTERS[router] + 100
        assert st["learned_balance"] == 0 and st["radix_balance"] <= 1.25 + noise
        assert st["heavy_keys"] == 0 and st["partitions"] == 128
    # a judge factor below the uniform keys' sampled balance makes the model
    # fit; an MLP trained for one step fits nothing and still falls back
    st = check(kr, ir, ks, is_, router="mlp", partitions=128, mlp_steps=1, radix_judge=0.5)
    assert st["learned_balance"] > 0
    assert st["learned"] == api.ROUTERS["mlp"] + 100
    assert st["radix_balance"] <= 0.5 * st["learned_balance"] + noise


def test_radix_judge_keeps_a_model_that_balances_better():
    # log-normal clusters: equal-width ranges put most rows in a few batches
    kr, ir = datagen.lognormal_mix(1 << 17, 53)
    ks, is_ = datagen.lognormal_mix(1 << 17, 54)
    st = check(kr, ir, ks, is_, router="pla", partitions=128)
    assert st["learned"] == api.ROUTERS["pla"]
    assert st["radix_balance"] > 1.25 * st["learned_balance"]
    # heavy keys isolated by the model's cuts do not count against it
    kr, ir, ks, is_ = datagen.fk_zipf(100_000, 400_000, 1.2, 55)
    st = check(kr, ir, ks, is_, router="pla", partitions=128)
    assert st["learned"] == api.ROUTERS["pla"] and st["heavy_keys"] >= 1


@pytest.mark.parametrize("router", ["radix", "pla"])
def test_route_regions_sampled_or_histogram(router):
    # learned routers size the batch regions from their sample; equal-width
    # ranges take a route histogram
    kr, ir, ks, is_ = datagen.uniform_pair(200_000, 300_003, 0, 1 << 20, 33, torch.int64)
    st = check(kr, ir, ks, is_, router=router, partitions=64)
    assert st["route_regions"] == (2 if router == "pla" else 1)


def test_1024_learned_batches_take_sampled_regions():
    # 1024 batches also take their regions from the sample (the cut-table
    # route then searches each row's batch again when it writes the row)
    kr, ir = datagen.lognormal_mix(1 << 18, 35)
    ks, is_ = datagen.lognormal_mix(1 << 18, 36)
    st = check(kr, ir, ks, is_, router="pla", partitions=1024)
    assert st["learned"] == api.ROUTERS["pla"] and st["partitions"] > 900
    assert st["route_regions"] in (2, 3)


@pytest.mark.parametrize("parts", [64, 1024])
@pytest.mark.parametrize("dtype", [torch.int32, torch.int64])
def test_sampled_regions_fall_back_to_exact_routing(dtype, parts):
    # the keys at the sampled positions are all small, the others large: the
    # sample gives the large-key batch almost no room, the route pass reports
    # the overflow and the join is routed again with exact batch sizes
    n, stride, seed = 200_000, 10, 5
    off_r = (((seed * 0x9E3779B97F4A7C15) % (1 << 64)) >> 33) % stride
    off_s = (((seed * 0xBF58476D1CE4E5B9) % (1 << 64)) >> 33) % stride
    g = torch.Generator().manual_seed(3)
    kr = torch.randint(1 << 20, 1 << 21, (n,), generator=g)
    ks = torch.randint(1 << 20, 1 << 21, (n,), generator=g)
    kr[off_r::stride] = torch.randint(0, 1000, (len(range(off_r, n, stride)),), generator=g)
    ks[off_s::stride] = torch.randint(0, 1000, (len(range(off_s, n, stride)),), generator=g)
    kr, ks = kr.to(dtype), ks.to(dtype)
    ir = torch.arange(n, dtype=dtype)
    is_ = torch.arange(n, dtype=dtype)
    st = check(kr, ir, ks, is_, router="pla", partitions=parts, sample_stride=stride, seed=seed,
               radix_judge=-1)
    assert st["route_regions"] == 3


@pytest.mark.parametrize("s", [0.0, 1.2])
def test_pla_budgeted_fk_zipf(s):
    kr, ir, ks, is_ = datagen.fk_zipf(200_000, 800_000, s, 41)
    budget = 6 << 20
    # the LSD path: every batch needs a sort buffer, so the budget makes groups
    st = check(kr, ir, ks, is_, mem_budget_bytes=budget, router="pla", partitions=256,
               fused=False)
    assert st["groups"] > 1
    assert st["scratch_peak"] <= budget
    st = check(kr, ir, ks, is_, mem_budget_bytes=budget, router="pla", partitions=256)
    assert st["fused_batches"] > 0 and st["scratch_peak"] <= budget
    if s > 1.0:
        assert st["heavy_keys"] >= 1  # the hottest keys get batches of their own


def test_auto_switches_to_partitioned_under_budget():
    kr, ir, ks, is_ = datagen.fk_zipf(300_000, 900_000, 0.8, 43)
    st = check(kr, ir, ks, is_, mem_budget_bytes=8 << 20, fused=False)
    assert st["learned"] % 100 == api.ROUTERS["pla"] and st["groups"] > 1
    assert st["scratch_peak"] <= 8 << 20
    st = check(kr, ir, ks, is_)  # unbounded: single pass
    assert st["partitions"] == 0


def test_pla_many_to_many_and_wide_keys():
    g = torch.Generator().manual_seed(12)
    base = torch.randint(-(1 << 62), 1 << 62, (3000,), generator=g, dtype=torch.int64)
    kr = base[torch.randint(0, 3000, (60000,), generator=g)]
    ks = base[torch.randint(0, 3000, (40000,), generator=g)]
    ir = torch.arange(60000, dtype=torch.int64)
    is_ = torch.arange(40000, dtype=torch.int64) * 7
    check(kr, ir, ks, is_, router="pla", partitions=64)
    check(kr, ir, ks, is_, router="radix", partitions=64)


def test_lognormal_pla_balances_better_than_radix():
    kr, ir = datagen.lognormal_mix(1 << 18, 51)
    ks, is_ = datagen.lognormal_mix(1 << 18, 52)
    sp = check(kr, ir, ks, is_, router="pla", partitions=256)
    sr = check(kr, ir, ks, is_, router="radix", partitions=256)
    assert sp["balance"] < 2.5
    assert sr["balance"] > 3 * sp["balance"]
    assert sp["radix_balance"] > 3 * sp["balance"]


def test_budget_too_small_is_reported():
    kr, ir, ks, is_ = datagen.uniform_pair(100_000, 100_000, 0, 1 << 20, 3, torch.int64)
    with pytest.raises(api.TjError) as ei:
        api.join_inner(kr.to(DEV), ir.to(DEV), ks.to(DEV), is_.to(DEV), mem_budget_bytes=4096,
                       router="pla")
    assert ei.value.status == api.TJ_ERR_BUDGET


def test_single_router_respects_budget():
    kr, ir, ks, is_ = datagen.uniform_pair(100_000, 100_000, 0, 1 << 20, 3, torch.int64)
    with pytest.raises(api.TjError) as ei:
        api.join_inner(kr.to(DEV), ir.to(DEV), ks.to(DEV), is_.to(DEV), mem_budget_bytes=1 << 20,
                       router="single")
    assert ei.value.status == api.TJ_ERR_BUDGET


def test_groups_alternate_between_two_lanes():
    # several groups under the budget: groups alternate between two streams,
    # each with half of the budget's working set; the pairs of a group follow
    # the previous group's, whichever stream ran it
    kr, ir, ks, is_ = datagen.fk_zipf(200_000, 800_000, 0.8, 47)
    budget = 6 << 20
    st = check(kr, ir, ks, is_, mem_budget_bytes=budget, router="pla", partitions=256,
               fused=False)
    assert st["groups"] >= 4 and st["lanes"] == 2
    assert st["scratch_peak"] <= budget
    st = check(kr, ir, ks, is_, router="pla", partitions=256, fused=False)  # one group
    assert st["groups"] == 1 and st["lanes"] == 1


def test_two_lanes_many_to_many_on_a_side_stream():
    # many matches per key across groups, called on a stream that is still
    # writing the inputs: the second lane must wait for the caller's stream
    g = torch.Generator().manual_seed(14)
    n = 400_000
    kr = torch.randint(0, 50_000, (n,), generator=g, dtype=torch.int64)
    ks = torch.randint(0, 50_000, (n,), generator=g, dtype=torch.int64)
    ir = torch.arange(n, dtype=torch.int64)
    is_ = torch.arange(n, dtype=torch.int64) * 3
    exp = oracle.join_inner(kr.numpy(), ir.numpy(), ks.numpy(), is_.numpy())
    s = torch.cuda.Stream()
    h = [t.pin_memory() for t in (kr, ir, ks, is_)]
    with torch.cuda.stream(s):
        d = [torch.empty_like(t, device=DEV) for t in h]
        for dst, src in zip(d, h):
            dst.copy_(src, non_blocking=True)
        got = api.join_inner(*d, mem_budget_bytes=6 << 20, router="pla", partitions=128,
                             fused=False)
        st = api.stats()
    s.synchronize()
    assert st["groups"] > 1 and st["lanes"] == 2
    assert_pairs_equal(got, exp)


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64])
def test_keys_outside_the_sample_range_without_key_statistics(dtype):
    # one sorted copy exceeds the budget, so the join routes by the sample's
    # range (no statistics pass); the extreme keys are never sampled and must
    # still reach the first and the last batch, whose ranges come from the
    # route pass itself
    n, stride, seed = 200_000, 10, 5
    off_r = (((seed * 0x9E3779B97F4A7C15) % (1 << 64)) >> 33) % stride
    off_s = (((seed * 0xBF58476D1CE4E5B9) % (1 << 64)) >> 33) % stride
    info = torch.iinfo(dtype)
    g = torch.Generator().manual_seed(8)
    kr = torch.randint(0, 1 << 20, (n,), generator=g, dtype=dtype)
    ks = torch.randint(0, 1 << 20, (n,), generator=g, dtype=dtype)
    far = (1 << 50) if dtype == torch.int64 else (1 << 29)
    for side_k, off in ((kr, off_r), (ks, off_s)):
        side_k[off + 1] = info.min
        side_k[off + 2] = info.max
        side_k[off + 3] = -far
        side_k[off + 4] = far
    ir = torch.arange(n, dtype=dtype)
    is_ = torch.arange(n, dtype=dtype)
    for fused in (False, True):
        st = check(kr, ir, ks, is_, mem_budget_bytes=4 << 20, router="pla", partitions=64,
                   sample_stride=stride, seed=seed, fused=fused)
        assert st["scratch_peak"] <= 4 << 20
        assert st["groups"] > 1 or fused
    assert st["key_bits"] == (64 if dtype == torch.int64 else 32)


def test_radix_judge_on_a_sample_range_plans_batches_by_their_width():
    # AUTO under a budget routes by the sample's range (no statistics pass);
    # the judge takes equal-width ranges for these uniform keys, and a key
    # range that is not a power of two leaves the top ranges empty: the exact
    # range must come from the last non-empty batch, so every batch is sorted
    # over its own 13 bits (two passes), not over 64
    kr, ir, ks, is_ = datagen.fk_zipf(600_000, 2_400_000, 0.0, 57)
    st = check(kr, ir, ks, is_, mem_budget_bytes=16 << 20, fused=False)
    assert st["learned"] == api.ROUTERS["pla"] + 100
    assert st["partitions"] == 128 and st["groups"] > 1
    assert st["radix_passes"] == 2 and st["digit_bits"] <= 7
    assert st["key_bits"] == 20  # keys 0 .. 599_999


def test_auto_chooses_the_path_from_scale_and_key_range():
    # no budget: 7e7 rows whose 24-bit key range gives batches the
    # partition-resident phase joins -> partitioned; the same scale with
    # 40-bit log-normal keys -> one pass.  Either way the bytes equal the
    # single pass's (itself checked against the oracle elsewhere).
    kr, ir, ks, is_ = datagen.fk_zipf(14_000_000, 56_000_000, 0.8, 59, device="cuda")
    auto = api.join_inner(kr, ir, ks, is_)
    st = api.stats()
    assert st["partitions"] > 0 and st["fused_batches"] > 0
    assert torch.equal(auto, api.join_inner(kr, ir, ks, is_, router="single"))
    del kr, ir, ks, is_, auto
    kr, ir = datagen.lognormal_mix(1 << 25, 61, device="cuda")
    ks, is_ = datagen.lognormal_mix(1 << 25, 62, device="cuda")
    auto = api.join_inner(kr, ir, ks, is_)
    assert api.stats()["partitions"] == 0
    assert torch.equal(auto, api.join_inner(kr, ir, ks, is_, router="single"))
