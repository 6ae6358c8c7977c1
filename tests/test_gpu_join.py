"""GPU parity of tj_join_inner against the CPU oracle, element by element.

Output order is fixed by the API (key, then S position, then R position), so
the comparison is exact.  Sizes span several sort tiles (3072 rows) and join
tiles (4096 rows) with ragged tails; edge cases cover empty inputs, a single
row, all-equal keys (no radix pass), disjoint key ranges, extreme and negative
keys, duplicate-heavy fan-out, S sparse against R (the out-of-chip R range
path) and a too-small output buffer.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_21237_gb300 import api, datagen
from gpu_util import DEV, assert_pairs_equal, np_of

pytestmark = pytest.mark.gpu


def check(kr, ir, ks, is_, **kw):
    got = api.join_inner(kr.to(DEV), ir.to(DEV), ks.to(DEV), is_.to(DEV), **kw)
    exp = oracle.join_inner(kr.numpy(), ir.numpy(), ks.numpy(), is_.numpy())
    assert_pairs_equal(got, exp)
    return got


def test_uniform_int32_1e6_full_size():
    # R and S of 1e6 rows, int32 keys uniform in [0, 2^20), ids = positions
    kr, ir, ks, is_ = datagen.uniform_pair(10**6, 10**6, 0, 1 << 20, datagen.BASE_SEED,
                                           torch.int32)
    got = check(kr, ir, ks, is_)
    assert api.stats()["radix_passes"] >= 1
    assert 800_000 < got.shape[0] < 1_100_000


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64])
@pytest.mark.parametrize("nr,ns", [(1, 1), (1, 5000), (4097, 1), (2047, 2049), (3072, 3073),
                                   (4096, 4096), (4097, 12289), (100003, 77777)])
def test_ragged_sizes(dtype, nr, ns):
    dom = max(4, (nr + ns) // 2)
    kr, ir, ks, is_ = datagen.uniform_pair(nr, ns, -dom, dom, 17 + nr + ns, dtype)
    check(kr, ir, ks, is_)


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64])
def test_full_width_keys(dtype):
    info = torch.iinfo(dtype)
    g = torch.Generator().manual_seed(5)
    base = torch.randint(info.min, info.max, (20000,), generator=g, dtype=torch.int64).to(dtype)
    kr = base[torch.randint(0, 20000, (30000,), generator=g)]
    ks = base[torch.randint(0, 20000, (50000,), generator=g)]
    kr[:3] = torch.tensor([info.min, info.max, 0], dtype=dtype)
    ks[:3] = torch.tensor([info.max, info.min, -1], dtype=dtype)
    ir = torch.arange(30000, dtype=dtype)
    is_ = torch.arange(50000, dtype=dtype)
    check(kr, ir, ks, is_)
    assert api.stats()["key_bits"] == (32 if dtype == torch.int32 else 64)


def test_all_equal_keys_no_radix_pass():
    kr = torch.full((300,), -7, dtype=torch.int64)
    ks = torch.full((500,), -7, dtype=torch.int64)
    ir = torch.arange(300, dtype=torch.int64) * 3
    is_ = torch.arange(500, dtype=torch.int64) * 5
    got = check(kr, ir, ks, is_)
    assert got.shape[0] == 150000
    assert api.stats()["radix_passes"] == 0


def test_disjoint_and_empty():
    kr = torch.arange(0, 10000, 2, dtype=torch.int32)
    ks = torch.arange(20000, 30000, 2, dtype=torch.int32)
    ids = torch.arange(5000, dtype=torch.int32)
    assert api.join_inner(kr.to(DEV), ids.to(DEV), ks.to(DEV), ids.to(DEV)).shape[0] == 0
    e = torch.zeros(0, dtype=torch.int32, device=DEV)
    assert api.join_inner(e, e, ks.to(DEV), ids.to(DEV)).shape[0] == 0
    assert api.join_inner(kr.to(DEV), ids.to(DEV), e, e).shape[0] == 0
    # interleaved, never equal
    ks2 = torch.arange(1, 10001, 2, dtype=torch.int32)
    check(kr, ids, ks2, ids)


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64])
def test_duplicate_fanout(dtype):
    g = torch.Generator().manual_seed(3)
    kr = torch.randint(0, 40, (6000,), generator=g).to(dtype)
    ks = torch.randint(0, 40, (9000,), generator=g).to(dtype)
    ir = torch.randint(-1000, 1000, (6000,), generator=g).to(dtype)
    is_ = torch.randint(-1000, 1000, (9000,), generator=g).to(dtype)
    got = check(kr, ir, ks, is_)
    assert got.shape[0] > 1_000_000


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64])
@pytest.mark.parametrize("dup", [1, 3])
@pytest.mark.parametrize("n_s", [1, 5000, 20000])
def test_s_sparse_against_r_uses_sampled_search(dtype, dup, n_s):
    # each S tile spans far more than the 4 x 2048 R rows kept on chip: the
    # bounds come from a strided sample of the R range, then one stride of R;
    # with dup > 1 every matching run has several R rows
    kr = (torch.arange(300000 * dup, dtype=torch.int64) // dup).to(dtype)
    ir = torch.arange(kr.numel(), dtype=dtype)
    g = torch.Generator().manual_seed(9 + n_s)
    ks = torch.randint(-1000, 301000, (n_s,), generator=g, dtype=torch.int64).to(dtype)
    is_ = torch.arange(n_s, dtype=dtype)
    check(kr, ir, ks, is_)


@pytest.mark.parametrize("s", [0.0, 0.8, 1.2])
@pytest.mark.parametrize("scattered", [False, True])
def test_fk_zipf_scaled(s, scattered):
    kr, ir, ks, is_ = datagen.fk_zipf(100_000, 400_000, s, datagen.BASE_SEED + 1,
                                      scattered=scattered)
    got = check(kr, ir, ks, is_)
    assert got.shape[0] == 400_000  # every S key is in R, R keys unique


def test_lognormal_mix_scaled():
    kr, ir = datagen.lognormal_mix(1 << 18, datagen.BASE_SEED + 2)
    ks, is_ = datagen.lognormal_mix(1 << 18, datagen.BASE_SEED + 12)
    check(kr, ir, ks, is_)


def test_capacity_error_reports_required_count():
    kr, ir, ks, is_ = datagen.uniform_pair(5000, 5000, 0, 100, 4, torch.int32)
    exp = oracle.join_inner(kr.numpy(), ir.numpy(), ks.numpy(), is_.numpy())
    out = torch.empty((10, 2), dtype=torch.int32, device=DEV)
    with pytest.raises(api.TjError) as ei:
        api.join_inner(kr.to(DEV), ir.to(DEV), ks.to(DEV), is_.to(DEV), out=out)
    assert ei.value.status == api.TJ_ERR_CAPACITY
    assert str(len(exp)) in ei.value.detail
    # the retry path of the binding gets the full result
    got = api.join_inner(kr.to(DEV), ir.to(DEV), ks.to(DEV), is_.to(DEV))
    assert_pairs_equal(got, exp)


def test_inputs_are_not_modified():
    kr, ir, ks, is_ = datagen.uniform_pair(9000, 7000, 0, 5000, 8, torch.int64)
    d = [x.to(DEV) for x in (kr, ir, ks, is_)]
    api.join_inner(*d)
    for a, b in zip(d, (kr, ir, ks, is_)):
        assert torch.equal(a.cpu(), b)


def test_nondefault_stream():
    kr, ir, ks, is_ = datagen.uniform_pair(20000, 30000, 0, 1 << 14, 21, torch.int32)
    st = torch.cuda.Stream()
    d = [x.to(DEV) for x in (kr, ir, ks, is_)]
    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        got = api.join_inner(*d, stream=st)
    st.synchronize()
    assert_pairs_equal(got, oracle.join_inner(kr.numpy(), ir.numpy(), ks.numpy(), is_.numpy()))


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64])
@pytest.mark.parametrize("dup", [1, 2])
def test_r_range_spans_several_chunks(dtype, dup):
    # the single 3000-row S tile spans 2-4 chunks of 2048 sorted R rows; with
    # dup > 1 runs of equal R keys straddle chunk boundaries
    g = torch.Generator().manual_seed(40 + dup)
    dom = 4000
    kr = torch.randint(0, dom, (dom * dup,), generator=g).to(dtype)
    ks = torch.randint(0, dom, (3000,), generator=g).to(dtype)
    ir = torch.arange(kr.numel(), dtype=dtype)
    is_ = torch.arange(ks.numel(), dtype=dtype)
    check(kr, ir, ks, is_)
