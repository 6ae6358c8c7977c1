"""Pins of the CPU oracle against things other than itself (no GPU needed).

Join (paper Sec. 4.1, result independent of the path, Sec. 3.3 / 5.1):
  * brute force over every (r, s) pair in pure Python on tiny inputs,
  * an independent dictionary hash join (Python) on inputs large enough to take
    the oracle's sort-merge branch,
  * the closed-form count sum_k c_R(k) * c_S(k),
  * special cases: all keys equal (n_r * n_s pairs in a known order), disjoint
    key sets (empty), empty sides, extreme and negative keys,
  * hand-worked fixtures in tests/golden/.
Sort (Sec. 4.2, read as stable): numpy's stable argsort, sortedness,
permutation, stability.
"""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brute_join(kr, ir, ks, is_):
    """Every (s, r) pair compared; order: key, S position, R position."""
    trip = []
    for s in range(len(ks)):
        for r in range(len(kr)):
            if int(ks[s]) == int(kr[r]):
                trip.append((int(ks[s]), s, r))
    trip.sort()
    return [(int(ir[r]), int(is_[s])) for _, s, r in trip]


def dict_join(kr, ir, ks, is_):
    """Independent hash join in Python (dict of R positions per key)."""
    rows = {}
    for r, k in enumerate(kr.tolist()):
        rows.setdefault(k, []).append(r)
    sorder = sorted(range(len(ks)), key=lambda s: (int(ks[s]), s))
    out = []
    for s in sorder:
        for r in rows.get(int(ks[s]), ()):
            out.append((int(ir[r]), int(is_[s])))
    return out


def closed_form_count(kr, ks):
    ur, cr = np.unique(kr, return_counts=True)
    us, cs = np.unique(ks, return_counts=True)
    common, ia, ib = np.intersect1d(ur, us, assume_unique=True, return_indices=True)
    return int(np.sum(cr[ia].astype(np.int64) * cs[ib].astype(np.int64)))


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("seed", range(6))
def test_join_vs_bruteforce_tiny(dtype, seed):
    rng = np.random.default_rng(seed)
    nr, ns = rng.integers(0, 60, size=2)
    dom = [3, 17, 100][seed % 3]
    kr = rng.integers(-dom, dom, nr).astype(dtype)
    ks = rng.integers(-dom, dom, ns).astype(dtype)
    ir = rng.integers(-1000, 1000, nr).astype(dtype)  # arbitrary ids, not positions
    is_ = rng.integers(-1000, 1000, ns).astype(dtype)
    got = oracle.join_inner(kr, ir, ks, is_)
    exp = brute_join(kr, ir, ks, is_)
    assert [tuple(map(int, p)) for p in got] == exp


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_join_sortmerge_branch_vs_dict_join(dtype):
    rng = np.random.default_rng(7)
    nr, ns = 1500, 2100  # n_r * n_s > 1e6: sort-merge branch
    kr = rng.integers(0, 700, nr).astype(dtype)
    ks = rng.integers(0, 700, ns).astype(dtype)
    ir = np.arange(nr, dtype=dtype)
    is_ = (np.arange(ns, dtype=np.int64) * 7 - 5).astype(dtype)
    got = oracle.join_inner(kr, ir, ks, is_)
    exp = dict_join(kr, ir, ks, is_)
    assert len(got) == len(exp) == closed_form_count(kr, ks)
    assert [tuple(map(int, p)) for p in got] == exp


@pytest.mark.parametrize("n", [10, 1000, 100000])
def test_join_count_closed_form(n):
    rng = np.random.default_rng(n)
    kr = rng.integers(0, max(2, n // 3), n).astype(np.int64)
    ks = rng.integers(0, max(2, n // 3), 2 * n).astype(np.int64)
    ir = np.arange(n, dtype=np.int64)
    is_ = np.arange(2 * n, dtype=np.int64)
    assert oracle.join_inner(kr, ir, ks, is_, count_only=True) == closed_form_count(kr, ks)


@pytest.mark.parametrize("nr,ns", [(3, 4), (40, 30), (1200, 900)])
def test_join_all_equal_keys(nr, ns):
    kr = np.full(nr, 5, np.int64)
    ks = np.full(ns, 5, np.int64)
    ir = np.arange(nr, dtype=np.int64) + 100
    is_ = np.arange(ns, dtype=np.int64) + 1000
    got = oracle.join_inner(kr, ir, ks, is_)
    assert got.shape == (nr * ns, 2)
    # S-major, then R: pair i*nr + j == (ir[j], is[i])
    assert np.array_equal(got[:, 0], np.tile(ir, ns))
    assert np.array_equal(got[:, 1], np.repeat(is_, nr))


def test_join_disjoint_and_empty():
    kr = np.arange(0, 1000, 2, dtype=np.int32)
    ks = np.arange(1, 1001, 2, dtype=np.int32)
    ids = np.arange(500, dtype=np.int32)
    assert oracle.join_inner(kr, ids, ks, ids).shape == (0, 2)
    e = np.zeros(0, np.int32)
    assert oracle.join_inner(e, e, ks, ids).shape == (0, 2)
    assert oracle.join_inner(kr, ids, e, e).shape == (0, 2)


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_join_extreme_keys(dtype):
    info = np.iinfo(dtype)
    vals = np.array([info.min, info.min + 1, -1, 0, 1, info.max - 1, info.max], dtype=dtype)
    rng = np.random.default_rng(3)
    kr = rng.choice(vals, 40).astype(dtype)
    ks = rng.choice(vals, 50).astype(dtype)
    ir = np.arange(40, dtype=dtype)
    is_ = np.arange(50, dtype=dtype)
    got = oracle.join_inner(kr, ir, ks, is_)
    assert [tuple(map(int, p)) for p in got] == brute_join(kr, ir, ks, is_)
    # key order: min first, max last, with the sign handled
    keys = kr[got[:, 0]]
    assert np.all(np.diff(keys.astype(np.float64)) >= 0)


def test_join_order_is_key_then_s_then_r():
    rng = np.random.default_rng(11)
    kr = rng.integers(0, 50, 400).astype(np.int64)
    ks = rng.integers(0, 50, 500).astype(np.int64)
    ir = np.arange(400, dtype=np.int64)
    is_ = np.arange(500, dtype=np.int64)
    got = oracle.join_inner(kr, ir, ks, is_)
    k = kr[got[:, 0]]
    assert np.array_equal(k, ks[got[:, 1]])
    trip = np.stack([k, got[:, 1], got[:, 0]], 1)
    order = np.lexsort((trip[:, 2], trip[:, 1], trip[:, 0]))
    assert np.array_equal(order, np.arange(len(order)))


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("n", [0, 1, 2, 17, 4096, 100003])
def test_sort_vs_numpy_stable(dtype, n):
    rng = np.random.default_rng(n + 1)
    info = np.iinfo(dtype)
    keys = rng.integers(info.min, info.max, n, dtype=dtype, endpoint=True)
    if n > 10:
        keys[: n // 3] = keys[0]  # many duplicates: exercises stability
        keys[n // 3] = info.min
        keys[n // 3 + 1] = info.max
    ids = np.arange(n, dtype=dtype)
    k, i = oracle.sort(keys, ids)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(k, keys[order])
    assert np.array_equal(i, ids[order])
    assert np.all(k[1:] >= k[:-1])
    same = k[1:] == k[:-1]
    assert np.all(i[1:][same] > i[:-1][same])  # stability (ids are positions)
    assert np.array_equal(np.sort(i), ids)  # permutation


def test_join_batch_matches_per_job():
    rng = np.random.default_rng(5)
    nr = [0, 5, 300, 40, 1]
    ns = [7, 0, 200, 900, 1]
    r_off = np.concatenate([[0], np.cumsum(nr)])
    s_off = np.concatenate([[0], np.cumsum(ns)])
    kr = rng.integers(0, 60, r_off[-1]).astype(np.int32)
    ks = rng.integers(0, 60, s_off[-1]).astype(np.int32)
    ir = np.concatenate([np.arange(n) for n in nr]).astype(np.int32)
    is_ = np.concatenate([np.arange(n) for n in ns]).astype(np.int32)
    out, off = oracle.join_batch(r_off, s_off, kr, ir, ks, is_)
    for j in range(len(nr)):
        a, b = r_off[j], r_off[j + 1]
        c, d = s_off[j], s_off[j + 1]
        exp = brute_join(kr[a:b], ir[a:b], ks[c:d], is_[c:d])
        got = [tuple(map(int, p)) for p in out[off[j]:off[j + 1]]]
        assert got == exp


def _read_golden(name):
    sec, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if line.startswith("[") and line.endswith("]"):
                cur = line[1:-1]
                sec[cur] = []
            else:
                sec[cur].append([int(t) for t in line.replace(",", " ").split()])
    return sec


@pytest.mark.parametrize("name", ["join_rabc_sbde.txt", "join_dup_negative.txt"])
def test_golden_join(name):
    g = _read_golden(name)
    R = np.array(g["R"], np.int64).reshape(-1, 2)
    S = np.array(g["S"], np.int64).reshape(-1, 2)
    exp = np.array(g["J"], np.int64).reshape(-1, 2)
    got = oracle.join_inner(R[:, 0], R[:, 1], S[:, 0], S[:, 1])
    assert np.array_equal(got, exp)


def test_golden_multi_attribute_join_with_late_gather():
    # R(A, B, C) joined with S(B, D, E) on B, the other attributes gathered
    # through the (r_id, s_id) pairs at the end (hand-worked fixture)
    g = _read_golden("join_payload_rabc_sbde.txt")
    R = np.array(g["R"], np.int64).reshape(-1, 3)
    S = np.array(g["S"], np.int64).reshape(-1, 3)
    exp = np.array(g["J"], np.int64).reshape(-1, 5)
    pairs = oracle.join_inner(R[:, 1], np.arange(len(R)), S[:, 0], np.arange(len(S)))
    (a, b, c), (d, e) = oracle.gather_pairs(pairs, [R[:, 0], R[:, 1], R[:, 2]],
                                            [S[:, 1], S[:, 2]])
    assert np.array_equal(np.stack([a, b, c, d, e], 1), exp)
    # a gather that takes an S column at r_id (sides swapped) is caught
    (d_wrong,), _ = oracle.gather_pairs(pairs, [S[:4, 1]], [])
    assert not np.array_equal(d_wrong, exp[:, 3])


def test_gather_rejects_ids_outside_the_relation():
    col = np.arange(5, dtype=np.int64)
    for bad in ([[5, 0]], [[-1, 0]]):
        with pytest.raises(ValueError):
            oracle.gather_pairs(np.array(bad, np.int64), [col], [])
    r, s = oracle.gather_pairs(np.zeros((0, 2), np.int64), [col], [col])
    assert r[0].size == 0 and s[0].size == 0


def test_golden_sort():
    g = _read_golden("sort_stable.txt")
    inp = np.array(g["IN"], np.int64).reshape(-1, 2)
    exp = np.array(g["OUT"], np.int64).reshape(-1, 2)
    k, i = oracle.sort(inp[:, 0], inp[:, 1])
    assert np.array_equal(np.stack([k, i], 1), exp)


def test_golden_sort_multi():
    g = _read_golden("sort_multi.txt")
    inp = np.array(g["IN"], np.int64).reshape(-1, 3)
    exp = np.array(g["OUT"], np.int64).reshape(-1, 3)
    (k0, k1), ids = oracle.sort_multi([inp[:, 0], inp[:, 1]], inp[:, 2])
    assert np.array_equal(np.stack([k0, k1, ids], 1), exp)
    # the keys in the wrong priority (k1 first) give another order
    (a, b), _ = oracle.sort_multi([inp[:, 1], inp[:, 0]], inp[:, 2])
    assert not np.array_equal(np.stack([b, a], 1), exp[:, :2])


def test_sort_multi_matches_brute_force():
    # brute force: Python's stable sorted() on the key tuples
    rng = np.random.default_rng(4)
    for n, m in ((1, 2), (50, 2), (200, 3)):
        cols = [rng.integers(-3, 4, n).astype(np.int64) for _ in range(m)]
        ids = rng.integers(0, 1 << 40, n).astype(np.int64)
        order = sorted(range(n), key=lambda i: tuple(int(c[i]) for c in cols))
        got, gids = oracle.sort_multi(cols, ids)
        for c, gc in zip(cols, got):
            assert np.array_equal(gc, c[order])
        assert np.array_equal(gids, ids[order])


def test_pins_catch_planted_mistakes():
    """Mutations of a correct result that a plausible oracle bug would produce
    are each rejected by one of the pins used above."""
    rng = np.random.default_rng(9)
    kr = rng.integers(0, 8, 30).astype(np.int64)
    ks = rng.integers(0, 8, 40).astype(np.int64)
    ir = np.arange(30, dtype=np.int64)
    is_ = np.arange(40, dtype=np.int64)
    good = [tuple(p) for p in brute_join(kr, ir, ks, is_)]
    # dropped pair -> closed-form count differs
    assert len(good[1:]) != closed_form_count(kr, ks)
    # ties in R-major instead of S-major order -> order pin differs
    trip = sorted((int(kr[r]), r, s) for r, s in good)
    rmajor = [(r, s) for _, r, s in trip]
    assert rmajor != good
    # ids swapped (transposed operands) -> brute force differs
    assert [(s, r) for r, s in good] != good
