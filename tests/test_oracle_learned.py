"""Pins of the learned-partitioner oracle (oracle/learned.py), CPU only.

Each function is checked against something other than itself: closed forms,
numpy routines for the special cases they reduce to, brute force, central
finite differences (for the network's gradient) and Adam's first-step closed
form.  The trained weights are parity-unpinned by design (fp32, order
dependent); everything they feed into routing is exact integer work.
"""
import numpy as np
import pytest

from oracle import learned as L


def test_sample_positions():
    for n, stride, off in [(1000, 100, 7), (99, 100, 0), (12345, 10, 9), (0, 100, 3)]:
        p = L.sample_positions(n, stride, off)
        assert len(p) == max(0, -(-(n - off) // stride))
        assert np.all(p % stride == off) and (len(p) == 0 or p[-1] < n)


def test_pla_knots_are_lower_quantiles():
    rng = np.random.default_rng(1)
    s = np.sort(rng.integers(-10**6, 10**6, 10001))
    t = L.pla_knots(s, 64)
    assert t[0] == s.min() and t[-1] == s.max()
    q = np.quantile(s, np.arange(65) / 64, method="lower")
    assert np.array_equal(t, q)
    assert np.all(np.diff(t) >= 0)


def test_pla_cdf_interpolates_knots():
    rng = np.random.default_rng(2)
    s = np.sort(rng.choice(10**7, 5000, replace=False))
    t = L.pla_knots(s, 128)
    assert len(np.unique(t)) == len(t)
    F = L.pla_cdf(t, t)
    assert np.allclose(F, np.arange(129) / 128)
    k = rng.integers(t[0], t[-1], 2000)
    assert np.allclose(L.pla_cdf(t, k), np.interp(k, t, np.arange(129) / 128))
    assert L.pla_cdf(t, np.array([t[0] - 5]))[0] == 0.0
    assert L.pla_cdf(t, np.array([t[-1] + 5]))[0] == 1.0


def test_boundaries_pla_satisfy_definition():
    rng = np.random.default_rng(3)
    s = np.sort(rng.integers(0, 10**9, 40000))
    t = L.pla_knots(s, 256)
    B = L.boundaries_pla(t, 64)
    for p, b in enumerate(B, start=1):
        assert L.pla_cdf(t, np.array([b]))[0] >= p / 64 - 1e-12
        assert L.pla_cdf(t, np.array([b - 1]))[0] < p / 64


def test_cuts_and_route_isolate_heavy_keys():
    rng = np.random.default_rng(4)
    s = np.sort(np.concatenate([rng.integers(0, 10**6, 9000), np.full(3000, 123456)]))
    t = L.pla_knots(s, 64)
    B = L.boundaries_pla(t, 32)
    c = L.cuts(B)
    assert np.all(np.diff(c) > 0)
    r = L.route(c, np.array([123455, 123456, 123457]))
    assert r[0] < r[1] < r[2]  # the heavy key sits alone in its partition
    keys = rng.integers(-10, 10**6 + 10, 5000)
    got = L.route(c, keys)
    brute = np.array([sum(1 for x in c if x <= k) for k in keys])
    assert np.array_equal(got, brute)
    order = np.argsort(keys, kind="stable")
    assert np.all(np.diff(got[order]) >= 0)  # partitions are key ranges


def test_cuts_at_int64_max_do_not_overflow():
    m = np.iinfo(np.int64).max
    c = L.cuts(np.array([5, m, m], dtype=np.int64))
    assert list(c) == [5, m]


def test_boundaries_radix():
    B = L.boundaries_radix(1000, 20, 4)
    assert list(B) == [1000 + p * (1 << 16) for p in range(1, 16)]


def test_mlp_forward_closed_form():
    th = np.zeros(L.N_PARAMS)
    b3, w1, b1, W2, b2, w3 = L.unpack(th)
    w1[0] = 1.0
    W2[0, 0] = 1.0
    w3[0] = 2.0
    th[0] = 0.5  # b3
    x = np.linspace(-1, 1, 11)
    assert np.allclose(L.mlp_forward(th, x), 2 * np.maximum(x, 0) + 0.5)


def test_mlp_grad_matches_finite_differences():
    rng = np.random.default_rng(5)
    th = rng.normal(0, 0.5, L.N_PARAMS)
    x = rng.random(64)
    y = rng.random(64)
    g = L.mlp_grad(th, x, y)
    eps = 1e-6
    num = np.empty_like(th)
    for i in range(len(th)):
        a, b = th.copy(), th.copy()
        a[i] += eps
        b[i] -= eps
        num[i] = (L.mlp_loss(a, x, y) - L.mlp_loss(b, x, y)) / (2 * eps)
    assert np.allclose(g, num, rtol=1e-5, atol=1e-8)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(6)
    th = rng.normal(size=50)
    g = rng.normal(size=50)
    new, m, v = L.adam_step(th, np.zeros(50), np.zeros(50), g, 1, lr=1e-3)
    assert np.allclose(new, th - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-10, atol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_table_boundaries_of_a_linear_cdf():
    T = 1024
    table = np.arange(T + 1) / T
    B = L.boundaries_table(table, 8, 0, (1 << 20) - 1)
    Lg = 20.0
    exp = [int(np.ceil(2 ** (p / 8 * Lg) - 1)) for p in range(1, 8)]
    assert list(B) == exp


def test_normalize_is_monotone_and_bounded():
    k = np.sort(np.random.default_rng(7).integers(0, 1 << 40, 1000))
    x = L.normalize_keys(k, k[0], k[-1])
    assert x[0] == 0.0 and abs(x[-1] - 1.0) < 1e-12 and np.all(np.diff(x) >= 0)


def test_normalize_keys_exact_values():
    # s1 - s0 + 1 = 2^20, so the denominator is log2(2^20) = 20 exactly and a
    # key s0 + 2^j - 1 maps to j / 20: exact in fp64.  A dropped "1 +" (log2 of
    # k - s0) or a wrong endpoint moves these values.
    for s0 in (0, -(1 << 30), 12345):
        s1 = s0 + (1 << 20) - 1
        ks = np.array([s0 + (1 << j) - 1 for j in range(0, 21)], dtype=np.int64)
        x = L.normalize_keys(ks, s0, s1)
        assert np.array_equal(x, np.arange(21) / 20.0)
        assert L.normalize_keys(np.array([s0 + (1 << 10) - 1]), s0, s1)[0] == 0.5
        # outside [s0, s1]: clipped to the ends
        assert list(L.normalize_keys(np.array([s0 - 7, s1 + 99]), s0, s1)) == [0.0, 1.0]
    # a single-key range has no width: everything maps to 0
    assert np.all(L.normalize_keys(np.array([3, 4, 5]), 4, 4) == 0.0)


def _two_unit_theta(a0, c0, a1, c1, v0, v1, b3=0.0):
    """Network whose output is v0 relu(a0 x + c0) + v1 relu(a1 x + c1) + b3 on
    x >= 0: hidden-1 units 0 and 1 feed hidden-2 units 0 and 1 through a unit
    weight (relu of a non-negative value is itself)."""
    th = np.zeros(L.N_PARAMS)
    b3_, w1, b1, W2, b2, w3 = L.unpack(th)
    w1[0], b1[0], w1[1], b1[1] = a0, c0, a1, c1
    W2[0, 0] = 1.0
    W2[1, 1] = 1.0
    w3[0], w3[1] = v0, v1
    th[0] = b3
    return th


def test_mlp_table_running_max_of_a_rise_and_fall():
    # f(x) = relu(x) - 2 relu(x - 1/2): rises to 1/2 at x = 1/2, then falls
    # back to 0 at x = 1.  The monotone table keeps the peak: min(u / T, 1/2).
    T = 64
    th = _two_unit_theta(1.0, 0.0, 1.0, -0.5, 1.0, -2.0)
    u = np.arange(T + 1)
    assert np.allclose(L.mlp_forward(th, u / T), np.where(u <= T // 2, u / T, 1 - u / T))
    assert np.allclose(L.mlp_table(th, T), np.minimum(u / T, 0.5), rtol=0, atol=1e-15)


def test_mlp_table_clips_to_unit_interval():
    # f(x) = 3 x - 1 - 3 relu(x - 0.9) ... below 0 until x = 1/3, above 1 from
    # x = 2/3 (up to 1.7 at x = 0.9, then down to 1.4): the table is
    # clip(3x - 1, 0, 1), flat at 1 after 2/3 whatever f does there.
    T = 90
    th = _two_unit_theta(3.0, 0.0, 1.0, -0.9, 1.0, -3.0, b3=-1.0)
    u = np.arange(T + 1)
    assert np.allclose(L.mlp_table(th, T), np.clip(3 * u / T - 1, 0.0, 1.0), rtol=0, atol=1e-12)


def test_boundaries_table_reads_the_first_grid_point():
    # table = min(u / T, 1/2) with T = 64: F reaches p / 8 at u = 8p for p <= 4
    # and never beyond 1/2, so the later boundaries take the last grid point,
    # which maps to s1.
    T = 64
    table = np.minimum(np.arange(T + 1) / T, 0.5)
    s0, s1 = 0, (1 << 20) - 1
    B = L.boundaries_table(table, 8, s0, s1)
    exp = [int(np.ceil(2.0 ** (8 * p / 64 * 20) - 1)) for p in range(1, 5)] + [s1] * 3
    assert list(B) == exp
