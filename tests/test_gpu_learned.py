"""GPU parity of the learned partitioner against its fp64 oracle
(oracle/learned.py): the network's gradient and Adam step, and joins routed
by the PLA and MLP models (exact); plus what the trained network gains over
the method without it (partition balance against equal-width radix ranges and
against the untrained network)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import learned as L
from paper_2602_21237_gb300 import api, datagen
from gpu_util import DEV, assert_pairs_equal

pytestmark = pytest.mark.gpu


def test_mlp_grad_matches_oracle():
    rng = np.random.default_rng(1)
    th = rng.normal(0, 0.4, L.N_PARAMS).astype(np.float32)
    for n in (1, 37, 256):
        x = rng.random(n).astype(np.float32)
        y = rng.random(n).astype(np.float32)
        g = api.mlp_grad(torch.from_numpy(th).to(DEV), torch.from_numpy(x).to(DEV),
                         torch.from_numpy(y).to(DEV)).cpu().numpy()
        ref = L.mlp_grad(th.astype(np.float64), x, y)
        # fp32 forward/backward and batch sums of <= 256 terms
        assert np.allclose(g, ref, rtol=2e-4, atol=2e-5 * np.abs(ref).max())


def test_adam_matches_oracle():
    rng = np.random.default_rng(2)
    th = rng.normal(size=L.N_PARAMS).astype(np.float32)
    m = (rng.normal(size=L.N_PARAMS) * 0.01).astype(np.float32)
    v = (rng.random(L.N_PARAMS) * 1e-4).astype(np.float32)
    g = rng.normal(size=L.N_PARAMS).astype(np.float32)
    for t in (1, 7):
        d = [torch.from_numpy(a.copy()).to(DEV) for a in (th, m, v, g)]
        # (1 - beta^t) is formed in fp32 on the device as well
        api.mlp_adam(d[0], d[1], d[2], d[3], t, 3e-3)
        # the oracle in fp64 with the constants the device holds (their fp32 values)
        f = lambda c: float(np.float32(c))  # noqa: E731
        b1, b2 = f(0.9), f(0.999)
        rt, rm, rv = L.adam_step(th.astype(np.float64), m.astype(np.float64),
                                 v.astype(np.float64), g.astype(np.float64), t, lr=f(3e-3),
                                 beta1=b1, beta2=b2, eps=f(1e-8))
        # fp32 bound: a few roundings (2^-24 each) of the summed terms' magnitudes
        eps = 4 * 2.0 ** -24
        tol_m = eps * (np.abs(b1 * m) + np.abs((1 - b1) * g))
        tol_v = eps * (np.abs(b2 * v) + np.abs((1 - b2) * g * g))
        assert np.all(np.abs(d[1].cpu().numpy() - rm) <= tol_m + 1e-30)
        assert np.all(np.abs(d[2].cpu().numpy() - rv) <= tol_v + 1e-30)
        # the step divides m by sqrt(v): relative error of a few 1e-7 of lr * |m / sqrt v|
        step = 3e-3 * np.abs(rm / (1 - 0.9 ** t)) / (np.sqrt(rv / (1 - 0.999 ** t)) + 1e-8)
        assert np.all(np.abs(d[0].cpu().numpy() - rt) <= 1e-5 * step + eps * np.abs(th) + 1e-12)


def _lognormal_pair(n, seed):
    kr, ir = datagen.lognormal_mix(n, seed)
    ks, is_ = datagen.lognormal_mix(n, seed + 1)
    return kr, ir, ks, is_


@pytest.mark.parametrize("router", ["pla", "mlp"])
def test_learned_join_parity(router):
    kr, ir, ks, is_ = _lognormal_pair(1 << 18, 61)
    got = api.join_inner(kr.to(DEV), ir.to(DEV), ks.to(DEV), is_.to(DEV), router=router,
                         partitions=256)
    assert_pairs_equal(got, oracle.join_inner(kr.numpy(), ir.numpy(), ks.numpy(), is_.numpy()))
    assert api.stats()["learned"] == api.ROUTERS[router]


def test_trained_network_gains_over_radix_and_untrained():
    kr, ir, ks, is_ = _lognormal_pair(1 << 19, 71)
    d = [x.to(DEV) for x in (kr, ir, ks, is_)]
    api.join_inner(*d, router="radix", partitions=256)
    radix = api.stats()["balance"]
    # the networks themselves (radix_judge < 0: no fallback to equal ranges)
    api.join_inner(*d, router="mlp", partitions=256, mlp_steps=1, radix_judge=-1)
    untrained = api.stats()["balance"]
    api.join_inner(*d, router="mlp", partitions=256, radix_judge=-1)
    trained = api.stats()["balance"]
    assert api.stats()["learned"] == api.ROUTERS["mlp"]
    # training ran until its loss levelled off: at least 150 steps, at most 600
    assert 150 <= api.stats()["mlp_steps"] <= 600
    assert trained < radix / 3, (trained, radix)
    assert trained < untrained, (trained, untrained)


def test_pla_boundaries_are_sample_quantiles():
    # route counts of the PLA router equal the oracle's routing of the same keys
    kr, ir, ks, is_ = _lognormal_pair(1 << 16, 81)
    api.join_inner(kr.to(DEV), ir.to(DEV), ks.to(DEV), is_.to(DEV), router="pla",
                   partitions=64, sample_stride=10, seed=5)
    st = api.stats()
    n = kr.numel()
    stride = 10
    off_r = ((5 * 0x9E3779B97F4A7C15) % (1 << 64) >> 33) % stride
    off_s = ((5 * 0xBF58476D1CE4E5B9) % (1 << 64) >> 33) % stride
    samp = np.sort(np.concatenate([kr.numpy()[L.sample_positions(n, stride, off_r)],
                                   ks.numpy()[L.sample_positions(n, stride, off_s)]]))
    knots = L.pla_knots(samp, 4096)
    cuts = L.cuts(L.boundaries_pla(knots, 64))
    parts = np.bincount(L.route(cuts, np.concatenate([kr.numpy(), ks.numpy()])),
                        minlength=len(cuts) + 1)
    assert st["partitions"] == len(cuts) + 1
    assert st["max_partition"] == parts.max()


def _fp32_forward_bound(th, x):
    """Forward error bound of the device's fp32 evaluation of the network at
    x (exact fp32 grid points): one rounding per fma (u = 2^-24), summed over
    each chain's terms, propagated through the 1-Lipschitz ReLUs; 1.1 covers
    the second-order terms."""
    u = 2.0 ** -24
    b3, w1, b1, W2, b2, w3 = L.unpack(np.asarray(th, np.float64))
    x = np.asarray(x, np.float64)
    z1 = x[:, None] * w1 + b1
    h1 = np.maximum(z1, 0)
    e1 = u * np.abs(z1)
    a = h1 @ W2 + b2
    ea = 33 * u * (np.abs(b2) + np.abs(h1) @ np.abs(W2)) + e1 @ np.abs(W2)
    h2 = np.maximum(a, 0)
    eo = 33 * u * (abs(b3) + np.abs(h2) @ np.abs(w3)) + ea @ np.abs(w3)
    return 1.1 * eo


@pytest.mark.parametrize("seed,T,parts,span", [(11, 4096, 128, (1 << 40) - 1),
                                               (12, 4096, 1024, 987_654_321_987),
                                               (13, 1024, 37, (1 << 20) - 1)])
def test_mlp_table_and_boundaries_match_oracle(seed, T, parts, span):
    rng = np.random.default_rng(seed)
    # a ramp with hinges at i / 32 whose slope changes at random: it dips
    # below 0, rises and falls (not monotone) and may pass 1, so the clip, the
    # running maximum and its plateaus are all exercised
    th = np.zeros(L.N_PARAMS, np.float32)
    th[1:33] = 1.0 + rng.normal(0, 0.05, 32)                                # w1
    th[33:65] = -np.arange(32) / 32.0                                       # b1
    th[65:1089] = (np.eye(32) + rng.normal(0, 0.03, (32, 32))).reshape(-1)  # W2
    th[1089:1121] = rng.normal(0, 0.01, 32)                                 # b2
    c = rng.normal(0, 1.2, 32)
    c[0] = 1.0
    th[1121:1153] = c                                                       # w3
    th[0] = -0.05
    s0 = int(rng.integers(-(1 << 40), 1 << 40))
    sample = np.sort(np.concatenate([[s0, s0 + span],
                                     s0 + rng.integers(0, span, 5000)])).astype(np.int64)
    table, bounds = api.mlp_table(torch.from_numpy(th).to(DEV), T, parts,
                                  torch.from_numpy(sample).to(DEV))
    table = table.cpu().numpy()
    bounds = bounds.cpu().numpy()
    # the table: within the fp32 bound of the fp64 oracle (the running maximum
    # and the clip are 1-Lipschitz, so the bound is the running max of the
    # pointwise one)
    ref = L.mlp_table(th.astype(np.float64), T)
    grid = np.arange(T + 1, dtype=np.float64) / T
    tol = np.maximum.accumulate(_fp32_forward_bound(th, grid))
    assert np.all(np.abs(table - ref) <= tol + 1e-30), float(np.max(np.abs(table - ref) - tol))
    assert np.all(np.diff(table) >= 0) and table.min() >= 0 and table.max() <= 1
    fwd = L.mlp_forward(th.astype(np.float64), grid)
    assert fwd.min() < 0 and np.any(np.diff(fwd) < 0) and ref[-1] > 0.9  # not degenerate
    # the boundaries: decided on the device's own table in fp32, mapped back in
    # fp64; the fp64 key equals the oracle's unless it lies within rounding of
    # an integer (exp2 and log2 may differ in the last bit)
    exp = L.boundaries_table(table, parts, int(sample[0]), int(sample[-1]), np.int64,
                             target_dtype=np.float32)
    Lg = np.log2(1.0 + float(sample[-1]) - float(sample[0]))
    for p in range(1, parts):
        if bounds[p - 1] == exp[p - 1]:
            continue
        tgt = np.float32(p) / np.float32(parts)
        uu = min(int(np.searchsorted(table.astype(np.float32), tgt, side="left")), T)
        k = float(sample[0]) + 2.0 ** (uu / T * Lg) - 1.0
        assert abs(k - round(k)) <= 1e-9 * max(1.0, abs(k)) and abs(int(bounds[p - 1]) - int(exp[p - 1])) == 1, \
            (p, bounds[p - 1], exp[p - 1], k)
    assert np.all(np.diff(bounds) >= 0)


def test_mlp_batch_option():
    # a smaller batch per step still routes exactly; more than 256 rows per
    # step is rejected before any work
    kr, ir, ks, is_ = _lognormal_pair(1 << 16, 81)
    d = [x.to(DEV) for x in (kr, ir, ks, is_)]
    got = api.join_inner(*d, router="mlp", partitions=64, mlp_batch=61, mlp_steps=50,
                         radix_judge=-1)
    assert_pairs_equal(got, oracle.join_inner(kr.numpy(), ir.numpy(), ks.numpy(), is_.numpy()))
    assert api.stats()["mlp_steps"] == 50  # below the first convergence check
    with pytest.raises(api.TjError) as ei:
        api.join_inner(*d, router="mlp", mlp_batch=257)
    assert ei.value.status == api.TJ_ERR_INVALID
