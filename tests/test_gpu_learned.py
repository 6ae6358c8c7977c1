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
    api.join_inner(*d, router="mlp", partitions=256, mlp_steps=1)
    untrained = api.stats()["balance"]
    api.join_inner(*d, router="mlp", partitions=256)
    trained = api.stats()["balance"]
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
