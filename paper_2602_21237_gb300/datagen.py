"""Seeded synthetic inputs for the join/sort workloads.

This module only draws random relations; it holds none of the join or sort
arithmetic, so both the CUDA path and the CPU oracle may use it.  Every
generator is deterministic for a given (seed, device): tests draw on the CPU and
copy to the GPU; the benchmark draws large inputs directly on the GPU.

Workloads (the paper prints no data of its own, Sec. 5.1 only says the inputs
were the same for both paths; these shapes stand in for them):

* ``uniform_pair``   -- R and S with keys uniform in [lo, hi), ids = positions.
* ``fk_zipf``        -- foreign-key join: R keys a random permutation of
  [0, n_r) (optionally scattered over 64 bits by a fixed bijection), S keys
  drawn Zipf(s) over R's keys, the rank -> key map an independent permutation.
* ``lognormal_mix``  -- 8 log-normal clusters (medians 2^(24+2c), log-sigma
  0.3 + 0.05c, weight 0.95/8 each) plus 5% uniform noise on [0, 2^40); draws
  at or above 2^40 wrap around modulo 2^40.
* ``batch_jobs``     -- many joins with |R|, |S| log-uniform, int32 keys
  uniform over [0, 2|R|).
* ``poisson_arrivals`` -- exponential inter-arrival times of a Poisson stream.
"""
from __future__ import annotations

import math

import torch

BASE_SEED = 20260221

_M1 = -7046029254386353131  # 0x9E3779B97F4A7C15 as signed int64 (odd)
_M2 = -4658895280553007687  # 0xBF58476D1CE4E5B9 as signed int64 (odd)


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _lsr(x: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 (torch's >> is arithmetic)."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def scatter64(x: torch.Tensor) -> torch.Tensor:
    """A fixed bijection of int64 (xor-shift / odd-multiply rounds): spreads
    dense keys over all 64 bits while keeping them distinct."""
    x = x.to(torch.int64)
    x = x ^ _lsr(x, 31)
    x = x * _M1
    x = x ^ _lsr(x, 29)
    x = x * _M2
    x = x ^ _lsr(x, 32)
    return x


def uniform_pair(n_r: int, n_s: int, lo: int, hi: int, seed: int, dtype=torch.int32,
                 device="cpu"):
    """R, S with keys uniform in [lo, hi) and ids = row positions."""
    g = _gen(seed, device)
    kr = torch.randint(lo, hi, (n_r,), generator=g, device=device, dtype=torch.int64).to(dtype)
    ks = torch.randint(lo, hi, (n_s,), generator=g, device=device, dtype=torch.int64).to(dtype)
    ir = torch.arange(n_r, device=device, dtype=dtype)
    is_ = torch.arange(n_s, device=device, dtype=dtype)
    return kr, ir, ks, is_


def zipf_ranks(n: int, m: int, s: float, g: torch.Generator, device, chunk: int = 1 << 26):
    """n ranks in [0, m) with P(rank = r) proportional to (r+1)^-s, by inverse
    CDF over the exact discrete distribution (fp64 cumulative sums)."""
    if s == 0.0:
        return torch.randint(0, m, (n,), generator=g, device=device, dtype=torch.int64)
    w = torch.arange(1, m + 1, device=device, dtype=torch.float64).pow_(-s)
    cdf = torch.cumsum(w, 0)
    del w
    cdf /= cdf[-1].clone()
    out = torch.empty(n, dtype=torch.int64, device=device)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        u = torch.rand(b - a, generator=g, device=device, dtype=torch.float64)
        idx = torch.searchsorted(cdf, u, right=True)
        out[a:b] = idx.clamp_(max=m - 1)
        del u, idx
    del cdf
    return out


def fk_zipf(n_r: int, n_s: int, s: float, seed: int, device="cpu", scattered: bool = False,
            dtype=torch.int64):
    """Foreign-key pair: R keys unique, S keys all drawn from R's keys."""
    g = _gen(seed, device)
    base = torch.randperm(n_r, generator=g, device=device, dtype=torch.int64)
    kr = scatter64(base) if scattered else base
    rank_to_row = torch.randperm(n_r, generator=g, device=device, dtype=torch.int64)
    ranks = zipf_ranks(n_s, n_r, s, g, device)
    ks = kr[rank_to_row[ranks]]
    del ranks, rank_to_row, base
    ir = torch.arange(n_r, device=device, dtype=dtype)
    is_ = torch.arange(n_s, device=device, dtype=dtype)
    return kr.to(dtype), ir, ks.to(dtype), is_


def lognormal_mix(n: int, seed: int, device="cpu", clusters: int = 8, noise: float = 0.05,
                  key_bits: int = 40):
    """n int64 keys: `clusters` log-normal clusters plus uniform noise."""
    g = _gen(seed, device)
    top = 1 << key_bits
    u = torch.rand(n, generator=g, device=device, dtype=torch.float64)
    comp = torch.clamp((u * clusters / (1.0 - noise)).to(torch.int64), max=clusters)
    med = torch.tensor([math.log(2.0 ** (24 + 2 * c)) for c in range(clusters)] + [0.0],
                       device=device, dtype=torch.float64)
    sig = torch.tensor([0.3 + 0.05 * c for c in range(clusters)] + [0.0], device=device,
                       dtype=torch.float64)
    z = torch.randn(n, generator=g, device=device, dtype=torch.float64)
    x = torch.exp(med[comp] + sig[comp] * z)
    # the upper tail of the widest clusters passes 2^key_bits: wrap it around
    # (clamping would pile ~2% of a cluster onto the single key 2^key_bits - 1)
    x = torch.remainder(torch.round(x), float(top)).to(torch.int64)
    noise_keys = torch.randint(0, top, (n,), generator=g, device=device, dtype=torch.int64)
    keys = torch.where(comp == clusters, noise_keys, x)
    return keys, torch.arange(n, device=device, dtype=torch.int64)


def log_uniform_sizes(n: int, lo: float, hi: float, seed: int) -> list:
    """n integers log-uniform in [lo, hi] (host-side, seeded)."""
    g = _gen(seed, "cpu")
    u = torch.rand(n, generator=g, dtype=torch.float64)
    v = torch.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))
    return [int(round(float(t))) for t in v]


def batch_jobs(n_jobs: int, lo: float, hi: float, seed: int, device="cpu",
               dtype=torch.int32):
    """n_jobs joins stored back to back.  Returns (r_off, s_off, kr, ir, ks, is)
    with offsets as python lists of length n_jobs + 1; ids are per-job row
    positions; keys of job j uniform over [0, 2|R_j|)."""
    nr = log_uniform_sizes(n_jobs, lo, hi, seed)
    ns = log_uniform_sizes(n_jobs, lo, hi, seed + 1)
    r_off, s_off = [0], [0]
    for a, b in zip(nr, ns):
        r_off.append(r_off[-1] + a)
        s_off.append(s_off[-1] + b)
    g = _gen(seed + 2, device)
    tr, ts = r_off[-1], s_off[-1]
    dom_r = torch.empty(tr, dtype=torch.float64, device=device)
    dom_s = torch.empty(ts, dtype=torch.float64, device=device)
    ir = torch.empty(tr, dtype=dtype, device=device)
    is_ = torch.empty(ts, dtype=dtype, device=device)
    for j in range(n_jobs):
        dom_r[r_off[j]:r_off[j + 1]] = 2.0 * nr[j]
        dom_s[s_off[j]:s_off[j + 1]] = 2.0 * nr[j]
        ir[r_off[j]:r_off[j + 1]] = torch.arange(nr[j], dtype=dtype, device=device)
        is_[s_off[j]:s_off[j + 1]] = torch.arange(ns[j], dtype=dtype, device=device)
    kr = (torch.rand(tr, generator=g, device=device, dtype=torch.float64) * dom_r).floor_()
    ks = (torch.rand(ts, generator=g, device=device, dtype=torch.float64) * dom_s).floor_()
    return r_off, s_off, kr.to(dtype), ir, ks.to(dtype), is_


def poisson_arrivals(rate: float, n: int, seed: int) -> list:
    """Arrival times (seconds) of n requests of a Poisson stream of `rate`/s."""
    g = _gen(seed, "cpu")
    u = torch.rand(n, generator=g, dtype=torch.float64).clamp_(min=1e-300)
    gaps = -torch.log(u) / rate
    return torch.cumsum(gaps, 0).tolist()
