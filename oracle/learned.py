"""fp64 oracle of the learned key-range partitioner -- TEST INFRASTRUCTURE ONLY.

The paper has no learned component; this is the partitioner that routes keys
to key-range partitions for the partitioned (multi-pass) join, whose
definition the library fixes as follows.  Plain numpy, one step per function,
in the order the library runs them:

1. ``sample_positions``: every ``stride``-th row starting at ``offset``
   (a 1% sample for stride 100), taken from R and from S and pooled.
2. ``pla_knots``: a piecewise-linear CDF with G segments whose knots are
   sample quantiles, t_i = s[floor(i (m - 1) / G)], i = 0..G.
3. ``pla_cdf``: F(k) = (i + (k - t_i) / (t_{i+1} - t_i)) / G with
   i = max{i < G : t_i <= k}; 0 below t_0, 1 from t_G on.
4. ``mlp_*``: the alternative model, a 1 -> 32 -> 32 -> 1 ReLU network on
   x = log2(1 + k - s_0) / log2(1 + s_{m-1} - s_0), fitted to the empirical CDF
   y_j = j / (m - 1) by mean squared error with Adam.  Forward, backward and
   the Adam step are written out here; the trained weights themselves are
   PARITY UNPINNED (fp32 on the device, order-dependent); their gradients and
   the Adam update are pinned by finite differences and a closed form.
5. ``boundaries_*``: B_p = the smallest key with F(key) >= p / P, p = 1..P-1
   (for the PLA with G = c P this is exactly t_{c p}; for the MLP, on its
   monotone tabulation).
6. ``cuts``: the sorted distinct boundaries, plus u + 1 for every boundary
   value u that repeats (a key holding at least one partition's worth of
   mass), so that such a key gets a partition of its own.
7. ``route``: partition(k) = #{c in cuts : c <= k}.  Partitions are key
   ranges [c_{j-1}, c_j) in key order.
"""
from __future__ import annotations

import numpy as np

HIDDEN = 32
N_PARAMS = 1 + HIDDEN + HIDDEN + HIDDEN * HIDDEN + HIDDEN + HIDDEN  # 1153 (b3 first)


def sample_positions(n: int, stride: int, offset: int) -> np.ndarray:
    return np.arange(offset, n, stride, dtype=np.int64)


def pla_knots(sorted_sample: np.ndarray, segments: int) -> np.ndarray:
    m = len(sorted_sample)
    idx = (np.arange(segments + 1, dtype=np.int64) * (m - 1)) // segments
    return sorted_sample[idx]


def pla_cdf(knots: np.ndarray, k) -> np.ndarray:
    t = knots.astype(np.float64)
    G = len(knots) - 1
    kk = np.asarray(k)
    out = np.empty(kk.shape, dtype=np.float64)
    flat = kk.reshape(-1)
    o = out.reshape(-1)
    for n, key in enumerate(flat):
        if key < knots[0]:
            o[n] = 0.0
        elif key >= knots[G]:
            o[n] = 1.0
        else:
            i = int(np.searchsorted(knots, key, side="right")) - 1  # max i with t_i <= key
            o[n] = (i + (float(key) - t[i]) / (t[i + 1] - t[i])) / G
    return out


def boundaries_pla(knots: np.ndarray, parts: int) -> np.ndarray:
    """Smallest key with F >= p / parts, p = 1..parts-1 (G divisible by parts)."""
    G = len(knots) - 1
    assert G % parts == 0
    c = G // parts
    return np.array([knots[c * p] for p in range(1, parts)], dtype=knots.dtype)


def boundaries_radix(lo: int, bits: int, parts_log2: int, dtype=np.int64) -> np.ndarray:
    """Equal-width key ranges: lo + p 2^(bits - parts_log2)."""
    sh = max(0, bits - parts_log2)
    n = 1 << min(parts_log2, bits)
    return np.array([lo + (p << sh) for p in range(1, n)], dtype=dtype)


def cuts(boundaries: np.ndarray) -> np.ndarray:
    b = np.asarray(boundaries)
    if b.size == 0:
        return b.copy()
    vals, counts = np.unique(b, return_counts=True)
    info = np.iinfo(b.dtype)
    extra = [int(v) + 1 for v, c in zip(vals, counts) if c >= 2 and int(v) < info.max]
    return np.unique(np.concatenate([vals, np.array(extra, dtype=b.dtype)])).astype(b.dtype)


def route(cut: np.ndarray, keys: np.ndarray) -> np.ndarray:
    return np.searchsorted(cut, keys, side="right").astype(np.int64)


# ---------------------------------------------------------------------------
# MLP 1 -> 32 -> 32 -> 1 (ReLU), parameters in one flat vector:
#   [b3 | w1(32) | b1(32) | W2(32x32, row i = from hidden-1 unit i) | b2(32) | w3(32)]
# ---------------------------------------------------------------------------
def unpack(theta):
    H = HIDDEN
    o = 0
    b3 = theta[o]; o += 1
    w1 = theta[o:o + H]; o += H
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].reshape(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    w3 = theta[o:o + H]; o += H
    return b3, w1, b1, W2, b2, w3


def mlp_forward(theta, x):
    b3, w1, b1, W2, b2, w3 = unpack(np.asarray(theta, np.float64))
    x = np.asarray(x, np.float64)
    z1 = x[:, None] * w1[None, :] + b1[None, :]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2[None, :]
    h2 = np.maximum(z2, 0.0)
    return h2 @ w3 + b3


def mlp_loss(theta, x, y):
    d = mlp_forward(theta, x) - np.asarray(y, np.float64)
    return float(np.mean(d * d))


def mlp_grad(theta, x, y):
    """Analytic gradient of the mean squared error (backpropagation)."""
    b3, w1, b1, W2, b2, w3 = unpack(np.asarray(theta, np.float64))
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    B = len(x)
    z1 = x[:, None] * w1[None, :] + b1[None, :]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2[None, :]
    h2 = np.maximum(z2, 0.0)
    out = h2 @ w3 + b3
    dy = 2.0 * (out - y) / B
    g_b3 = dy.sum()
    g_w3 = h2.T @ dy
    dz2 = (dy[:, None] * w3[None, :]) * (z2 > 0)
    g_W2 = h1.T @ dz2
    g_b2 = dz2.sum(0)
    dz1 = (dz2 @ W2.T) * (z1 > 0)
    g_w1 = (x[:, None] * dz1).sum(0)
    g_b1 = dz1.sum(0)
    return np.concatenate([[g_b3], g_w1, g_b1, g_W2.reshape(-1), g_b2, g_w3])


def adam_step(theta, m, v, g, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015) at step t >= 1.  Returns new
    (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def normalize_keys(keys, s0, s1):
    """x = log2(1 + k - s0) / log2(1 + s1 - s0), clipped to [0, 1]."""
    k = np.asarray(keys, np.float64)
    L = np.log2(1.0 + float(s1) - float(s0))
    if L <= 0:
        return np.zeros_like(k)
    return np.clip(np.log2(1.0 + np.maximum(k - float(s0), 0.0)) / L, 0.0, 1.0)


def mlp_table(theta, T: int = 4096):
    """Monotone tabulation on x = u / T: running maximum of the network output,
    clipped to [0, 1]."""
    x = np.arange(T + 1, dtype=np.float64) / T
    y = np.clip(mlp_forward(theta, x), 0.0, 1.0)
    return np.maximum.accumulate(y)


def boundaries_table(table, parts: int, s0: int, s1: int, dtype=np.int64,
                     target_dtype=np.float64):
    """B_p from a monotone tabulated CDF on the normalised axis: the first grid
    point u with table[u] >= p / parts, mapped back to a key (ceil).  The
    comparison is made in `target_dtype` (the library tabulates in fp32 and
    compares there; a check of its kernels takes the decision in the same
    precision)."""
    T = len(table) - 1
    L = np.log2(1.0 + float(s1) - float(s0))
    tab = np.asarray(table).astype(target_dtype)
    out = []
    for p in range(1, parts):
        target = target_dtype(p) / target_dtype(parts)
        u = int(np.searchsorted(tab, target, side="left"))
        u = min(u, T)
        x = u / T
        out.append(int(np.ceil(s0 + (2.0 ** (x * L) - 1.0))))
    return np.minimum(np.array(out, dtype=np.float64), float(s1)).astype(dtype)
