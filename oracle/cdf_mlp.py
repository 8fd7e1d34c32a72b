"""CPU oracle of the learned splitter proposal: a 1-32-32-1 CDF network.

TEST INFRASTRUCTURE ONLY (like the rest of this package): the test suite and
the smoke check import it; the product library never does.

The paper proposes no learned model; its splitter rounds (Sec. 4.2.2) accept
any set of candidate cuts, and a model of the key distribution is one source
of such cuts before round 1.  This file restates, in numpy float64, the
textbook definitions the CUDA kernels implement in float32:

  * feature map phi(key): the order-preserving key bits u (the sign bit
    flipped for int64 keys), mapped affinely onto [0, 1] either directly
    (LINEAR) or through log2(1 + u) (LOG), then clipped to [0, 1];
  * the network  y = w3 . relu(W2 relu(w1 x + b1) + b2) + b3  (32 hidden
    units per layer, ReLU with derivative 0 at 0, linear output);
  * the loss  L = (1/n) sum_b (y_b - t_b)^2  with targets t_b = rank_b / N
    (the empirical CDF at the training keys);
  * its gradient by the chain rule (reverse mode, written out by hand);
  * the Adam update (Kingma and Ba, ICLR 2015) with bias correction;
  * the proposal: for each splitter i = 1..p-1 and each of `per` targets
    tau = i/p + delta (2k/(per-1) - 1) around it, bisection on x in [0, 1]
    for the smallest x with y(x) >= tau, mapped back to a key.

Parameter vector (1153 floats), in this order: w1[32], b1[32], W2[32*32]
(row-major, W2[i, j] = weight from hidden-1 unit j to hidden-2 unit i),
b2[32], w3[32], b3.
"""
from __future__ import annotations

import numpy as np

H = 32
NPARAM = H + H + H * H + H + H + 1  # 1153
LINEAR, LOG = 0, 1
BETA1, BETA2, ADAM_EPS = 0.9, 0.999, 1e-8
SIGN = np.uint64(1 << 63)


INIT_TAG = 0x43444621  # fourth counter word of the initialisation draws
INIT_SCALE = float(np.sqrt(6.0 / H))


def init(seed: int):
    """Initial parameters from Philox4x32-10 words: parameter k draws
    u = (x0 >> 8) 2^-24 from counter (k, 0, 0, INIT_TAG) and key = the seed
    halves.  Hidden-1 units alternate in sign with |w1| in [4, 8) and knots
    -b1/w1 spread evenly over [0, 1] (a 1-D piecewise-linear basis); the
    other weights are uniform in +-sqrt(6/32); b2 = 0.1, b3 = 0.5."""
    from . import philox4x32_10
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    u = np.empty(NPARAM)
    for k in range(NPARAM):
        x = philox4x32_10((k, 0, 0, INIT_TAG), key)
        u[k] = float(int(x[0]) >> 8) * 2.0 ** -24
    w1 = np.array([(1.0 if i % 2 == 0 else -1.0) * (1.0 + u[i]) * 4.0 for i in range(H)])
    b1 = np.array([-w1[i] * (i + 0.5) / H for i in range(H)])
    W2 = ((2.0 * u[2 * H:2 * H + H * H] - 1.0) * INIT_SCALE).reshape(H, H)
    b2 = np.full(H, 0.1)
    o = 2 * H + H * H + H
    w3 = (2.0 * u[o:o + H] - 1.0) * INIT_SCALE
    return pack(w1, b1, W2, b2, w3, 0.5)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (NPARAM,)
    o = 0
    w1 = theta[o:o + H]; o += H
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].reshape(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    w3 = theta[o:o + H]; o += H
    b3 = theta[o]
    return w1, b1, W2, b2, w3, b3


def pack(w1, b1, W2, b2, w3, b3):
    return np.concatenate([np.ravel(w1), np.ravel(b1), np.ravel(W2), np.ravel(b2), np.ravel(w3),
                           np.array([b3], dtype=np.float64)]).astype(np.float64)


def ordered_bits(keys, key_type="u64"):
    k = np.ascontiguousarray(keys)
    if key_type == "i64":
        return k.astype(np.int64).view(np.uint64) ^ SIGN
    return k.astype(np.uint64)


def raw_feature(u, mode):
    """The feature before the affine map: u itself or log2(1 + u), as float64."""
    u = np.asarray(u, dtype=np.uint64)
    f = u.astype(np.float64)
    return np.log2(1.0 + f) if mode == LOG else f


def feature(keys, mode, lo, hi, key_type="u64"):
    """phi(key) in [0, 1]: (raw - lo) / (hi - lo), clipped."""
    r = raw_feature(ordered_bits(keys, key_type), mode)
    return np.clip((r - lo) / (hi - lo), 0.0, 1.0)


def forward(theta, x):
    """Network output and the activations the backward pass needs."""
    w1, b1, W2, b2, w3, b3 = unpack(theta)
    x = np.asarray(x, dtype=np.float64)
    z1 = np.outer(x, w1) + b1          # (n, 32)
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2                # (n, 32)
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3                   # (n,)
    return y, (x, h1, h2)


def loss(theta, x, t):
    y, _ = forward(theta, x)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def grad(theta, x, t):
    """dL/dtheta of the mean squared error, by the chain rule."""
    w1, b1, W2, b2, w3, b3 = unpack(theta)
    y, (x, h1, h2) = forward(theta, x)
    n = x.shape[0]
    d = 2.0 * (y - np.asarray(t, dtype=np.float64)) / n   # dL/dy_b
    g_b3 = d.sum()
    g_w3 = h2.T @ d
    dz2 = np.outer(d, w3) * (h2 > 0.0)                     # dL/dz2
    g_b2 = dz2.sum(axis=0)
    g_W2 = dz2.T @ h1                                      # (32, 32): [i, j] = sum_b dz2[b, i] h1[b, j]
    dz1 = (dz2 @ W2) * (h1 > 0.0)                          # dL/dz1
    g_b1 = dz1.sum(axis=0)
    g_w1 = dz1.T @ x
    return pack(g_w1, g_b1, g_W2, g_b2, g_w3, g_b3), float(np.mean((y - t) ** 2))


def adam_step(theta, m, v, g, step, lr):
    """One Adam update; step counts from 1.  Returns (theta, m, v)."""
    m = BETA1 * m + (1.0 - BETA1) * g
    v = BETA2 * v + (1.0 - BETA2) * g * g
    mhat = m / (1.0 - BETA1 ** step)
    vhat = v / (1.0 - BETA2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + ADAM_EPS), m, v


def train(theta, x, t, steps, lr, m=None, v=None, step0=0):
    """`steps` full-batch Adam steps; returns (theta, m, v, last loss)."""
    m = np.zeros(NPARAM) if m is None else m
    v = np.zeros(NPARAM) if v is None else v
    L = None
    for k in range(steps):
        g, L = grad(theta, x, t)
        theta, m, v = adam_step(theta, m, v, g, step0 + k + 1, lr)
    return theta, m, v, L


def round_bf16(theta):
    """Each parameter as a bfloat16 network uses it: its float32 value rounded
    to the nearest bfloat16 (the top 16 bits of a float32), ties to even,
    returned as float64.  Rounding adds 0x7FFF plus the lowest kept bit to
    the float32 bit pattern and clears the 16 dropped bits."""
    b = np.asarray(theta, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def targets(p, per, delta):
    """CDF targets of the proposed cuts: for splitter i = 1..p-1 and
    k = 0..per-1, i/p + delta (2k/(per-1) - 1) (just i/p when per = 1),
    clipped to [0, 1]; splitter-major order."""
    out = []
    for i in range(1, p):
        for k in range(per):
            off = 0.0 if per == 1 else delta * (2.0 * k / (per - 1) - 1.0)
            out.append(min(1.0, max(0.0, i / p + off)))
    return np.array(out, dtype=np.float64)


def propose(theta, p, mode, lo, hi, key_type="u64", iters=40, per=1, delta=0.0):
    """Keys of the proposed cuts: for each target tau (see targets), bisection
    for the smallest x in [0, 1] with y(x) >= tau, then the inverse feature
    map."""
    tau_all = targets(p, per, delta)
    out = np.empty(tau_all.shape[0], dtype=np.uint64)
    for q, tau in enumerate(tau_all):
        a, b = 0.0, 1.0
        for _ in range(iters):
            mid = 0.5 * (a + b)
            if forward(theta, np.array([mid]))[0][0] < tau:
                a = mid
            else:
                b = mid
        out[q] = key_of_feature(b, mode, lo, hi)
    if key_type == "i64":
        return (out ^ SIGN).view(np.int64)
    return out


def key_of_feature(x, mode, lo, hi):
    """Inverse of the feature map (ordered key bits), clamped to [0, 2^64 - 1]."""
    r = lo + x * (hi - lo)
    u = (2.0 ** r) - 1.0 if mode == LOG else r
    if not u > 0.0:
        return np.uint64(0)
    if u >= 18446744073709551615.0:
        return np.uint64(2**64 - 1)
    return np.uint64(int(u))
