"""FP64 CPU oracle of the learned threshold proposer.

TEST INFRASTRUCTURE ONLY (see the package docstring): the GPU proposer's
features, forward pass, loss, gradients and optimiser step are checked
against these plain numpy definitions. Nothing here is imported by the
product package.

The proposer is not part of the paper (whose method is the exhaustive
search of section II-C); it is a network that reads a coarse view of a
histogram and proposes thresholds, so that the exact search can be confined
to a window of candidates. Its definition, written out here once:

  features  x_k = log1p(sum_{j=16k}^{16k+15} h_j) / log1p(N), k = 0..255,
            for a 4096-level histogram h with N counts (all zero if N = 0);
  network   z1 = W1 x + b1, a1 = GELU(z1), z2 = W2 a1 + b2, a2 = GELU(z2),
            z3 = W3 a2 + b3 (4096 logits, one per threshold level), with
            W1, W2: 256 x 256, W3: 4096 x 256, GELU(z) = z Phi(z) =
            z (1 + erf(z / sqrt 2)) / 2;
  loss      mean over the batch of the cross-entropy -sum_t y_t log
            softmax(z3)_t against a target distribution y;
  target    uniform over the thresholds that give the exact search's
            partition: t* and the empty levels that follow it;
  optimiser Adam (Kingma & Ba 2015) with bias correction.

The 2-D search's proposer is the same network reading a 256 x 256 grey x
mean histogram: x_f = log1p(count of the 16 x 16 block f) / log1p(N) with
f = 16 * (grey block) + (mean block), and its 4096 logits score cells of
4 x 4 threshold pairs, cell 64 * (t // 4) + s // 4; its target is the cell of
the exact search's pair.

Parameters travel as one flat float vector in the order W1, b1, W2, b2, W3,
b3, each matrix row-major [out][in].
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

NIN, NHID, NOUT = 256, 256, 4096
GROUP = 16                      # histogram levels per feature
SHAPES = [("W1", (NHID, NIN)), ("b1", (NHID,)), ("W2", (NHID, NHID)), ("b2", (NHID,)),
          ("W3", (NOUT, NHID)), ("b3", (NOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(flat):
    """Flat parameter vector -> dict of FP64 arrays (views reshaped)."""
    flat = np.asarray(flat, np.float64)
    assert flat.size == NPARAM, flat.size
    out, o = {}, 0
    for name, s in SHAPES:
        n = int(np.prod(s))
        out[name] = flat[o:o + n].reshape(s)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SHAPES])


def features(h):
    """x[nh][256] from histograms h[nh][4096]: the log of the counts of each
    group of 16 levels, over the log of the total count."""
    h = np.asarray(h, np.float64).reshape(-1, NOUT)
    s = h.reshape(h.shape[0], NIN, GROUP).sum(axis=2)
    n = h.sum(axis=1, keepdims=True)
    den = np.log1p(n)
    return np.divide(np.log1p(s), den, out=np.zeros_like(s), where=den > 0)   # empty histogram: all zero


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    """d GELU / dz = Phi(z) + z phi(z)."""
    phi = np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * phi


def forward(params, x):
    """Logits z3[B][4096] and the intermediate values (z1, a1, z2, a2)."""
    p = unpack(params)
    x = np.asarray(x, np.float64)
    z1 = x @ p["W1"].T + p["b1"]
    a1 = gelu(z1)
    z2 = a1 @ p["W2"].T + p["b2"]
    a2 = gelu(z2)
    z3 = a2 @ p["W3"].T + p["b3"]
    return z3, (z1, a1, z2, a2)


def log_softmax(z):
    m = z.max(axis=1, keepdims=True)
    return z - m - np.log(np.exp(z - m).sum(axis=1, keepdims=True))


def loss(z3, y):
    """Mean cross-entropy of targets y[B][4096] against logits z3."""
    return float(-(np.asarray(y, np.float64) * log_softmax(z3)).sum() / z3.shape[0])


def grads(params, x, y):
    """(loss, flat gradient) by the chain rule, written out layer by layer."""
    p = unpack(params)
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    z3, (z1, a1, z2, a2) = forward(params, x)
    B = x.shape[0]
    d3 = (np.exp(log_softmax(z3)) - y) / B        # dL/dz3
    g = {"W3": d3.T @ a2, "b3": d3.sum(axis=0)}
    da2 = d3 @ p["W3"]
    d2 = da2 * gelu_grad(z2)
    g["W2"] = d2.T @ a1
    g["b2"] = d2.sum(axis=0)
    da1 = d2 @ p["W2"]
    d1 = da1 * gelu_grad(z1)
    g["W1"] = d1.T @ x
    g["b1"] = d1.sum(axis=0)
    return loss(z3, y), pack(g)


def targets(h, t_star):
    """Target distributions y[nh][4096]: uniform over t* and the empty
    levels after it (the thresholds that give t*'s partition). t* = -1
    (no valid threshold) gives an all-zero row."""
    h = np.asarray(h).reshape(-1, NOUT)
    y = np.zeros(h.shape, np.float64)
    for i, t in enumerate(np.asarray(t_star).reshape(-1)):
        if t < 0:
            continue
        e = t + 1
        while e < NOUT - 1 and h[i, e] == 0:
            e += 1
        y[i, t:e] = 1.0 / (e - t)
    return y


def adam_step(params, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1): returns (params, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as FP64: the
    weights the GPU forward pass multiplies with."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def features2d(h2):
    """2-D proposer features [n][256] of 2-D histograms [n][256][256] (zero
    for an empty histogram)."""
    h = np.asarray(h2, np.float64).reshape(-1, 256, 256)
    blocks = h.reshape(-1, 16, 16, 16, 16).sum(axis=(2, 4)).reshape(-1, 256)
    n = h.reshape(h.shape[0], -1).sum(axis=1, keepdims=True)
    return np.divide(np.log1p(blocks), np.log1p(n), out=np.zeros_like(blocks), where=n > 0)


def cell2d(t, s):
    """Cell of a 2-D threshold pair: 64 * (t // 4) + s // 4."""
    return 64 * (np.asarray(t) // 4) + np.asarray(s) // 4
