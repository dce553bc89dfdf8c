"""CPU oracle of the surrogate MLP: forward, MSE loss, backward, Adam in FP64.

TEST INFRASTRUCTURE ONLY (tests, smoke, bench CPU baseline); shares no code
with the CUDA kernels. Textbook formulas:
  z_l = W_l h_{l-1} + b_l, h_l = GELU(z_l) = z Phi(z) (Phi the standard normal CDF, exact
  via erf), y = w5 . h_4 + b5, L = mean (y - t)^2;
  dL/dy = 2 (y - t) / n; dz_4 = dy w5 * GELU'(z_4); dz_{l-1} = (W_l^T dz_l) * GELU'(z_{l-1});
  dW_l = sum_rows dz_l h_{l-1}^T, db_l = sum_rows dz_l; GELU'(z) = Phi(z) + z phi(z);
  Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
  w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
With bf16=True, the values the method stores in BF16 (inputs, weights, activations h_l
and the back-propagated dz_l) are rounded to BF16 (via FP32, round-to-nearest-even) at
the same points; all arithmetic stays FP64.
"""

import math

import numpy as np

from workloads import mlp as L

_erf = np.vectorize(math.erf, otypes=[np.float64])


def bf16(x):
    """Round to bfloat16 (through float32, round to nearest even), returned as float64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    rounded = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def _r(x, on):
    return bf16(x) if on else np.asarray(x, dtype=np.float64)


def forward(p, X, bf=True):
    """p: one member's parameter dict; X: [n, 128]. Returns (y, cache)."""
    h = _r(X, bf)
    cache = {"h0": h}
    for l in range(1, 5):
        W = _r(p[f"W{l}"], bf)
        z = h @ W.T + np.asarray(p[f"b{l}"], np.float64)
        h = _r(gelu(z), bf)
        cache[f"z{l}"], cache[f"h{l}"] = z, h
    y = h @ np.asarray(p["w5"], np.float64) + float(p["b5"][0])
    return y, cache


def loss_and_grads(p, X, t, bf=True):
    """MSE loss and gradients (dict like p) for one member on rows X, targets t."""
    n = len(t)
    y, c = forward(p, X, bf)
    e = y - np.asarray(t, np.float64)
    loss = float(np.mean(e * e))
    dy = 2.0 * e / n
    g = {}
    w5 = np.asarray(p["w5"], np.float64)
    g["w5"] = dy @ c["h4"]
    g["b5"] = np.array([dy.sum()])
    dz = _r(np.outer(dy, w5) * gelu_grad(c["z4"]), bf)
    for l in range(4, 0, -1):
        g[f"W{l}"] = dz.T @ c[f"h{l - 1}"]
        g[f"b{l}"] = dz.sum(axis=0)
        if l > 1:
            W = _r(p[f"W{l}"], bf)
            dz = _r((dz @ W) * gelu_grad(c[f"z{l - 1}"]), bf)
    return loss, y, g


def adam(w, g, m, v, t, lr, b1, b2, eps):
    """One Adam step on flat float64 arrays; returns (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    w = w - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return w, m, v


def flatten(g, members_flat_shape=None):
    """Pack a gradient dict into the flat per-member layout (float64, length L.P)."""
    out = np.zeros(L.P, dtype=np.float64)
    for l, (fin, fout) in enumerate(L.LAYERS):
        out[L.OFF_W[l]:L.OFF_W[l] + fin * fout] = np.asarray(g[f"W{l + 1}"]).ravel()
        out[L.OFF_B[l]:L.OFF_B[l] + fout] = g[f"b{l + 1}"]
    out[L.OFF_W5:L.OFF_W5 + L.WID] = g["w5"]
    out[L.OFF_B5] = g["b5"][0]
    return out
