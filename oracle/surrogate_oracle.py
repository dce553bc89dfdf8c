"""CPU oracle of the surrogate MLP: forward, MSE loss, backward, Adam in FP64.

TEST INFRASTRUCTURE ONLY (tests, smoke, bench CPU baseline); shares no code
with the CUDA kernels. Textbook formulas:
  z_l = W_l h_{l-1} + b_l, h_l = GELU(z_l), GELU in its tanh form (Hendrycks & Gimpel):
  GELU(z) = z/2 (1 + tanh(u)), u = sqrt(2/pi) (z + 0.044715 z^3); y = w5 . h_4 + b5,
  L = mean (y - t)^2;
  dL/dy = 2 (y - t) / n; dz_4 = dy w5 * GELU'(z_4); dz_{l-1} = (W_l^T dz_l) * GELU'(z_{l-1});
  dW_l = sum_rows dz_l h_{l-1}^T, db_l = sum_rows dz_l;
  GELU'(z) = (1 + tanh u)/2 + z/2 (1 - tanh^2 u) sqrt(2/pi) (1 + 3 * 0.044715 z^2);
  Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
  w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
With bf16=True, the values the method stores in BF16 (inputs, weights, activations h_l
and the back-propagated dz_l) are rounded to BF16 (via FP32, round-to-nearest-even) at
the same points; all arithmetic stays FP64.

FP8 inference (forward_fp8): layers 2-4 take E4M3 operands (OCP FP8: 4 exponent bits,
bias 7, 3 mantissa bits, largest finite 448, subnormal spacing 2^-9). Each weight matrix
has one scale: s = max_{n,k} |W[n][k]| / 448 (1 if the matrix is zero), code = E4M3(W / s),
both steps in FP32 as the kernel takes them (the codes are integers: both sides decide
them in the same precision); activations are quantised with scale 1/2 (codes of 2 h).
Rounding to E4M3 is to nearest, ties to even, saturating at +-448.
"""

import math

import numpy as np

from workloads import mlp as L



def bf16(x):
    """Round to bfloat16 (through float32, round to nearest even), returned as float64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    rounded = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


GELU_K = math.sqrt(2.0 / math.pi)
GELU_C = 0.044715


def gelu(z):
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * z * (1.0 + np.tanh(GELU_K * (z + GELU_C * z ** 3)))


def gelu_grad(z):
    z = np.asarray(z, dtype=np.float64)
    t = np.tanh(GELU_K * (z + GELU_C * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_K * (1.0 + 3.0 * GELU_C * z * z)


E4M3_MAX = 448.0


def e4m3(x):
    """Round to the E4M3 grid (nearest, ties to even, saturating at +-448); float64 values."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    _, e = np.frexp(a)                           # a = m 2^e, m in [0.5, 1)
    E = np.maximum(e - 1, -6)                    # binade exponent; below 2^-6 the subnormal spacing
    step = np.ldexp(1.0, E - 3)                  # 3 mantissa bits
    q = np.minimum(np.rint(a / step) * step, E4M3_MAX)
    return np.copysign(q, x)


def quantize_matrix(W):
    """E4M3 quantisation of a weight matrix with one scale, in FP32 like the kernel:
    (codes, scale)."""
    W32 = np.asarray(W, dtype=np.float32)
    amax = np.float32(np.max(np.abs(W32)))
    s = np.float32(amax / np.float32(E4M3_MAX)) if amax > 0 else np.float32(1.0)
    return e4m3(W32 / s), s


def _r(x, on):
    return bf16(x) if on else np.asarray(x, dtype=np.float64)


def forward(p, X, bf=True):
    """p: one member's parameter dict; X: [n, 64]. Returns (y, cache)."""
    h = _r(X, bf)
    cache = {"h0": h}
    for l in range(1, 5):
        W = _r(p[f"W{l}"], bf)
        z = h @ W.T + np.asarray(p[f"b{l}"], np.float64)
        h = _r(gelu(z), bf)
        cache[f"z{l}"], cache[f"h{l}"] = z, h
    y = h @ np.asarray(p["w5"], np.float64) + float(p["b5"][0])
    return y, cache


def forward_fp8(p, X):
    """Forward with layer 1 in BF16 and layers 2-4 on E4M3 codes (see the module header):
    z_l = (s_l / 2) (E4M3(2 h_{l-1}) . codes_l) + b_l; the head reads h_4 unrounded."""
    h = bf16(X)
    z = h @ bf16(p["W1"]).T + np.asarray(p["b1"], np.float64)
    h = gelu(z)
    for l in range(2, 5):
        q, s = quantize_matrix(p[f"W{l}"])
        z = (e4m3(2.0 * h) @ q.T) * (0.5 * np.float64(s)) + np.asarray(p[f"b{l}"], np.float64)
        h = gelu(z)
    return h @ np.asarray(p["w5"], np.float64) + float(p["b5"][0])


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
