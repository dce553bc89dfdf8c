"""Pins of the MLP oracle: GELU values, gradients by central differences,
Adam's first step in closed form, BF16 and E4M3 rounding against torch's
conversions, the FP8 forward against the FP64 forward."""

import math

import numpy as np
import pytest

from oracle import surrogate_oracle as S
from workloads import mlp as L


def test_gelu_values():
    torch = pytest.importorskip("torch")
    z = np.concatenate([np.linspace(-8, 8, 161), [1.0, -1.0, 0.5, 30.0, -30.0]])
    want = torch.nn.functional.gelu(torch.tensor(z, dtype=torch.float64), approximate="tanh").numpy()
    assert np.allclose(S.gelu(z), want, rtol=1e-14, atol=1e-15)
    # tanh form against the erf definition z Phi(z): Phi(1) = 0.8413447460685429; the two
    # forms differ by less than 1e-3 everywhere (Hendrycks & Gimpel)
    assert abs(S.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-3
    exact = np.array([0.5 * x * (1 + math.erf(x / math.sqrt(2))) for x in z])
    assert np.max(np.abs(S.gelu(z) - exact)) < 1e-3
    assert S.gelu(np.array([0.0]))[0] == 0.0
    assert S.gelu_grad(np.array([0.0]))[0] == 0.5
    zz = np.linspace(-4, 4, 33)
    h = 1e-6
    fd = (S.gelu(zz + h) - S.gelu(zz - h)) / (2 * h)
    assert np.allclose(S.gelu_grad(zz), fd, atol=1e-8)


def test_e4m3_rounding():
    """E4M3 (OCP FP8): against torch's float8_e4m3fn conversion inside the finite range, ties to
    even, subnormals, saturation."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(50000) * 50, rng.standard_normal(50000) * 0.01,
                        rng.uniform(-448, 448, 20000)]).astype(np.float32)
    want = torch.tensor(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(S.e4m3(x), want)
    # 1 + 1/16 lies halfway between 1 and 1.125 (even: 1); 1 + 3/16 between 1.125 and 1.25 (even: 1.25)
    cases = {1 + 1 / 16: 1.0, 1 + 3 / 16: 1.25, 2.0 ** -9: 2.0 ** -9, 2.0 ** -10: 0.0, 3 * 2.0 ** -10: 2.0 ** -8,
             448.0: 448.0, 460.0: 448.0, 1e6: 448.0, -1e6: -448.0, 0.0: 0.0, 240.0: 240.0, 250.0: 256.0}
    for a, b in cases.items():
        assert S.e4m3(np.array([a]))[0] == b, a


def test_fp8_quantization_and_forward():
    flat = L.init_params(1, [5])
    p = L.unpack(flat, 1)[0]
    q, s = S.quantize_matrix(p["W2"])
    assert q.shape == (256, 256) and s.dtype == np.float32
    assert np.max(np.abs(q)) == 448.0                        # the largest weight maps to 448
    assert np.array_equal(q, S.e4m3(q))                     # codes lie on the grid
    W = np.asarray(p["W2"], np.float64)
    err = np.abs(q * np.float64(s) - W)
    # half a step of 3 mantissa bits relative to each weight, or half the subnormal spacing 2^-9
    # of the codes for the few weights below the normal range
    assert np.all(err <= np.maximum(2.0 ** -4 * np.abs(W), 2.0 ** -10 * s) * 1.0001)
    X = np.zeros((300, L.IN))
    X[:, :L.FEATURES] = np.random.default_rng(1).standard_normal((300, L.FEATURES))
    y8 = S.forward_fp8(p, X)
    y, _ = S.forward(p, X, bf=False)
    err = np.abs(y8 - y)
    assert np.max(err) < 0.1 * (1 + np.max(np.abs(y))) and np.median(err) < 0.02, (err.max(), np.median(err))


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.concatenate([np.array([1.0, 1.00390625, 1.01171875, -2.5e-3, 3.0e5, 0.0]),
                        np.random.default_rng(0).standard_normal(2000) * 10.0])
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(S.bf16(x), want)
    assert S.bf16(np.array([1.00390625]))[0] == 1.0        # halfway, rounds to even
    assert S.bf16(np.array([1.01171875]))[0] == 1.015625   # halfway, rounds to even


def _net(seed=3):
    flat = L.init_params(1, [seed]).astype(np.float64)
    p = L.unpack(flat, 1)[0]
    for k in p:
        p[k] = p[k].copy()
    rng = np.random.default_rng(seed)
    for l in range(1, 5):
        p[f"b{l}"] += 0.1 * rng.standard_normal(p[f"b{l}"].shape)
    p["b5"][0] = 0.3
    X = np.zeros((6, L.IN))
    X[:, :L.FEATURES] = rng.standard_normal((6, L.FEATURES))
    t = rng.standard_normal(6)
    return p, X, t


def test_backward_matches_central_differences():
    """Exact-arithmetic mode: analytic gradients equal central differences of the loss."""
    p, X, t = _net()
    loss, _, g = S.loss_and_grads(p, X, t, bf=False)
    rng = np.random.default_rng(1)
    h = 1e-6
    for name in ["W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4", "w5", "b5"]:
        arr = p[name]
        for _ in range(4):
            idx = tuple(rng.integers(0, s) for s in arr.shape)
            if name == "W1":
                idx = (idx[0], idx[1] % L.FEATURES)
            old = arr[idx]
            arr[idx] = old + h
            lp = S.loss_and_grads(p, X, t, bf=False)[0]
            arr[idx] = old - h
            lm = S.loss_and_grads(p, X, t, bf=False)[0]
            arr[idx] = old
            fd = (lp - lm) / (2 * h)
            assert g[name][idx] == pytest.approx(fd, rel=1e-5, abs=1e-9), (name, idx)


def test_adam_first_step_closed_form():
    """t = 1: bias-corrected m = g and v = g^2, so the step is lr g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    w0 = np.array([1.0, 1.0, 1.0, 1.0])
    w, m, v = S.adam(w0, g, np.zeros(4), np.zeros(4), 1, 1e-3, 0.9, 0.999, 1e-8)
    assert np.allclose(w, w0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-14, atol=0)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_flat_layout_round_trip():
    p, X, t = _net()
    _, _, g = S.loss_and_grads(p, X, t, bf=False)
    flat = S.flatten(g)
    back = L.unpack(flat, 1)[0]
    for k in g:
        assert np.array_equal(np.asarray(back[k]).ravel(), np.asarray(g[k]).ravel())


def test_fp8_forward_worked_example():
    """A single path through the network, worked by hand: W1[0][0] = 1, W2[0][0] = 1/2,
    W3[0][0] = -1/4, W4[0][0] = 2, w5[0] = 1, b5 = 1/2, every other weight and bias zero.
    Each one-entry matrix quantises to the code +-448 with scale |w| / 448 (zeros stay code 0),
    so layer l gives z = (s / 2) E4M3(2 h) (+-448) = (w / 2) E4M3(2 h).
    Input x = 1:
      h1 = gelu(1) = 0.84119..., 2 h1 = 1.68238 = 13.46 steps of 1/8 -> 13/8 = 1.625,
      z2 = 1.625 / 4 = 0.40625; h2 = gelu(z2) = 0.26719, 2 h2 = 0.53440 = 8.55 steps of
      1/16 -> 9/16 = 0.5625, z3 = -0.5625 / 8 = -0.0703125; h3 = gelu(z3) = -0.033186,
      2 h3 = -0.066371 = -8.4955 steps of 2^-7 -> -8/128 = -0.0625, z4 = -0.0625,
      y = gelu(-0.0625) + 1/2.
    Input x = 2:
      2 gelu(2) = 3.9092 = 15.64 steps of 1/4 -> 4.0, z2 = 1; 2 gelu(1) -> 1.625 as above,
      z3 = -0.203125; 2 gelu(z3) = -0.17043 = -10.91 steps of 2^-6 -> -11/64, z4 = -11/64,
      y = gelu(-11/64) + 1/2.
    The scale |w| / 448 is rounded to FP32 (as the kernel takes it), so these hold to about
    2^-24 relative. The FP64 forward without quantisation differs (z2 = gelu(1) / 2 etc.) by
    far more, so the example fixes where E4M3 rounding happens and the 2h scaling."""
    def g(z):
        return 0.5 * z * (1.0 + math.tanh(math.sqrt(2.0 / math.pi) * (z + 0.044715 * z ** 3)))

    flat = np.zeros(L.P, dtype=np.float32)
    p = L.unpack(flat, 1)[0]
    p["W1"][0, 0], p["W2"][0, 0], p["W3"][0, 0], p["W4"][0, 0] = 1.0, 0.5, -0.25, 2.0
    p["w5"][0], p["b5"][0] = 1.0, 0.5
    X = np.zeros((2, L.IN))
    X[0, 0], X[1, 0] = 1.0, 2.0
    y = S.forward_fp8(p, X)
    assert abs(y[0] - (g(-0.0625) + 0.5)) < 1e-8
    assert abs(y[1] - (g(-11.0 / 64.0) + 0.5)) < 1e-8
    # the intermediate values stated above
    assert abs(g(1.0) - 0.8411919906) < 1e-9 and abs(g(0.40625) - 0.2671909895) < 1e-9
    y_bf, _ = S.forward(p, X, bf=False)
    assert abs(y_bf[0] - y[0]) > 1e-4 and abs(y_bf[1] - y[1]) > 1e-4
