"""Pins of the MLP oracle: GELU values, gradients by central differences,
Adam's first step in closed form, BF16 rounding against torch's conversion."""

import math

import numpy as np
import pytest

from oracle import surrogate_oracle as S
from workloads import mlp as L


def test_gelu_values():
    # GELU(z) = z Phi(z): Phi(1) = 0.8413447460685429, Phi(-1) = 0.15865525393145707
    assert S.gelu(np.array([1.0]))[0] == pytest.approx(0.8413447460685429, rel=1e-15)
    assert S.gelu(np.array([-1.0]))[0] == pytest.approx(-0.15865525393145707, rel=1e-15)
    assert S.gelu(np.array([0.0]))[0] == 0.0
    assert S.gelu_grad(np.array([0.0]))[0] == 0.5
    z = np.linspace(-4, 4, 33)
    h = 1e-6
    fd = (S.gelu(z + h) - S.gelu(z - h)) / (2 * h)
    assert np.allclose(S.gelu_grad(z), fd, atol=1e-8)


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
