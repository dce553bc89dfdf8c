"""GPU parity of the fused ensemble forward (one persistent tcgen05 launch per
call, BF16 or with layers 2-4 on E4M3 codes) with the FP64 oracle.

Tolerances. BF16: as for the layer-by-layer forward (one BF16 step, 2^-8, per
stored activation, through four layers): |dy| <= 2e-2 (1 + |y|). FP8: the
E4M3 codes of the weights are integers decided in FP32 on both sides and must
match exactly; the activation codes follow values that the GPU computes in
FP32 with the hardware tanh (about 2^-11 relative) and the oracle in FP64, so a code can land one E4M3 step (2^-3 relative) away.
Perturbing the oracle's pre-quantisation activations by up to 2^-8 moves its
outputs by at most 0.034 on these models (0.003 median); the test allows
|dy| <= 5e-2 (1 + |y|) and a median of 1e-2.
"""

import numpy as np
import pytest

from oracle import surrogate_oracle as S
from workloads import mlp as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch

    from paper_1701_08547_gb300 import build

    build.build()
    assert torch.cuda.is_available()
    return torch.device("cuda:0")


def feats(n, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    X = np.zeros((n, L.IN))
    X[:, :L.FEATURES] = scale * rng.standard_normal((n, L.FEATURES))
    return S.bf16(X)


def to_dev(X, dev):
    import torch

    return torch.from_numpy(X.astype(np.float32)).to(torch.bfloat16).to(dev)


def make(members, seed0=5):
    from paper_1701_08547_gb300.surrogate import Surrogate

    s = Surrogate(members=members, batch=512)
    flat = L.init_params(members, [seed0 + m for m in range(members)])
    rng = np.random.default_rng(seed0)
    a = flat.reshape(members, L.P)
    for l in range(4):
        a[:, L.OFF_B[l]:L.OFF_B[l] + L.WID] = 0.1 * rng.standard_normal((members, L.WID))
    a[:, L.OFF_B5] = 0.25
    s.set_params(a.ravel())
    return s, a.ravel()


@pytest.mark.parametrize("n", [1, 127, 1000])
def test_fused_bf16_matches_oracle(dev, n):
    s, flat = make(3)
    X = feats(n, 1)
    s.set_forward_mode(s.FWD_FUSED_BF16)
    pred = s.forward(to_dev(X, dev)).cpu().numpy()
    s.check()
    for m, p in enumerate(L.unpack(flat, 3)):
        y, _ = S.forward(p, X, bf=True)
        err = np.abs(pred[m] - y)
        assert np.all(err <= 2e-2 * (1 + np.abs(y))), err.max()
        assert np.median(err) < 2e-3


def test_fused_and_layered_agree(dev):
    """Same BF16 operands, FP32 accumulation in tensor memory in both; the head sums
    in a different order."""
    s, _ = make(5)
    X = to_dev(feats(3000, 9), dev)
    s.set_forward_mode(s.FWD_LAYERED)
    a = s.forward(X).cpu().numpy()
    s.set_forward_mode(s.FWD_FUSED_BF16)
    b = s.forward(X).cpu().numpy()
    s.check()
    assert np.all(np.abs(a - b) <= 1e-2 * (1 + np.abs(a))), np.abs(a - b).max()
    assert np.median(np.abs(a - b)) < 1e-3


def test_fused_many_units_per_cta(dev):
    """40,000 rows x 5 members = 1,565 (tile, member) units: several units per CTA on
    both chains, a ragged last tile; sampled rows against the oracle."""
    s, flat = make(5)
    n = 40000
    X = feats(n, 4)
    s.set_forward_mode(s.FWD_FUSED_BF16)
    pred = s.forward(to_dev(X, dev)).cpu().numpy()
    s.check()
    rows = np.concatenate([np.arange(0, 256), np.random.default_rng(2).choice(n, 600, replace=False),
                           np.arange(n - 200, n)])
    for m, p in enumerate(L.unpack(flat, 5)):
        y, _ = S.forward(p, X[rows], bf=True)
        err = np.abs(pred[m, rows] - y)
        assert np.all(err <= 2e-2 * (1 + np.abs(y))), (m, err.max())


def test_fp8_codes_match_oracle(dev):
    import torch

    s, flat = make(2)
    for step in range(2):  # before and after an Adam step (the codes follow the master weights)
        master = s.get(s.GET_PARAMS).reshape(2, L.P)
        codes = s.get(s.GET_FP8_CODES).reshape(2, 3, 256, 256)
        scales = s.get(s.GET_FP8_SCALES).reshape(2, 3, 256)
        for m, p in enumerate(L.unpack(master.ravel(), 2)):
            for l in range(3):
                q, sc = S.quantize_matrix(p[f"W{l + 2}"])
                assert np.array_equal(scales[m, l], np.full(256, sc, np.float32)), (step, m, l)
                assert np.array_equal(codes[m, l], q), (step, m, l)
        X = to_dev(feats(256, 3), dev)
        t = torch.randn(256, device=dev)
        s.train_step(X, t, apply_update=True)


@pytest.mark.parametrize("n", [100, 5000])
def test_fused_fp8_matches_oracle(dev, n):
    s, flat = make(3)
    X = feats(n, 6)
    s.set_forward_mode(s.FWD_FUSED_FP8)
    pred = s.forward(to_dev(X, dev)).cpu().numpy()
    s.check()
    for m, p in enumerate(L.unpack(flat, 3)):
        y = S.forward_fp8(p, X)
        err = np.abs(pred[m] - y)
        assert np.all(err <= 5e-2 * (1 + np.abs(y))), err.max()
        assert np.median(err) < 1e-2


def test_fused_empty_input(dev):
    import torch

    s, _ = make(2)
    pred = torch.full((2, 0), 7.0, device=dev)
    s.forward(torch.empty((0, L.IN), dtype=torch.bfloat16, device=dev), pred)
    s.check()
