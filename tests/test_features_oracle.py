"""Pins of the oracle's surrogate features by hand-worked values (each feature
is a fixed scaling of a quantity pinned elsewhere)."""

import math

import numpy as np
import pytest

from workloads import archs, gen


def test_features_hand_worked(oracle):
    a = archs.arch("sm_103")
    d = gen.descriptors(1, 1, "dense")
    d["n"][0] = [128.0, 2.0, 64.0, 32.0, 32.0, 32.0, 16.0]  # n_c = IPC_c: one cycle per class
    d["r0"][0], d["s0"][0], d["d"][0] = 16, 0, np.float32(0.25)
    f = oracle.features(a, d[0], 256, 2432, 1, 100)
    # occupancy: T=256 -> 8 warps -> G_W = 8; R=16 -> 512 regs/warp -> 128 warps -> G_R = 16;
    # S=0 -> 1 KB per block -> 228 blocks; B* = 8 (warp-limited), W* = 64
    assert f[19] == 8 / 32 and f[26] == 8 / 32 and f[27] == 16 / 32 and f[28] == 64 / 32
    assert f[29] == 8 / 32 and f[30] == 1.0 and f[31] == 1.0
    assert (f[32], f[33], f[34]) == (1.0, 0.0, 0.0)
    assert f[18] == pytest.approx(0.8) and f[21] == pytest.approx(math.log2(2432) / 16)
    assert f[22] == 1 / 8 and f[23] == 1.0 and f[24] == 16 / 255 and f[25] == 512 / 8192
    # G = 2 full waves of 152 x 8 slots: waves = 2, par = n_SM, hide = 1, lane = 1
    assert f[35] == pytest.approx(0.1) and f[36] == 1.0 and f[37] == 1 / 32 and f[20] == 1.0
    # cost = 1.25 * 1024 * 7 / 152 (closed form); C_nm = 1.25 * 1024 * 5, C_m = 1.25 * 1024 * 2
    assert f[38] == pytest.approx(math.log2(1.25 * 1024 * 7 / 152 + 1) / 40)
    assert f[39] == pytest.approx(math.log2(1.25 * 1024 * 5 + 1) / 40)
    assert f[40] == pytest.approx(math.log2(1.25 * 1024 * 2 + 1) / 40)
    assert f[42] == 233472 / 233472 and f[43] == 1024 / 65536
    assert f[7] == pytest.approx(128 / (306 + 1)) and f[0] == pytest.approx(math.log2(129) / 20)
    assert f[14] == pytest.approx(math.log2(131 / 65) / 10)
    assert f[44] == pytest.approx(math.log2(33) / 20)
    # residuals of the cost features under BF16 storage: f38 = log2(59.947...) / 40 =
    # 0.1476406..., which lies in [1/8, 1/4) where BF16 (8 significant bits) has spacing
    # 2^-10; it rounds to 151 / 1024 = 0.1474609375, so f45 = 256 (0.1476406... - 151 / 1024)
    # = 0.0459...
    cost = 1.25 * 1024 * 7 / 152
    want38 = math.log2(cost + 1) / 40
    assert abs(want38 - 0.1476406) < 1e-7
    assert f[45] == pytest.approx(256 * (want38 - 151 / 1024), rel=1e-9)
    assert abs(f[45] - 0.0459969) < 1e-6
    for j, fj in ((45, f[38]), (46, f[39]), (47, f[40])):
        step = 2.0 ** (math.floor(math.log2(fj)) - 7)  # BF16 spacing at fj
        assert abs(f[j]) <= 128 * step                  # at most half a BF16 step, times 256
        assert (fj - f[j] / 256) / step == pytest.approx(round((fj - f[j] / 256) / step), abs=1e-9)


def test_bf16_residual_features_reconstruct_the_cost_terms(oracle):
    """f38 + f45 / 256 (and 39/46, 40/47) gives the cost features back to about 2^-16 once
    every feature is stored in BF16 (the surrogate's input precision)."""
    from oracle import surrogate_oracle as S

    a, ax = archs.arch("sm_103"), gen.axes()
    d = gen.descriptors(30, 9, "uneven")
    rng = np.random.default_rng(1)
    worst = 0.0
    for i in range(30):
        n = int(gen.space_sizes(d[i:i + 1])[0])
        for p in rng.integers(0, n, 20):
            f = oracle.features(a, d[i], *oracle.decode_point(d[i], ax, p))
            if f[29] == 0:
                continue
            b = S.bf16(f)
            for hi, lo in ((38, 45), (39, 46), (40, 47)):
                rec = b[hi] + b[lo] / 256
                worst = max(worst, abs(rec - f[hi]) / f[hi])
                assert abs(b[hi] - f[hi]) / f[hi] > 2.0 ** -30 or b[lo] == 0  # hi alone is coarse
    assert worst < 2.0 ** -15, worst


def test_invalid_point_features(oracle):
    a = archs.arch("sm_103")
    d = gen.descriptors(1, 1, "dense")
    d["r0"][0] = 300
    f = oracle.features(a, d[0], 256, 64, 1, 100)
    assert f[29] == 0 and f[30] == 0 and f[38] == 0 and f[32:35].sum() == 0
