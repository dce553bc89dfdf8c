"""Oracle checks by invariants, brute force and library routines.

* occupancy: a search over block counts that allocates warps, registers and
  shared memory one block at a time (a different formulation from the
  closed forms of Eqs. 3-5) must find the same B*; B* never rises with more
  registers (or more shared memory at the same capacity) and never falls
  with a larger carveout.
* enumeration: the per-point output at canonical index i equals a direct
  evaluation of the configuration that i decodes to (carveout fastest).
* selection: the oracle's top-k equals numpy's lexsort of its own per-point
  FP32 costs; segmented top-k equals a stable argsort per segment.
"""

import numpy as np
import pytest

from workloads import archs, gen

ARCH_NAMES = list(archs.ARCHS)


def brute_force_blocks(a, T, R, S, carveout):
    """Largest block count that fits, by trying B = B_mp, B_mp-1, ..., 0."""
    warp = a["warp_size"]
    if T > a["max_threads_block"] or R > a["regs_thread_max"] or S > a["smem_block_max"]:
        return 0
    wb = -(-T // warp)
    s_alloc = -(-(S + a["smem_reserved_block"]) // a["smem_alloc_unit"]) * a["smem_alloc_unit"]
    caps = [c for c in a["smem_caps"] if 100 * c >= carveout * a["smem_caps"][-1] and c >= s_alloc]
    cap = caps[0] if caps else None
    for B in range(a["max_blocks_sm"], 0, -1):
        if B * wb > a["max_warps_sm"]:
            continue
        if R > 0:
            if a["reg_alloc_mode"] == 0:
                per_warp = -(-R * warp // a["reg_alloc_unit"]) * a["reg_alloc_unit"]
                if per_warp * wb > a["regs_block_max"]:
                    return 0
                gran = a["warp_alloc_gran"]
                groups = -(-(B * wb) // gran)  # warps are handed out in groups of `gran`
                if groups * gran * per_warp > a["regs_sm"]:
                    continue
            else:
                per_block = -(-R * warp * wb // a["reg_alloc_unit"]) * a["reg_alloc_unit"]
                if per_block > a["regs_block_max"] or B * per_block > a["regs_sm"]:
                    continue
        if s_alloc > 0:
            if cap is None or B * s_alloc > cap:
                continue
        return B
    return 0


@pytest.mark.parametrize("name", ARCH_NAMES)
def test_occupancy_matches_brute_force(oracle, name):
    a = archs.arch(name)
    rng = np.random.default_rng(7)
    Ts = list(range(32, 1025, 32)) + [1, 33, 48, 100, 1000, 1056]
    for _ in range(1500):
        T = int(rng.choice(Ts))
        R = int(rng.integers(0, a["regs_thread_max"] + 3))
        S = int(rng.integers(0, a["smem_block_max"] + 600)) if rng.random() < 0.8 else 0
        C = int(rng.choice([0, 10, 25, 50, 75, 100]))
        o = oracle.occupancy(a, T, R, S, C)
        assert o["B"] == brute_force_blocks(a, T, R, S, C), (T, R, S, C)


@pytest.mark.parametrize("name", ARCH_NAMES)
def test_occupancy_monotone(oracle, name):
    """B* non-increasing in R, and in S while the chosen capacity stays the
    same; non-decreasing in carveout; W* <= W_mp; B* <= B_mp."""
    a = archs.arch(name)
    rng = np.random.default_rng(3)
    for _ in range(300):
        T = int(rng.integers(1, 33)) * 32
        R = int(rng.integers(1, 100))
        S = int(rng.integers(0, 40000))
        C = int(rng.choice([0, 25, 50, 100]))
        o = oracle.occupancy(a, T, R, S, C)
        assert o["W"] <= a["max_warps_sm"] and o["B"] <= a["max_blocks_sm"]
        assert oracle.occupancy(a, T, R + 1, S, C)["B"] <= o["B"]
        assert oracle.occupancy(a, T, R + 8, S, C)["B"] <= o["B"]
        for dS in (1, 4096):
            o2 = oracle.occupancy(a, T, R, S + dS, C)
            assert o2["cap"] != o["cap"] or o2["B"] <= o["B"]
            assert o2["cap"] >= o["cap"] or not o2["valid"]
        for C2 in (25, 50, 100):
            if C2 >= C:
                assert oracle.occupancy(a, T, R, S, C2)["B"] >= o["B"]


def test_capacity_raised_to_fit_one_block(oracle):
    """Fermi at carveout 0 %: a 16 KB split holds one 12000-byte block; a
    16400-byte block (16512 after rounding to 128 B) does not fit it, so the
    48 KB split is used and two blocks fit (the preferred split is a hint,
    not a limit)."""
    a = archs.arch("sm_20")
    o1 = oracle.occupancy(a, 64, 16, 12000, 0)
    o2 = oracle.occupancy(a, 64, 16, 16400, 0)
    assert (o1["cap"], o1["G_S"]) == (16384, 1)
    assert (o2["cap"], o2["G_S"]) == (49152, 2)


def decode_index(desc, ax, i):
    """Canonical index -> (T, G, U, C) for a descriptor's space, carveout fastest."""
    m = int(desc["space_mask"])
    pos = lambda sh, w: [b for b in range(w) if (m >> (sh + b)) & 1]
    tp, gp, up, cp = pos(0, 32), pos(32, 16), pos(48, 8), pos(56, 4)
    i, ic = divmod(i, len(cp))
    i, iu = divmod(i, len(up))
    it, ig = divmod(i, len(gp))
    return ax["t"][tp[it]], ax["g"][gp[ig]], ax["u"][up[iu]], ax["c"][cp[ic]]


def test_enumeration_canonical_order(oracle):
    a = archs.arch("sm_103")
    ax = gen.axes()
    d = gen.descriptors(6, 5, "uneven")
    off = gen.point_offsets(d)
    r = oracle.evaluate(a, ax, d, 3, emit=True, offsets=off)
    rng = np.random.default_rng(1)
    for kk in range(len(d)):
        size = off[kk + 1] - off[kk]
        for i in rng.integers(0, size, 40):
            T, G, U, C = decode_index(d[kk], ax, int(i))
            R = int(d[kk]["r0"]) + 4 * (U - 1)
            o = oracle.occupancy(a, T, R, int(d[kk]["s0"]), C)
            at = off[kk] + i
            assert r["B"][at] == o["B"] and r["W"][at] == o["W"]
            if o["valid"]:
                c = oracle.cost32(a, d[kk]["n"], d[kk]["d"], U, T, G, o["B"], o["W"])
                assert np.float32(c) == r["cost32"][at]
            else:
                assert np.isinf(r["cost32"][at])


@pytest.mark.parametrize("space,k", [("dense128", 5), ("uneven", 7), ("dense", 16)])
def test_topk_equals_lexsort(oracle, space, k):
    a = archs.arch("sm_103")
    d = gen.descriptors(12, 2, space)
    off = gen.point_offsets(d)
    r = oracle.evaluate(a, gen.axes(), d, k, emit=True, offsets=off)
    for kk in range(len(d)):
        c = r["cost32"][off[kk]:off[kk + 1]]
        idx = np.arange(len(c))
        ok = np.isfinite(c)
        order = np.lexsort((idx[ok], c[ok]))[:k]
        want_i = np.full(k, -1, np.int32)
        want_c = np.full(k, np.inf, np.float32)
        want_i[:len(order)] = idx[ok][order]
        want_c[:len(order)] = c[ok][order]
        assert np.array_equal(r["idx"][kk], want_i)
        assert np.array_equal(r["cost"][kk], want_c)


def test_topk_pads_when_few_valid(oracle):
    """A kernel whose space is mostly invalid (too many registers) pads with (-1, +inf)."""
    a = archs.arch("sm_103")
    d = gen.descriptors(1, 9, "dense128")
    d["r0"] = 254            # only U=1 fits 255 registers, and then only blocks of <= 8 warps
    r = oracle.evaluate(a, gen.axes(), d, 16)
    n_valid = int(np.sum(r["idx"][0] >= 0))
    assert n_valid < 16 and np.all(np.isinf(r["cost"][0][n_valid:]))
    d["r0"] = 300            # every point invalid
    r = oracle.evaluate(a, gen.axes(), d, 4)
    assert np.all(r["idx"] == -1) and np.all(np.isinf(r["cost"]))


def test_permutation_invariance(oracle):
    a = archs.arch("sm_103")
    d = gen.descriptors(20, 4, "uneven")
    perm = np.random.default_rng(0).permutation(20)
    r1 = oracle.evaluate(a, gen.axes(), d, 5)
    r2 = oracle.evaluate(a, gen.axes(), d[perm], 5)
    assert np.array_equal(r1["idx"][perm], r2["idx"])
    assert np.array_equal(r1["cost"][perm], r2["cost"])


def test_segmented_topk_matches_argsort(oracle):
    rng = np.random.default_rng(0)
    lens = [0, 1, 3, 17, 100, 1000, 4097]
    off = np.zeros(len(lens) + 1, np.int64)
    off[1:] = np.cumsum(lens)
    s = gen.scores(int(off[-1]), 3)
    s[rng.integers(0, len(s), 50)] = np.inf
    s[100:110] = s[100]          # ties
    r = oracle.topk(s, off, 8)
    for i in range(len(lens)):
        seg = s[off[i]:off[i + 1]]
        idx = np.arange(len(seg))
        ok = np.isfinite(seg)
        order = np.argsort(seg[ok], kind="stable")[:8]
        want = np.full(8, -1)
        want[:len(order)] = idx[ok][order]
        assert np.array_equal(r["idx"][i], want)


def test_rejects_mask_outside_axes(oracle):
    ax = gen.axes()
    ax["u"] = ax["u"][:4]
    d = gen.descriptors(1, 1, "dense")
    assert oracle.space_size(ax, d[0]) == -1
    with pytest.raises(ValueError):
        oracle.evaluate(archs.arch("sm_103"), ax, d, 3)
