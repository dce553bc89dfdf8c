"""The search oracle (random and Nelder-Mead search with the static cost as the
objective) against fixed points outside itself: SplitMix64's reference outputs,
the exhaustive optimum of the C oracle's full sort, the uniformity of the draws,
the pruned thread-count set of the suggestion oracle, and the invariants any
search must keep. The Nelder-Mead trajectory itself has no published values
(parity unpinned beyond these invariants; the GPU matches it bit for bit)."""

import math

import numpy as np
import pytest

from oracle import oracle as O
from oracle import search_oracle as S
from oracle import suggest_oracle as SG
from workloads import archs, gen


def test_splitmix64_reference_outputs():
    # SplitMix64 from state 0: the first three outputs of the reference generator
    # (Steele, Lea and Flood 2014) are 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f.
    assert [S.mix64(j * S.GAMMA) for j in (1, 2, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                          0x06C45D188009454F]


def test_draws_are_uniform():
    key = S.mix64(7)
    n = 10
    counts = np.bincount([S.draw_below(key, 3, j, n) for j in range(20000)], minlength=n)
    chi2 = float(((counts - 2000.0) ** 2 / 2000.0).sum())
    assert chi2 < 30.0  # 9 degrees of freedom: p < 0.0005 above 30


@pytest.fixture(scope="module")
def small(oracle):
    a, ax = archs.arch("sm_103"), gen.axes()
    d = gen.descriptors(40, 51, "uneven")
    sizes = gen.space_sizes(d)
    d = d[(sizes > 0) & (sizes <= 600)][:12]
    off = gen.point_offsets(d)
    ev = oracle.evaluate(a, ax, d, 1, emit=True, offsets=off)
    return a, ax, d, off, ev


def test_random_search_with_a_large_budget_finds_the_exhaustive_optimum(small):
    a, ax, d, off, ev = small
    sizes = gen.space_sizes(d)
    budget = int(40 * sizes.max())  # P(miss) <= exp(-40) per kernel
    r = S.search(a, ax, d, "random", budget, 11, offsets=off, costs=ev["cost32"])
    assert np.array_equal(r["idx"], ev["idx"][:, 0])
    assert np.array_equal(r["cost"].view(np.uint32), ev["cost"][:, 0].view(np.uint32))
    assert np.all(r["evals"] == budget)


@pytest.mark.parametrize("method", ["random", "nelder_mead"])
@pytest.mark.parametrize("budget", [1, 7, 40])
def test_search_invariants(small, method, budget):
    a, ax, d, off, ev = small
    r = S.search(a, ax, d, method, budget, 5, offsets=off, costs=ev["cost32"])
    assert np.all(r["evals"] <= budget) and np.all(r["evals"] >= 1)
    for i in range(len(d)):
        c = ev["cost32"][off[i]:off[i + 1]]
        if r["idx"][i] < 0:  # no evaluated point had a valid configuration
            assert math.isinf(r["cost"][i])
            continue
        assert r["idx"][i] < len(c) and np.isfinite(r["cost"][i])
        assert r["cost"][i] == c[r["idx"][i]]
        assert r["cost"][i] >= ev["cost"][i, 0]  # never better than the exhaustive optimum


def test_nelder_mead_improves_on_its_start(small):
    a, ax, d, off, ev = small
    one = S.search(a, ax, d, "nelder_mead", 1, 9, offsets=off, costs=ev["cost32"])
    many = S.search(a, ax, d, "nelder_mead", 60, 9, offsets=off, costs=ev["cost32"])
    # the first evaluation is the start point; more evaluations can only keep or lower the best
    assert np.all(many["cost"] <= one["cost"])
    assert np.mean(many["cost"] < one["cost"]) > 0.3


def test_pruned_search_stays_in_the_kept_thread_counts(small):
    a, ax, d, off, ev = small
    keep = np.array([SG.suggest(a, ax, desc)["t_star"] for desc in d], dtype=np.uint64)
    for method in ("random", "nelder_mead"):
        r = S.search(a, ax, d, method, 30, 3, t_keep=keep, offsets=off, costs=ev["cost32"])
        for i in range(len(d)):
            if r["idx"][i] < 0:  # nothing kept, or no valid point among those evaluated
                assert math.isinf(r["cost"][i])
                continue
            T, G, U, C = O.decode_point(d[i], ax, int(r["idx"][i]))
            assert (int(keep[i]) >> ax["t"].index(T)) & 1


def test_empty_space():
    a, ax = archs.arch("sm_103"), gen.axes()
    d = gen.descriptors(3, 2, "dense128")
    d["space_mask"][1] = np.uint64(0)
    off = gen.point_offsets(d)
    ev = O.evaluate(a, ax, d, 1, emit=True, offsets=off)
    r = S.search(a, ax, d, "nelder_mead", 10, 1, offsets=off, costs=ev["cost32"])
    assert r["idx"][1] == -1 and math.isinf(r["cost"][1]) and r["evals"][1] == 0
