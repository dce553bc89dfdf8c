"""Static search-space pruning: the oracle against Table "Suggested parameters"
and the search-space reductions of Section IV-C; the GPU (tune_suggest, through
the C ABI) against the oracle."""

import numpy as np
import pytest

from conftest import read_golden
from oracle import suggest_oracle as SO
from workloads import archs, gen


def paper_desc(r_u, flops_heavy=True):
    d = gen.descriptors(1, 1, "dense")
    d["r0"], d["s0"] = r_u, 0
    d["space_mask"] = np.uint64(gen.mask_bits(range(32), [0], [0], [3]))  # all 32 thread counts
    d["n"][0] = [5000.0, 0, 100, 1000, 0, 100, 10] if flops_heavy else [100.0, 0, 100, 1000, 0, 100, 10]
    return d


@pytest.mark.parametrize("row", read_golden("table_suggested_params.txt"), ids=lambda r: f"{r[0]}-{r[1]}")
def test_suggest_reproduces_table(oracle, row):
    kern, name, tstar, Ru, Rstar, Sstar, occstar, cols = row
    a, ax = archs.arch(name), gen.axes()
    o = SO.suggest(a, ax, paper_desc(int(Ru))[0])
    want_t = sum(1 << (int(T) // 32 - 1) for T in tstar.split(","))
    assert o["t_star"] == want_t
    if "occ" in cols:
        assert abs(o["occ_star"] - float(occstar)) < 0.005
    if "R" in cols:
        assert o["r_headroom"] == int(Rstar)
    if "S" in cols:
        assert o["s_star"] == int(Sstar)


def test_search_space_reduction():
    """5,120 variants; T* keeps 4 of 32 thread counts on Kepler (640, 87.5 %) and 5 on
    Fermi/Maxwell (84 %); the intensity rule keeps 2 (93.8 %)."""
    g = {r[0]: float(r[1]) for r in read_golden("search_space.txt")}
    ax = gen.axes()
    for name, frac in (("sm_35", g["kepler_saving_pct"]), ("sm_20", g["fermi_maxwell_saving_pct"]),
                       ("sm_52", g["fermi_maxwell_saving_pct"])):
        o = SO.suggest(archs.arch(name), ax, paper_desc(16)[0])
        kept = bin(o["t_star"]).count("1")
        assert round(100 * (1 - kept / 32), 1 if name == "sm_35" else 0) == frac
        if name == "sm_35":
            assert g["variants"] * kept / 32 == g["kepler_after_static"]
        kept_rule = bin(o["t_rule"]).count("1")
        assert round(100 * (1 - kept_rule / 32), 1) == g["static_plus_rule_saving_pct"]


def test_rule_picks_upper_or_lower_half():
    ax = gen.axes()
    a = archs.arch("sm_60")
    up = SO.suggest(a, ax, paper_desc(16, True)[0])
    lo = SO.suggest(a, ax, paper_desc(16, False)[0])
    assert up["t_star"] == lo["t_star"]
    star = [p for p in range(32) if up["t_star"] >> p & 1]
    assert [p for p in range(32) if up["t_rule"] >> p & 1] == star[-2:]
    assert [p for p in range(32) if lo["t_rule"] >> p & 1] == star[:2]


@pytest.mark.gpu
@pytest.mark.parametrize("name", list(archs.ARCHS))
def test_gpu_suggest_matches_oracle(oracle, name):
    import torch

    import paper_1701_08547_gb300 as T
    from paper_1701_08547_gb300 import build

    build.build()
    a, ax = archs.arch(name), gen.axes()
    d = gen.descriptors(150, 17, "uneven")
    d["r0"] = np.minimum(d["r0"], 60)
    d = np.concatenate([d, paper_desc(27)])
    g = T.tune_suggest(a, ax, T.descs_to_device(d, torch.device("cuda:0")))
    g = {k: v.cpu().numpy() for k, v in g.items()}
    for i in range(len(d)):
        o = SO.suggest(a, ax, d[i])
        assert int(g["t_star"][i]) & 0xffffffff == o["t_star"], i
        assert g["occ_star"][i] == np.float32(o["occ_star"]), i
        assert g["r_headroom"][i] == o["r_headroom"] and g["s_star"][i] == o["s_star"], i
        assert int(g["t_rule"][i]) & 0xffffffff == o["t_rule"], i


@pytest.mark.gpu
def test_gpu_pruning_against_measured_times():
    """Pruned spaces against timed variants on this GPU: the report is complete and
    self-consistent (the rule keeps a subset of T*, so it cannot do better)."""
    import torch

    from paper_1701_08547_gb300 import build
    from paper_1701_08547_gb300 import surrogate_data as SD

    build.build()
    a, ax = archs.arch("sm_103"), gen.axes()
    r = SD.evaluate_pruning(a, ax, gen.descriptors(40, 41, "dense"), torch.device("cuda:0"))
    assert r["kernels"] >= 30
    st, ru = r["static_t_star"], r["rule"]
    assert st["kept_thread_counts"] == 5.0 and ru["kept_thread_counts"] == 2.0
    assert 1.0 <= st["median_slowdown"] <= ru["median_slowdown"]
    assert ru["hit"] <= st["hit"] <= 1.0
