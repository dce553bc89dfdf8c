"""Pins of the CPU oracle against what the paper prints and what the
mathematics fixes (closed forms), independent of the oracle's own code.

Occupancy (Eqs. 1-5) is pinned by the paper's Table "Suggested parameters to
achieve theoretical occupancy" (T*, register and shared-memory headroom,
occ*) and Table "Statistics for autotuned kernels" (occupancy modes); the
cost (Eq. 6 plus the launch-configuration terms) by special cases whose
value is known in closed form.
"""

import math

import numpy as np
import pytest

from conftest import read_golden
from workloads import archs

TC = list(range(32, 1025, 32))  # Orio TC = range(32,1025,32), Fig. "Performance tuning specification"


def occ_ratio(O, row, T, R, S, carveout=100):
    o = O.occupancy(row, T, R, S, carveout)
    return o["W"] / row["max_warps_sm"], o


def test_arch_rows_match_table_gpus():
    """The paper's four arch rows carry Table "GPUs used in this experiment" verbatim."""
    names = ["sm_20", "sm_35", "sm_52", "sm_60"]
    for field, *vals in read_golden("table_gpus.txt"):
        for name, v in zip(names, vals):
            assert archs.arch(name)[field] == int(v), (name, field)


def test_arch_ipc_match_table_ipc():
    """Per-class IPC of the paper rows = Table "Instruction throughput per number of cycles"."""
    names = ["sm_20", "sm_35", "sm_52", "sm_60"]
    for cls, *vals in read_golden("table_ipc.txt"):
        c = archs.CLASSES.index(cls)
        for name, v in zip(names, vals):
            assert archs.arch(name)["ipc"][c] == float(v), (name, cls)


def table_rows():
    return read_golden("table_suggested_params.txt")


@pytest.mark.parametrize("row", table_rows(), ids=lambda r: f"{r[0]}-{r[1]}")
def test_table_suggested_params(oracle, row):
    """Reproduce the pinned columns of Table "Suggested parameters" (Section IV-C)."""
    kern, name, tstar, Ru, Rstar, Sstar, occstar, cols = row
    a = archs.arch(name)
    cols = cols.split(",")
    Ru, Rstar, Sstar, occstar = int(Ru), int(Rstar), int(Sstar), float(occstar)
    tstar = [int(x) for x in tstar.split(",")]

    # T*: thread counts of the Orio range whose warp limit alone reaches full occupancy.
    full = [T for T in TC if occ_ratio(oracle, a, T, 16, 0)[0] == 1.0]
    assert full == tstar

    # occ*: best occupancy over T* with the kernel's registers.
    def best(R, S=0):
        return max(occ_ratio(oracle, a, T, R, S)[0] for T in tstar)

    occ_u = best(Ru)
    if "occ" in cols:
        assert abs(occ_u - occstar) < 0.005
    if "R" in cols:
        # R^u + R*: the largest register count that keeps the same best occupancy.
        assert best(Ru + Rstar) == occ_u
        assert best(Ru + Rstar + 1) < occ_u
    if "S" in cols:
        # S*: the largest per-block shared memory that keeps B* at the best T.
        T_best = next(T for T in tstar if occ_ratio(oracle, a, T, Ru, 0)[0] == occ_u)
        B0 = oracle.occupancy(a, T_best, Ru, 0)["B"]
        assert oracle.occupancy(a, T_best, Ru, Sstar)["B"] == B0
        assert oracle.occupancy(a, T_best, Ru, Sstar + 1)["B"] < B0


def test_table_breakdown_modes_reachable(oracle):
    """Every occupancy mode of Table "Statistics for autotuned kernels" is a
    value the calculation produces on that GPU for some thread count and
    register count (theoretical occupancy = W*/W_mp)."""
    for name, *modes in read_golden("table_breakdown_modes.txt"):
        a = archs.arch(name)
        reach = set()
        for T in TC:
            for R in range(16, a["regs_thread_max"] + 1, 1):
                r, o = occ_ratio(oracle, a, T, R, 0)
                if o["valid"]:
                    reach.add(round(100 * r, 2))
        for m in modes:
            m = float(m)
            assert any(abs(m - x) <= 0.011 for x in reach), (name, m)


def test_search_space_arithmetic(oracle):
    """Section IV-C: 5,120 variants, 640 after keeping T* on Kepler (87.5 %),
    84 % saved on Fermi/Maxwell (5 of 32 thread counts kept)."""
    g = {r[0]: float(r[1]) for r in read_golden("search_space.txt")}
    n_tc, n_bc, n_uif, n_pl, n_flags = 32, len(range(24, 193, 24)), len(range(1, 6)), 2, 2
    assert n_tc * n_bc * n_uif * n_pl * n_flags == g["variants"]
    kept = {}
    for name in ("sm_20", "sm_35", "sm_52"):
        a = archs.arch(name)
        kept[name] = sum(occ_ratio(oracle, a, T, 16, 0)[0] == 1.0 for T in TC)
    assert g["variants"] * kept["sm_35"] / n_tc == g["kepler_after_static"]
    assert 100 * (1 - kept["sm_35"] / n_tc) == g["kepler_saving_pct"]
    for name in ("sm_20", "sm_52"):
        assert round(100 * (1 - kept[name] / n_tc)) == g["fermi_maxwell_saving_pct"]


# ---- closed forms for individual terms -------------------------------------------------


def test_occupancy_hand_worked_kepler_384(oracle):
    """Eq. 3 on Kepler: T=384 -> 12 warps -> floor(64/12)=5 blocks -> 60 of 64 warps."""
    o = oracle.occupancy(archs.arch("sm_35"), 384, 16, 0)
    assert (o["W_B"], o["G_W"], o["B"], o["W"]) == (12, 5, 5, 60)


def test_occupancy_register_limit_warp_mode(oracle):
    """Eq. 4, per-warp allocation on Pascal: R=38 -> 38*32=1216 rounded to 1280
    registers per warp -> floor(65536/1280)=51 warps -> 48 (granularity 4) ->
    6 blocks of 8 warps -> 48 of 64 warps."""
    o = oracle.occupancy(archs.arch("sm_60"), 256, 38, 0)
    assert (o["G_R"], o["B"], o["W"]) == (6, 6, 48)


def test_occupancy_register_limit_block_mode(oracle):
    """Eq. 4, per-block allocation on Fermi: R=27, T=192 -> 27*192=5184 registers
    (a multiple of 64) -> floor(32768/5184)=6 blocks (36 of 48 warps, occ .75)."""
    o = oracle.occupancy(archs.arch("sm_20"), 192, 27, 0)
    assert (o["G_R"], o["B"], o["W"]) == (6, 6, 36)


def test_occupancy_cases(oracle):
    """Eqs. 4-5 case 1 (over the per-thread / per-block maximum -> 0), case 3
    (nothing requested -> B_mp), and the thread-per-block maximum."""
    a = archs.arch("sm_60")
    assert oracle.occupancy(a, 256, 256, 0)["G_R"] == 0
    assert not oracle.occupancy(a, 256, 256, 0)["valid"]
    assert oracle.occupancy(a, 256, 0, 0)["G_R"] == a["max_blocks_sm"]
    assert oracle.occupancy(a, 256, 32, 49153)["G_S"] == 0
    assert oracle.occupancy(a, 256, 32, 0)["G_S"] == a["max_blocks_sm"]
    assert not oracle.occupancy(a, 1056, 16, 0)["valid"]
    # Shared memory case 2: 48 KB / roundup(5000, 256)=5120 -> 9 blocks.
    assert oracle.occupancy(a, 64, 16, 5000)["G_S"] == 9


def test_occupancy_carveout_sm103(oracle):
    """Carveout reading on sm_103: capacity = smallest supported capacity that
    is >= carveout% of 228 KB and holds one block (s0 + 1 KB reserved,
    rounded to 128 B)."""
    a = archs.arch("sm_103")
    # s0 = 0: 1 KB per block. 0 % -> smallest capacity holding a block = 8 KB -> 8 blocks.
    o = oracle.occupancy(a, 64, 16, 0, 0)
    assert (o["cap"], o["G_S"]) == (8 * 1024, 8)
    # 25 % of 228 KB = 57 KB -> 64 KB; s0 = 7000 -> 8024 -> 8064 B per block -> 8 blocks.
    o = oracle.occupancy(a, 64, 16, 7000, 25)
    assert (o["cap"], o["G_S"]) == (64 * 1024, 8)
    # 50 % -> 114 KB -> 132 KB; 100 % -> 228 KB.
    assert oracle.occupancy(a, 64, 16, 7000, 50)["cap"] == 132 * 1024
    assert oracle.occupancy(a, 64, 16, 7000, 100)["G_S"] == (228 * 1024) // 8064


def _n_unit(a):
    """Counts giving n_c / IPC_c = 1 for every class."""
    return [float(x) for x in a["ipc"]]


def test_cost_closed_form_full_waves(oracle):
    """U=1, d=0, T a multiple of 32 (lane = 1), W* >= W_sat (hide = 1) and G a
    whole number of waves (par = n_SM):  cost = K * sum_c n_c/IPC_c / n_SM.
    With n_c = IPC_c every class contributes one cycle: 7 * 1024 / 152."""
    a = archs.arch("sm_103")
    B, W, T = 8, 64, 256
    G = 2 * a["n_sm"] * B
    c = oracle.cost64(a, _n_unit(a), 0.0, 1, T, G, B, W)
    assert c == pytest.approx(7 * 1024 / 152, rel=1e-15)


def test_cost_terms_scale_as_defined(oracle):
    """Each factor of the cost, checked by a ratio of two evaluations."""
    a = archs.arch("sm_103")
    n = [3.0e4, 1.0e3, 7.0e4, 2.0e4, 5.0e3, 9.0e3, 1.1e3]
    B, W, T, G = 8, 64, 256, 2 * 152 * 8
    base = oracle.cost64(a, n, 0.0, 1, T, G, B, W)
    # divergence: cost scales by (1 + d)
    assert oracle.cost64(a, n, 0.25, 1, T, G, B, W) == pytest.approx(1.25 * base, rel=1e-14)
    # unrolling amortises only the branch count: n_BRANCH / U
    only_br = [0, 0, 0, 0, 0, 9.0e3, 0]
    assert oracle.cost64(a, only_br, 0.0, 4, T, G, B, W) == pytest.approx(
        oracle.cost64(a, only_br, 0.0, 1, T, G, B, W) / 4, rel=1e-14)
    only_fp = [5.0e4, 0, 0, 0, 0, 0, 0]
    assert oracle.cost64(a, only_fp, 0.0, 4, T, G, B, W) == oracle.cost64(a, only_fp, 0.0, 1, T, G, B, W)
    # memory latency hiding: W* = 8 warps -> hide = 32/8 = 4 on memory classes only
    only_mem = [0, 0, 0, 2.0e4, 5.0e3, 0, 0]
    assert oracle.cost64(a, only_mem, 0.0, 1, T, G, 1, 8) == pytest.approx(
        4 * oracle.cost64(a, only_mem, 0.0, 1, T, G, 1, 32), rel=1e-14)
    assert oracle.cost64(a, only_mem, 0.0, 1, T, G, 1, 64) == oracle.cost64(a, only_mem, 0.0, 1, T, G, 1, 32)
    assert oracle.cost64(a, only_fp, 0.0, 1, T, G, 1, 8) == oracle.cost64(a, only_fp, 0.0, 1, T, G, 1, 32)
    # partial warps: T = 48 occupies 2 warps -> lane = 64/48
    c48 = oracle.cost64(a, only_fp, 0.0, 1, 48, G, B, 2 * B)
    c64 = oracle.cost64(a, only_fp, 0.0, 1, 64, G, B, 2 * B)
    assert c48 == pytest.approx(c64 * 64 / 48, rel=1e-14)
    # tail wave: G = slots + 1 -> 2 waves -> par = n_SM (slots+1) / (2 slots)
    slots = 152 * B
    par = 152 * (slots + 1) / (2 * slots)
    assert oracle.cost64(a, only_fp, 0.0, 1, T, slots + 1, B, W) == pytest.approx(
        5.0e4 * 1024 / 128 / par, rel=1e-14)
    # one block: G = 1 fills 1 of the n_SM * B* block slots -> par = 1 / B*
    assert oracle.cost64(a, only_fp, 0.0, 1, T, 1, B, W) == pytest.approx(5.0e4 * 1024 / 128 * B, rel=1e-14)


def test_cost_per_class_weights(oracle):
    """One class at a time: cost = K * n_c / IPC_c / n_SM (full waves, W* >= 32),
    so a swapped class order or IPC column shows up here."""
    a = archs.arch("sm_103")
    B, W, T, G = 8, 64, 256, 152 * 8
    for c in range(7):
        n = [0.0] * 7
        n[c] = 1000.0
        want = 1024 * 1000.0 / a["ipc"][c] / 152
        assert oracle.cost64(a, n, 0.0, 1, T, G, B, W) == pytest.approx(want, rel=1e-14), c


def test_cost32_within_bound_of_cost64(oracle):
    """The FP32 evaluation stays within 1e-5 relative of FP64 (a compensated
    sum plus at most a dozen rounded operations: a few ulp)."""
    from workloads import gen

    a = archs.arch("sm_103")
    d = gen.descriptors(8, 11, "dense")
    off = gen.point_offsets(d)
    r = oracle.evaluate(a, gen.axes(), d, 4, emit=True, offsets=off)
    ok = np.isfinite(r["cost64"])
    rel = np.abs(r["cost32"][ok].astype(np.float64) - r["cost64"][ok]) / r["cost64"][ok]
    assert rel.max() < 2e-6
    assert np.array_equal(np.isfinite(r["cost32"]), ok)
