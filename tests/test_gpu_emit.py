"""The synthetic variants behind the surrogate's labels (tune_emit_measure), on the GPU.

* Each sample's canonical point index decodes to the (T, G, U, C) the oracle's
  canonical order gives (the order tune_eval's indices follow, bit-exact with the
  oracle elsewhere), so a label belongs to the point the ranking names.
* Every thread runs the same per-thread work at every launch shape, so time per
  unit of work (time / (G T)) is what the static cost ranks: the analytic cost and
  the measured per-unit time must be rank-correlated on fully timed spaces.
* Each class's executed operations (an instrumented build of the variants) equal
  what the descriptor asks for at that launch.
* Failure paths made on the host: an injected compile failure returns
  TUNE_ECOMPILE and the next call works; one repetition made a second slower is
  discarded by the median of three (and shows with a single repetition).
"""

import numpy as np
import pytest

from workloads import archs, gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch

    from paper_1701_08547_gb300 import build

    build.build()
    assert torch.cuda.is_available()
    return torch.device("cuda:0")


def _ranks(x):
    r = np.empty(len(x))
    r[np.argsort(x, kind="stable")] = np.arange(len(x))
    return r


def spearman(a, b):
    ra, rb = _ranks(a), _ranks(b)
    ra -= ra.mean()
    rb -= rb.mean()
    return float(np.sum(ra * rb) / np.sqrt(np.sum(ra * ra) * np.sum(rb * rb)))


def test_emitted_points_decode_canonically(dev, oracle):
    from paper_1701_08547_gb300 import surrogate_data as SD

    ax = gen.axes()
    d = gen.descriptors(40, 61, "uneven")
    sizes = gen.space_sizes(d)
    rng = np.random.default_rng(2)
    kern = rng.integers(0, len(d), 120)
    pt = np.array([rng.integers(0, sizes[k]) for k in kern], dtype=np.int32)
    # tiny per-thread work and one repetition: only the decode is checked here
    _, _, cfg = SD.measure(ax, d, kern, pt, scale=1e-6, reps=1, launched=True)
    for i in range(len(kern)):
        assert tuple(cfg[i]) == tuple(oracle.decode_point(d[kern[i]], ax, pt[i])), i


def test_analytic_cost_ranks_timed_variants(dev, oracle):
    """Spearman correlation, per kernel, between the model's FP32 cost and the measured time
    per unit of work over its fully timed held-out space (80 points): positive on average
    and for most kernels (chance gives 0)."""
    from paper_1701_08547_gb300 import surrogate_data as SD

    a, ax = archs.arch("sm_103"), gen.axes()
    d, ns = SD.timed_spaces(ax, gen.descriptors(24, 62, "dense"))
    o = oracle.evaluate(a, ax, d, 1, emit=True, offsets=gen.point_offsets(d))
    size = ns.shape[1]
    rho = []
    for i in range(len(d)):
        c = o["cost32"][i * size:(i + 1) * size].astype(np.float64)
        ok = np.isfinite(c) & np.isfinite(ns[i])
        if ok.sum() >= 20:
            rho.append(spearman(c[ok], ns[i][ok]))
    rho = np.array(rho)
    print("spearman per kernel", np.round(rho, 2))
    assert len(rho) >= 16
    assert rho.mean() > 0.3 and np.mean(rho > 0) >= 0.8, rho


def test_injected_compile_failure(dev):
    import paper_1701_08547_gb300 as T
    from paper_1701_08547_gb300 import native
    from paper_1701_08547_gb300 import surrogate_data as SD

    ax = gen.axes()
    d = gen.descriptors(2, 63, "dense128")
    kern, pt = np.array([0, 1]), np.array([5, 77], dtype=np.int32)
    T.tune_inject_fault(native.TUNE_FAULT_COMPILE, 1)
    with pytest.raises(T.TuneError) as e:
        SD.measure(ax, d, kern, pt, scale=1e-6, reps=1)
    assert e.value.code == native.TUNE_ECOMPILE
    us, _ = SD.measure(ax, d, kern, pt, scale=1e-6, reps=1)  # the fault was used up
    assert np.all(np.isfinite(us))


def test_injected_slow_repetition_is_discarded_by_the_median(dev):
    import paper_1701_08547_gb300 as T
    from paper_1701_08547_gb300 import native
    from paper_1701_08547_gb300 import surrogate_data as SD

    ax = gen.axes()
    d = gen.descriptors(1, 64, "dense128")
    kern, pt = np.array([0]), np.array([40], dtype=np.int32)
    base, _ = SD.measure(ax, d, kern, pt, reps=3)
    T.tune_inject_fault(native.TUNE_FAULT_SLOW_REP, 1)
    med, _ = SD.measure(ax, d, kern, pt, reps=3)
    T.tune_inject_fault(native.TUNE_FAULT_SLOW_REP, 1)
    single, _ = SD.measure(ax, d, kern, pt, reps=1)
    T.tune_inject_fault(native.TUNE_FAULT_SLOW_REP, 0)
    assert base[0] < 1e5 and med[0] < 1e5, (base, med)   # well under the injected second
    assert single[0] >= 1e6                             # the fault itself was live


def _expected_counts(desc, T, G, items, scale):
    """Operations per class a variant's threads must execute: each thread runs `items` items of
    round(n_c scale) operations per class (computed in FP32 as the library does); shared
    loads/stores only with at least 4 bytes of shared memory; lanes below round(32 d) of every
    warp repeat the FP32 loop."""
    n = np.floor(np.float32(desc["n"]) * np.float32(scale) + np.float32(0.5)).astype(np.int64)
    if int(desc["s0"]) // 4 == 0:
        n[4] = 0
    div = int(np.floor(np.float32(desc["d"]) * np.float32(32.0) + np.float32(0.5)))
    lanes_div = sum(1 for t in range(T) if (t & 31) < div)
    e = n * G * T * items
    e[0] += n[0] * G * lanes_div * items
    return e


def test_executed_instruction_counts_match_the_descriptors(dev, oracle):
    """The dynamic side of the static-versus-dynamic instruction mix (Section IV): every class's
    executed operations, tallied in an instrumented build of each variant, equal what its
    descriptor asks for at that launch (so the labels time the work the features describe);
    with divergence the dynamic mix departs from the static one only by the repeated FP32
    loop, which the mix error shows."""
    from paper_1701_08547_gb300 import surrogate_data as SD

    ax = gen.axes()
    d = gen.descriptors(30, 65, "dense")
    d["space_mask"] = np.uint64(gen.mask_bits([0, 1, 4, 7, 31], [0, 3, 6], [0, 3], [3]))
    d["s0"][:3] = [0, 3, 5]  # no shared memory, or less than one word
    d["d"][3] = np.float32(0.0)
    d["d"][4] = np.float32(1.0)
    sizes = gen.space_sizes(d)
    rng = np.random.default_rng(6)
    kern = np.arange(len(d))
    pt = np.array([rng.integers(0, sizes[k]) for k in kern], dtype=np.int32)
    items, scale = 2, 1.0 / 2048
    cnt = SD.count_ops(ax, d, kern, pt, items=items, scale=scale)
    checked = 0
    for i in range(len(kern)):
        if np.all(cnt[i] == np.iinfo(np.uint64).max):
            continue
        T_, G_, U_, C_ = oracle.decode_point(d[kern[i]], ax, pt[i])
        want = _expected_counts(d[kern[i]], T_, G_, items, scale)
        assert np.array_equal(cnt[i].astype(np.int64), want), (i, cnt[i], want)
        checked += 1
    assert checked >= 25
    # mix error against the emitted (rounded) counts: none without divergence; with every lane
    # repeating the FP32 loop (d = 1) only the FLOPS share moves (and with it the others')
    rounded = lambda i: np.floor(np.float32(d["n"][i]) * np.float32(scale) + np.float32(0.5))
    e0 = SD.mix_error(rounded(3), cnt[3])
    e1 = SD.mix_error(rounded(4), cnt[4])
    assert all(v < 1e-9 for c, v in e0.items() if c != "intensity"), e0
    assert rounded(4)[0] == 0 or e1["FLOPS"] > 0.0
