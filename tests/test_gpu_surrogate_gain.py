"""What the learned surrogate gains over the analytic model alone, and the sanity case.

Measured labels: this GPU's times of the library's synthetic variants
(tune_emit_measure), per unit of per-thread work (every thread runs the
descriptor's counts, so time / (G T) is what the static cost ranks). The ensemble
is trained by the library's kernels; on held-out kernels whose small spaces
(80 points) are timed completely, hit@5 = the measured-best point is among a
ranking's 5 picks. The analytic model must beat 5 uniform random picks among the
launchable points. Between the ensemble and the analytic model the hit rates differ by
a few kernels in 200, inside the run-to-run spread of the measured best (a 95 %
interval spans about +-0.06), so on hit@5 the ensemble (with its analytic fallback at
std/mean 0.1, and without fallback) must be not significantly worse: the analytic
rate lies at or below the upper end of the ensemble's 95 % Wilson interval. Without
the fallback the ensemble's first pick must be closer to the measured best (median
slowdown) than the analytic model's.

Sanity case: trained on the analytic model's own costs as labels (128 K sampled
points, 120 epochs: at 60 the fit depended on the initial draws, 0.93-0.965 within
1 %), the ensemble must reproduce the analytic choice: on held-out kernels, one of its top 5 points
is within 1 % of the least analytic cost for at least 95 % of them. (The held-out
spaces hold a median of 4 points within 1 % of the best and 12 within 5 %, and
exact ties are common; a regression fit to a few % cannot order points that
close, and a measured label could not either: median-of-3 timings vary by more.
The exact-best rate is asserted at 0.8 and printed.)
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
    return torch.device("cuda:0")


def test_surrogate_beats_analytic_on_measured_best(dev):
    from paper_1701_08547_gb300 import surrogate_data as SD

    a, ax = archs.arch("sm_103"), gen.axes()
    data = SD.build_set(a, ax, gen.descriptors(800, 4, "dense"), 64, 4, dev)
    assert data["n"] > 0.6 * data["measured"]
    sur, trace = SD.train(data, members=5, epochs=60, dev=dev)
    assert trace[-1].mean() < 0.1 * trace[0, 0].mean()
    timed = SD.timed_spaces(ax, gen.descriptors(200, 40, "dense"))
    with_fb = SD.evaluate(sur, a, ax, None, dev, k=5, thresh=0.1, timed=timed)
    no_fb = SD.evaluate(sur, a, ax, None, dev, k=5, thresh=1e30, timed=timed)
    print(with_fb, no_fb)
    assert with_fb["kernels"] >= 150
    assert with_fb["hit_analytic"] > with_fb["hit_random"]
    assert with_fb["hit_analytic"] <= with_fb["hit_surrogate_ci95"][1]
    assert no_fb["hit_analytic"] <= no_fb["hit_surrogate_ci95"][1]
    assert no_fb["first_pick_slowdown_surrogate"] <= no_fb["first_pick_slowdown_analytic"]


def test_surrogate_trained_on_analytic_labels_reproduces_the_analytic_choice(dev):
    import torch

    import paper_1701_08547_gb300 as T
    from paper_1701_08547_gb300 import surrogate_data as SD

    a, ax = archs.arch("sm_103"), gen.axes()
    data = SD.analytic_set(a, ax, gen.descriptors(2000, 44, "dense"), 64, 44, dev)
    sur, trace = SD.train(data, members=5, epochs=120, dev=dev)
    held = SD.eval_spaces(gen.descriptors(200, 45, "dense"))
    off = gen.point_offsets(held)
    dd = T.descs_to_device(held, dev)
    s_idx, _, _ = sur.infer(a, ax, dd, off, 5, thresh=1e30)
    pc = torch.empty(int(off[-1]), dtype=torch.float32, device=dev)
    T.tune_eval(a, ax, dd, 1, flags=T.TUNE_EMIT_POINTS, pt_cost=pc, pt_offsets=torch.from_numpy(off).to(dev))
    cost = pc.cpu().numpy().reshape(len(held), -1)
    s_idx = s_idx.cpu().numpy()
    ok = np.isfinite(cost).any(axis=1)
    def hits(tol):
        # a hit: one of the 5 picks costs at most (1 + tol) times the least analytic cost
        return np.array([(cost[i, s_idx[i][s_idx[i] >= 0]] <= (1 + tol) * np.nanmin(np.where(
            np.isfinite(cost[i]), cost[i], np.nan))).any() for i in range(len(held))])[ok]

    exact, within1 = hits(0.0).mean(), hits(0.01).mean()
    print("sanity hit@5 exact", exact, "within 1 %", within1, "kernels", ok.sum(), "final loss", trace[-1].mean())
    assert ok.sum() >= 150
    assert within1 >= 0.95 and exact >= 0.8
