"""GPU parity of tune_search (random and Nelder-Mead search with the static cost as
the objective) against the search oracle, through the C ABI: best index, best FP32
cost and evaluation count bit for bit, over full and statically pruned spaces."""

import numpy as np
import pytest

from oracle import search_oracle as S
from oracle import suggest_oracle as SG
from workloads import archs, gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch

    from paper_1701_08547_gb300 import build

    build.build()
    assert torch.cuda.is_available()
    return torch.device("cuda:0")


def run(dev, a, ax, d, method, budget, seed, keep=None):
    import torch

    import paper_1701_08547_gb300 as T

    dd = T.descs_to_device(d, dev)
    kt = None if keep is None else torch.from_numpy(keep.astype(np.uint32)).to(dev)
    ws = T.workspace(0, 0, 1, dev)
    i, c, e = T.tune_search(a, ax, dd, method, budget, seed, t_keep=kt, workspace_buf=ws)
    T.tune_check(ws)
    return i.cpu().numpy(), c.cpu().numpy(), e.cpu().numpy()


def check(dev, oracle, a, ax, d, method, budget, seed, keep=None):
    off = gen.point_offsets(d)
    ev = oracle.evaluate(a, ax, d, 1, emit=True, offsets=off)
    o = S.search(a, ax, d, method, budget, seed, t_keep=keep, offsets=off, costs=ev["cost32"])
    gi, gc, ge = run(dev, a, ax, d, method, budget, seed, keep)
    bad = np.nonzero((gi != o["idx"]) | (ge != o["evals"]))[0]
    assert len(bad) == 0, (bad[:5], gi[bad[:5]], o["idx"][bad[:5]], ge[bad[:5]], o["evals"][bad[:5]])
    assert np.array_equal(gc.view(np.uint32), o["cost"].view(np.uint32))
    return gi, gc, ge


@pytest.mark.parametrize("method", ["random", "nelder_mead"])
@pytest.mark.parametrize("budget", [1, 16, 100])
def test_dense128(dev, oracle, method, budget):
    a, ax = archs.arch("sm_103"), gen.axes()
    d = gen.descriptors(64, 1, "dense128")
    check(dev, oracle, a, ax, d, method, budget, 1234)


@pytest.mark.parametrize("method", ["random", "nelder_mead"])
def test_uneven_spaces(dev, oracle, method):
    a, ax = archs.arch("sm_103"), gen.axes()
    d = gen.descriptors(400, 61, "uneven")
    d["space_mask"][::37] = np.uint64(0)  # some empty spaces
    check(dev, oracle, a, ax, d, method, 64, 99)


@pytest.mark.parametrize("method", ["random", "nelder_mead"])
def test_dense_full_size_spaces(dev, oracle, method):
    a, ax = archs.arch("sm_103"), gen.axes()
    d = gen.descriptors(24, 2, "dense")
    check(dev, oracle, a, ax, d, method, 256, 7)


@pytest.mark.parametrize("row", ["sm_35", "sm_20"])
def test_other_rows(dev, oracle, row):
    a, ax = archs.arch(row), gen.axes()
    d = gen.descriptors(64, 5, "dense128")
    check(dev, oracle, a, ax, d, "nelder_mead", 48, 3)


@pytest.mark.parametrize("method", ["random", "nelder_mead"])
def test_pruned_space(dev, oracle, method):
    a, ax = archs.arch("sm_103"), gen.axes()
    d = gen.descriptors(80, 8, "dense")
    keep = np.array([SG.suggest(a, ax, desc)["t_star"] for desc in d], dtype=np.uint64)
    check(dev, oracle, a, ax, d, method, 64, 21, keep)


def test_repeatable_and_seeded(dev):
    a, ax = archs.arch("sm_103"), gen.axes()
    d = gen.descriptors(200, 9, "uneven")
    r1 = run(dev, a, ax, d, "nelder_mead", 40, 5)
    r2 = run(dev, a, ax, d, "nelder_mead", 40, 5)
    r3 = run(dev, a, ax, d, "nelder_mead", 40, 6)
    assert all(np.array_equal(x, y) for x, y in zip(r1, r2))
    assert not np.array_equal(r1[0], r3[0])
