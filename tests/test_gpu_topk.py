"""GPU parity of tune_topk (segmented top-k over external scores) against the
CPU oracle, through the C ABI: indices and scores bit for bit."""

import numpy as np
import pytest

from workloads import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch

    from paper_1701_08547_gb300 import build

    build.build()
    assert torch.cuda.is_available()
    return torch.device("cuda:0")


def run(dev, scores, off, k):
    import torch

    import paper_1701_08547_gb300 as T

    s = torch.from_numpy(scores).to(dev)
    o = torch.from_numpy(off).to(dev)
    idx, val = T.tune_topk(s, o, k)
    return idx.cpu().numpy(), val.cpu().numpy()


def check(dev, oracle, scores, off, k):
    gi, gv = run(dev, scores, off, k)
    o = oracle.topk(scores, off, k)
    assert np.array_equal(gi, o["idx"]), np.argwhere(gi != o["idx"])[:5]
    assert np.array_equal(gv, o["cost"])  # -0.0 and +0.0 compare equal


@pytest.mark.parametrize("k", [1, 5, 8, 9, 16])
def test_uneven_segments(dev, oracle, k):
    rng = np.random.default_rng(k)
    lens = np.concatenate([[0, 1, 2, 31, 32, 33, 127, 128, 129], rng.integers(0, 20000, 300)])
    off = np.zeros(len(lens) + 1, np.int64)
    off[1:] = np.cumsum(lens)
    s = gen.scores(int(off[-1]), 17)
    check(dev, oracle, s, off, k)


def test_ties_inf_nan_negative(dev, oracle):
    rng = np.random.default_rng(1)
    lens = rng.integers(1, 3000, 200)
    off = np.zeros(len(lens) + 1, np.int64)
    off[1:] = np.cumsum(lens)
    n = int(off[-1])
    s = np.round(gen.scores(n, 5, 1.0, 20.0)).astype(np.float32)  # many exact ties
    s[rng.integers(0, n, n // 10)] = np.inf
    s[rng.integers(0, n, n // 50)] = np.nan
    s[rng.integers(0, n, n // 50)] *= -1.0
    s[rng.integers(0, n, 20)] = -np.inf
    s[rng.integers(0, n, 20)] = -0.0
    check(dev, oracle, s, off, 12)


def test_all_invalid_and_short_segments(dev, oracle):
    off = np.array([0, 0, 3, 3, 10], np.int64)
    s = np.array([np.inf, np.nan, np.inf, 1, 2, 3, 4, 5, 6, 7], np.float32)
    check(dev, oracle, s, off, 16)


def test_large_segments(dev, oracle):
    lens = np.array([1 << 20, 3, (1 << 20) + 5, 77777])
    off = np.zeros(len(lens) + 1, np.int64)
    off[1:] = np.cumsum(lens)
    check(dev, oracle, gen.scores(int(off[-1]), 9), off, 10)


@pytest.mark.parametrize("shift", [1, 2, 3])
def test_unaligned_base(dev, oracle, shift):
    """Scores that start 4, 8 or 12 bytes past a 16-byte boundary: every segment's
    aligned body, head and tail move."""
    import torch

    import paper_1701_08547_gb300 as T

    rng = np.random.default_rng(40 + shift)
    lens = np.concatenate([[0, 1, 3, 4, 5, 7, 515, 4099], rng.integers(0, 9000, 60)])
    off = np.zeros(len(lens) + 1, np.int64)
    off[1:] = np.cumsum(lens)
    n = int(off[-1])
    s = gen.scores(n, 23 + shift)
    buf = torch.empty(n + shift, dtype=torch.float32, device=dev)
    buf[shift:] = torch.from_numpy(s).to(dev)
    view = buf[shift:]
    assert view.data_ptr() % 16 == 4 * shift
    gi, gv = T.tune_topk(view, torch.from_numpy(off).to(dev), 7)
    o = oracle.topk(s, off, 7)
    assert np.array_equal(gi.cpu().numpy(), o["idx"])
    assert np.array_equal(gv.cpu().numpy(), o["cost"])
