"""GPU check of the real-kernel variants (tune_real_measure, through the C ABI): the
timed matVec2D, ATAX and BiCG variants compute A x, A^T (A x), A p and A^T r of the
documented operands (compared with an FP64 product on the host), and every launchable
configuration gets a positive time."""

import numpy as np
import pytest

from paper_1701_08547_gb300 import realkernels as R
from workloads import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch

    from paper_1701_08547_gb300 import build

    build.build()
    assert torch.cuda.is_available()
    return torch.device("cuda:0")


def operands(n):
    i = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    A = (((7 * i + 13 * j) % 17) - 8) * 0.125
    x = (((5 * np.arange(n)) % 11) - 5) * 0.25
    r = (((5 * np.arange(n) + 3) % 11) - 5) * 0.25
    return A, x, r


@pytest.mark.parametrize("kind", ["matvec", "atax", "bicg"])
def test_results_and_times(dev, kind):
    n = 300
    ax = gen.axes()
    us, regs, res = R.measure(kind, n, ax, reps=1, with_result=True)
    A, x, r = operands(n)
    if kind == "matvec":
        want = A @ x
        got = res[:n]
    elif kind == "atax":
        want = A.T @ (A @ x)
        got = res[:n]
    else:
        want = np.concatenate([A @ x, A.T @ r])
        got = res[:2 * n]
    # FP32 accumulation over n terms of magnitude <= 1.25 (ATAX: a second product of such sums)
    tol = 1e-5 * n * (np.abs(A).max() * np.abs(x).max()) * (n if kind == "atax" else 1)
    assert np.max(np.abs(got - want)) <= tol
    assert np.all(regs > 0)
    ok = np.isfinite(us)
    assert ok.mean() > 0.9 and np.all(us[ok] > 0)
