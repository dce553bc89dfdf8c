"""Schedules, the autotuner and CUDA-graph replay all give the oracle's top-k."""

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


def _same(gi, gc, o):
    assert np.array_equal(gi, o["idx"])
    assert np.array_equal(gc.view(np.uint32), o["cost"].view(np.uint32))


@pytest.mark.parametrize("chunk", [None, 0, 3, 8])
@pytest.mark.parametrize("ctas", [0, 1, 3])
def test_warp_schedule_knobs(dev, oracle, chunk, ctas):
    import paper_1701_08547_gb300 as T

    a, ax = archs.arch("sm_103"), gen.axes()
    d = gen.descriptors(3000, 4, "uneven")
    o = oracle.evaluate(a, ax, d, 6)
    fl = T.TUNE_SCHED_WARP | (0 if chunk is None else T.TUNE_SCHED_CHUNK(chunk)) | (T.TUNE_SCHED_CTAS(ctas) if ctas else 0)
    ws = T.workspace(0, len(d), 6, dev)
    i, c = T.tune_eval(a, ax, T.descs_to_device(d, dev), 6, flags=fl, workspace_buf=ws)
    T.tune_check(ws)
    _same(i.cpu().numpy(), c.cpu().numpy(), o)


def test_autotune_picks_a_valid_schedule(dev, oracle):
    import paper_1701_08547_gb300 as T

    a, ax = archs.arch("sm_103"), gen.axes()
    d = gen.descriptors(20000, 3, "uneven")
    flags, ms, i, c = T.tune_autotune(a, ax, T.descs_to_device(d, dev), 5, reps=2)
    assert ms > 0 and flags & (T.TUNE_SCHED_WARP | T.TUNE_SCHED_THREAD)
    pick = np.arange(0, 20000, 97)
    o = oracle.evaluate(a, ax, d[pick], 5)
    _same(i.cpu().numpy()[pick], c.cpu().numpy()[pick], o)


def test_cuda_graph_replay(dev, oracle):
    """tune_eval captured in a CUDA graph (status reset + one persistent launch)
    and replayed: every replay gives the oracle's result."""
    import torch

    import paper_1701_08547_gb300 as T

    a, ax = archs.arch("sm_103"), gen.axes()
    d = gen.descriptors(5000, 3, "uneven")
    dd = T.descs_to_device(d, dev)
    k = 5
    ws = T.workspace(0, len(d), k, dev)
    idx = torch.empty((len(d), k), dtype=torch.int32, device=dev)
    cost = torch.empty((len(d), k), dtype=torch.float32, device=dev)
    fl = T.TUNE_SCHED_WARP | T.TUNE_SCHED_CHUNK(2)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        T.tune_eval(a, ax, dd, k, flags=fl, topk_idx=idx, topk_cost=cost, workspace_buf=ws, stream=s)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        T.tune_eval(a, ax, dd, k, flags=fl, topk_idx=idx, topk_cost=cost, workspace_buf=ws, stream=s)
    o = oracle.evaluate(a, ax, d, k)
    for _ in range(2):
        idx.fill_(7)
        g.replay()
        torch.cuda.synchronize()
        T.tune_check(ws)
        _same(idx.cpu().numpy(), cost.cpu().numpy(), o)
