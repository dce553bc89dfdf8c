"""tune_eval_host (descriptors and results in host memory, copies overlapped with the
evaluation in chunks) against tune_eval and the oracle: bit for bit for every chunk size,
schedule and the status word."""

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


def host_eval(d, k, chunk, flags=0):
    import torch

    import paper_1701_08547_gb300 as T

    a, ax = archs.arch("sm_103"), gen.axes()
    hd = torch.from_numpy(np.ascontiguousarray(d).view(np.uint8).reshape(-1, 64)).pin_memory()
    hi = torch.empty((len(d), k), dtype=torch.int32).pin_memory()
    hc = torch.empty((len(d), k), dtype=torch.float32).pin_memory()
    s = torch.cuda.current_stream()
    scratch = T.tune_eval_host(a, ax, hd, k, chunk, hi, hc, flags=flags, stream=s)
    T.tune_check(scratch, s)
    torch.cuda.synchronize()
    return hi.numpy().copy(), hc.numpy().copy()


@pytest.mark.parametrize("chunk", [1, 7, 1000, 4999, 100000])
def test_matches_oracle_for_every_chunk(dev, oracle, chunk):
    d = gen.descriptors(5000 if chunk > 1 else 300, 81, "uneven")
    gi, gc = host_eval(d, 5, chunk)
    o = oracle.evaluate(archs.arch("sm_103"), gen.axes(), d, 5)
    assert np.array_equal(gi, o["idx"])
    assert np.array_equal(gc.view(np.uint32), o["cost"].view(np.uint32))


@pytest.mark.parametrize("flags", [0, 0x10 | (1 << 8), 0x10 | (3 << 8) | (2 << 12)])
def test_schedules_and_dense_spaces(dev, flags):
    import paper_1701_08547_gb300 as T

    d = gen.descriptors(3000, 2, "dense")
    gi, gc = host_eval(d, 10, 777, flags)
    ti, tc = T.tune_eval(archs.arch("sm_103"), gen.axes(), T.descs_to_device(d, dev), 10)
    assert np.array_equal(gi, ti.cpu().numpy())
    assert np.array_equal(gc.view(np.uint32), tc.cpu().numpy().view(np.uint32))


def test_malformed_descriptor_and_empty_call(dev):
    import paper_1701_08547_gb300 as T

    d = gen.descriptors(600, 3, "dense128")
    d["space_mask"][450] = np.uint64(1 << 62)  # bits outside the axes
    with pytest.raises(Exception):
        host_eval(d, 4, 128)
    gi, gc = host_eval(d[:0], 4, 128)
    assert gi.shape == (0, 4)
