"""tune_eval_host (descriptors and results in host memory, copies overlapped with the
evaluation in chunks, or read and written in place with TUNE_HOST_DIRECT) against tune_eval
and the oracle: bit for bit for every chunk size, schedule and the status word."""

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


DIRECT = 0x40  # TUNE_HOST_DIRECT


@pytest.mark.parametrize("flags", [DIRECT, DIRECT | 0x10 | (3 << 8) | (2 << 12)])
def test_direct_matches_oracle(dev, oracle, flags):
    d = gen.descriptors(5000, 82, "uneven")
    gi, gc = host_eval(d, 5, 1000, flags)
    o = oracle.evaluate(archs.arch("sm_103"), gen.axes(), d, 5)
    assert np.array_equal(gi, o["idx"])
    assert np.array_equal(gc.view(np.uint32), o["cost"].view(np.uint32))


def test_direct_status_and_empty_call(dev):
    d = gen.descriptors(600, 3, "dense128")
    d["space_mask"][450] = np.uint64(1 << 62)  # bits outside the axes
    with pytest.raises(Exception):
        host_eval(d, 4, 128, DIRECT)
    gi, gc = host_eval(d[:0], 4, 128, DIRECT)
    assert gi.shape == (0, 4)


def test_direct_refuses_pageable_buffers(dev):
    """Pageable host buffers are refused before any launch (the device is never pointed
    at memory it cannot address)."""
    import torch

    import paper_1701_08547_gb300 as T
    from paper_1701_08547_gb300.native import TuneError

    d = gen.descriptors(100, 4, "dense")
    hd = torch.from_numpy(np.ascontiguousarray(d).view(np.uint8).reshape(-1, 64).copy())  # pageable
    hi = torch.empty((len(d), 4), dtype=torch.int32)
    hc = torch.empty((len(d), 4), dtype=torch.float32)
    with pytest.raises(TuneError):
        T.tune_eval_host(archs.arch("sm_103"), gen.axes(), hd, 4, 100, hi, hc, flags=DIRECT,
                         stream=torch.cuda.current_stream())
