"""tune_eval_noalloc: the workspace-free entry point for hosts that cannot
allocate device memory for this library (runtimes that own all device
memory, or a budget fixed at start-up). Its scratch is a static array inside
the library, so its results must equal tune_eval's, bit for bit, call after
call: the array keeps the previous call's contents, which each call clears.

Marked run_last (tests/conftest.py moves such tests to the end of the run; the
file name also sorts last), so a failure here cannot hide failures elsewhere in
a run that stops at the first one.
"""

import ctypes as C

import numpy as np
import pytest

from workloads import archs, gen

pytestmark = [pytest.mark.gpu, pytest.mark.run_last]


@pytest.fixture(scope="module")
def lib():
    import torch

    from paper_1701_08547_gb300 import build, native

    build.build()
    assert torch.cuda.is_available()
    return native.load_noalloc()


def _noalloc(lib, arch, axes, d_dev, n, k, stream):
    import torch

    from paper_1701_08547_gb300 import native

    idx = torch.full((n, k), 7, dtype=torch.int32, device=d_dev.device)
    cost = torch.full((n, k), 7.0, dtype=torch.float32, device=d_dev.device)
    a, x = native.make_arch(arch), native.make_axes(axes)
    rc = lib.tune_eval_noalloc(C.byref(a), C.byref(x), C.c_void_p(d_dev.data_ptr()), n, k, 0,
                               C.c_void_p(idx.data_ptr()), C.c_void_p(cost.data_ptr()), None, None,
                               None, None, C.c_void_p(stream.cuda_stream))
    return rc, idx.cpu().numpy(), cost.cpu().numpy()


def test_noalloc_matches_tune_eval_twice(lib):
    import torch

    import paper_1701_08547_gb300 as T

    stream = torch.cuda.current_stream()
    for space, n, k, seed in (("uneven", 700, 5, 3), ("dense", 300, 10, 2)):
        a, ax = archs.arch("sm_103"), gen.axes()
        d = T.descs_to_device(gen.descriptors(n, seed, space))
        ws = T.workspace(0, n, k)
        ref_i, ref_c = T.tune_eval(a, ax, d, k, workspace_buf=ws, stream=stream)
        T.tune_check(ws, stream)
        ref_i, ref_c = ref_i.cpu().numpy(), ref_c.cpu().numpy()
        for _ in range(2):  # two calls in a row share the static scratch
            rc, gi, gc = _noalloc(lib, a, ax, d, n, k, stream)
            assert rc == 0, lib.tune_last_error()
            assert np.array_equal(gi, ref_i)
            assert np.array_equal(gc.view(np.uint32), ref_c.view(np.uint32))


def test_noalloc_reports_malformed_then_recovers(lib):
    """A malformed descriptor is reported; the next call starts from a cleared status."""
    import torch

    import paper_1701_08547_gb300 as T

    stream = torch.cuda.current_stream()
    a, ax = archs.arch("sm_103"), gen.axes()
    bad = gen.descriptors(4, 5, "dense128")
    bad["space_mask"][2] = np.uint64(1 << 61)
    rc, gi, _ = _noalloc(lib, a, ax, T.descs_to_device(bad), 4, 3, stream)
    assert rc == -1 and "malformed" in lib.tune_last_error().decode()
    assert np.all(gi[2] == -1)
    good = gen.descriptors(4, 5, "dense128")
    rc, gi, gc = _noalloc(lib, a, ax, T.descs_to_device(good), 4, 3, stream)
    assert rc == 0
    ref_i, _ = T.tune_eval(a, ax, T.descs_to_device(good), 3, stream=stream)
    assert np.array_equal(gi, ref_i.cpu().numpy())


def test_noalloc_rejects_bad_arguments(lib):
    from paper_1701_08547_gb300 import native

    a, x = native.make_arch(archs.arch("sm_103")), native.make_axes(gen.axes())
    fake = C.c_void_p(16)
    rc = lib.tune_eval_noalloc(C.byref(a), C.byref(x), fake, 1, 17, 0, fake, fake, None, None, None,
                               None, None)
    assert rc == -1


def test_noalloc_emit_points_match_tune_eval(lib):
    """TUNE_EMIT_POINTS through the static scratch: per-point B*, W* and cost equal
    tune_eval's bit for bit, with one of the three per-point arrays NULL (left untouched),
    on two calls in a row."""
    import torch

    import paper_1701_08547_gb300 as T
    from paper_1701_08547_gb300 import native

    stream = torch.cuda.current_stream()
    a, ax = archs.arch("sm_103"), gen.axes()
    d = gen.descriptors(90, 9, "uneven")
    off = gen.point_offsets(d)
    total, k = int(off[-1]), 4
    dd = T.descs_to_device(d)
    po = torch.from_numpy(off).cuda()
    ref = [torch.empty(total, dtype=dt, device="cuda") for dt in (torch.int32, torch.int32, torch.float32)]
    ref_i, ref_c = T.tune_eval(a, ax, dd, k, flags=T.TUNE_EMIT_POINTS, pt_blocks=ref[0], pt_warps=ref[1],
                               pt_cost=ref[2], pt_offsets=po, stream=stream)
    ref_np = [r.cpu().numpy() for r in ref]
    for null in (1, 2):  # pt_warps NULL, then pt_cost NULL
        pts = [torch.full((total,), 7, dtype=dt, device="cuda") for dt in (torch.int32, torch.int32, torch.float32)]
        ptr = [C.c_void_p(t.data_ptr()) for t in pts]
        ptr[null] = None
        idx = torch.empty((90, k), dtype=torch.int32, device="cuda")
        cost = torch.empty((90, k), dtype=torch.float32, device="cuda")
        ax_, a_ = native.make_axes(ax), native.make_arch(a)
        rc = lib.tune_eval_noalloc(C.byref(a_), C.byref(ax_), C.c_void_p(dd.data_ptr()), 90, k,
                                   native.TUNE_EMIT_POINTS, C.c_void_p(idx.data_ptr()),
                                   C.c_void_p(cost.data_ptr()), ptr[0], ptr[1], ptr[2],
                                   C.c_void_p(po.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.tune_last_error()
        assert np.array_equal(idx.cpu().numpy(), ref_i.cpu().numpy())
        assert np.array_equal(cost.cpu().numpy().view(np.uint32), ref_c.cpu().numpy().view(np.uint32))
        got = [t.cpu().numpy() for t in pts]
        for j in range(3):
            if j == null:
                assert np.all(got[j] == 7)
            else:
                assert np.array_equal(got[j].view(np.uint32), ref_np[j].view(np.uint32)), j
