"""GB300-native static autotuning: occupancy + instruction-mix cost over whole
tuning spaces, and per-kernel top-k (Lim, Norris & Malony, Section III).

The functions here mirror the C ABI of libtune.so (include/tune.h) with the
same names; they marshal PyTorch tensors (device memory) and the current
CUDA stream into the C calls and nothing else.
"""

import ctypes as C

from . import native
from .native import (TUNE_EMIT_POINTS, TUNE_SCHED_CHUNK, TUNE_SCHED_CTAS,  # noqa: F401
                     TUNE_SCHED_THREAD, TUNE_SCHED_WARP, TuneError)

__all__ = ["tune_eval", "tune_eval_archs", "tune_topk", "tune_autotune", "tune_features", "tune_suggest", "tune_search", "tune_eval_host", "tune_workspace_bytes", "tune_check", "tune_inject_fault",
           "descs_to_device", "TUNE_EMIT_POINTS", "TUNE_SCHED_WARP", "TUNE_SCHED_THREAD",
           "TUNE_SCHED_CHUNK", "TUNE_SCHED_CTAS", "TuneError"]


def _torch():
    import torch

    return torch


def _stream(stream):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def tune_workspace_bytes(call, n, k):
    return native.load().tune_workspace_bytes(int(call), int(n), int(k))


def workspace(call, n, k, device="cuda"):
    torch = _torch()
    nbytes = tune_workspace_bytes(call, n, k)
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def descs_to_device(descs, device="cuda"):
    """Copy a numpy descriptor array (64-byte records) to a uint8 device tensor [n, 64]."""
    torch = _torch()
    import numpy as np

    raw = np.ascontiguousarray(descs).view(np.uint8).reshape(-1, 64)
    return torch.from_numpy(raw).to(device)


def tune_eval(arch, axes, descs, k, flags=0, topk_idx=None, topk_cost=None, pt_blocks=None,
              pt_warps=None, pt_cost=None, pt_offsets=None, workspace_buf=None, stream=None):
    """Evaluate every point of every kernel's space and select each kernel's top-k.

    descs: contiguous device tensor holding n 64-byte descriptor records.
    Returns (topk_idx int32 [n, k], topk_cost float32 [n, k]).
    """
    torch = _torch()
    L = native.load()
    assert descs.is_cuda and descs.is_contiguous() and descs.numel() * descs.element_size() % 64 == 0
    n = descs.numel() * descs.element_size() // 64
    dev = descs.device
    if topk_idx is None:
        topk_idx = torch.empty((n, k), dtype=torch.int32, device=dev)
    if topk_cost is None:
        topk_cost = torch.empty((n, k), dtype=torch.float32, device=dev)
    if workspace_buf is None:
        workspace_buf = workspace(native.TUNE_CALL_EVAL, n, k, dev)
    a = native.make_arch(arch)
    x = native.make_axes(axes)
    rc = L.tune_eval(C.byref(a), C.byref(x), _ptr(descs), n, int(k), int(flags), _ptr(topk_idx),
                     _ptr(topk_cost), _ptr(pt_blocks), _ptr(pt_warps), _ptr(pt_cost),
                     _ptr(pt_offsets), _ptr(workspace_buf), workspace_buf.numel(), _stream(stream))
    native.check(rc)
    return topk_idx, topk_cost


def tune_eval_archs(archs, axes, descs, k, flags=0, workspace_buf=None, stream=None):
    """tune_eval against several architecture rows in one launch.
    Returns (topk_idx int32 [n_arch, n, k], topk_cost float32 [n_arch, n, k])."""
    torch = _torch()
    L = native.load()
    assert descs.is_cuda and descs.is_contiguous() and descs.numel() * descs.element_size() % 64 == 0
    n = descs.numel() * descs.element_size() // 64
    dev = descs.device
    na = len(archs)
    topk_idx = torch.empty((na, n, k), dtype=torch.int32, device=dev)
    topk_cost = torch.empty((na, n, k), dtype=torch.float32, device=dev)
    if workspace_buf is None:
        workspace_buf = workspace(native.TUNE_CALL_EVAL, 0, k, dev)
    rows = (native.TuneArch * na)(*[native.make_arch(a) for a in archs])
    x = native.make_axes(axes)
    rc = L.tune_eval_archs(rows, na, C.byref(x), _ptr(descs), n, int(k), int(flags), _ptr(topk_idx),
                           _ptr(topk_cost), _ptr(workspace_buf), workspace_buf.numel(), _stream(stream))
    native.check(rc)
    return topk_idx, topk_cost


def tune_topk(scores, seg_offsets, k, topk_idx=None, topk_score=None, workspace_buf=None,
              stream=None):
    """Segmented top-k (smallest scores, ties -> lower index) over device float32 scores."""
    torch = _torch()
    L = native.load()
    n_seg = seg_offsets.numel() - 1
    dev = scores.device
    if topk_idx is None:
        topk_idx = torch.empty((n_seg, k), dtype=torch.int32, device=dev)
    if topk_score is None:
        topk_score = torch.empty((n_seg, k), dtype=torch.float32, device=dev)
    if workspace_buf is None:
        workspace_buf = workspace(native.TUNE_CALL_TOPK, n_seg, k, dev)
    rc = L.tune_topk(_ptr(scores), _ptr(seg_offsets), n_seg, int(k), _ptr(topk_idx),
                     _ptr(topk_score), _ptr(workspace_buf), workspace_buf.numel(), _stream(stream))
    native.check(rc)
    return topk_idx, topk_score


def tune_autotune(arch, axes, descs, k, reps=3, topk_idx=None, topk_cost=None, workspace_buf=None,
                  stream=None):
    """Time tune_eval's candidate schedules on these descriptors; returns
    (best_flags, best_ms, topk_idx, topk_cost)."""
    torch = _torch()
    L = native.load()
    n = descs.numel() * descs.element_size() // 64
    dev = descs.device
    if topk_idx is None:
        topk_idx = torch.empty((n, k), dtype=torch.int32, device=dev)
    if topk_cost is None:
        topk_cost = torch.empty((n, k), dtype=torch.float32, device=dev)
    if workspace_buf is None:
        workspace_buf = workspace(native.TUNE_CALL_EVAL, n, k, dev)
    a = native.make_arch(arch)
    x = native.make_axes(axes)
    bf, bms = C.c_uint32(0), C.c_float(0.0)
    rc = L.tune_autotune(C.byref(a), C.byref(x), _ptr(descs), n, int(k), int(reps), _ptr(topk_idx),
                         _ptr(topk_cost), _ptr(workspace_buf), workspace_buf.numel(), C.byref(bf),
                         C.byref(bms), _stream(stream))
    native.check(rc)
    return bf.value, bms.value, topk_idx, topk_cost


def tune_features(arch, axes, descs, sample_kernel, sample_point, feats=None, workspace_buf=None,
                  stream=None):
    """Surrogate input features (device bfloat16 [n, 64]) of listed (kernel, point) samples."""
    torch = _torch()
    L = native.load()
    n = sample_kernel.numel()
    dev = descs.device
    if feats is None:
        feats = torch.empty((n, native.TUNE_SURROGATE_INPUTS), dtype=torch.bfloat16, device=dev)
    if workspace_buf is None:
        workspace_buf = workspace(native.TUNE_CALL_EVAL, 0, 1, dev)
    a = native.make_arch(arch)
    x = native.make_axes(axes)
    rc = L.tune_features(C.byref(a), C.byref(x), _ptr(descs), _ptr(sample_kernel), _ptr(sample_point), n,
                         _ptr(feats), _ptr(workspace_buf), workspace_buf.numel(), _stream(stream))
    native.check(rc)
    return feats


def tune_suggest(arch, axes, descs, workspace_buf=None, stream=None):
    """Static pruning per kernel: dict of device tensors t_star, occ_star, r_headroom, s_star, t_rule."""
    torch = _torch()
    L = native.load()
    n = descs.numel() * descs.element_size() // 64
    dev = descs.device
    out = {"t_star": torch.empty(n, dtype=torch.int32, device=dev),
           "occ_star": torch.empty(n, dtype=torch.float32, device=dev),
           "r_headroom": torch.empty(n, dtype=torch.int32, device=dev),
           "s_star": torch.empty(n, dtype=torch.int32, device=dev),
           "t_rule": torch.empty(n, dtype=torch.int32, device=dev)}
    if workspace_buf is None:
        workspace_buf = workspace(native.TUNE_CALL_EVAL, 0, 1, dev)
    a = native.make_arch(arch)
    x = native.make_axes(axes)
    rc = L.tune_suggest(C.byref(a), C.byref(x), _ptr(descs), n, _ptr(out["t_star"]), _ptr(out["occ_star"]),
                        _ptr(out["r_headroom"]), _ptr(out["s_star"]), _ptr(out["t_rule"]), _ptr(workspace_buf),
                        workspace_buf.numel(), _stream(stream))
    native.check(rc)
    return out


def tune_search(arch, axes, descs, method, budget, seed, t_keep=None, workspace_buf=None, stream=None):
    """Random (method "random") or Nelder-Mead ("nelder_mead") search per kernel with the
    static cost as the objective; t_keep: optional device uint32 mask per kernel of the
    thread-count positions to search. Returns (best_idx, best_cost, evals) device tensors."""
    torch = _torch()
    L = native.load()
    m = {"random": native.TUNE_SEARCH_RANDOM, "nelder_mead": native.TUNE_SEARCH_NELDER_MEAD}[method]
    n = descs.numel() * descs.element_size() // 64
    dev = descs.device
    best_idx = torch.empty(n, dtype=torch.int32, device=dev)
    best_cost = torch.empty(n, dtype=torch.float32, device=dev)
    evals = torch.empty(n, dtype=torch.int32, device=dev)
    if workspace_buf is None:
        workspace_buf = workspace(native.TUNE_CALL_EVAL, 0, 1, dev)
    a = native.make_arch(arch)
    x = native.make_axes(axes)
    rc = L.tune_search(C.byref(a), C.byref(x), _ptr(descs), n, int(m), int(budget), int(seed) & (2 ** 64 - 1),
                       _ptr(t_keep) if t_keep is not None else None, _ptr(best_idx), _ptr(best_cost), _ptr(evals),
                       _ptr(workspace_buf), workspace_buf.numel(), _stream(stream))
    native.check(rc)
    return best_idx, best_cost, evals


def tune_eval_host(arch, axes, host_descs, k, chunk, topk_idx, topk_cost, scratch=None, flags=0, stream=None):
    """tune_eval from and to host memory with the copies overlapping the evaluation, or,
    with flags | TUNE_HOST_DIRECT and pinned buffers, in place over the host link in one
    launch. host_descs: host uint8 tensor [n, 64] (pinned for overlap); topk_idx /
    topk_cost: host int32 / float32 tensors [n, k] (pinned); scratch: device uint8 tensor of
    tune_eval_host_scratch_bytes(chunk, k) bytes, 256 in the direct mode (allocated here if
    None). Enqueues on `stream`; returns the scratch (its header holds the status word)."""
    torch = _torch()
    L = native.load()
    n = host_descs.numel() // 64
    nbytes = 256 if flags & native.TUNE_HOST_DIRECT else L.tune_eval_host_scratch_bytes(int(chunk), int(k))
    if scratch is None:
        scratch = torch.empty(nbytes, dtype=torch.uint8, device=torch.device("cuda", torch.cuda.current_device()))
    a = native.make_arch(arch)
    x = native.make_axes(axes)
    rc = L.tune_eval_host(C.byref(a), C.byref(x), _ptr(host_descs), n, int(k), int(flags), _ptr(topk_idx),
                          _ptr(topk_cost), int(chunk), _ptr(scratch), scratch.numel(), _stream(stream))
    native.check(rc)
    return scratch


def tune_inject_fault(kind, count=1):
    """Set `count` pending injected faults of one kind (native.TUNE_FAULT_COMPILE,
    TUNE_FAULT_SLOW_REP or TUNE_FAULT_WAIT; 0 clears), to exercise failure paths."""
    native.check(native.load().tune_inject_fault(int(kind), int(count)))


def tune_check(workspace_buf, stream=None):
    """Wait for the stream and raise if a kernel flagged malformed input."""
    return native.check(native.load().tune_check(_ptr(workspace_buf), _stream(stream)))


def tune_eval_noalloc(arch, axes, descs, k, flags=0, topk_idx=None, topk_cost=None, pt_blocks=None,
                      pt_warps=None, pt_cost=None, pt_offsets=None, stream=None):
    """tune_eval without a workspace, for hosts that cannot allocate device memory
    for the library: scratch lives in a static 4 KB device array inside libtune.so.
    Waits for the stream before returning. Output tensors must be given by callers
    that cannot allocate; when omitted they are created here for convenience."""
    torch = _torch()
    L = native.load_noalloc()
    n = descs.numel() * descs.element_size() // 64
    dev = descs.device
    if topk_idx is None:
        topk_idx = torch.empty((n, k), dtype=torch.int32, device=dev)
    if topk_cost is None:
        topk_cost = torch.empty((n, k), dtype=torch.float32, device=dev)
    a = native.make_arch(arch)
    x = native.make_axes(axes)
    rc = L.tune_eval_noalloc(C.byref(a), C.byref(x), _ptr(descs), n, int(k), int(flags),
                             _ptr(topk_idx), _ptr(topk_cost), _ptr(pt_blocks), _ptr(pt_warps),
                             _ptr(pt_cost), _ptr(pt_offsets), _stream(stream))
    native.check(rc)
    return topk_idx, topk_cost
