"""The paper's dense benchmark kernels as a tuning workload on this GPU.

matVec2D (y = A x), ATAX (y = A^T (A x)) and BiCG (q = A p, s = A^T r) from the
paper's kernel table (Section IV-A): each kernel's descriptor is written from its loop
structure (the static instruction counts a binary analysis would report), its
variants over a tuning sub-space are timed with tune_real_measure, and the static
model's ranking (tune_eval), its pruning (tune_suggest) and its searches (tune_search)
are compared with the measured times. Driver code: every step runs in the library.
"""

import ctypes as C

import numpy as np

from . import native
from workloads import gen

KINDS = {"matvec": native.TUNE_REAL_MATVEC, "atax": native.TUNE_REAL_ATAX, "bicg": native.TUNE_REAL_BICG}
# Tuning sub-space of the default axes: every thread count, grid sizes 64..4096 blocks,
# unroll 1, 2, 4, 8, carveouts 0 and 100 % (32 x 4 x 4 x 2 = 1,024 variants).
SUB = {"t": None, "g": [64, 256, 1024, 4096], "u": [1, 2, 4, 8], "c": [0, 100]}


def space_mask(axes):
    t_idx = range(len(axes["t"]))
    g_idx = [axes["g"].index(v) for v in SUB["g"]]
    u_idx = [axes["u"].index(v) for v in SUB["u"]]
    c_idx = [axes["c"].index(v) for v in SUB["c"]]
    return gen.mask_bits(t_idx, g_idx, u_idx, c_idx)


def descriptor(kind, n, r0, axes):
    """Descriptor of one kernel at matrix order n. Per output element a product runs n
    inner iterations of one FMA (FP32), two loads (matrix and vector element, GLDST), one
    index increment (INT) and one loop branch (BRANCH), plus one store and four index
    operations; matVec2D has one product, ATAX and BiCG two."""
    p = 1 if kind == "matvec" else 2
    d = np.zeros(1, dtype=gen.DESC_DTYPE)
    d["n"][0] = np.array([p * n, 0, p * (n + 4), p * (2 * n + 1), 0, p * n, 0], dtype=np.float32)
    d["r0"] = r0
    d["s0"] = 0
    d["d"] = 0.0
    d["space_mask"] = np.uint64(space_mask(axes))
    return d


def points(axes):
    """(T, G, U, C) of every point of the sub-space in canonical order (C fastest)."""
    out = []
    for T in axes["t"]:
        for G in SUB["g"]:
            for U in SUB["u"]:
                for Cv in SUB["c"]:
                    out.append((T, G, U, Cv))
    return np.array(out, dtype=np.int32)


def measure(kind, n, axes, reps=3, stream=None, with_result=False):
    """Median microseconds and registers of every variant of the sub-space (canonical order)."""
    L = native.load()
    pts = points(axes)
    cols = [np.ascontiguousarray(pts[:, j]) for j in range(4)]
    us = np.empty(len(pts), np.float32)
    regs = np.empty(len(pts), np.int32)
    res = np.empty(2 * n, np.float32) if with_result else None
    s = C.c_void_p(stream.cuda_stream) if stream is not None else None
    rc = L.tune_real_measure(KINDS[kind], n, *[c.ctypes.data for c in cols], len(pts), reps, us.ctypes.data,
                             regs.ctypes.data, res.ctypes.data if res is not None else None, s)
    native.check(rc)
    return us, regs, res


def evaluate(arch, axes, dev, n=6144, reps=3, k=5, surrogate=None):
    """Per kernel: the measured best variant; where the static model ranks it (tune_eval
    over the whole sub-space); whether the model's top-k holds it (hit@k); the measured
    time of the model's first pick over the best; whether static pruning (T*) keeps the
    best thread count; and the same for the learned surrogate when given."""
    import torch

    import paper_1701_08547_gb300 as T

    out = {}
    pts = points(axes)
    for kind in KINDS:
        us, regs, _ = measure(kind, n, axes, reps)
        ok = np.isfinite(us)
        best = int(np.argmin(np.where(ok, us, np.inf)))
        d = descriptor(kind, n, int(regs[pts[:, 2] == 1][0]), axes)
        dd = T.descs_to_device(d, dev)
        size = len(pts)
        idx, cost = T.tune_eval(arch, axes, dd, 16)
        ai = idx.cpu().numpy()[0]
        top = [int(i) for i in ai[:k] if i >= 0]
        first = top[0] if top else -1
        # model rank of the measured best: its position in the model's full (cost, index) order
        emit_B = torch.empty(size, dtype=torch.int32, device=dev)
        emit_W = torch.empty(size, dtype=torch.int32, device=dev)
        emit_c = torch.empty(size, dtype=torch.float32, device=dev)
        T.tune_eval(arch, axes, dd, 1, flags=native.TUNE_EMIT_POINTS, pt_blocks=emit_B, pt_warps=emit_W,
                    pt_cost=emit_c, pt_offsets=torch.tensor([0, size], dtype=torch.int64, device=dev))
        mc = emit_c.cpu().numpy()
        order = np.lexsort((np.arange(size), mc))
        rank = int(np.nonzero(order == best)[0][0]) + 1
        keep = int(T.tune_suggest(arch, axes, dd)["t_star"].cpu().numpy()[0]) & 0xFFFFFFFF
        t_best = axes["t"].index(int(pts[best, 0]))
        rec = {"variants": int(ok.sum()), "best": dict(zip("TGUC", map(int, pts[best]))),
               "best_us": float(us[best]), "model_rank_of_best": rank, f"model_hit@{k}": best in top,
               "model_first_pick_slowdown": float(us[first] / us[best]) if first >= 0 and ok[first] else None,
               "t_star": [axes["t"][p] for p in range(32) if (keep >> p) & 1],
               "t_star_keeps_best": bool((keep >> t_best) & 1),
               "median_over_best": float(np.median(us[ok]) / us[best])}
        # Nelder-Mead over the model (64 evaluations, 6 % of the sub-space), full and T*-pruned
        kt = torch.from_numpy(np.array([keep], dtype=np.uint32).view(np.int32)).to(dev)
        for name, tk in (("search_nm", None), ("search_nm_t_star", kt)):
            bi, _, _ = T.tune_search(arch, axes, dd, "nelder_mead", 64, 17, t_keep=tk)
            b = int(bi.cpu().numpy()[0])
            rec[f"{name}_slowdown"] = float(us[b] / us[best]) if b >= 0 and ok[b] else None
        if surrogate is not None:
            s_idx, _, _ = surrogate.infer(arch, axes, dd, np.array([0, size], np.int64), k, 1e30)
            si = [int(i) for i in s_idx.cpu().numpy()[0] if i >= 0]
            rec[f"surrogate_hit@{k}"] = best in si
            rec["surrogate_first_pick_slowdown"] = float(us[si[0]] / us[best]) if si and ok[si[0]] else None
        out[kind] = rec
    return out
