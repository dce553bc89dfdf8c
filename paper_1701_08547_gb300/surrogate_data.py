"""Surrogate data generation, training and evaluation on the GPU (driver code).

* label generation: tune_emit_measure times synthetic variants of sampled
  (descriptor, point) pairs on this GPU. Every thread of a variant runs the
  descriptor's per-thread work, so a launch of G blocks of T threads does
  G T units of it; the label is ln(nanoseconds per unit of work) =
  ln(1000 us / (G T ITEMS)), the quantity the static model's cost ranks (its
  counts are per thread; its launch-shape terms spread G T units of work over
  the busy SMs);
* features: tune_features (the analyzer's internals for each sample);
* training: surrogate_train (the library's BF16 kernels) over seeded epochs;
* evaluation: held-out descriptors whose small spaces are timed completely;
  hit@5 = the measured-best point (least time per unit of work) is among the
  5 a ranking picks, for the ensemble (with its analytic fallback), for the
  analytic model alone, and for 5 uniform random picks (the chance floor),
  each with a 95 % Wilson interval over the kernels.

All random choices (descriptors, sampled points, epoch orders, initial
weights) are seeded; the seeds are arguments.
"""

import ctypes as C

import numpy as np

from . import native
from . import descs_to_device, tune_eval, tune_features, tune_suggest
from .surrogate import Surrogate

ITEMS = 1                 # work items per thread
COUNT_SCALE = 1.0 / 1024.0
# Sub-space sampled for labels: threads >= 64, grid 64 .. 2048 blocks (axis positions), so
# that every variant finishes within about a millisecond.
T_MIN_POS, G_MIN_POS, G_MAX_POS = 1, 6, 11
# Held-out spaces, fully timed: 5 thread counts x 4 grids x unroll {1, 4} x carveout {0, 100}
EVAL_T, EVAL_G, EVAL_U, EVAL_C = [1, 3, 7, 15, 31], [7, 9, 11, 13], [0, 3], [0, 3]
# Pruning spaces, fully timed: all 32 thread counts x grids {512, 2048} x unroll 1 x carveout 100
PRUNE_T, PRUNE_G, PRUNE_U, PRUNE_C = list(range(32)), [9, 11], [0], [3]


def _emit_lib():
    L = native.load()
    if not getattr(L, "_emit_declared", False):
        vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
        L.tune_emit_measure.argtypes = [C.POINTER(native.TuneAxes), vp, i64, vp, vp, i64, i32, C.c_float, i32,
                                        vp, vp, vp, vp]
        L.tune_emit_measure.restype = C.c_int
        L.tune_emit_count.argtypes = [C.POINTER(native.TuneAxes), vp, i64, vp, vp, i64, i32, C.c_float, vp, vp]
        L.tune_emit_count.restype = C.c_int
        L._emit_declared = True
    return L


def measure(axes, descs, skern, spoint, items=ITEMS, scale=COUNT_SCALE, reps=3, stream=None, launched=False):
    """Median launch time (us; NaN where not launchable) and registers of each sample's variant;
    with launched=True also the (T, G, U, C) each sample decoded to (int32 [n, 4])."""
    import torch

    L = _emit_lib()
    d = np.ascontiguousarray(descs)
    sk = np.ascontiguousarray(skern, dtype=np.int32)
    sp = np.ascontiguousarray(spoint, dtype=np.int32)
    us = np.empty(len(sk), dtype=np.float32)
    regs = np.empty(len(sk), dtype=np.int32)
    cfg = np.zeros((len(sk), 4), dtype=np.int32)
    s = torch.cuda.current_stream() if stream is None else stream
    x = native.make_axes(axes)
    native.check(L.tune_emit_measure(C.byref(x), d.ctypes.data, len(d), sk.ctypes.data, sp.ctypes.data, len(sk),
                                     int(items), float(scale), int(reps), us.ctypes.data, regs.ctypes.data,
                                     cfg.ctypes.data, C.c_void_p(s.cuda_stream)))
    return (us, regs, cfg) if launched else (us, regs)


def count_ops(axes, descs, skern, spoint, items=ITEMS, scale=COUNT_SCALE, stream=None):
    """Operations executed per class (FP32, FP64, INT, GLDST, SLDST, BRANCH, SFU) by all threads
    of each sample's variant, uint64 [n, 7] (all ones where the launch is not possible)."""
    import torch

    L = _emit_lib()
    d = np.ascontiguousarray(descs)
    sk = np.ascontiguousarray(skern, dtype=np.int32)
    sp = np.ascontiguousarray(spoint, dtype=np.int32)
    out = np.empty((len(sk), 7), dtype=np.uint64)
    s = torch.cuda.current_stream() if stream is None else stream
    x = native.make_axes(axes)
    native.check(L.tune_emit_count(C.byref(x), d.ctypes.data, len(d), sk.ctypes.data, sp.ctypes.data, len(sk),
                                   int(items), float(scale), out.ctypes.data, C.c_void_p(s.cuda_stream)))
    return out


CATEGORIES = {"FLOPS": (0, 1, 6), "MEM": (3, 4), "CTRL": (5,), "INT": (2,)}


def mix_error(static, dynamic):
    """Section IV's comparison of a static and a dynamic instruction mix, per category
    (FLOPS = FP32 + FP64 + SFU, MEM = global + shared loads/stores, CTRL = branches, INT):
    the squared difference of the two mixes' category shares in percent, (100 f_s - 100 f_d)^2,
    and the intensity FLOPS / MEM of the static mix."""
    st = np.asarray(static, np.float64)
    dy = np.asarray(dynamic, np.float64)
    out = {}
    for name, cls in CATEGORIES.items():
        fs = st[list(cls)].sum() / st.sum()
        fd = dy[list(cls)].sum() / dy.sum()
        out[name] = float((100 * fs - 100 * fd) ** 2)
    out["intensity"] = float(st[[0, 1, 6]].sum() / max(st[[3, 4]].sum(), 1e-30))
    return out


def per_unit_ns(us, cfg, items=ITEMS):
    """Nanoseconds per unit of per-thread work: 1000 us / (G T items) (NaN stays NaN)."""
    return 1000.0 * np.asarray(us, np.float64) / (cfg[:, 1].astype(np.float64) * cfg[:, 0] * items)


def sample_points(descs, per_desc, seed):
    """per_desc random canonical point indices per descriptor, restricted to T >= 64 and
    64 <= G <= 2048."""
    rng = np.random.default_rng(seed)
    skern, spoint = [], []
    for i, d in enumerate(descs):
        m = int(d["space_mask"])
        tp = [b for b in range(32) if (m >> b) & 1 and b >= T_MIN_POS]
        gp = [b for b in range(16) if (m >> (32 + b)) & 1 and G_MIN_POS <= b <= G_MAX_POS]
        up = [b for b in range(8) if (m >> (48 + b)) & 1]
        cp = [b for b in range(4) if (m >> (56 + b)) & 1]
        if not (tp and gp and up and cp):
            continue
        allt = [b for b in range(32) if (m >> b) & 1]
        allg = [b for b in range(16) if (m >> (32 + b)) & 1]
        for _ in range(per_desc):
            t, g = allt.index(rng.choice(tp)), allg.index(rng.choice(gp))
            u, c = rng.integers(len(up)), rng.integers(len(cp))
            skern.append(i)
            spoint.append(((t * len(allg) + g) * len(up) + u) * len(cp) + c)
    return np.array(skern, dtype=np.int64), np.array(spoint, dtype=np.int32)


def build_set(arch, axes, descs, per_desc, seed, dev):
    """Measured training set: features (device bf16), labels ln(ns per unit of work) (device),
    kept samples."""
    import torch

    skern, spoint = sample_points(descs, per_desc, seed)
    us, _, cfg = measure(axes, descs, skern, spoint, launched=True)
    ns = per_unit_ns(us, cfg)
    feats = tune_features(arch, axes, descs_to_device(descs, dev), torch.from_numpy(skern).to(dev),
                          torch.from_numpy(spoint).to(dev))
    valid = feats[:, 29].float().cpu().numpy() > 0  # B* > 0 under the model
    keep = np.isfinite(ns) & (ns > 0) & valid
    idx = torch.from_numpy(np.nonzero(keep)[0]).to(dev)
    return {"feats": feats[idx].contiguous(),
            "labels": torch.from_numpy(np.log(ns[keep]).astype(np.float32)).to(dev),
            "n": int(keep.sum()), "measured": len(us), "us": us}


def analytic_set(arch, axes, descs, per_desc, seed, dev):
    """Training set labelled by the analytic model itself (the surrogate's sanity case): the
    same sampled points and features as build_set, label (ln(cost) - median) / std from
    tune_eval's per-point costs (a positive affine map of the label keeps the ranking; the
    members' std / mean is not used with these labels); points without a valid configuration
    are dropped."""
    import torch

    from workloads import gen

    skern, spoint = sample_points(descs, per_desc, seed)
    dd = descs_to_device(descs, dev)
    off = gen.point_offsets(descs)
    total = int(off[-1])
    pc = torch.empty(total, dtype=torch.float32, device=dev)
    tune_eval(arch, axes, dd, 1, flags=native.TUNE_EMIT_POINTS, pt_cost=pc,
              pt_offsets=torch.from_numpy(off).to(dev))
    cost = pc.cpu().numpy()[off[skern] + spoint].astype(np.float64)
    feats = tune_features(arch, axes, dd, torch.from_numpy(skern).to(dev), torch.from_numpy(spoint).to(dev))
    keep = np.isfinite(cost) & (cost > 0)
    idx = torch.from_numpy(np.nonzero(keep)[0]).to(dev)
    lab = np.log(cost[keep])
    shift, scale = float(np.median(lab)), float(np.std(lab)) or 1.0
    return {"feats": feats[idx].contiguous(),
            "labels": torch.from_numpy(((lab - shift) / scale).astype(np.float32)).to(dev),
            "n": int(keep.sum()), "measured": len(cost), "label_shift": shift, "label_scale": scale}


def train(data, members=5, epochs=20, batch=8192, lr=1e-3, seed=5, dev="cuda"):
    """Train an ensemble on a measured set; returns (Surrogate, loss trace [epochs, steps, members])."""
    import torch

    from workloads import mlp as L

    n = data["n"]
    batch = min(batch, max(128, (n // 128) * 128))
    sur = Surrogate(members=members, batch=batch, lr=lr)
    sur.set_params(L.init_params(members, [seed + m for m in range(members)]))
    rng = np.random.default_rng(seed)
    order = torch.from_numpy(np.concatenate([rng.permutation(n) for _ in range(epochs)]).astype(np.int32)).to(dev)
    steps = (n + batch - 1) // batch
    trace = torch.zeros(epochs * steps * members, dtype=torch.float32, device=dev)
    sur.train(data["feats"], data["labels"], order, epochs, trace)
    torch.cuda.synchronize()
    return sur, trace.cpu().numpy().reshape(epochs, steps, members)


def eval_spaces(descs):
    from workloads import gen

    out = descs.copy()
    out["space_mask"] = np.uint64(gen.mask_bits(EVAL_T, EVAL_G, EVAL_U, EVAL_C))
    return out


def wilson(hits, n, z=1.96):
    """95 % Wilson score interval of a binomial proportion hits / n."""
    if n == 0:
        return [0.0, 1.0]
    p = hits / n
    c = (p + z * z / (2 * n)) / (1 + z * z / n)
    h = z * np.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / (1 + z * z / n)
    return [float(max(0.0, c - h)), float(min(1.0, c + h))]


def timed_spaces(axes, descs):
    """Time every point of each descriptor's held-out space: (descriptors with those spaces,
    ns per unit of work [n, size], NaN where not launchable)."""
    from workloads import gen

    d = eval_spaces(descs)
    size = int(gen.space_sizes(d[:1])[0])
    skern = np.repeat(np.arange(len(d)), size)
    spoint = np.tile(np.arange(size), len(d)).astype(np.int32)
    us, _, cfg = measure(axes, d, skern, spoint, launched=True)
    return d, per_unit_ns(us, cfg).reshape(len(d), size)


def evaluate(sur, arch, axes, descs, dev, k=5, thresh=0.1, timed=None):
    """Against the measured best (least time per unit of work) of fully timed held-out spaces:
    hit@k (best among the k picks), overlap of the k picks with the measured k best, and the
    median slowdown of the first pick, for the ensemble (with its analytic fallback at
    `thresh`) and for the analytic model; the chance floor of k uniform picks among the
    launchable points; 95 % Wilson intervals of the hit rates. `timed` reuses timed_spaces()."""
    from workloads import gen

    d, us = timed if timed is not None else timed_spaces(axes, descs)
    size = us.shape[1]
    dd = descs_to_device(d, dev)
    a_idx, _ = tune_eval(arch, axes, dd, k)
    s_idx, _, fb = sur.infer(arch, axes, dd, gen.point_offsets(d), k, thresh)
    a_idx, s_idx, fb = a_idx.cpu().numpy(), s_idx.cpu().numpy(), fb.cpu().numpy()
    t = np.where(np.isfinite(us), us, np.inf)  # unlaunchable points never win and count as misses
    ok = np.sum(np.isfinite(us), axis=1) >= k
    best = np.argmin(t, axis=1)
    meas_top = np.argsort(t, axis=1, kind="stable")[:, :k]

    def stats(idx):
        hit = np.array([best[i] in idx[i] for i in range(len(d))])[ok]
        ov = np.array([len(set(idx[i]) & set(meas_top[i])) / k for i in range(len(d))])[ok]
        first = np.array([t[i, idx[i, 0]] / t[i, best[i]] if idx[i, 0] >= 0 else np.inf
                          for i in range(len(d))])[ok]
        return float(hit.mean()), int(hit.sum()), float(ov.mean()), float(np.median(first))

    n_ok = int(ok.sum())
    hs, ns_, os_, rs = stats(s_idx)
    ha, na, oa, ra = stats(a_idx)
    launchable = np.sum(np.isfinite(us), axis=1)[ok]
    floor = float(np.mean(np.minimum(1.0, k / launchable)))
    return {"kernels": n_ok, "k": k, "thresh": thresh, "hit_surrogate": hs, "hit_analytic": ha,
            "hit_random": floor, "hit_surrogate_ci95": wilson(ns_, n_ok), "hit_analytic_ci95": wilson(na, n_ok),
            "overlap_surrogate": os_, "overlap_analytic": oa, "first_pick_slowdown_surrogate": rs,
            "first_pick_slowdown_analytic": ra, "fallback_rate": float(fb[ok].mean())}


def evaluate_pruning(arch, axes, descs, dev):
    """Static pruning (tune_suggest) against measured times: every point of spaces with all 32
    thread counts is timed; per kernel, is the measured-best thread count in T* (and in the
    rule's half of T*), and how much slower is the best point left in the pruned space."""
    from workloads import gen

    d = descs.copy()
    d["space_mask"] = np.uint64(gen.mask_bits(PRUNE_T, PRUNE_G, PRUNE_U, PRUNE_C))
    size = int(gen.space_sizes(d[:1])[0])
    n_g = len(PRUNE_G)
    us, _, cfg = measure(axes, d, np.repeat(np.arange(len(d)), size), np.tile(np.arange(size), len(d)).astype(np.int32),
                         launched=True)
    ns = per_unit_ns(us, cfg)
    t = np.where(np.isfinite(ns), ns, np.inf).reshape(len(d), len(PRUNE_T), n_g)  # canonical order: T, then G
    sug = tune_suggest(arch, axes, descs_to_device(d, dev))
    star = sug["t_star"].cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    rule = sug["t_rule"].cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    ok = np.isfinite(t.min(axis=(1, 2))) & (star != 0)
    best_t = t.min(axis=2)                       # per kernel, per thread count
    overall = best_t.min(axis=1)

    def stats(mask):
        sel = np.array([[(m >> p) & 1 for p in PRUNE_T] for m in mask], dtype=bool)
        pruned = np.where(sel, best_t, np.inf).min(axis=1)
        hit = (pruned == overall)[ok]
        slow = (pruned / overall)[ok]
        return {"hit": float(hit.mean()), "median_slowdown": float(np.median(slow)),
                "p90_slowdown": float(np.quantile(slow, 0.9)), "kept_thread_counts": float(sel[ok].sum(1).mean())}

    return {"kernels": int(ok.sum()), "thread_counts": len(PRUNE_T), "grids": [int(axes["g"][p]) for p in PRUNE_G],
            "static_t_star": stats(star), "rule": stats(rule)}
