"""Throughput of the static-autotuning hot path on GB300.

One step = tune_eval over the whole workload: every point of every kernel's
tuning space gets occupancy + cost, then each kernel's top-k is selected.
Default workload: 100,000 synthetic kernels x 16,384-point dense spaces
(threads 32..1024/32 x grid 2^0..2^15 x unroll 1..8 x carveout {0,25,50,100}%),
top-10 per kernel, sm_103 architecture row.

Prints one JSON line (rank 0). Under torchrun each rank evaluates its own
100,000 kernels (weak scaling, no data-path collective); the timing is the
max over ranks.

--impl reference times the CPU oracle (the plain FP64 + FP32-mirror C
implementation) on a bounded sample of the same workload, on the host cores.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import archs, gen  # noqa: E402

METRIC = "tuning points evaluated/sec + top-k"
WORKLOADS = {
    # name: (n_kernels per rank, space, k, seed)
    "dense": (100_000, "dense", 10, 2),
    "dense128": (64, "dense128", 5, 1),
    "uneven": (1_000_000, "uneven", 5, 3),
    "topk": (100_000, None, 10, 11),
    "surfwd": (1 << 20, None, 0, 12),
    "surtrain": (1 << 16, None, 0, 13),
    "search": (100_000, "dense", 1, 2),
}
ISSUE_LANES_PER_SM_CLK = 4 * 32  # 4 schedulers x 32 lanes per SM and clock
# Thread-instructions of a per-point evaluation after the per-kernel hoists (decode ~3,
# 2 IMNMX, 1 IMAD, 2 table loads, 1 FFMA + 2 FMUL, 1 compare); reported beside the
# headline for reference.
PER_POINT_EVAL_INSTR = 12
# Thread-instructions of pricing one point from scratch (occupancy limits, cost sums,
# launch-shape terms): one evaluation of a search.
UNHOISTED_INSTR_PER_POINT = 60
L2_FLUSH_BYTES = 256 << 20       # larger than the 126.5 MB L2


def space_counts(descs):
    """(points, (T, U, C) triples) of every kernel's space."""
    sizes = gen.space_sizes(descs)
    m = np.asarray(descs["space_mask"], dtype=np.uint64)
    n_g = np.zeros(len(m), np.int64)
    for b in range(16):
        n_g += ((m >> np.uint64(32 + b)) & np.uint64(1)).astype(np.int64)
    triples = np.where(n_g > 0, sizes // np.maximum(n_g, 1), 0)
    return sizes, triples


def algorithmic_instructions(descs, axes):
    """Thread-instructions of evaluating every point once the grid-independent work is
    factored out: grid size does not enter the occupancy (Eqs. 1-5), so B*, W* and the
    cost factor X(T,U,C) are per (T, U, C) triple (B* min, W* multiply, hide lookup,
    FFMA, lane-efficiency multiply = 5), and each point then costs X * ipar(B*, G) (1
    multiply) and one compare with the running k-th best (1): 2 per point + 5 per triple.
    """
    sizes, triples = space_counts(descs)
    return int(2 * sizes.sum() + 5 * triples.sum())


def triple_instructions(descs):
    """Lower figure for a ranking that never prices individual points: 8 per triple (the
    5 above, the triple's cheapest point X * min_G ipar (lookup + multiply), 1 compare)."""
    _, triples = space_counts(descs)
    return int(8 * triples.sum())


def kernel_source_hash():
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_1701_08547_gb300", "csrc", "tune_eval.cu"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def recorded_profile(workload):
    """Figures of the committed ncu summary of this workload's launch, if it was taken on
    the current kernel source (else {}): bytes_per_launch (DRAM read + write) and
    issue_active (fraction of issue slots used)."""
    path = os.path.join(ROOT, "profiles", f"tune_eval_{workload}.md")
    if not os.path.exists(path):
        return {}
    vals = {}
    with open(path) as f:
        for line in f:
            if line.startswith("bench-traffic:"):
                for kv in line.split(":", 1)[1].split():
                    k, v = kv.split("=")
                    vals[k] = v
    if vals.get("source_sha256") != kernel_source_hash():
        return {}
    return {k: float(v) for k, v in vals.items() if k != "source_sha256"}


def recorded_traffic(workload):
    """DRAM bytes per launch from the committed ncu summary (None if stale or absent)."""
    return recorded_profile(workload).get("bytes_per_launch")


class ClockSampler:
    """SM clock and clock-event reasons sampled during the timed region.

    Read-only NVML queries from a polling thread (every 2 ms), so that short
    timed regions still get samples; falls back to nvidia-smi if NVML is not
    loadable.
    """

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, uuid=None, index=0):
        self.uuid, self.index = uuid, index
        self.sm, self.mx, self.reasons = [], [], set()
        self._stop = None

    def _nvml(self):
        import ctypes as C

        lib = C.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            return None, None
        h = C.c_void_p()
        ok = False
        if self.uuid:
            ok = lib.nvmlDeviceGetHandleByUUID(self.uuid.encode(), C.byref(h)) == 0
        if not ok:
            ok = lib.nvmlDeviceGetHandleByIndex_v2(self.index, C.byref(h)) == 0
        return (lib, h) if ok else (None, None)

    def _poll(self):
        import ctypes as C

        lib, h = self._nvml()
        if lib is None:
            return
        clk, mx, rs = C.c_uint(), C.c_uint(), C.c_ulonglong()
        lib.nvmlDeviceGetMaxClockInfo(h, 1, C.byref(mx))
        while not self._stop.is_set():
            if lib.nvmlDeviceGetClockInfo(h, 1, C.byref(clk)) == 0:
                self.sm.append(float(clk.value))
                self.mx.append(float(mx.value))
            if lib.nvmlDeviceGetCurrentClocksEventReasons(h, C.byref(rs)) == 0:
                for bit, name in self.REASONS.items():
                    if rs.value & bit:
                        self.reasons.add(name)
            self._stop.wait(0.002)

    def __enter__(self):
        import threading

        self._stop = threading.Event()
        self._thread = threading.Thread(target=self._poll, daemon=True)
        try:
            self._thread.start()
        except RuntimeError:
            self._thread = None
        return self

    def __exit__(self, *exc):
        self._stop.set()
        if self._thread is not None:
            self._thread.join(timeout=5)

    def summary(self):
        if not self.sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": sorted(self.reasons), "samples": 0}
        return {"sm_mhz": statistics.median(self.sm), "sm_max_mhz": max(self.mx),
                "reasons": sorted(self.reasons), "samples": len(self.sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard(n, seed, space, rank):
    """Rank r's kernels: descriptors r n .. (r + 1) n - 1 of the seeded workload (weak
    scaling; kernels are independent, so the ranks exchange no data)."""
    return gen.descriptors(n, seed, space, first=rank * n)


def max_over_ranks(value, world, device):
    """The largest of the ranks' values (the step time of the slowest rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"sm_max_mhz": 2070.0}, "fallback"


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1701_08547_gb300 as T
    from paper_1701_08547_gb300 import build as B

    rank, world, local = dist_env()
    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    n, space, k, seed = WORKLOADS[args.workload]
    n = args.kernels or n
    a, ax = archs.arch("sm_103"), gen.axes()
    descs = shard(n, seed, space, rank)
    points = int(gen.space_sizes(descs).sum())
    algo_instr = algorithmic_instructions(descs, ax)
    triple_instr = triple_instructions(descs)

    d_dev = T.descs_to_device(descs, dev)
    ws = T.workspace(0, n, k, dev)
    topi = torch.empty((n, k), dtype=torch.int32, device=dev)
    topc = torch.empty((n, k), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)

    # Schedule: chosen by the library's autotuner on this workload (untimed), or forced.
    if args.flags:
        sched, tuned_ms = int(args.flags, 16), None
    elif args.sched == "auto":
        sched, tuned_ms, _, _ = T.tune_autotune(a, ax, d_dev, k, reps=3, topk_idx=topi, topk_cost=topc,
                                                workspace_buf=ws, stream=stream)
    else:
        sched, tuned_ms = {"warp": 0x10, "thread": 0x20}[args.sched], None

    def step():
        T.tune_eval(a, ax, d_dev, k, flags=sched, topk_idx=topi, topk_cost=topc, workspace_buf=ws,
                    stream=stream)

    step()  # first call outside capture (occupancy queries are cached here)
    torch.cuda.synchronize()
    graph = None
    if not args.no_graph:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            step()
    run_step = graph.replay if graph is not None else step

    for _ in range(args.warmup):
        flush.zero_()
        run_step()
    torch.cuda.synchronize()
    T.tune_check(ws, stream)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    uuid = f"GPU-{uuid}" if uuid is not None and not str(uuid).startswith("GPU-") else uuid
    with ClockSampler(uuid, local) as clk:
        for i in range(args.steps):
            flush.zero_()  # L2 flush between timed steps (outside the event pair)
            starts[i].record(stream)
            run_step()
            ends[i].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    T.tune_check(ws, stream)
    step_ms = [s_.elapsed_time(e) for s_, e in zip(starts, ends)]
    ms = max_over_ranks(sum(step_ms) / len(step_ms), world, dev)

    # ---- end to end through the public API with host buffers (pinned), transfers timed.
    # Direct: one launch reads the descriptors from and writes the top-k into the pinned
    # (mapped) host buffers over the host link while it evaluates. Staged: tune_eval_host
    # copies chunks in and out on library streams while it evaluates (reported beside).
    host_d = torch.from_numpy(np.ascontiguousarray(descs).view(np.uint8).reshape(-1, 64)).pin_memory()
    host_i = torch.empty((n, k), dtype=torch.int32).pin_memory()
    host_c = torch.empty((n, k), dtype=torch.float32).pin_memory()
    # staged: one chunk per 250,000 kernels at least (a launch needs enough kernels per warp
    # to pay for its set-up), four chunks for larger inputs
    e2e_chunk = args.e2e_chunk or max(1, min(n, max(250_000, (n + 3) // 4)))

    def e2e_time(extra_flags):
        e_start = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        e_end = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        scratch = None
        for i in range(args.warmup + args.steps):
            flush.zero_()
            if i >= args.warmup:
                e_start[i - args.warmup].record(stream)
            scratch = T.tune_eval_host(a, ax, host_d, k, e2e_chunk, host_i, host_c, scratch=scratch,
                                       flags=sched | extra_flags, stream=stream)
            if i >= args.warmup:
                e_end[i - args.warmup].record(stream)
        torch.cuda.synchronize()
        T.tune_check(scratch, stream)
        # the host results are the device run's, bit for bit
        if not (torch.equal(host_i, topi.cpu()) and torch.equal(host_c, topc.cpu())):
            raise RuntimeError("tune_eval_host results differ from tune_eval")
        return max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(e_start, e_end)) / args.steps, world, dev)

    e2e_staged_ms = e2e_time(0)
    e2e_call = ("tune_eval_host with TUNE_HOST_DIRECT (one launch reads and writes the pinned host buffers "
                "over NVLink-C2C while it evaluates)")
    try:
        e2e_ms = e2e_time(T.native.TUNE_HOST_DIRECT)
    except T.native.TuneError as err:  # pinned memory not mapped on this system: staged copies only
        e2e_ms, e2e_call = e2e_staged_ms, f"tune_eval_host, staged ({err})"
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return None

    peaks, peak_kind = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * ISSUE_LANES_PER_SM_CLK * peaks["sm_max_mhz"] * 1e6 / 1e12  # Tinstr/s
    achieved = algo_instr / (ms * 1e-3) / 1e12
    achieved_12 = PER_POINT_EVAL_INSTR * points / (ms * 1e-3) / 1e12
    achieved_triple = triple_instr / (ms * 1e-3) / 1e12
    line = {
        "metric": METRIC,
        "value": world * points / (ms * 1e-3),
        "unit": "points/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32+f32",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {n} kernels x {points // n} points, top-{k}, sm_103 row",
                   "kernels_per_gpu": n, "points_per_gpu": points, "k": k,
                   "l2": "flushed between timed steps (256 MB write outside the timed events)",
                   "parallelism": f"replicas x{world} (kernel ranges)",
                   "schedule_flags": hex(sched),
                   "schedule": "forced" if args.flags else ("autotuned" if args.sched == "auto" else args.sched),
                   "cuda_graph": graph is not None},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tinstr/s",
                     "frac": achieved / peak, "traffic": recorded_traffic(args.workload),
                     "peak_source": f"{sms} SMs x 128 lanes x {peaks['sm_max_mhz']} MHz ({peak_kind})",
                     "instr_per_point": algo_instr / points,
                     "instr_definition": "2 per point (cost multiply, compare) + 5 per (T,U,C) triple",
                     "frac_12_per_point": achieved_12 / peak,
                     "issue_active_ncu": recorded_profile(args.workload).get("issue_active"),
                     "frac_8_per_triple": achieved_triple / peak},
        "e2e": {"value": world * points / (e2e_ms * 1e-3), "unit": "points/s",
                "h2d_bytes_per_step": n * 64, "d2h_bytes_per_step": n * k * 8,
                "ms_per_step": e2e_ms,
                "call": e2e_call,
                "staged_ms_per_step": e2e_staged_ms,
                "staged_call": f"tune_eval_host, {e2e_chunk} kernels per chunk copied in and out on library streams"},
        "clocks": clk.summary(),
        "gpu_launches": args.steps,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_sample)
    if not args.no_surrogate:
        line["surrogate"] = surrogate_section(args, dev, a, ax, peaks)
    return line


# FLOPs per sample and member of the surrogate MLP (128 -> 256 x 4 -> 1): forward
# 2 (128*256 + 3*256*256 + 256); training = forward + backward (2x forward).
MLP_FWD_FLOP = 2 * (128 * 256 + 3 * 256 * 256 + 256)
MLP_TRAIN_FLOP = 3 * MLP_FWD_FLOP


def surrogate_section(args, dev, a, ax, peaks):
    """Learned surrogate at bounded size: measured labels, training and inference
    throughput against the BF16 tensor peak, top-5 agreement with the measured best
    (held-out, fully timed spaces) and with the analytic model (dense points)."""
    import torch

    import paper_1701_08547_gb300 as T
    from paper_1701_08547_gb300 import surrogate_data as SD

    members = 5
    t0 = time.perf_counter()
    data = SD.build_set(a, ax, gen.descriptors(args.sur_descs, 4, "dense"), 64, 4, dev)
    gen_s = time.perf_counter() - t0
    epochs = 20
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sur, trace = SD.train(data, members=members, epochs=epochs, dev=dev)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    samples = data["n"] * epochs
    train_tflops = samples * members * MLP_TRAIN_FLOP / train_s / 1e12
    # inference over every point of dense kernels (features, ensemble, ranking, fallback)
    nk = args.sur_infer_kernels
    d = gen.descriptors(nk, 2, "dense")
    off = gen.point_offsets(d)
    dd = T.descs_to_device(d, dev)
    inf_sur = SD.Surrogate(members=members, batch=65536)
    inf_sur.set_params(sur.get(sur.GET_PARAMS))
    inf_sur.infer(a, ax, dd, off, 5, 0.1)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s_idx, _, fb = inf_sur.infer(a, ax, dd, off, 5, 0.1)
    torch.cuda.synchronize()
    infer_s = time.perf_counter() - t0
    pts = int(off[-1])
    infer_tflops = pts * members * MLP_FWD_FLOP / infer_s / 1e12
    a_idx, _ = T.tune_eval(a, ax, dd, 5)
    si, ai = s_idx.cpu().numpy(), a_idx.cpu().numpy()
    agree_overlap = float(np.mean([len(set(si[i]) & set(ai[i])) / 5 for i in range(nk)]))
    agree_hit = float(np.mean([ai[i, 0] in si[i] for i in range(nk)]))
    held_out = gen.descriptors(args.sur_eval, 40, "dense")
    ev = SD.evaluate(sur, a, ax, held_out, dev, k=5, thresh=0.1)
    ev_nofb = SD.evaluate(sur, a, ax, held_out, dev, k=5, thresh=1e30)
    pruning = SD.evaluate_pruning(a, ax, held_out, dev)
    from paper_1701_08547_gb300 import realkernels as RK

    t0 = time.perf_counter()
    real = RK.evaluate(a, ax, dev, n=args.real_n, surrogate=inf_sur)
    real["seconds"] = time.perf_counter() - t0
    real["matrix_order"] = args.real_n
    peak = peaks.get("bf16_tflops", 1900.0)
    return {
        "members": members,
        "labels": {"samples_measured": data["measured"], "samples_kept": data["n"], "seconds": gen_s,
                   "kind": "this GPU's median-of-3 times of emitted variants"},
        "train": {"samples_per_s": samples / train_s, "epochs": epochs, "seconds": train_s,
                  "tflops": train_tflops, "frac_bf16_peak": train_tflops / peak,
                  "final_mse_ln_us": float(trace[-1].mean())},
        "infer": {"points_per_s": pts / infer_s, "points": pts, "kernels": nk, "seconds": infer_s,
                  "tflops": infer_tflops, "frac_bf16_peak": infer_tflops / peak,
                  "fallback_rate": float(fb.float().mean().item())},
        "top5_vs_analytic": {"overlap": agree_overlap, "analytic_best_in_surrogate_top5": agree_hit},
        "top5_vs_measured_best": {"thresh_0.1": ev, "no_fallback": ev_nofb},
        "static_pruning_vs_measured_best": pruning,
        "real_kernels": real,
    }


def run_surfwd(args):
    """Surrogate forward throughput: 2^20 rows x 5 members, CUDA events, four paths:
    the fused persistent kernel in BF16 (headline) and with layers 2-4 on E4M3 codes,
    and the layer-by-layer tcgen05 and mma.sync GEMMs; against the measured BF16 tensor
    peak (FP8: twice that, the nominal FP8/BF16 ratio)."""
    import torch

    from paper_1701_08547_gb300 import build as B
    from paper_1701_08547_gb300.surrogate import Surrogate
    from workloads import mlp as L

    B.build()
    dev = torch.device("cuda", 0)
    sur = Surrogate(members=5, batch=65536)
    sur.set_params(L.init_params(5))
    n = args.kernels or (1 << 20)
    g = torch.Generator(device=dev)
    g.manual_seed(12)
    X = torch.randn(n, 128, generator=g, device=dev).to(torch.bfloat16)
    pred = torch.empty((5, n), device=dev)
    peaks, kind = measured_peaks()
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    out = {}
    paths = (("fused_bf16", Surrogate.FWD_FUSED_BF16, True), ("fused_fp8", Surrogate.FWD_FUSED_FP8, True),
             ("layered_tcgen05", Surrogate.FWD_LAYERED, True), ("layered_mma_sync", Surrogate.FWD_LAYERED, False))
    for name, mode, tc in paths:
        sur.set_forward_mode(mode)
        sur.use_tcgen05(tc)
        for _ in range(args.warmup):
            sur.forward(X, pred)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
        for i in range(args.steps):
            ev[2 * i].record()
            sur.forward(X, pred)
            ev[2 * i + 1].record()
        torch.cuda.synchronize()
        ms = sum(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(args.steps)) / args.steps
        tf = n * 5 * MLP_FWD_FLOP / (ms * 1e-3) / 1e12
        peak = 2 * bf16_peak if mode == Surrogate.FWD_FUSED_FP8 else bf16_peak
        out[name] = {"ms": ms, "rows_per_s": n / (ms * 1e-3), "tflops": tf, "peak_tflops": peak,
                     "frac": tf / peak}
    sur.check()
    head = out["fused_bf16"]
    return {"metric": "surrogate forward rows/sec (5 members)", "value": head["rows_per_s"],
            "unit": "rows/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": head["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"surfwd: {n} rows x 5 members, 128 -> 256 x 4 -> 1, fused BF16 kernel"},
            "roofline": {"bound": "tensor", "achieved": head["tflops"], "peak": bf16_peak, "unit": "TFLOP/s",
                         "frac": head["frac"], "traffic": None, "peak_source": kind},
            "paths": out}


def train_step_bytes(rows, members):
    """Algorithmic HBM bytes of one training step of the tcgen05 path (what the design must
    move): forward X read, G = gelu'(Z) (FP16) and H (BF16) of four layers written; head
    backward G4 and H4 read, dZ4 written; fused input gradients dZ4 and G3..G1 read, dZ3..dZ1
    written; weight gradients dZ of four layers and their inputs (H1..H3, X) read; Adam over
    the parameters (master, gradient and both moments read, master, moments and the BF16 copy
    written)."""
    from workloads import mlp as L

    act = rows * members * L.WID  # elements of one layer's activations
    x = rows * 128 * 2
    fwd = x + 4 * act * 2 + 4 * act * 2
    head = act * 2 + act * 2 + act * 2
    bwd = act * 2 + 3 * act * 2 + 3 * act * 2
    wgrad = 4 * act * 2 + 3 * act * 2 + x
    adam = members * L.P * (16 + 14)
    return fwd + head + bwd + wgrad + adam


def run_surtrain(args):
    """Surrogate training throughput: 5 members, 8,192-row batches of 65,536 synthetic rows
    (48 standard-normal features zero-padded to 128, standard-normal labels), one step =
    forward, MSE loss, backward and Adam for every member (tcgen05 path), CUDA events per
    step; against the HBM roofline of the step's algorithmic bytes (the step moves far more
    bytes than its 0.2 TFLOP needs tensor time for)."""
    import torch

    from paper_1701_08547_gb300 import build as B
    from paper_1701_08547_gb300.surrogate import Surrogate
    from workloads import mlp as L

    B.build()
    dev = torch.device("cuda", 0)
    members, batch = 5, 8192
    n = args.kernels or (1 << 16)
    n -= n % batch
    sur = Surrogate(members=members, batch=batch)
    sur.set_params(L.init_params(members))
    g = torch.Generator(device=dev)
    g.manual_seed(13)
    X = torch.zeros(n, 128, device=dev)
    X[:, :L.FEATURES] = torch.randn(n, L.FEATURES, generator=g, device=dev)
    X = X.to(torch.bfloat16)
    y = torch.randn(n, generator=g, device=dev)
    nb = n // batch

    def step(i):
        b = i % nb
        sur.train_step(X[b * batch:(b + 1) * batch], y[b * batch:(b + 1) * batch], apply_update=True)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
    for i in range(args.steps):
        ev[2 * i].record()
        step(args.warmup + i)
        ev[2 * i + 1].record()
    torch.cuda.synchronize()
    sur.check()
    ms = sum(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(args.steps)) / args.steps
    peaks, kind = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    bytes_step = train_step_bytes(batch, members)
    gbs = bytes_step / (ms * 1e-3) / 1e9
    tflops = batch * members * MLP_TRAIN_FLOP / (ms * 1e-3) / 1e12
    return {"metric": "surrogate training samples/sec (5 members)", "value": batch / (ms * 1e-3),
            "unit": "samples/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"surtrain: {n} rows in {batch}-row steps x {members} members, "
                                   "128 -> 256 x 4 -> 1, tcgen05 forward and backward, Adam"},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                         "traffic": None, "algorithmic_bytes_per_step": bytes_step, "peak_source": kind},
            "tflops": tflops, "frac_bf16_peak": tflops / peaks.get("bf16_tflops", 1900.0)}


def run_search(args):
    """Random and Nelder-Mead search per kernel with the static cost as the objective, over
    the full space and over the statically pruned one (T*): kernels searched per second and
    how often the search finds the exhaustive optimum (tune_eval's top-1)."""
    import torch

    import paper_1701_08547_gb300 as T
    from paper_1701_08547_gb300 import build as B

    B.build()
    dev = torch.device("cuda", 0)
    n, space, _, seed = WORKLOADS["search"]
    n = args.kernels or n
    a, ax = archs.arch("sm_103"), gen.axes()
    descs = gen.descriptors(n, seed, space)
    d_dev = T.descs_to_device(descs, dev)
    budget = args.budget
    ws = T.workspace(0, n, 1, dev)
    opt_i, opt_c = T.tune_eval(a, ax, d_dev, 1, workspace_buf=ws)
    keep = T.tune_suggest(a, ax, d_dev)["t_star"]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    peaks, kind = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * ISSUE_LANES_PER_SM_CLK * peaks["sm_max_mhz"] * 1e6 / 1e12
    out = {}
    for method in ("random", "nelder_mead"):
        for pruned in (False, True):
            kt = keep if pruned else None
            for _ in range(args.warmup):
                T.tune_search(a, ax, d_dev, method, budget, 1, t_keep=kt, workspace_buf=ws)
            torch.cuda.synchronize()
            times, evals = [], 0
            for i in range(args.steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                bi, bc, ev = T.tune_search(a, ax, d_dev, method, budget, 100 + i, t_keep=kt, workspace_buf=ws)
                e1.record()
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
                evals = int(ev.sum().item())
            T.tune_check(ws)
            ms = sum(times) / len(times)
            valid = torch.isfinite(opt_c[:, 0])
            hit = float(((bi == opt_i[:, 0]) & valid).sum().item() / max(1, int(valid.sum().item())))
            ratio = (bc / opt_c[:, 0])[valid & torch.isfinite(bc)]
            achieved = UNHOISTED_INSTR_PER_POINT * evals / (ms * 1e-3) / 1e12
            out[f"{method}{'_pruned' if pruned else ''}"] = {
                "ms": ms, "kernels_per_s": n / (ms * 1e-3), "evaluations_per_s": evals / (ms * 1e-3),
                "evals_per_kernel": evals / n, "hit_exhaustive_top1": hit,
                "median_cost_ratio": float(ratio.median().item()) if ratio.numel() else None,
                "p90_cost_ratio": float(ratio.quantile(0.9).item()) if ratio.numel() else None,
                "frac_issue_at_60_per_eval": achieved / peak}
    head = out["nelder_mead"]
    return {"metric": "kernels searched/sec (Nelder-Mead, static cost objective)", "value": head["kernels_per_s"],
            "unit": "kernels/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32+f32",
            "data": "synthetic",
            "config": {"workload": f"search: {n} dense kernels x 16384 points, budget {budget} evaluations per kernel",
                       "l2": "flushed between timed steps"},
            "roofline": {"bound": "alu", "achieved": UNHOISTED_INSTR_PER_POINT * head["evaluations_per_s"] / 1e12,
                         "peak": peak, "unit": "Tinstr/s", "frac": head["frac_issue_at_60_per_eval"],
                         "traffic": None, "instr_per_point": UNHOISTED_INSTR_PER_POINT,
                         "peak_source": f"{sms} SMs x 128 lanes x {peaks['sm_max_mhz']} MHz ({kind})"},
            "methods": out, "gpu_launches": args.steps}


def run_topk(args):
    """Segmented top-k over external scores: 100,000 segments x 16,384 float32
    scores (the dense workload's point count), top-10; HBM-bound."""
    import torch

    import paper_1701_08547_gb300 as T
    from paper_1701_08547_gb300 import build as B

    rank, world, local = dist_env()
    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n_seg = args.kernels or 100_000
    seg, k = 16384, 10
    total = n_seg * seg
    g = torch.Generator(device=dev)
    g.manual_seed(11)  # seeded log-uniform scores in [1, 1e6], made on the device (6.6 GB)
    scores = torch.rand(total, generator=g, device=dev, dtype=torch.float32)
    scores.mul_(float(np.log(1e6))).exp_()
    off = torch.arange(0, total + 1, seg, dtype=torch.int64, device=dev)
    ws = T.workspace(1, n_seg, k, dev)
    oi = torch.empty((n_seg, k), dtype=torch.int32, device=dev)
    ov = torch.empty((n_seg, k), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        T.tune_topk(scores, off, k, oi, ov, ws, stream)
    torch.cuda.synchronize()
    st = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    en = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    uuid = f"GPU-{uuid}" if uuid is not None and not str(uuid).startswith("GPU-") else uuid
    with ClockSampler(uuid, local) as clk:
        for i in range(args.steps):
            st[i].record(stream)
            T.tune_topk(scores, off, k, oi, ov, ws, stream)
            en[i].record(stream)
        torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in zip(st, en)) / args.steps
    peaks, kind = measured_peaks()
    nbytes = total * 4 + (n_seg + 1) * 8 + n_seg * k * 8
    gbs = nbytes / (ms * 1e-3) / 1e9
    return {"metric": "segmented top-k scores/sec", "value": total / (ms * 1e-3), "unit": "scores/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"topk: {n_seg} segments x {seg} scores, top-{k}",
                       "l2": f"input {nbytes / 1e9:.1f} GB, larger than L2"},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks.get("hbm_gbs", 6800.0),
                         "unit": "GB/s", "frac": gbs / peaks.get("hbm_gbs", 6800.0), "traffic": None,
                         "peak_source": kind},
            "clocks": clk.summary(), "gpu_launches": args.steps}


def cpu_baseline(workload, sample):
    from oracle import oracle as O

    n, space, k, seed = WORKLOADS[workload]
    sample = min(sample, n)
    descs = gen.descriptors(sample, seed, space)
    a, ax = archs.arch("sm_103"), gen.axes()
    threads = O.threads_available()
    O.evaluate(a, ax, descs[:8], k, nthreads=threads)  # load + warm
    t0 = time.perf_counter()
    O.evaluate(a, ax, descs, k, nthreads=threads)
    dt = time.perf_counter() - t0
    pts = int(gen.space_sizes(descs).sum())
    return {"value": pts / dt, "unit": "points/s", "cores": threads, "kind": "oracle",
            "sample": f"first {sample} kernels of the {workload} workload ({pts} points), "
                      f"{dt:.2f} s wall on {threads} threads"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    from oracle import oracle as O

    n, space, k, seed = WORKLOADS[args.workload]
    a, ax = archs.arch("sm_103"), gen.axes()
    sample = min(args.cpu_sample, n)
    descs = gen.descriptors(sample, seed, space)
    pts = int(gen.space_sizes(descs).sum())
    threads = O.threads_available()
    for _ in range(args.warmup):
        O.evaluate(a, ax, descs[: max(1, sample // 8)], k, nthreads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.evaluate(a, ax, descs, k, nthreads=threads)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = pts / (ms * 1e-3)
    sample_desc = f"first {sample} kernels of the {args.workload} workload ({pts} points) per step"
    return {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "points/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int64+f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {n} kernels x {pts // sample} points, top-{k}, sm_103 row",
                   "kernels_per_gpu": n, "k": k},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": threads, "kind": "oracle",
                         "sample": sample_desc},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=list(WORKLOADS), default="dense")
    p.add_argument("--cpu-sample", type=int, default=16000)
    p.add_argument("--kernels", type=int, default=0, help="override the kernel count (small ncu cases)")
    p.add_argument("--sched", choices=["auto", "warp", "thread"], default="auto")
    p.add_argument("--no-graph", action="store_true", help="plain launches instead of graph replays")
    p.add_argument("--flags", default="", help="tune_eval schedule flags in hex (skips the autotuner)")
    p.add_argument("--no-surrogate", action="store_true", help="skip the learned-surrogate section")
    p.add_argument("--sur-descs", type=int, default=1000, help="descriptors for surrogate labels (x64 points)")
    p.add_argument("--sur-infer-kernels", type=int, default=500, help="dense kernels scored by the ensemble")
    p.add_argument("--sur-eval", type=int, default=150, help="held-out kernels with fully timed spaces")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--budget", type=int, default=128, help="search workload: evaluations per kernel")
    p.add_argument("--real-n", type=int, default=4096, help="matrix order of the real-kernel variants")
    p.add_argument("--e2e-chunk", type=int, default=0, help="kernels per host-transfer chunk (0: chosen)")
    args = p.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        line = run_reference(args)
    elif args.workload == "topk":
        line = run_topk(args)
    elif args.workload == "surfwd":
        line = run_surfwd(args)
    elif args.workload == "surtrain":
        line = run_surtrain(args)
    elif args.workload == "search":
        line = run_search(args)
    else:
        line = run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
