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
    "mix": (12, "dense", 0, 67),
    "emit": (100_000, "dense", 10, 2),
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
    """Hash of the evaluation kernel's sources (tune_eval.cu and the arithmetic it includes)."""
    h = hashlib.sha256()
    for name in ("tune_eval.cu", "eval_common.cuh"):
        with open(os.path.join(ROOT, "paper_1701_08547_gb300", "csrc", name), "rb") as f:
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


def _uuid(dev):
    import torch

    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    return f"GPU-{uuid}" if uuid is not None and not str(uuid).startswith("GPU-") else uuid


def issue_peak(dev):
    """(Tinstr/s, description): SMs x 4 schedulers x 32 lanes x the measured maximum SM clock."""
    import torch

    peaks, kind = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return (sms * ISSUE_LANES_PER_SM_CLK * peaks["sm_max_mhz"] * 1e6 / 1e12,
            f"{sms} SMs x 128 lanes x {peaks['sm_max_mhz']} MHz ({kind})")


def eval_workload(args, name, dev, stream, flush, rank, world, local, n=None, with_e2e=True, with_clocks=False):
    """One tune_eval workload timed the way the headline is: schedule from the library's
    autotuner (untimed), one step captured in a CUDA graph, W warm-up replays, K timed
    replays with an L2 flush before each (outside the events), max over ranks; then the
    end-to-end call from and to pinned host buffers (transfers inside the timed region).
    Returns the measurement dict and the device results of the last step."""
    import torch

    import paper_1701_08547_gb300 as T

    n0, space, k, seed = WORKLOADS[name]
    n = n or n0
    a, ax = archs.arch("sm_103"), gen.axes()
    descs = shard(n, seed, space, rank)
    points = int(gen.space_sizes(descs).sum())
    d_dev = T.descs_to_device(descs, dev)
    ws = T.workspace(0, n, k, dev)
    topi = torch.empty((n, k), dtype=torch.int32, device=dev)
    topc = torch.empty((n, k), dtype=torch.float32, device=dev)

    if args.flags:
        sched, tuned_ms = int(args.flags, 16), None
    elif args.sched == "auto":
        sched, tuned_ms, _, _ = T.tune_autotune(a, ax, d_dev, k, reps=3, topk_idx=topi, topk_cost=topc,
                                                workspace_buf=ws, stream=stream)
    else:
        sched, tuned_ms = {"warp": 0x10, "thread": 0x20}[args.sched], None

    def step():
        T.tune_eval(a, ax, d_dev, k, flags=sched, topk_idx=topi, topk_cost=topc, workspace_buf=ws, stream=stream)

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
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(_uuid(dev), local) as clk:
        for i in range(args.steps):
            flush.zero_()  # L2 flush between timed steps (outside the event pair)
            starts[i].record(stream)
            run_step()
            ends[i].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    T.tune_check(ws, stream)
    ms = max_over_ranks(sum(s_.elapsed_time(e) for s_, e in zip(starts, ends)) / args.steps, world, dev)
    out = {"descs": descs, "n": n, "k": k, "points": points, "ms": ms, "sched": sched, "tuned_ms": tuned_ms,
           "graph": graph is not None, "clocks": clk.summary(), "topi": topi, "topc": topc}
    if with_e2e:
        out["e2e"] = e2e_eval(args, descs, n, k, points, sched, dev, stream, flush, world, topi, topc)
    return out


def e2e_eval(args, descs, n, k, points, sched, dev, stream, flush, world, topi, topc):
    """End to end through the public API with host buffers (pinned), transfers timed. Direct:
    one launch reads the descriptors from and writes the top-k into the pinned (mapped) host
    buffers over the host link while it evaluates. Staged: tune_eval_host copies chunks in and
    out on library streams while it evaluates (reported beside). Results are checked equal to
    the device run's."""
    import torch

    import paper_1701_08547_gb300 as T

    a, ax = archs.arch("sm_103"), gen.axes()
    host_d = torch.from_numpy(np.ascontiguousarray(descs).view(np.uint8).reshape(-1, 64)).pin_memory()
    host_i = torch.empty((n, k), dtype=torch.int32).pin_memory()
    host_c = torch.empty((n, k), dtype=torch.float32).pin_memory()
    # staged: one chunk per 250,000 kernels at least (a launch needs enough kernels per warp
    # to pay for its set-up), four chunks for larger inputs
    chunk = args.e2e_chunk or max(1, min(n, max(250_000, (n + 3) // 4)))

    def timed(extra_flags):
        e_start = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        e_end = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        scratch = None
        for i in range(args.warmup + args.steps):
            flush.zero_()
            if i >= args.warmup:
                e_start[i - args.warmup].record(stream)
            scratch = T.tune_eval_host(a, ax, host_d, k, chunk, host_i, host_c, scratch=scratch,
                                       flags=sched | extra_flags, stream=stream)
            if i >= args.warmup:
                e_end[i - args.warmup].record(stream)
        torch.cuda.synchronize()
        T.tune_check(scratch, stream)
        if not (torch.equal(host_i, topi.cpu()) and torch.equal(host_c, topc.cpu())):
            raise RuntimeError("tune_eval_host results differ from tune_eval")
        return max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(e_start, e_end)) / args.steps, world, dev)

    staged_ms = timed(0)
    call = ("tune_eval_host with TUNE_HOST_DIRECT (one launch reads and writes the pinned host buffers "
            "over NVLink-C2C while it evaluates)")
    try:
        ms = timed(T.native.TUNE_HOST_DIRECT)
    except T.native.TuneError as err:  # pinned memory not mapped on this system: staged copies only
        ms, call = staged_ms, f"tune_eval_host, staged ({err})"
    return {"value": world * points / (ms * 1e-3), "unit": "points/s", "h2d_bytes_per_step": n * 64,
            "d2h_bytes_per_step": n * k * 8, "ms_per_step": ms, "call": call, "staged_ms_per_step": staged_ms,
            "staged_call": f"tune_eval_host, {chunk} kernels per chunk copied in and out on library streams"}


def eval_roofline(r, dev, workload):
    """Issue roofline of one tune_eval measurement. Algorithmic figure: the scope table's 12
    thread-instructions per point of a per-point evaluation after the per-kernel hoists. The
    kernel ranks exactly without pricing most points (a (T,U,C) triple's cheapest point bounds
    all of its grid sizes; only candidate triples are walked), so it can exceed that figure's
    issue bound; the executed instructions per point (ncu) and the issue-slot use are given
    beside it."""
    peak, peak_source = issue_peak(dev)
    ms, points = r["ms"], r["points"]
    achieved_12 = PER_POINT_EVAL_INSTR * points / (ms * 1e-3) / 1e12
    prof = recorded_profile(workload)
    out = {"bound": "alu", "achieved": achieved_12, "peak": peak, "unit": "Tinstr/s", "frac": achieved_12 / peak,
           "traffic": prof.get("bytes_per_launch"), "peak_source": peak_source,
           "instr_per_point": PER_POINT_EVAL_INSTR,
           "instr_definition": ("12 thread-instructions per point of a per-point evaluation (scope table); the "
                                "kernel is an exact top-k by (T,U,C)-triple bounds that prices only candidate "
                                "triples' points, so frac > 1 means it beats per-point evaluation"),
           "executed_instr_per_point_ncu": prof.get("thread_instr_per_point"),
           "issue_active_ncu": prof.get("issue_active"),
           "frac_2_per_point_5_per_triple": algorithmic_instructions(r["descs"], None) / (ms * 1e-3) / 1e12 / peak}
    return out


def eval_line(args, name, r, dev, world, cpu=True):
    """The JSON object of one tune_eval workload (headline or sub-object)."""
    n, k, points = r["n"], r["k"], r["points"]
    line = {
        "metric": METRIC,
        "value": world * points / (r["ms"] * 1e-3),
        "unit": "points/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": r["ms"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32+f32",
        "data": "synthetic",
        "config": {"workload": f"{name}: {n} kernels x {points / n:.0f} points (mean), top-{k}, sm_103 row",
                   "kernels_per_gpu": n, "points_per_gpu": points, "k": k,
                   "l2": "flushed between timed steps (256 MB write outside the timed events)",
                   "parallelism": f"replicas x{world} (kernel ranges)",
                   "schedule_flags": hex(r["sched"]),
                   "schedule": "forced" if args.flags else ("autotuned" if args.sched == "auto" else args.sched),
                   "cuda_graph": r["graph"]},
        "roofline": eval_roofline(r, dev, name),
        "clocks": r["clocks"],
        "gpu_launches": args.steps,
    }
    if "e2e" in r:
        line["e2e"] = r["e2e"]
    if cpu and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(name, CPU_SAMPLE.get(name, args.cpu_sample))
    return line


def emit_points(args, dev, stream, flush, world):
    """Every point priced and written (TUNE_EMIT_POINTS): B*, W* (int32) and the FP32 cost of
    each of the dense workload's points, 12 bytes per point, plus the top-k. HBM-bound:
    algorithmic bytes = 12 per point written + the 64-byte descriptor and the 8-byte offset
    read + 8 k bytes of top-k written per kernel."""
    import torch

    import paper_1701_08547_gb300 as T

    n0, space, k, seed = WORKLOADS["dense"]
    n = args.emit_kernels or n0
    a, ax = archs.arch("sm_103"), gen.axes()
    descs = gen.descriptors(n, seed, space)
    off = gen.point_offsets(descs)
    points = int(off[-1])
    d_dev = T.descs_to_device(descs, dev)
    po = torch.from_numpy(off).to(dev)
    pb = torch.empty(points, dtype=torch.int32, device=dev)
    pw = torch.empty(points, dtype=torch.int32, device=dev)
    pc = torch.empty(points, dtype=torch.float32, device=dev)
    ws = T.workspace(0, n, k, dev)
    topi = torch.empty((n, k), dtype=torch.int32, device=dev)
    topc = torch.empty((n, k), dtype=torch.float32, device=dev)

    def step():
        T.tune_eval(a, ax, d_dev, k, flags=T.TUNE_EMIT_POINTS, topk_idx=topi, topk_cost=topc, pt_blocks=pb,
                    pt_warps=pw, pt_cost=pc, pt_offsets=po, workspace_buf=ws, stream=stream)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    T.tune_check(ws, stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
    for i in range(args.steps):
        flush.zero_()
        ev[2 * i].record(stream)
        step()
        ev[2 * i + 1].record(stream)
    torch.cuda.synchronize()
    T.tune_check(ws, stream)
    ms = max_over_ranks(sum(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(args.steps)) / args.steps,
                        world, dev)
    # the emitted points agree with the oracle on sampled kernels (bit for bit)
    from oracle import oracle as O

    pick = np.random.default_rng(7).choice(n, 16, replace=False)
    o = O.evaluate(a, ax, descs[pick], k, emit=True, offsets=gen.point_offsets(descs[pick]))
    for j, i in enumerate(pick):
        got = pc[int(off[i]):int(off[i + 1])].cpu().numpy()
        want = o["cost32"][j * 16384:(j + 1) * 16384]
        if not np.array_equal(got.view(np.uint32), want.view(np.uint32)):
            raise RuntimeError("emitted per-point costs differ from the oracle")
    peaks, kind = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    nbytes = 12 * points + 72 * n + 8 + 8 * k * n
    gbs = nbytes / (ms * 1e-3) / 1e9
    prof = recorded_profile("emit")
    line = {"metric": "tuning points priced and written/sec (B*, W*, cost of every point)",
            "value": world * points / (ms * 1e-3), "unit": "points/s", "ms_per_step": ms, "steps": args.steps,
            "warmup": args.warmup,
            "config": {"workload": f"emit: dense {n} kernels x 16384 points, every point's B*, W* and FP32 cost "
                                   f"written ({12 * points / 1e9:.1f} GB), top-{k}",
                       "l2": "outputs far larger than L2; 256 MB flush between timed steps"},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                         "traffic": prof.get("bytes_per_launch_scaled"), "algorithmic_bytes": nbytes,
                         "peak_source": kind},
            "gpu_launches": args.steps, "check": "16 sampled kernels' per-point costs equal the oracle's bit for bit"}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline("dense", 4000, emit=True)
    return line


def run_emit(args):
    """The every-point path alone (TUNE_EMIT_POINTS on the dense workload; --kernels sets a
    smaller case for profiling)."""
    import torch

    from paper_1701_08547_gb300 import build as B

    B.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    a2 = argparse.Namespace(**vars(args))
    a2.emit_kernels = args.kernels or 0
    return emit_points(a2, dev, stream, flush, 1)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1701_08547_gb300 import build as B

    rank, world, local = dist_env()
    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)

    head = eval_workload(args, args.workload, dev, stream, flush, rank, world, local, n=args.kernels or None)
    subs = {}
    if not args.headline_only and args.workload == "dense":
        for name in ("dense128", "uneven"):
            subs[name] = eval_workload(args, name, dev, stream, flush, rank, world, local)
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return None
    line = eval_line(args, args.workload, head, dev, world)
    if not args.headline_only and args.workload == "dense":
        line["configs"] = {"C1_dense128": eval_line(args, "dense128", subs["dense128"], dev, world),
                           "C3_uneven": eval_line(args, "uneven", subs["uneven"], dev, world)}
        line["configs"]["C2_emit_every_point"] = emit_points(args, dev, stream, flush, world)
    if not args.no_surrogate:
        peaks, _ = measured_peaks()
        line["surrogate"] = surrogate_section(args, dev, archs.arch("sm_103"), gen.axes(), peaks, stream)
    if not args.headline_only and args.workload == "dense":
        line["other_kernels"] = other_workloads(args)
    return line


# Algorithmic FLOPs per sample and member of the surrogate MLP (48 features -> 256 x 4 -> 1):
# forward 2 (48*256 + 3*256*256 + 256) = 418,304 (the zero padding of the inputs is not
# counted); training = forward + backward (2x forward).
MLP_FWD_FLOP = 2 * (48 * 256 + 3 * 256 * 256 + 256)
MLP_TRAIN_FLOP = 3 * MLP_FWD_FLOP


def surrogate_section(args, dev, a, ax, peaks, stream):
    """The learned path at the scope table's configurations 4 and 5: labels measured on this
    GPU (s1), training throughput (C4), inference over every point of the dense workload in
    BF16 and FP8 with the analytic fallback (C5), and the top-5 agreement with the measured
    best (held-out, fully timed spaces) and with the analytic model."""
    import torch

    import paper_1701_08547_gb300 as T
    from paper_1701_08547_gb300 import surrogate_data as SD
    from workloads import mlp as L

    members = 5
    t0 = time.perf_counter()
    data = SD.build_set(a, ax, gen.descriptors(args.sur_descs, 4, "dense"), 64, 4, dev)
    gen_s = time.perf_counter() - t0
    out = {"members": members,
           "labels": {"samples_measured": data["measured"], "samples_kept": data["n"], "seconds": gen_s,
                      "kind": "this GPU's median-of-3 times of emitted variants, per unit of per-thread work"}}
    out["C4_train"], sur = train_section(args, dev, data, members, peaks, stream)

    # ---- C5: every point of the dense workload scored by the ensemble, BF16 and FP8
    nk = args.sur_infer_kernels
    d = gen.descriptors(nk, 2, "dense")
    off = gen.point_offsets(d)
    pts = int(off[-1])
    inf_sur = SD.Surrogate(members=members, batch=65536)
    inf_sur.set_params(sur.get(sur.GET_PARAMS))
    host_d = torch.from_numpy(np.ascontiguousarray(d).view(np.uint8).reshape(-1, 64)).pin_memory()
    dd = torch.empty_like(host_d, device=dev)
    dd.copy_(host_d)
    a_idx, _ = T.tune_eval(a, ax, dd, 5, stream=stream)
    ai = a_idx.cpu().numpy()
    warm = gen.descriptors(max(1, nk // 16), 2, "dense")
    warm_d = T.descs_to_device(warm, dev)
    timed = SD.timed_spaces(ax, gen.descriptors(args.sur_eval, 40, "dense"))
    c5 = {}
    sustained = peaks.get("bf16_tflops_sustained", 1700.0)
    for name, mode in (("bf16", SD.Surrogate.FWD_FUSED_BF16), ("fp8", SD.Surrogate.FWD_FUSED_FP8)):
        inf_sur.set_forward_mode(mode)
        for _ in range(args.warmup):
            inf_sur.infer(a, ax, warm_d, gen.point_offsets(warm), 5, 0.1, stream=stream)
        torch.cuda.synchronize()
        hi = torch.empty((nk, 5), dtype=torch.int32).pin_memory()
        hf = torch.empty(nk, dtype=torch.uint8).pin_memory()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        with ClockSampler(_uuid(dev), dev.index or 0) as clk:
            ev[0].record(stream)
            with torch.cuda.stream(stream):
                dd.copy_(host_d, non_blocking=True)
            ev[1].record(stream)
            s_idx, _, fb = inf_sur.infer(a, ax, dd, off, 5, 0.1, stream=stream)
            ev[2].record(stream)
            with torch.cuda.stream(stream):
                hi.copy_(s_idx, non_blocking=True)
                hf.copy_(fb, non_blocking=True)
            ev[3].record(stream)
            torch.cuda.synchronize()
        ms = ev[1].elapsed_time(ev[2])
        e2e_ms = ev[0].elapsed_time(ev[3])
        inf_sur.check()
        si, fbn = hi.numpy(), hf.numpy()
        tf = pts * members * MLP_FWD_FLOP / (ms * 1e-3) / 1e12
        peak = sustained * (2 if name == "fp8" else 1)
        ev_fb = SD.evaluate(inf_sur, a, ax, None, dev, k=5, thresh=0.1, timed=timed)
        ev_nofb = SD.evaluate(inf_sur, a, ax, None, dev, k=5, thresh=1e30, timed=timed)
        c5[name] = {
            "metric": "tuning points scored by the surrogate ensemble/sec + top-k (fallback at std/mean 0.1)",
            "value": pts / (ms * 1e-3), "unit": "points/s", "ms_per_step": ms, "steps": 1,
            "warmup": args.warmup, "dtype": "bf16" if name == "bf16" else "e4m3 layers 2-4, bf16 layer 1",
            "config": {"workload": f"C5: dense {nk} kernels x 16384 points ({pts} points), 5 members, top-5, "
                                   "fallback per kernel where a pick's std/mean > 0.1",
                       "warmup": f"{args.warmup} passes over {len(warm)} kernels"},
            "roofline": {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                         "traffic": None,
                         "flop_definition": "418,304 FLOP per point and member (48 -> 256 x 4 -> 1 forward); "
                                            "the whole call (features, ensemble, ranking, fallback) is timed",
                         "peak_source": "measured sustained BF16 GEMM" + (" x 2 (nominal FP8/BF16)" if name == "fp8"
                                                                           else "")},
            "e2e": {"value": pts / (e2e_ms * 1e-3), "unit": "points/s", "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": nk * 64, "d2h_bytes_per_step": nk * (5 * 4 + 1),
                    "call": "descriptors copied from pinned host memory, surrogate_infer, top-5 and fallback "
                            "flags copied back, all inside the timed region"},
            "fallback_rate": float(fbn.mean()),
            "top5_vs_analytic": {"overlap": float(np.mean([len(set(si[i]) & set(ai[i])) / 5 for i in range(nk)])),
                                 "analytic_best_in_top5": float(np.mean([ai[i, 0] in si[i] for i in range(nk)]))},
            "top5_vs_measured_best": {"thresh_0.1": ev_fb, "no_fallback": ev_nofb},
            "clocks": clk.summary(),
            # the analytic top-k (1), then per chunk of 64 kernels (2^20 points): offsets, features,
            # the fused ensemble forward, scores, segmented top-k, fallback (6)
            "gpu_launches": 1 + 6 * ((nk + 63) // 64),
        }
        if not args.no_cpu_baseline and name == "bf16":
            c5[name]["cpu_baseline"] = surrogate_cpu_baseline(a, ax, inf_sur, members)
    out["C5_infer"] = c5
    out["static_pruning_vs_measured_best"] = SD.evaluate_pruning(a, ax, gen.descriptors(args.sur_eval, 40, "dense"),
                                                                 dev)
    from paper_1701_08547_gb300 import realkernels as RK

    inf_sur.set_forward_mode(SD.Surrogate.FWD_FUSED_BF16)
    t0 = time.perf_counter()
    real = RK.evaluate(a, ax, dev, n=args.real_n, surrogate=inf_sur)
    real["seconds"] = time.perf_counter() - t0
    real["matrix_order"] = args.real_n
    out["real_kernels"] = real
    return out


def train_section(args, dev, data, members, peaks, stream):
    """C4: the library's training (surrogate_train: BF16 tcgen05 forward and backward, Adam) on
    the measured labels, timed with CUDA events; and end to end with the features, labels and
    epoch orders copied from pinned host memory and the loss trace copied back."""
    import torch

    from paper_1701_08547_gb300 import surrogate_data as SD
    from workloads import mlp as L

    epochs = args.sur_epochs
    n = data["n"]
    batch = 8192
    rng = np.random.default_rng(5)
    order_h = torch.from_numpy(np.concatenate([rng.permutation(n) for _ in range(epochs)]).astype(np.int32))
    steps = (n + batch - 1) // batch
    feats_h = data["feats"].cpu().pin_memory()
    labels_h = data["labels"].cpu().pin_memory()
    order_h = order_h.pin_memory()

    def run(e2e):
        sur = SD.Surrogate(members=members, batch=batch)
        sur.set_params(L.init_params(members, [5 + m for m in range(members)]))
        trace = torch.zeros(epochs * steps * members, dtype=torch.float32, device=dev)
        trace_h = torch.empty(trace.numel(), dtype=torch.float32).pin_memory()
        f, lab, o = data["feats"], data["labels"], order_h.to(dev)
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record(stream)
        with torch.cuda.stream(stream):
            if e2e:
                f = feats_h.to(dev, non_blocking=True)
                lab = labels_h.to(dev, non_blocking=True)
                o = order_h.to(dev, non_blocking=True)
            sur.train(f, lab, o, epochs, trace, stream=stream)
            if e2e:
                trace_h.copy_(trace, non_blocking=True)
        e[1].record(stream)
        torch.cuda.synchronize()
        sur.check()
        return sur, e[0].elapsed_time(e[1]), trace.cpu().numpy().reshape(epochs, steps, members)

    run(False)  # warm-up (module load, first launches)
    sur, ms, trace = run(False)
    _, e2e_ms, _ = run(True)
    samples = n * epochs
    step_ms = ms / (epochs * steps)
    hbm = peaks.get("hbm_gbs", 6800.0)
    gbs = train_step_bytes(batch, members) / (step_ms * 1e-3) / 1e9
    tf = samples * members * MLP_TRAIN_FLOP / (ms * 1e-3) / 1e12
    line = {"metric": "surrogate training samples/sec (5 members)", "value": samples / (ms * 1e-3),
            "unit": "samples/s", "ms_per_step": step_ms, "steps": epochs * steps, "warmup": 1,
            "dtype": "bf16 (FP32 accumulation and master weights)",
            "config": {"workload": f"C4: {n} measured labels x {epochs} epochs in {batch}-row steps, {members} "
                                   "members, 48 -> 256 x 4 -> 1, Adam",
                       "labels": "64 K measured here instead of 20 M (timing 20 M variants takes hours); the "
                                 "step time does not depend on the label count"},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                         "traffic": None, "algorithmic_bytes_per_step": train_step_bytes(batch, members),
                         "tensor_tflops": tf, "tensor_frac_sustained": tf / peaks.get("bf16_tflops_sustained", 1700.0),
                         "flop_definition": "3 x 418,304 FLOP per sample and member"},
            "e2e": {"value": samples / (e2e_ms * 1e-3), "unit": "samples/s", "ms": e2e_ms,
                    "h2d_bytes_per_step": (feats_h.numel() * 2 + labels_h.numel() * 4 + order_h.numel() * 4) /
                    (epochs * steps),
                    "d2h_bytes_per_step": 4 * members,
                    "call": "features, labels and epoch orders copied from pinned host memory, surrogate_train, "
                            "loss trace copied back, all inside the timed region"},
            "final_mse": float(trace[-1].mean()),
            # per step: batch gather, fused forward, loss (2), head backward (2), weight transpose and
            # fused input-gradient chain (2), four weight-gradient passes with their reductions (8), Adam
            "gpu_launches": 17 * epochs * steps}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = train_cpu_baseline(members)
    return line, sur


def train_cpu_baseline(members, rows=2048):
    """The FP64 oracle's forward + backward (+ Adam) on one batch, per sample and member."""
    from oracle import surrogate_oracle as S
    from workloads import mlp as L

    rng = np.random.default_rng(0)
    X = np.zeros((rows, L.IN))
    X[:, :L.FEATURES] = rng.standard_normal((rows, L.FEATURES))
    X = S.bf16(X)
    t = rng.standard_normal(rows)
    flat = L.init_params(members)
    t0 = time.perf_counter()
    for p in L.unpack(flat, members):
        S.loss_and_grads(p, X, t, bf=True)
    dt = time.perf_counter() - t0
    return {"value": rows / dt, "unit": "samples/s", "cores": os.cpu_count() or 1, "kind": "oracle",
            "sample": f"one {rows}-row batch, {members} members, FP64 forward + backward (numpy), {dt:.2f} s"}


def surrogate_cpu_baseline(a, ax, sur, members, kernels=8, per_kernel=1000):
    """The oracle's inference (features in FP64, FP64 forward of every member on the BF16
    weights, mean and spread) on `per_kernel` points of each of `kernels` dense kernels."""
    from oracle import oracle as O
    from oracle import surrogate_oracle as S
    from workloads import mlp as L

    d = gen.descriptors(kernels, 2, "dense")
    flat = sur.get(sur.GET_PARAMS)
    rng = np.random.default_rng(3)
    t0 = time.perf_counter()
    for i in range(kernels):
        X = np.zeros((per_kernel, L.IN))
        for r, p in enumerate(rng.integers(0, 16384, per_kernel)):
            X[r, :48] = O.features(a, d[i], *O.decode_point(d[i], ax, p))
        X = S.bf16(X)
        preds = np.stack([S.forward(prm, X, bf=True)[0] for prm in L.unpack(flat, members)])
        r = np.exp(preds)
        _ = r.std(0) / r.mean(0)
    dt = time.perf_counter() - t0
    n = kernels * per_kernel
    return {"value": n / dt, "unit": "points/s", "cores": os.cpu_count() or 1, "kind": "oracle",
            "sample": f"{per_kernel} random points of each of {kernels} dense kernels ({n} points), {dt:.2f} s"}


def other_workloads(args):
    """The remaining kernels of the path, each timed alone (their own JSON objects): the
    segmented top-k (a8), the fused ensemble forward (s3) in BF16 and FP8, one training step
    (s4), and the search drivers."""
    import copy

    out = {}
    for name, fn in (("topk", run_topk), ("surfwd", run_surfwd), ("surtrain", run_surtrain),
                     ("search", run_search)):
        a2 = copy.copy(args)
        a2.kernels = 0
        a2.workload = name
        r = fn(a2)
        for key in ("n_gpus", "higher_is_better", "scaling", "vs_baseline", "data"):
            r.pop(key, None)
        out[name] = r
    return out


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
    X = torch.zeros(n, L.IN, device=dev)  # 48 standard-normal features, zero padding as tune_features writes
    X[:, :L.FEATURES] = torch.randn(n, L.FEATURES, generator=g, device=dev)
    X = X.to(torch.bfloat16)
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
            "config": {"workload": f"surfwd: {n} rows x 5 members, 64 -> 256 x 4 -> 1, fused BF16 kernel"},
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
    x = rows * L.IN * 2
    fwd = x + 4 * act * 2 + 4 * act * 2
    head = act * 2 + act * 2 + act * 2
    bwd = act * 2 + 3 * act * 2 + 3 * act * 2
    wgrad = 4 * act * 2 + 3 * act * 2 + x
    adam = members * L.P * (16 + 14)
    return fwd + head + bwd + wgrad + adam


def run_surtrain(args):
    """Surrogate training throughput: 5 members, 8,192-row batches of 65,536 synthetic rows
    (48 standard-normal features zero-padded to 64, standard-normal labels), one step =
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
    X = torch.zeros(n, L.IN, device=dev)
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
                                   "64 -> 256 x 4 -> 1, tcgen05 forward and backward, Adam"},
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


MIX_POINT = (256, 64, 2, 100)  # (T, G, U, carveout %) at which the mix samples are launched


def run_mix(args):
    """Static versus dynamic instruction mix (Section IV, Table "Error rates when estimating
    dynamic instruction mixes from static mixes"), the launches for an ncu capture: 12 dense
    descriptors' variants at one point (one untimed and one timed launch each) and the three
    real kernels at (T = 128, G = 1024, U = 4, C = 100 %) (one untimed and one timed run each).
    Prints, per variant, the descriptor's counts (scaled as emitted), the executed operations per
    class tallied by an instrumented build (tune_emit_count) and their mix error; per real
    kernel, its descriptor. The SASS-level dynamic mix comes from ncu's per-class counters of
    the same launches (`kernel name` variant / rows / cols, in this order)."""
    import torch

    from paper_1701_08547_gb300 import build as B
    from paper_1701_08547_gb300 import realkernels as RK
    from paper_1701_08547_gb300 import surrogate_data as SD

    B.build()
    torch.cuda.set_device(0)
    ax = gen.axes()
    d = gen.descriptors(12, 67, "dense")
    d["d"][:6] = np.float32(0.0)  # half without divergence
    T_, G_, U_, C_ = MIX_POINT
    p = (((ax["t"].index(T_) * 16 + ax["g"].index(G_)) * 8 + ax["u"].index(U_)) * 4 + ax["c"].index(C_))
    kern = np.arange(len(d))
    pt = np.full(len(d), p, dtype=np.int32)
    cnt = SD.count_ops(ax, d, kern, pt)
    us, _, cfg = SD.measure(ax, d, kern, pt, reps=1, launched=True)
    scaled = np.floor(d["n"].astype(np.float32) * np.float32(SD.COUNT_SCALE) + np.float32(0.5)).astype(np.int64)
    variants = []
    for i in range(len(d)):
        variants.append({"launch": list(map(int, cfg[i])), "us": float(us[i]),
                         "static_per_thread": scaled[i].tolist(), "d": float(d["d"][i]),
                         "executed": cnt[i].astype(np.int64).tolist(),
                         "mix_error_executed": SD.mix_error(scaled[i], cnt[i])})
    real = {}
    n = 2048
    for kind in RK.KINDS:
        pts = np.array([[128, 1024, 4, 100]], dtype=np.int32)
        cols = [np.ascontiguousarray(pts[:, j]) for j in range(4)]
        usr = np.empty(1, np.float32)
        regs = np.empty(1, np.int32)
        from paper_1701_08547_gb300 import native

        native.check(native.load().tune_real_measure(RK.KINDS[kind], n, *[c.ctypes.data for c in cols], 1, 1,
                                                     usr.ctypes.data, regs.ctypes.data, None, None))
        desc = RK.descriptor(kind, n, int(regs[0]), ax)
        real[kind] = {"n": n, "launch": [128, 1024, 4, 100], "us": float(usr[0]),
                      "static_per_item": desc["n"][0].astype(np.int64).tolist(),
                      "items": n if kind == "matvec" else 2 * n}
    return {"metric": "static vs dynamic instruction mix (launches for ncu)", "value": None, "unit": None,
            "classes": ["FP32", "FP64", "INT", "GLDST", "SLDST", "BRANCH", "SFU"],
            "count_scale": SD.COUNT_SCALE, "variants": variants, "real_kernels": real}


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


# Oracle samples per workload for the CPU baseline (about 1-2 s on 16 Grace cores each).
CPU_SAMPLE = {"dense": 16000, "dense128": 64, "uneven": 10000}
CPU_SAMPLE_1CORE = 1000  # kernels of the single-thread run, extrapolated per point


def cpu_baseline(workload, sample, emit=False):
    """The CPU oracle (plain C, FP64 cost + FP32 mirror, full sort per kernel, OpenMP over
    kernels) timed on the host cores on the first `sample` kernels of the workload, and on one
    core on the first 1,000 (points/s of each; the workload's points per kernel are the same
    distribution, so the rates extrapolate to the whole workload)."""
    from oracle import oracle as O

    n, space, k, seed = WORKLOADS[workload]
    sample = min(sample, n)
    descs = gen.descriptors(sample, seed, space)
    a, ax = archs.arch("sm_103"), gen.axes()
    threads = O.threads_available()

    def run(d, nt):
        kw = dict(emit=True, offsets=gen.point_offsets(d)) if emit else {}
        t0 = time.perf_counter()
        O.evaluate(a, ax, d, k, nthreads=nt, **kw)
        return time.perf_counter() - t0

    run(descs[:8], threads)  # load + warm
    dt = run(descs, threads)
    pts = int(gen.space_sizes(descs).sum())
    one = descs[:min(CPU_SAMPLE_1CORE, sample)]
    dt1 = run(one, 1)
    pts1 = int(gen.space_sizes(one).sum())
    what = "every point's B*, W*, FP32 and FP64 cost written, " if emit else ""
    return {"value": pts / dt, "unit": "points/s", "cores": threads, "kind": "oracle",
            "sample": f"first {sample} kernels of the {workload} workload ({pts} points), {what}"
                      f"{dt:.2f} s wall on {threads} threads",
            "one_core": {"value": pts1 / dt1, "unit": "points/s", "cores": 1,
                         "sample": f"first {len(one)} kernels ({pts1} points), {dt1:.2f} s on 1 thread; "
                                   f"extrapolated to the whole workload: "
                                   f"{n * (pts1 / len(one)) / (pts1 / dt1):.0f} s"}}


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
    p.add_argument("--headline-only", action="store_true",
                   help="only the selected workload (no sub-configurations or other kernels)")
    p.add_argument("--emit-kernels", type=int, default=0, help="kernels of the every-point run (0: 100,000)")
    p.add_argument("--sur-epochs", type=int, default=20, help="training epochs over the measured labels")
    p.add_argument("--sur-descs", type=int, default=1000, help="descriptors for surrogate labels (x64 points)")
    p.add_argument("--sur-infer-kernels", type=int, default=100_000, help="dense kernels scored by the ensemble")
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
    elif args.workload == "mix":
        line = run_mix(args)
    elif args.workload == "emit":
        line = run_emit(args)
    else:
        line = run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
