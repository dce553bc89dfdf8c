/*
 * tune.h — C ABI of the GB300 static-autotuning library (libtune.so).
 *
 * The library evaluates, for every point of many kernels' tuning spaces
 * (threads per block x grid size x unroll x shared-memory carveout), the
 * occupancy calculation of Lim, Norris & Malony, "Autotuning GPU Kernels
 * via Static and Predictive Analysis" (Section III-A, Eqs. 1-5) and its
 * instruction-mix cost (Section III-B, Eq. 6, extended with launch-shape
 * terms), then selects each kernel's k cheapest configurations.
 *
 * Conventions for every entry point:
 *  - Pointers marked "device" are CUDA device pointers owned by the caller;
 *    the library never frees or retains them after the call returns.
 *    Pointers marked "host" are read during the call only.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and the call returns without synchronising. Errors found on
 *    the host are returned at once; errors found by a kernel (malformed
 *    descriptor contents) are written to the status word in `workspace`
 *    and returned by tune_check().
 *  - Return value: TUNE_OK (0) or a negative TUNE_E* code; a message for the
 *    last error on the calling thread is available from tune_last_error().
 *  - The library never allocates device memory in these calls: scratch
 *    space is the caller's `workspace` of at least tune_workspace_bytes().
 */
#ifndef TUNE_H
#define TUNE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st* tune_stream_t; /* identical to cudaStream_t */

enum {
    TUNE_OK = 0,
    TUNE_EINVAL = -1,   /* bad argument or malformed input record */
    TUNE_ENOMEM = -2,   /* workspace too small */
    TUNE_ECUDA = -3,    /* a CUDA runtime call failed */
    TUNE_ETIMEOUT = -4, /* a bounded device-side wait gave up */
    TUNE_ECOMPILE = -5, /* run-time compilation failed */
    TUNE_EUNSUPPORTED = -6
};

enum { TUNE_NCLASS = 7 }; /* FP32, FP64, INT, GLDST, SLDST, BRANCH, SFU */

/*
 * Architecture row: the limits of Table "GPUs used in this experiment"
 * (Section III-A) and the per-class throughputs of Table "Instruction
 * throughput per number of cycles" (Section III-B), plus the allocation
 * details the occupancy calculation needs on current GPUs. Host memory.
 * Limits: warp_size = 32, max_warps_sm <= 64, max_blocks_sm <= 32,
 * 1 <= n_smem_caps <= 16 with smem_caps ascending, ipc[c] finite and
 * >= 2^-16, 1 <= w_sat <= 2^20, 1 <= work_scale <= 2^24. (With the
 * descriptor ranges below these bounds keep every cost of a valid point
 * under 2^114, so an FP32 cost never overflows: +inf always means "no
 * valid configuration".) A row outside them is refused with TUNE_EINVAL.
 */
typedef struct tune_arch {
    int32_t cc;                  /* compute capability x 10 */
    int32_t n_sm;                /* multiprocessors */
    int32_t warp_size;           /* T_W */
    int32_t max_threads_block;   /* T_B */
    int32_t max_warps_sm;        /* W_mp */
    int32_t max_blocks_sm;       /* B_mp */
    int32_t regs_sm;             /* register file per SM */
    int32_t regs_block_max;      /* registers per block, maximum */
    int32_t regs_thread_max;     /* R_T */
    int32_t reg_alloc_unit;      /* register allocation unit */
    int32_t reg_alloc_mode;      /* 0: per warp, 1: per block */
    int32_t warp_alloc_gran;     /* warps per register-allocation group */
    int32_t smem_block_max;      /* S_B, bytes */
    int32_t smem_reserved_block; /* bytes reserved per block by the runtime */
    int32_t smem_alloc_unit;     /* shared-memory allocation unit, bytes */
    int32_t n_smem_caps;         /* supported per-SM shared-memory capacities */
    int32_t smem_caps[16];       /* bytes, ascending */
    float ipc[TUNE_NCLASS];      /* instructions per cycle per SM, per class */
    int32_t w_sat;               /* warps per SM that hide memory latency */
    int32_t work_scale;          /* K: work items per instruction count */
} tune_arch;

/*
 * Tuning axes: the values that descriptor space-mask bits select. Host
 * memory. 1 <= n_t <= 32, 1 <= n_g <= 16, 1 <= n_u <= 8, 1 <= n_c <= 4;
 * t in [1, 4096], g >= 1 with n_sm * g < 2^24, u in [1, 64], c in [0, 100].
 */
typedef struct tune_axes {
    int32_t n_t, n_g, n_u, n_c;
    int32_t t[32]; /* threads per block */
    int32_t g[16]; /* grid size, blocks */
    int32_t u[8];  /* unroll factor; registers/thread = r0 + 4 (u - 1) */
    int32_t c[4];  /* preferred shared-memory carveout, percent of the largest capacity */
} tune_axes;

/*
 * Kernel descriptor, 64 bytes, 16-byte aligned: the static facts the
 * paper's front end extracts (Section III, "Static Analysis": registers and
 * shared memory from ptxas, instruction counts from the binary).
 * space_mask bits 0..31 select t[], 32..47 g[], 48..55 u[], 56..59 c[];
 * bits 60..63 and bits beyond each axis length must be zero. A record
 * outside the field ranges below, or whose mask breaks these rules, is
 * malformed (see tune_eval).
 */
typedef struct tune_kernel_desc {
    float n[TUNE_NCLASS]; /* static instruction counts per class, in [0, 2^40] */
    int32_t r0;           /* registers per thread at unroll 1, in [0, 2^24) */
    int32_t s0;           /* shared memory per block, bytes, in [0, 2^30) */
    float d;              /* branch-divergence fraction, in [0, 1] */
    uint64_t space_mask;
    int32_t reserved[4];
} tune_kernel_desc;

/* tune_eval flags */
#define TUNE_EMIT_POINTS 0x1u   /* also write per-point B*, W*, cost (pt_* arrays) */
#define TUNE_SCHED_WARP 0x10u   /* schedule: one warp per descriptor (the default) */
#define TUNE_SCHED_THREAD 0x20u /* schedule: one thread per descriptor (not with EMIT) */
#define TUNE_HOST_DIRECT 0x40u  /* tune_eval_host: evaluate in place in mapped host memory */
/* Warp schedule knobs (tune_autotune picks them): a work queue handing each warp
 * 2^c consecutive descriptors per grab (c in 0..14; default: a static stride),
 * and at most m resident CTAs per SM (m in 1..15; default: as many as fit). */
#define TUNE_SCHED_CHUNK(c) ((((uint32_t)(c)) + 1u) << 8)
#define TUNE_SCHED_CTAS(m) (((uint32_t)(m)) << 12)

/* Calls for tune_workspace_bytes(). */
enum { TUNE_CALL_EVAL = 0, TUNE_CALL_TOPK = 1 };

/*
 * tune_eval — evaluate every point of every kernel's space and select each
 * kernel's k best.
 *
 * For kernel i and each point (T, G, U, C) of its space, in canonical order
 * (row-major over T, G, U, C restricted to the mask, C fastest):
 *   R  = r0 + 4 (U - 1)
 *   B* = min(G_W, G_R, G_S)  (Eqs. 1, 3, 4, 5), W* = B* ceil(T/32)  (Eq. 2);
 *   invalid if B* = 0 or T > max_threads_block.
 *   cost = (C_nm + C_m hide) lane / par  (Eq. 6 with c_x = 1 / IPC_x, plus
 *   the library's launch-shape terms hide, lane, par), computed in FP32 in
 *   a fixed operation order with compensated sums.
 * Outputs (device):
 *   topk_idx  int32[n_kernels * k]  canonical point indices, best first;
 *                                   equal costs -> lower index first;
 *                                   -1 past the last valid point
 *   topk_cost float[n_kernels * k]  their costs (+inf for padding)
 *   pt_blocks, pt_warps (int32), pt_cost (float): optional, only with
 *   TUNE_EMIT_POINTS; indexed pt_offsets[i] + canonical index, where
 *   pt_offsets (device int64[n_kernels + 1]) is the exclusive scan of space
 *   sizes. Invalid points get B* = W* = 0, cost = +inf. Any of the three may
 *   be NULL.
 * Arguments: arch, axes (host); descs (device, 16-byte aligned,
 * n_kernels records); 1 <= k <= 16; workspace (device) of at least
 * tune_workspace_bytes(TUNE_CALL_EVAL, n_kernels, k) bytes.
 * n_kernels = 0 is valid and enqueues only the status reset.
 * A malformed descriptor (mask selecting values outside the axes, or a
 * field outside its range: a count above 2^40, negative or not a number,
 * d outside [0, 1], r0 or s0 out of range) gets padding outputs and sets
 * TUNE_EINVAL in the status word; the other descriptors are unaffected.
 */
int tune_eval(const tune_arch* arch, const tune_axes* axes, const tune_kernel_desc* descs,
              int64_t n_kernels, int32_t k, uint32_t flags, int32_t* topk_idx, float* topk_cost,
              int32_t* pt_blocks, int32_t* pt_warps, float* pt_cost, const int64_t* pt_offsets,
              void* workspace, size_t ws_bytes, tune_stream_t stream);

/*
 * tune_eval_noalloc — tune_eval for callers that cannot provide a workspace.
 * The paper has no counterpart; this is a library convenience.
 *
 * Some programs cannot allocate device memory on this library's behalf: hosts
 * that own all device memory and give plugins no way to request a buffer
 * (serving runtimes, framework allocators), and programs whose device-memory
 * budget is fixed at start-up. This entry point takes the same inputs and
 * outputs as tune_eval but keeps its scratch (status word and counters) in a
 * static device array of 4096 bytes inside the library, which every GPU that
 * loads the library holds until the process exits. It calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *  - A call whose scratch need, tune_workspace_bytes(TUNE_CALL_EVAL, n, k),
 *    exceeds 4096 bytes is rejected with TUNE_ENOMEM. (Every call of this
 *    version needs the 256-byte header only, so the limit is not reached.)
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before starting any stream capture.
 *  - That address is kept for the life of the process. It belongs to the
 *    device's primary context: after cudaDeviceReset (or anything else that
 *    destroys and recreates that context) it is stale, so do not use this
 *    entry point across a device reset.
 *  - Every call shares the array and clears the part it uses at the start;
 *    calls that overlap on the GPU (for example on two streams) race on it.
 *  - The call waits for `stream` before returning, so that it can return
 *    TUNE_EINVAL for malformed descriptors found by the kernel.
 */
int tune_eval_noalloc(const tune_arch* arch, const tune_axes* axes, const tune_kernel_desc* descs,
                      int64_t n_kernels, int32_t k, uint32_t flags, int32_t* topk_idx,
                      float* topk_cost, int32_t* pt_blocks, int32_t* pt_warps, float* pt_cost,
                      const int64_t* pt_offsets, tune_stream_t stream);

/*
 * tune_autotune — choose tune_eval's schedule for a workload by measurement.
 * (Library tooling; the paper autotunes the kernels it analyses, not itself.)
 * Runs tune_eval on the given descriptors with each candidate schedule — the
 * warp schedule with a static stride or a work queue of 1, 4, 16 or 64
 * descriptors per grab at full residency or 2 / 3 CTAs per SM, and the thread
 * schedule — times `reps` runs of each with CUDA events on `stream` (after one
 * untimed run) and keeps the fastest run's time. Returns the winner's schedule
 * bits in *best_flags (OR them into tune_eval's flags) and its time in
 * *best_ms; topk_idx / topk_cost hold the winner's results. Arguments as for
 * tune_eval, 1 <= reps <= 100. Waits for `stream` before returning.
 */
int tune_autotune(const tune_arch* arch, const tune_axes* axes, const tune_kernel_desc* descs,
                  int64_t n_kernels, int32_t k, int32_t reps, int32_t* topk_idx, float* topk_cost,
                  void* workspace, size_t ws_bytes, uint32_t* best_flags, float* best_ms,
                  tune_stream_t stream);

/*
 * tune_topk — segmented top-k over an external score array (device): the
 * ranking step of the paper's autotuning (Section IV-A: the variants of a
 * kernel are sorted by time, ascending, and the best ranks are kept), here
 * over any per-point score, e.g. a surrogate's predicted runtimes.
 * For segment s = [seg_offsets[s], seg_offsets[s+1]) of `scores`, the k
 * smallest scores that are not +inf or NaN, equal scores -> lower index;
 * topk_idx holds indices within the segment (-1 for padding), topk_score
 * the scores (+inf for padding). seg_offsets: device int64[n_seg + 1],
 * non-decreasing, segment lengths < 2^31. 1 <= k <= 16.
 */
int tune_topk(const float* scores, const int64_t* seg_offsets, int64_t n_seg, int32_t k,
              int32_t* topk_idx, float* topk_score, void* workspace, size_t ws_bytes,
              tune_stream_t stream);

/* ---- learned surrogate (Section VII: machine learning for the static models) ----
 *
 * An ensemble of MLPs predicting the logarithm of a tuning point's runtime (in
 * the labels' unit) from 48 static features (zero-padded to TUNE_SURROGATE_INPUTS
 * = 64 inputs, one 128-byte BF16 row): 64 -> 256 -> 256 -> 256 -> 256 -> 1 with
 * GELU (tanh form), BF16 weights and activations, FP32
 * accumulation, FP32 master weights, Adam, MSE loss. All members are trained
 * together on the same batches by the library's BF16 tensor-core kernels.
 * Unlike the tune_* calls, a surrogate handle owns device memory (weights,
 * optimiser state, activations for one batch), allocated by
 * surrogate_create and released by surrogate_free. Feature arrays are BF16
 * (uint16_t bit patterns), [n, 64], row-major, device.
 *
 * Parameter layout per member (floats; surrogate_param_count() = 214336 per
 * member, members back to back): W1 [256 x 64] at 0, b1 [256] at 16384, W2 at
 * 16640, b2 at 82176, W3 at 82432, b3 at 147968, W4 at 148224, b4 at 213760,
 * w5 [256] at 214016, b5 at 214272; W[o][i] row-major (output-major).
 */
#define TUNE_SURROGATE_INPUTS 64
typedef struct tune_surrogate tune_surrogate;
typedef struct tune_surrogate_cfg {
    int32_t members; /* ensemble size, 1..16 */
    int32_t batch;   /* rows per training step, multiple of 128, <= 65536 */
    float lr, beta1, beta2, eps; /* Adam */
} tune_surrogate_cfg;

int surrogate_create(tune_surrogate** h, const tune_surrogate_cfg* cfg);
void surrogate_free(tune_surrogate* h);
/* Floats per member in the parameter layout. */
int surrogate_param_count(void);
/* Copy master weights (host, members x surrogate_param_count() floats); resets Adam. Synchronous. */
int surrogate_set_params(tune_surrogate* h, const float* host, int64_t n);
/* Copy to host: what = 0 master weights, 1 gradients of the last step, 2 Adam m, 3 Adam v
 * (members x param_count floats), 4 last loss per member (members floats), 5 last
 * predictions (members x batch), 6 the E4M3 codes of W2..W4 as their values (members x 3
 * x 256 x 256), 7 the scales of those codes (members x 3 x 256: one per matrix, repeated for each
 * of its rows). Synchronous. */
int surrogate_get(tune_surrogate* h, int what, float* host, int64_t n);
/* pred (device, [members, n]) = each member's output for feats (device bf16 [n, 64]).
 * By default one persistent launch runs every member over 128-row tiles with the
 * activations kept on chip (option 1). feats must be 16-byte aligned. */
int surrogate_forward(tune_surrogate* h, const uint16_t* feats, int64_t n, float* pred, tune_stream_t stream);
/* One step on rows feats[0..n), labels[0..n) (device), 1 <= n <= batch: forward, MSE
 * loss, backward into the gradient buffer, and (apply_update != 0) one Adam step. */
int surrogate_train_step(tune_surrogate* h, const uint16_t* feats, const float* labels, int64_t n,
                         int32_t apply_update, tune_stream_t stream);
/* `epochs` passes over n rows in the order given (device int32 [epochs, n], a
 * permutation of 0..n-1 per epoch), batch rows per step; loss_trace (device,
 * nullable) receives [epochs, steps, members] losses. */
int surrogate_train(tune_surrogate* h, const uint16_t* feats, const float* labels, int64_t n,
                    const int32_t* order, int32_t epochs, float* loss_trace, tune_stream_t stream);

/* Ensemble size of a handle (0 for NULL). */
int surrogate_members(const tune_surrogate* h);
/* Options: 0 = layer-by-layer forward on tcgen05 tensor cores (value 1, the default) or
 * on mma.sync (value 0); 1 = how surrogate_forward / surrogate_infer run the ensemble:
 * 0 layer by layer (option 0 picks the GEMM), 1 fused BF16 (default), 2 fused with
 * layers 2-4 on E4M3 codes: each of W2..W4 quantised with one scale (max |w| over the matrix
 * / 448; codes nearest-even, saturating), activations as codes of 2 h, FP32 accumulation;
 * 2 = training's backward pass: 0 one mma.sync GEMM per input and weight gradient;
 * 1 (default, with option 0 on) the chain dZ4 -> dZ3 -> dZ2 -> dZ1 (products with W4,
 * W3, W2) in one fused tcgen05 launch and the weight and bias gradients of every layer on
 * tcgen05 in one launch (both operands MN-major, one CTA per 128 x 64 gradient tile and
 * member accumulating the whole batch; the bias sums by a second MMA with an all-ones
 * operand). */
int surrogate_set_option(tune_surrogate* h, int option, int value);
/* Synchronous: TUNE_ETIMEOUT if a bounded wait inside a surrogate kernel gave up since the
 * last check; the check clears the handle's status word. */
int surrogate_status(tune_surrogate* h);

/*
 * tune_features — the surrogate's 48 input features (zero-padded to 64 BF16
 * columns) of listed tuning points: sample i is point sample_point[i]
 * (canonical index) of descriptor sample_kernel[i]. Features are fixed
 * scalings of the descriptor, the launch parameters and the occupancy and
 * cost internals of Eqs. 3-6 (see csrc/features.cuh for the list). feats:
 * device BF16 [n, 64]. Invalid samples set TUNE_EINVAL in the status word.
 */
int tune_features(const tune_arch* arch, const tune_axes* axes, const tune_kernel_desc* descs,
                  const int64_t* sample_kernel, const int32_t* sample_point, int64_t n, uint16_t* feats,
                  void* workspace, size_t ws_bytes, tune_stream_t stream);

/*
 * surrogate_infer — rank every point of every kernel's space by the ensemble's
 * predicted runtime (mean over members of exp(prediction), in microseconds);
 * per kernel, if any of the surrogate's k best points has a member spread
 * (std / mean of the predicted runtimes) above `thresh`, return the analytic
 * top-k instead (tune_eval's cost values) and set used_fallback[kernel] = 1.
 * pt_offsets_host: host int64 [n_kernels + 1], exclusive scan of space sizes
 * (each space <= 2^20 points). Outputs (device): topk_idx, topk_score
 * [n_kernels, k], used_fallback uint8 [n_kernels]. workspace of at least
 * surrogate_infer_workspace_bytes(members, n_kernels, k). Synchronous.
 */
int surrogate_infer(tune_surrogate* h, const tune_arch* arch, const tune_axes* axes,
                    const tune_kernel_desc* descs, int64_t n_kernels, const int64_t* pt_offsets_host,
                    int32_t k, float thresh, int32_t* topk_idx, float* topk_score, uint8_t* used_fallback,
                    void* workspace, size_t ws_bytes, tune_stream_t stream);
size_t surrogate_infer_workspace_bytes(int members, int64_t n_kernels, int32_t k);

/*
 * tune_emit_measure — the surrogate's labels: run synthetic code variants on
 * this GPU and time them. (The paper's autotuner times generated variants,
 * Section IV-A; these variants are the library's own, not Orio's.)
 * For sample i, descriptor descs[sample_kernel[i]] at point sample_point[i]
 * (canonical index) becomes a kernel compiled at run time (NVRTC, sm_103a)
 * in which every thread executes `items` work items; per item and
 * instruction class it runs a dependent loop of round(n_c * count_scale)
 * operations, unrolled U times, keeps registers live according to r0, uses
 * s0 bytes of dynamic shared memory, and repeats its FP32 loop on round(32 d)
 * lanes of each warp. The per-thread work is therefore the same at every
 * (T, G): the descriptor's counts are per thread, as in Eq. 6, and a launch of
 * G blocks does G T items of work (time / (G T items) is what the model's
 * cost ranks). It is launched with G blocks of T threads at carveout C: one
 * untimed launch, then `reps` launches timed with CUDA events.
 *   us[i]       median time of the launch in microseconds (NaN where the
 *               launch is not possible, e.g. too many registers for T)
 *   regs[i]     the variant's registers per thread
 *   launched    NULL or int32[4 * n_samples]: the (T, G, U, C) the sample's
 *               canonical index decoded to (row-major over T, G, U, C
 *               restricted to the mask, C fastest), written before the launch
 * descs, sample arrays and outputs are host memory; the call allocates two
 * 4 MB device buffers for its duration and is synchronous. Returns
 * TUNE_ECOMPILE if a variant fails to compile.
 */
int tune_emit_measure(const tune_axes* axes, const tune_kernel_desc* descs, int64_t n_kernels,
                      const int32_t* sample_kernel, const int32_t* sample_point, int64_t n_samples,
                      int32_t items, float count_scale, int32_t reps, float* us, int32_t* regs,
                      int32_t* launched, tune_stream_t stream);

/*
 * tune_emit_count — the executed instruction mix of tune_emit_measure's variants (the
 * dynamic side of Section IV's comparison of static and dynamic instruction mixes, Table
 * "Error rates when estimating dynamic instruction mixes from static mixes"). Sample i's
 * variant is built with per-class tallies (one per executed iteration of a class's loop:
 * FP32 FMA, FP64 FMA, integer step, global load, shared load-store, branch, SFU sine) and
 * launched once as tune_emit_measure launches it; counts[7 i + c] = the operations of class c
 * executed by all its threads (UINT64_MAX where the launch is not possible). Arguments as
 * for tune_emit_measure; counts is host memory; synchronous; allocates its buffers (two 4 MB,
 * one 56 B) for the duration of the call.
 */
int tune_emit_count(const tune_axes* axes, const tune_kernel_desc* descs, int64_t n_kernels,
                    const int32_t* sample_kernel, const int32_t* sample_point, int64_t n_samples,
                    int32_t items, float count_scale, uint64_t* counts, tune_stream_t stream);

/*
 * tune_eval_archs — tune_eval of the same descriptors against n_arch
 * architecture rows (1..8) in one launch (a sweep over GPU generations:
 * Eqs. 1-6 with each row's limits and throughputs). archs: host array
 * [n_arch]. Outputs topk_idx / topk_cost [n_arch][n_kernels][k]; row i's
 * results equal tune_eval(&archs[i], ...) bit for bit. flags: TUNE_SCHED_WARP
 * with its chunk and CTA fields only. Workspace: the 256-byte header (status
 * word and one queue counter per row).
 */
int tune_eval_archs(const tune_arch* archs, int32_t n_arch, const tune_axes* axes, const tune_kernel_desc* descs,
                    int64_t n_kernels, int32_t k, uint32_t flags, int32_t* topk_idx, float* topk_cost,
                    void* workspace, size_t ws_bytes, tune_stream_t stream);

/*
 * tune_suggest — static search-space pruning (Section III-C "Static Search
 * Analysis", Section IV-C Table "Suggested parameters to achieve theoretical
 * occupancy"). Per kernel, at its registers r0 and shared memory s0 and the
 * largest shared-memory capacity:
 *   t_star[i]     mask over the thread-count axis: the thread counts of the
 *                 kernel's space reaching the best theoretical occupancy
 *   occ_star[i]   that occupancy, W* / W_mp
 *   r_headroom[i] registers that can be added while some thread count of
 *                 T* still reaches occ* (R*)
 *   s_star[i]     the largest shared memory per block keeping the block count
 *                 at the smallest thread count of T* (S*)
 *   t_rule[i]     the rule-based reduction: intensity (FP32 + FP64 counts over
 *                 GLDST + SLDST counts) > 4.0 keeps the upper half of T*
 *                 (floor(|T*| / 2) values, at least one), else the lower half.
 * All outputs device arrays [n_kernels]; -1 headrooms for kernels with no valid point.
 */
int tune_suggest(const tune_arch* arch, const tune_axes* axes, const tune_kernel_desc* descs,
                 int64_t n_kernels, uint32_t* t_star, float* occ_star, int32_t* r_headroom,
                 int32_t* s_star, uint32_t* t_rule, void* workspace, size_t ws_bytes,
                 tune_stream_t stream);

/*
 * tune_search — random or Nelder-Mead simplex search over each kernel's tuning
 * space, with the static model's cost as the objective. The paper's autotuner
 * explores the space left after static pruning with one of its search methods
 * (Section III-C lists its methods; Section IV-C: exhaustive, or random or
 * Nelder-Mead simplex to bound the tuning time); with the model as the
 * objective no variant is run.
 *   method   TUNE_SEARCH_RANDOM or TUNE_SEARCH_NELDER_MEAD
 *   budget   objective evaluations per kernel, 1..2^20
 *   seed     random draws: draw j of kernel i is the SplitMix64 output of the state
 *            mix64(seed) + (i 2^32 + j + 1) 0x9E3779B97F4A7C15, mapped to [0, n) as
 *            ((x >> 32) n) >> 32
 *   t_keep   device uint32[n_kernels] or NULL: thread-count positions to search
 *            (e.g. tune_suggest's t_star or t_rule), intersected with the kernel's
 *            mask; NULL searches the whole space
 * A point is a rank vector over the searched lists (thread counts, grid sizes,
 * unroll factors, carveouts); its objective is the FP32 cost of the point as
 * tune_eval computes it (+inf without a valid configuration), points ordered by
 * (cost, canonical index in the kernel's full space).
 *   random: evaluation j draws rank d from draw 4 j + d.
 *   Nelder-Mead: five vertices in fixed point (8 fractional bits), rounded to the
 *   nearest rank (floor of v + 1/2) and clamped; start x0 from draws 0..3, vertex
 *   d + 1 = x0 moved max(1, n_d / 4) ranks along axis d (backwards where forwards
 *   leaves the list); vertices ordered by (cost, index, vertex number); centroid c
 *   of the best four (sum >> 2); reflection 2c - w; if it beats the best,
 *   expansion 3c - 2w (the better of the two replaces w); else if it beats the
 *   second worst it replaces w; else contraction c + ((r - c) >> 1) if the
 *   reflection r beats w, else c + ((w - c) >> 1), replacing w if it beats the
 *   better of r and w (resp. w); else every vertex moves halfway to the best
 *   (v = b + ((v - b) >> 1)) and is evaluated. Every evaluation counts; the
 *   search stops when the budget is spent or a shrink leaves all vertices on one
 *   point.
 * Outputs (device, [n_kernels]): best_idx (canonical index of the best point seen,
 * -1 if no evaluated point has a valid configuration), best_cost (+inf then),
 * evals (evaluations made). Asynchronous on
 * `stream`; workspace: the 256-byte header (status word; malformed descriptors set
 * TUNE_EINVAL, read with tune_check).
 */
#define TUNE_SEARCH_RANDOM 1
#define TUNE_SEARCH_NELDER_MEAD 2
int tune_search(const tune_arch* arch, const tune_axes* axes, const tune_kernel_desc* descs, int64_t n_kernels,
                int32_t method, int32_t budget, uint64_t seed, const uint32_t* t_keep, int32_t* best_idx,
                float* best_cost, int32_t* evals, void* workspace, size_t ws_bytes, tune_stream_t stream);

/*
 * tune_real_measure — the paper's dense benchmark kernels (Section IV-A, Table
 * "Kernel specifications") as tuning variants timed on this GPU: matVec2D y = A x,
 * ATAX y = A^T (A x), BiCG q = A p and s = A^T r, for an n x n FP32 matrix.
 * Each product is a grid-stride loop over output elements (a thread per row of A x,
 * per column of A^T x) whose inner loop over n is unrolled U times. Variant v runs
 * the kernel's launches with G[v] blocks of T[v] threads at carveout C[v] percent:
 * one untimed run, then `reps` runs timed with CUDA events; us[v] = median run time
 * in microseconds (NaN where the configuration cannot launch), regs[v] = registers
 * per thread of the unroll's module. Operands are fixed: A[i][j] = ((7i + 13j) mod
 * 17 - 8) / 8, x = p: ((5j) mod 11 - 5) / 4, r: ((5j + 3) mod 11 - 5) / 4.
 * result: NULL or host float[n] (matVec2D: y; ATAX: y) / [2n] (BiCG: q then s), the
 * outputs of variant 0. Arrays T, G, U, C, us, regs are host memory; the call
 * allocates the operands (n^2 + 4n floats) for its duration and is synchronous.
 * Returns TUNE_ECOMPILE if a module fails to compile.
 */
#define TUNE_REAL_MATVEC 0
#define TUNE_REAL_ATAX 1
#define TUNE_REAL_BICG 2
int tune_real_measure(int32_t kernel, int32_t n, const int32_t* T, const int32_t* G, const int32_t* U,
                      const int32_t* C, int32_t n_variants, int32_t reps, float* us, int32_t* regs, float* result,
                      tune_stream_t stream);

/*
 * tune_eval_host — tune_eval with the descriptors and the top-k results in host
 * memory: the kernels are cut into chunks of `chunk`; chunk i is copied to the device
 * on a library stream, evaluated on `stream`, and its results copied back on a second
 * library stream while chunk i + 1 is copied in and evaluated, so that the transfers
 * overlap the evaluation (two staging buffers in dev_scratch). Host buffers should be
 * pinned for the copies to run asynchronously. Results equal tune_eval's bit for bit.
 * With TUNE_HOST_DIRECT the three host buffers must be pinned and mapped into the
 * device's address space (cudaHostAlloc / cudaMallocHost, or cudaHostRegister with
 * mapping; checked with cudaPointerGetAttributes, TUNE_EINVAL otherwise): one launch
 * then reads the descriptors from and writes the top-k into host memory over the
 * host link while it evaluates (no staging copies; chunk is not used, and dev_scratch
 * needs only the 256-byte status header).
 *   host_descs      host tune_kernel_desc[n_kernels]
 *   host_topk_idx   host int32[n_kernels * k];  host_topk_cost  host float[n_kernels * k]
 *   dev_scratch     device memory, 256-byte aligned, of tune_eval_host_scratch_bytes(chunk, k)
 *                   bytes; its first 256 bytes are the status header (read with tune_check)
 *   flags           TUNE_SCHED_WARP with its chunk / CTA fields, TUNE_HOST_DIRECT
 * Enqueues the work and returns; `stream` completes once the last result is in host
 * memory. Calls on one device use the same two library streams and must not run
 * concurrently from several host threads.
 */
size_t tune_eval_host_scratch_bytes(int64_t chunk, int32_t k);
int tune_eval_host(const tune_arch* arch, const tune_axes* axes, const tune_kernel_desc* host_descs, int64_t n_kernels,
                   int32_t k, uint32_t flags, int32_t* host_topk_idx, float* host_topk_cost, int64_t chunk,
                   void* dev_scratch, size_t scratch_bytes, tune_stream_t stream);

/* Bytes of device workspace the call needs (at least 256). */
size_t tune_workspace_bytes(int call, int64_t n, int32_t k);

/*
 * tune_check — wait for `stream`, then return the status word the last
 * call on this workspace left (TUNE_OK, TUNE_EINVAL, TUNE_ETIMEOUT).
 */
int tune_check(const void* workspace, tune_stream_t stream);

/* Message for the last error returned on the calling thread ("" if none). */
const char* tune_last_error(void);

/* Library version, e.g. 100 for 0.1.0. */
int tune_version(void);

/*
 * tune_inject_fault — make the library's failure paths run on purpose, for
 * testing a caller's error handling (library tooling; the paper has no
 * counterpart). Sets the number of pending faults of one kind (0 clears);
 * each fault is used up once. Nothing here faults or hangs the GPU: the
 * failures are made on the host, or by a kernel that leaves a copy unissued
 * and gives up its bounded wait on it early.
 *   TUNE_FAULT_COMPILE   the next `count` variant modules that tune_emit_measure
 *                        or tune_real_measure request fail as if run-time
 *                        compilation had rejected them (TUNE_ECOMPILE; nothing
 *                        is cached)
 *   TUNE_FAULT_SLOW_REP  the next `count` timed repetitions of those calls
 *                        read one second longer, as if the GPU had been taken
 *                        away meanwhile (the median of reps >= 3 discards a
 *                        single such repetition)
 *   TUNE_FAULT_WAIT      the next `count` launches of the surrogate's per-layer
 *                        tcgen05 forward GEMM (option 1 = 0, option 0 = 1)
 *                        leave their first operand copy unissued, so its wait
 *                        gives up after a short bound: every CTA records the
 *                        timeout, waits for the copies it did issue, frees its
 *                        tensor memory and returns without writing its output;
 *                        surrogate_status then returns TUNE_ETIMEOUT
 */
#define TUNE_FAULT_COMPILE 1
#define TUNE_FAULT_SLOW_REP 2
#define TUNE_FAULT_WAIT 3
int tune_inject_fault(int kind, int count);

#ifdef __cplusplus
}
#endif

#endif /* TUNE_H */
