// tune_eval: occupancy (Eqs. 1-5) + instruction-mix cost (Eq. 6 with launch-shape
// terms) over every point of every kernel's tuning space, then per-kernel top-k.
//
// Work decomposition (GB300, CUDA cores only; the path is integer/FP32 issue-bound):
//  * one warp evaluates one kernel descriptor; CTAs of 8 warps stride over the
//    descriptors (grid = SMs x resident CTAs);
//  * per CTA, once: tables that depend only on the architecture row and the
//    axes (W_B, G_W, lane by thread count; hide by W*; waves/slots factor by
//    (B*, G); floor(w / W_B) for the register limit);
//  * per kernel, lane-parallel: the per-unroll cost sums C_nm(U), C_m(U)
//    (compensated FP32 sums), register-limited warps, per-carveout G_S, and
//    the (T, U) block limit min(G_W, G_R);
//  * pre-pass: a lane walks (T, U, C) triples; occupancy B*, W* come from
//    two table lookups and a min (grid size does not enter Eqs. 1-5); every
//    grid size G of a triple costs X(T,U,C) * ipar(B*, G), and since a product
//    by X > 0 is monotone under round-to-nearest the triple's cheapest point
//    is exactly X * min_G ipar(B*, G): one FP32 multiply per triple. A value
//    that k distinct triple minima do not exceed (tau0, from each lane's two
//    smallest (T, U)-pair minima counted with their multiplicities) bounds the
//    kernel's k-th best cost; each triple's minimum is kept in shared memory;
//  * main pass: lanes scan the minima; only triples that can still beat the
//    bound are re-evaluated, and the warp merges their grid sizes in
//    increasing (cost, index) order into a warp-wide exact top-k list (lane j
//    holds the j-th best); ties go to the lower canonical index.
//  * with TUNE_EMIT_POINTS the main pass instead computes and writes every
//    point's B*, W* and cost.
#include <math.h>
#include <stdint.h>

#include <string.h>

#include <algorithm>
#include <limits>
#include <mutex>

#include "eval_common.cuh"
#include "tune_internal.h"

namespace {

using namespace tune_dev;

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kMaxB = 32;  // blocks per SM supported by the tables
constexpr int kIparStride = 17;  // words per ipar row (16 grid positions and one of padding)
constexpr unsigned kFull = 0xffffffffu;



constexpr int kMaxArch = 8;  // architecture rows of one launch (blockIdx.y)

struct CtaTables {
    // (waves*slots)/(n_sm*G) by (B*-1, g position); +inf padding. Rows of 17 words, so that a
    // warp reading one g position of 32 rows (lane = row) touches 32 distinct banks.
    float ipar[kMaxB][kIparStride];
    float rcp[8];                    // 1 / IPC per class
    float rcpn[33];                  // 1 / n for n = 1..32 (axis-subset sizes; [0] unused)
    float hide[kMaxW + 1];           // max(1, W_sat / W*)
    float lane[32];                  // (32 * W_B) / T by t position
    int wb[32];                      // W_B = ceil(T / 32) by t position
    int gw[32];                      // G_W by t position (0 if T > max threads per block)
    unsigned char divt[kMaxW + 1][32];  // floor(w / W_B) by (w, t position)
    unsigned char perm[kMaxB][16];   // g positions of ipar row b in increasing (value, g) order
    float iparmin[kMaxB];            // min of ipar row b over all axis grid sizes
    unsigned short rwarps[256];      // register-limited warps by R (Eq. 4, per-warp allocation)
    unsigned short rwbmax[256];      // largest W_B whose block fits the per-block register limit, by R
    int cap_lo[4];                   // first capacity index allowed by carveout position c
    int order_safe;                  // 1: distinct ipar values of a row differ by more than 2^-21 relative
    int unit_shift;                  // log2 of the shared-memory allocation unit, or -1
};

// Parameters of one launch. For a single architecture row the host builds the CTA tables
// (they depend on the row and the axes only) and passes them here, 6.6 KB of kernel
// parameters each CTA copies to shared memory; with several rows (blockIdx.y) every CTA
// builds its row's tables itself.
struct EvalParams {
    tune_arch a[kMaxArch];
    int n_arch;
    tune_axes x;
    int64_t n_kernels;
    int k;
    int chunk;        // dynamic work queue: kernels per grab (0 = static stride)
    int host_tables;  // 1: tab holds row 0's tables
    CtaTables tab;
};

struct WarpTables {
    float iparmin[kMaxB + 1];  // by B*: min over the kernel's grid sizes of ipar(B*, G); [0] = NaN
    unsigned char gwr[32][8];  // min(G_W, G_R) by (t rank, u rank)
    float cnm[8], cm[8];     // by u rank
    int regs[8];             // R by u rank
    int gs[4];               // G_S by c rank
    int4 tinfo[32];          // by t rank: W_B, lane efficiency (float bits), t position, G_W
    int ru[8];               // by u rank: register-limited warps | (largest W_B that fits) << 8
    int gpos[16];            // g position by g rank
    union {
        float key[32 * 32];  // ranking pass: each triple's minimum cost, by (row, lane)
        struct {             // emitting pass:
            float iparc[kMaxB][kIparStride];  // ipar rows compacted to the kernel's grid sizes
            float4 uc[32];   // by (u rank * n_C + c rank): C_nm, C_m, u rank, G_S
        };
    };
};

// The same tables, built on the host for a single architecture row (IEEE single-precision
// divisions and multiplications, each rounded to nearest as __fdiv_rn / __fmul_rn round them on
// the device, so the values are bit for bit those of build_cta_tables below).
void host_cta_tables(const tune_arch& a, const tune_axes& x, CtaTables& ct)
{
    memset(&ct, 0, sizeof(ct));
    const float inf = std::numeric_limits<float>::infinity();
    for (int b = 0; b < kMaxB; ++b)
        for (int g = 0; g < 16; ++g) {
            float v = inf;
            if (b < a.max_blocks_sm && g < x.n_g) {
                const int slots = a.n_sm * (b + 1), G = x.g[g];
                const int waves = (G + slots - 1) / slots;
                v = (float)(waves * slots) / (float)(a.n_sm * G);
            }
            ct.ipar[b][g] = v;
        }
    for (int w = 0; w <= kMaxW; ++w)
        for (int t = 0; t < 32; ++t) {
            const int wb = t < x.n_t ? (x.t[t] + 31) / 32 : 1;
            ct.divt[w][t] = (unsigned char)(w / wb);
        }
    ct.order_safe = 1;
    const int u = a.smem_alloc_unit;
    ct.unit_shift = (u & (u - 1)) == 0 ? __builtin_ctz((unsigned)u) : -1;
    for (int b = 0; b < kMaxB; ++b) {
        float mn = inf;
        for (int g = 0; g < x.n_g; ++g) mn = std::min(mn, ct.ipar[b][g]);
        ct.iparmin[b] = mn;
        unsigned char* ord = ct.perm[b];
        for (int g = 0; g < x.n_g; ++g) {
            const float v = ct.ipar[b][g];
            int j = g;
            while (j > 0 && ct.ipar[b][ord[j - 1]] > v) {
                ord[j] = ord[j - 1];
                --j;
            }
            ord[j] = (unsigned char)g;
        }
        for (int r = 0; r + 1 < x.n_g; ++r) {
            const float v1 = ct.ipar[b][ord[r]], v2 = ct.ipar[b][ord[r + 1]];
            const volatile float gap = v2 - v1, tol = v1 * 0x1p-21f;  // two roundings, no fused form
            if (v2 != v1 && gap <= tol) ct.order_safe = 0;
        }
    }
    for (int t = 0; t < 32; ++t) {
        int wb = 1, gw = 0;
        float ln = 1.0f;
        if (t < x.n_t) {
            const int T = x.t[t];
            wb = (T + 31) / 32;
            gw = T <= a.max_threads_block ? std::min(a.max_blocks_sm, a.max_warps_sm / wb) : 0;
            ln = (float)(32 * wb) / (float)T;
        }
        ct.wb[t] = wb;
        ct.gw[t] = gw;
        ct.lane[t] = ln;
    }
    for (int w = 0; w <= kMaxW; ++w) ct.hide[w] = std::max(1.0f, w > 0 ? (float)a.w_sat / (float)w : 1.0f);
    for (int c = 0; c < 8; ++c) ct.rcp[c] = c < TUNE_NCLASS ? 1.0f / a.ipc[c] : 0.0f;
    for (int n = 1; n <= 32; ++n) ct.rcpn[n] = 1.0f / (float)n;
    for (int c = 0; c < 4; ++c) {
        const long long need = c < x.n_c ? (long long)x.c[c] * a.smem_caps[a.n_smem_caps - 1] : 0;
        int i = 0;
        while (i < a.n_smem_caps && 100LL * a.smem_caps[i] < need) ++i;
        ct.cap_lo[c] = i;
    }
    for (int R = 0; R < 256; ++R) {
        int warps, wbmax;
        reg_params(a, R, warps, wbmax);
        ct.rwarps[R] = (unsigned short)warps;
        ct.rwbmax[R] = (unsigned short)std::min(wbmax, 65535);
    }
}

// host_cta_tables for the launch's row 0, reusing the last result of the calling thread when the
// row and the axes are the same (compared byte for byte).
void fill_host_tables(EvalParams& q)
{
    struct Last {
        bool valid = false;
        tune_arch a;
        tune_axes x;
        CtaTables t;
    };
    static thread_local Last last;
    if (!last.valid || memcmp(&last.a, &q.a[0], sizeof(tune_arch)) != 0 ||
        memcmp(&last.x, &q.x, sizeof(tune_axes)) != 0) {
        last.a = q.a[0];
        last.x = q.x;
        host_cta_tables(last.a, last.x, last.t);
        last.valid = true;
    }
    q.tab = last.t;
    q.host_tables = 1;
}

// Row 0's tables from the launch parameters into shared memory (a word per thread and step).
__device__ __forceinline__ void copy_cta_tables(const CtaTables& src, CtaTables& ct)
{
    const uint32_t* s = reinterpret_cast<const uint32_t*>(&src);
    uint32_t* d = reinterpret_cast<uint32_t*>(&ct);
    for (int i = threadIdx.x; i < (int)(sizeof(CtaTables) / 4); i += blockDim.x) d[i] = s[i];
}

__device__ void build_cta_tables(const EvalParams& p, const tune_arch& a, CtaTables& ct)
{
    if (p.host_tables) {
        copy_cta_tables(p.tab, ct);
        return;
    }
    const tune_axes& x = p.x;
    for (int i = threadIdx.x; i < kMaxB * 16; i += blockDim.x) {
        int b = i >> 4, g = i & 15;
        float v = __int_as_float(0x7f800000);
        if (b < a.max_blocks_sm && g < x.n_g) {
            int slots = a.n_sm * (b + 1);
            int G = x.g[g];
            int waves = ceil_div(G, slots);
            v = __fdiv_rn((float)(waves * slots), (float)(a.n_sm * G));
        }
        ct.ipar[b][g] = v;
    }
    for (int i = threadIdx.x; i < (kMaxW + 1) * 32; i += blockDim.x) {
        int w = i >> 5, t = i & 31;
        int wb = t < x.n_t ? ceil_div(x.t[t], 32) : 1;
        ct.divt[w][t] = (unsigned char)(w / wb);
    }
    int tid = threadIdx.x;
    if (tid == 0) {
        ct.order_safe = 1;
        const int u = a.smem_alloc_unit;
        ct.unit_shift = (u & (u - 1)) == 0 ? __ffs(u) - 1 : -1;
    }
    __syncthreads();
    if (tid < kMaxB) {  // insertion sort of row tid by (ipar value, g position), in place
        float mn = __int_as_float(0x7f800000);
        for (int g = 0; g < x.n_g; ++g) mn = fminf(mn, ct.ipar[tid][g]);
        ct.iparmin[tid] = mn;
        unsigned char* ord = ct.perm[tid];
        for (int g = 0; g < x.n_g; ++g) {
            const float v = ct.ipar[tid][g];
            int j = g;
            while (j > 0 && ct.ipar[tid][ord[j - 1]] > v) {
                ord[j] = ord[j - 1];
                --j;
            }
            ord[j] = (unsigned char)g;
        }
        // With distinct values this far apart, X * v keeps their order strictly for every
        // X > 0 (no underflow), so a walk in perm order meets equal costs only from
        // equal values, in increasing g (and index) order.
        for (int r = 0; r + 1 < x.n_g; ++r) {
            const float v1 = ct.ipar[tid][ord[r]], v2 = ct.ipar[tid][ord[r + 1]];
            if (v2 != v1 && __fsub_rn(v2, v1) <= __fmul_rn(v1, 0x1p-21f)) ct.order_safe = 0;
        }
    }
    if (tid < 32) {
        int wb = 1, gw = 0;
        float ln = 1.0f;
        if (tid < x.n_t) {
            int T = x.t[tid];
            wb = ceil_div(T, 32);
            gw = T <= a.max_threads_block ? min(a.max_blocks_sm, a.max_warps_sm / wb) : 0;
            ln = __fdiv_rn((float)(32 * wb), (float)T);
        }
        ct.wb[tid] = wb;
        ct.gw[tid] = gw;
        ct.lane[tid] = ln;
    } else if (tid < 32 + kMaxW + 1) {
        int w = tid - 32;
        float h = w > 0 ? __fdiv_rn((float)a.w_sat, (float)w) : 1.0f;
        ct.hide[w] = fmaxf(1.0f, h);
    } else if (tid < 32 + kMaxW + 1 + 8) {
        int c = tid - 32 - kMaxW - 1;
        ct.rcp[c] = c < TUNE_NCLASS ? __fdiv_rn(1.0f, a.ipc[c]) : 0.0f;
    } else if (tid < 32 + kMaxW + 1 + 8 + 4) {
        // capacities are ascending: those at or above index cap_lo satisfy the carveout
        const int c = tid - 32 - kMaxW - 1 - 8;
        const long long need = c < x.n_c ? (long long)x.c[c] * a.smem_caps[a.n_smem_caps - 1] : 0;
        int i = 0;
        while (i < a.n_smem_caps && 100LL * a.smem_caps[i] < need) ++i;
        ct.cap_lo[c] = i;
    }
    for (int R = tid; R < 256; R += blockDim.x) {
        int warps, wbmax;
        reg_params(a, R, warps, wbmax);
        ct.rwarps[R] = (unsigned short)warps;
        ct.rwbmax[R] = (unsigned short)min(wbmax, 65535);
    }
    if (tid < 33) ct.rcpn[tid] = tid > 0 ? __frcp_rn((float)tid) : 0.0f;
}

// q = floor(n / d) for 0 <= n < 2^25 and 1 <= d < 2^25: a single-precision estimate
// (within 2 of q) corrected with exact integer remainders.
__device__ __forceinline__ int udiv_small(int n, int d)
{
    int q = __float2int_rz(__fmul_rn((float)n, __frcp_rn((float)d)));
    int r = n - q * d;
    while (r < 0) {
        --q;
        r += d;
    }
    while (r >= d) {
        ++q;
        r -= d;
    }
    return q;
}

// G_S (Eq. 5) as smem_blocks(), starting the capacity search at the carveout's
// first admissible capacity (carveout position cp).
__device__ __forceinline__ int smem_blocks_from(const tune_arch& a, const CtaTables& ct, int s0, int cp)
{
    if (s0 > a.smem_block_max) return 0;
    const int need = s0 + a.smem_reserved_block;
    const int unit = a.smem_alloc_unit;
    const int s_alloc = ct.unit_shift >= 0 ? ((need + unit - 1) >> ct.unit_shift) << ct.unit_shift
                                           : ceil_div(need, unit) * unit;
    if (s_alloc == 0) return a.max_blocks_sm;
    for (int i = ct.cap_lo[cp]; i < a.n_smem_caps; ++i) {
        const int ci = a.smem_caps[i];
        if (ci >= s_alloc) return udiv_small(ci, s_alloc);
    }
    return 0;
}

// G_R (Eq. 4) for R registers and blocks of W_B warps (t position tp).
__device__ __forceinline__ int reg_blocks(const tune_arch& a, const CtaTables& ct, int R, int wb, int tp,
                                          int warps, int wbmax)
{
    if (R > a.regs_thread_max) return 0;
    if (R <= 0) return a.max_blocks_sm;
    if (a.reg_alloc_mode == 0) return wb > wbmax ? 0 : ct.divt[warps][tp];
    const long long rpb = (long long)ceil_div(R * 32 * wb, a.reg_alloc_unit) * a.reg_alloc_unit;
    return rpb > a.regs_block_max ? 0 : (int)(a.regs_sm / rpb);
}

// Sorted insert of (c, i) into a lane's register list (ascending; strict "<"
// keeps earlier = lower-index entries first among equal costs).
// (cost, index) keys ordered lexicographically; costs are >= 0, so their bit
// patterns order like the values.
__device__ __forceinline__ bool key_less(float c, int i, float c2, int i2)
{
    return c < c2 || (c == c2 && i < i2);
}


template <int N>
struct IntC {
    static constexpr int value = N;
};

// floor(n / d) for 0 <= n < 8192 and 1 <= d <= 32, given rcp = 1/d rounded to
// nearest: (n + 1/2) / d lies at least 1/64 away from an integer, far more than
// the rounding error of the product, so truncation is exact.
__device__ __forceinline__ int small_div(int n, float rcp)
{
    return __float2int_rz(__fmul_rn((float)n + 0.5f, rcp));
}

// Warp-wide top-k list: lane j < k holds the j-th best (cost, index), ascending.
// Inserts one key (the same on every lane); returns nothing, updates the list
// and the k-th key (tau) on every lane.
__device__ __forceinline__ void warp_list_insert(float& lc, int& li, float& tau_c, int& tau_i, float c,
                                                 int i, int k, int lane)
{
    const unsigned below = __ballot_sync(kFull, lane < k && key_less(lc, li, c, i));
    const int pos = __popc(below);
    const float up_c = __shfl_up_sync(kFull, lc, 1);
    const int up_i = __shfl_up_sync(kFull, li, 1);
    if (lane < k) {
        if (lane == pos) {
            lc = c;
            li = i;
        } else if (lane > pos) {
            lc = up_c;
            li = up_i;
        }
    }
    tau_c = __shfl_sync(kFull, lc, k - 1);
    tau_i = __shfl_sync(kFull, li, k - 1);
}

template <bool EMIT, bool MULTI>
__global__ void __maxnreg__(64)
    tune_eval_kernel(const __grid_constant__ EvalParams p, const int4* __restrict__ descs,
                     int32_t* __restrict__ topk_idx, float* __restrict__ topk_cost,
                     int32_t* __restrict__ pt_b, int32_t* __restrict__ pt_w,
                     float* __restrict__ pt_c, const int64_t* __restrict__ pt_off,
                     int* __restrict__ status, unsigned long long* __restrict__ queue)
{
    __shared__ CtaTables ct;
    __shared__ WarpTables wts[kWarps];
    // with several architecture rows, blockIdx.y selects the row; its results and work queue
    // follow those of the rows before it (one row: the row's fields are kernel constants)
    const tune_arch& a = p.a[MULTI ? blockIdx.y : 0];
    if (MULTI) {
        topk_idx += (int64_t)blockIdx.y * p.n_kernels * p.k;
        topk_cost += (int64_t)blockIdx.y * p.n_kernels * p.k;
        queue += blockIdx.y;
    }
    build_cta_tables(p, a, ct);
    __syncthreads();

    const tune_axes& x = p.x;
    const int lane = threadIdx.x & 31;
    WarpTables& w = wts[threadIdx.x >> 5];
    const float kInf = __int_as_float(0x7f800000);
    const int k = p.k;
    const int64_t n_k = p.n_kernels;
    const uint32_t g_ok = (1u << x.n_g) - 1u;

    // Work distribution: a static stride over descriptors, or (chunk > 0) a queue
    // from which each warp takes `chunk` consecutive descriptors at a time. The next
    // descriptor's words, and in queue mode the start of the chunk after the current
    // one, are fetched while the current descriptor is evaluated.
    const int64_t stride = (int64_t)gridDim.x * kWarps;
    unsigned long long grabbed = 0;  // lane 0: start of the next chunk, once grabbed
    auto grab = [&]() {
        if (lane == 0) grabbed = atomicAdd(queue, (unsigned long long)p.chunk);
    };
    int64_t kid, q_end = 0;
    if (p.chunk == 0) {
        kid = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    } else {
        grab();
        kid = (int64_t)__shfl_sync(kFull, grabbed, 0);
        q_end = min(kid + p.chunk, n_k);
        if (kid < n_k) grab();
    }
    // lanes 0..3 hold the four 16-byte words of the descriptor (lane & 3)
    int4 v = kid < n_k ? __ldg(descs + kid * 4 + (lane & 3)) : make_int4(0, 0, 0, 0);
    while (kid < n_k) {
        int64_t nk;
        if (p.chunk == 0) {
            nk = kid + stride;
        } else if (kid + 1 < q_end) {
            nk = kid + 1;
        } else {
            nk = (int64_t)__shfl_sync(kFull, grabbed, 0);
            q_end = min(nk + p.chunk, n_k);
            if (nk < n_k) grab();
        }
        const int4 v_next = nk < n_k ? __ldg(descs + nk * 4 + (lane & 3)) : make_int4(0, 0, 0, 0);

        do {  // evaluate descriptor kid (break = done)
            int4 vw[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                vw[q] = make_int4(__shfl_sync(kFull, v.x, q), __shfl_sync(kFull, v.y, q),
                                  __shfl_sync(kFull, v.z, q), __shfl_sync(kFull, v.w, q));
            Desc kd;
            unpack(vw, kd);
            const int r0 = kd.r0, s0 = kd.s0;
            const uint32_t tm = kd.tm, gm = kd.gm, um = kd.um, cm = kd.cm;
            const bool bad = desc_bad(kd, x);
            const int nT = __popc(tm), nG = __popc(gm), nU = __popc(um), nC = __popc(cm);
            if (bad || nT * nG * nU * nC == 0) {
                if (bad && lane == 0) atomicOr(status, tune::kStatusInvalid);
                if (lane < k) {
                    topk_idx[kid * k + lane] = -1;
                    topk_cost[kid * k + lane] = kInf;
                }
                break;
            }
            const int nUC = nU * nC;
            const int g_stride = nG * nUC;

            // ---- per-axis tables, lane = axis position: per unroll the cost sums and
            // register limits, per carveout G_S.
            const uint32_t below = (1u << lane) - 1u;
            if (lane < 16 && ((gm >> lane) & 1u)) w.gpos[__popc(gm & below)] = lane;
            if (lane < 8 && ((um >> lane) & 1u)) {
                const int ur = __popc(um & below);
                const int U = x.u[lane];
                const int R = r0 + 4 * (U - 1);
                unit_costs(kd.n, kd.d, U, ct.rcp, a.work_scale, w.cnm[ur], w.cm[ur]);
                w.regs[ur] = R;
                int warps, wbmax;
                if (R >= 0 && R < 256) {
                    warps = ct.rwarps[R];
                    wbmax = ct.rwbmax[R];
                } else {
                    reg_params(a, R, warps, wbmax);
                }
                w.ru[ur] = warps | (wbmax << 8);
            }
            if (lane < 4 && ((cm >> lane) & 1u)) w.gs[__popc(cm & below)] = smem_blocks_from(a, ct, s0, lane);
            // Per-warp register allocation with R > 0 for every unroll (r0 > 0): the (T, U)
            // block limit is min(G_W, W_B > wbmax ? 0 : floor(warps / W_B)) and is formed
            // where it is used; otherwise (per-block allocation, R = 0) it is tabulated.
            const bool simple = !EMIT && a.reg_alloc_mode == 0 && r0 > 0;
            __syncwarp();
            // ---- per thread count (lane = t position): W_B, lane efficiency, G_W by t rank
            // (and the tabulated block limit min(G_W, G_R)).
            if ((tm >> lane) & 1u) {
                const int tr = __popc(tm & below);
                const int wb = ct.wb[lane];
                const int gw = ct.gw[lane];
                w.tinfo[tr] = make_int4(wb, __float_as_int(ct.lane[lane]), lane, gw);
                if (!simple) {
                    for (int ur = 0; ur < nU; ++ur) {
                        const int ru = w.ru[ur];
                        const int gr = reg_blocks(a, ct, w.regs[ur], wb, lane, ru & 0xff, ru >> 8);
                        w.gwr[tr][ur] = (unsigned char)min(gw, gr);
                    }
                }
            }
            // min(G_W, G_R) of (t rank, u rank); ti = tinfo[t rank]
            auto block_limit = [&](int t_r, const int4& ti, int u_r) -> int {
                if (!simple) return w.gwr[t_r][u_r];
                const int ru = w.ru[u_r];
                return min(ti.w, ti.x > (ru >> 8) ? 0 : (int)ct.divt[ru & 0xff][ti.z]);
            };
            // ---- (U, C) pair table for the emitting pass; lane = pair rank.
            if (EMIT && lane < nUC) {
                const int ur = lane / nC, cr = lane - (lane / nC) * nC;
                w.uc[lane] = make_float4(w.cnm[ur], w.cm[ur], __int_as_float(ur), __int_as_float(w.gs[cr]));
            }
            // ---- waves/slots factor rows, compacted to this kernel's grid sizes, and
            // their minima.
            const bool g_dense = gm == g_ok;
            if (lane == 0) w.iparmin[0] = __int_as_float(0x7fc00000);  // B* = 0: no valid configuration
            if (lane < kMaxB) {
                if (g_dense) {
                    w.iparmin[lane + 1] = ct.iparmin[lane];
                } else if (EMIT) {
                    float mn = kInf;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float f = j < nG ? ct.ipar[lane][w.gpos[j]] : kInf;
                        w.iparc[lane][j] = f;
                        mn = fminf(mn, f);
                    }
                    w.iparmin[lane + 1] = mn;
                } else {
                    // the kernel's nG grid sizes only (a warp-uniform trip count)
                    const float* row = ct.ipar[lane];
                    float mn = kInf;
                    for (int j = 0; j < nG; ++j) mn = fminf(mn, row[w.gpos[j]]);
                    w.iparmin[lane + 1] = mn;
                }
            }
            __syncwarp();

            float lc = kInf;  // this lane's entry of the warp's top-k list (lanes < k)
            int li = -1;
            float tau_c = kInf;  // the list's k-th key
            int tau_i = -1;
            float tau0 = kInf;   // bound from the pre-pass

            // Merge: each candidate lane walks its triple's grid sizes in increasing
            // cost (the order of X * ipar(B*, G) over G depends on B* only); the warp
            // repeatedly takes the smallest head and inserts it while it beats the k-th
            // entry. A lane's walk is in (cost, index) order unless two nearly equal
            // ipar values round to one cost, or X underflows; then (relaxed) equal
            // costs are walked on until a head costs more than the k-th entry.
            auto merge = [&](bool any, int B, float X, int base) {
                const bool relaxed = !ct.order_safe || __any_sync(kFull, any && !(X >= 0x1p-100f));
                int r = 0;
                float hc = kInf;
                int hi = 0x7fffffff;
                auto advance = [&]() {
                    hc = kInf;
                    hi = 0x7fffffff;
                    if (g_dense) {  // every axis grid size present: rank = position
                        if (r < x.n_g) {
                            const int g = ct.perm[B - 1][r++];
                            hc = __fmul_rn(X, ct.ipar[B - 1][g]);
                            hi = base + g * nUC;
                        }
                        return;
                    }
                    while (r < x.n_g) {
                        const int g = ct.perm[B - 1][r++];
                        if ((gm >> g) & 1u) {
                            hc = __fmul_rn(X, ct.ipar[B - 1][g]);
                            hi = base + __popc(gm & ((1u << g) - 1u)) * nUC;
                            break;
                        }
                    }
                };
                if (any) advance();
                for (;;) {
                    const unsigned mc = __reduce_min_sync(kFull, __float_as_uint(hc));
                    const float mcf = __uint_as_float(mc);
                    const unsigned mi = __reduce_min_sync(kFull, hc == mcf ? (unsigned)hi : 0xffffffffu);
                    if (mc >= 0x7f800000u || mcf > tau0 || mcf > tau_c) break;
                    const bool enters = key_less(mcf, (int)mi, tau_c, tau_i);
                    if (!enters && !relaxed) break;
                    if (enters) warp_list_insert(lc, li, tau_c, tau_i, mcf, (int)mi, k, lane);
                    if (hc == mcf && hi == (int)mi) advance();
                }
            };

            if (!EMIT) {
                // ---- pre-pass over (T, U) pairs, lane = pair rank mod 32, carveouts inner.
                // Every grid size G of a triple costs X(T,U,C) * ipar(B*, G); a product by
                // X > 0 is monotone under round-to-nearest, so the triple's cheapest point
                // is exactly X * min_G ipar(B*, G). Each lane keeps the two smallest pair minima
                // (the smallest triple minimum over a (T, U) pair's carveouts) of its pairs, each
                // with its multiplicity (the pair's carveouts whose minimum equals it: the
                // carveouts of a pair often share B* and so their cost); tau0 is the smallest
                // value at which these entries, in increasing order, count k triples, and so
                // bounds the kernel's k-th best cost (k distinct triples each own a point
                // <= tau0). Each minimum is also stored at its triple rank (t rank * nUC +
                // u rank * nC + c rank), so that the carveouts of one (T, U) pair sit in
                // neighbouring lanes of the scan.
                const int nP = nT * nU;
                const int n_prow = (nP + 31) >> 5;
                const int n_blk = (nP * nC + 127) >> 7;  // blocks of 128 triples for the scan
                const float rcp_u = ct.rcpn[nU], rcp_c = ct.rcpn[nC], rcp_uc = ct.rcpn[nUC];
                {  // tail of the last block: no triple (NaN)
                    const float nan = __int_as_float(0x7fc00000);
                    *reinterpret_cast<float4*>(&w.key[((n_blk - 1) << 7) + 4 * lane]) = make_float4(nan, nan, nan, nan);
                }
                __syncwarp();
                float m0 = kInf, m1 = kInf;  // this lane's two smallest pair minima, ascending
                int c0 = 0, c1 = 0;          // their multiplicities
                // one body per carveout count, so that G_S stays in registers and a pair's
                // minima are stored with one vector store
                auto pairs = [&](auto nc_tag) {
                    constexpr int NC = decltype(nc_tag)::value;
                    int gs[NC];
#pragma unroll
                    for (int c = 0; c < NC; ++c) gs[c] = w.gs[c];
                    // pair pr = lane + 32 j = t_r nU + u_r, advanced by 32 pairs per step
                    const int dq = small_div(32, rcp_u), dr = 32 - dq * nU;
                    int t_r = small_div(lane, rcp_u), u_r = lane - t_r * nU;
                    for (int j = 0; j < n_prow; ++j, t_r += dq, u_r += dr) {
                        const int pr = lane + (j << 5);
                        if (pr >= nP) break;
                        if (u_r >= nU) {
                            u_r -= nU;
                            ++t_r;
                        }
                        const int4 ti = w.tinfo[t_r];
                        const int wb = ti.x;
                        const float ln = __int_as_float(ti.y);
                        const int gwr = block_limit(t_r, ti, u_r);
                        const float cnm = w.cnm[u_r], cmv = w.cm[u_r];
                        float key[NC];
                        float pm = kInf;
#pragma unroll
                        for (int c = 0; c < NC; ++c) {
                            // branch-free: a triple without a valid configuration (B* = 0) reads
                            // hide[0] and iparmin[0] = NaN, so it is keyed NaN (never a
                            // candidate, not counted in the bound); W* = B* W_B <= W_mp <= kMaxW
                            // for a valid triple. X is finite (counts <= 2^40).
                            const int B = min(gwr, gs[c]);
                            const float X = __fmul_rn(__fmaf_rn(cmv, ct.hide[B * wb], cnm), ln);
                            key[c] = __fmul_rn(X, w.iparmin[B]);
                            pm = fminf(pm, key[c]);
                        }
                        int mult = 0;
#pragma unroll
                        for (int c = 0; c < NC; ++c) mult += key[c] == pm ? 1 : 0;
                        {
                            const bool lt0 = pm < m0, lt1 = pm < m1;
                            m1 = lt0 ? m0 : (lt1 ? pm : m1);
                            c1 = lt0 ? c0 : (lt1 ? mult : c1);
                            m0 = lt0 ? pm : m0;
                            c0 = lt0 ? mult : c0;
                        }
                        float* krow = &w.key[pr * NC];
                        if constexpr (NC == 4) {
                            *reinterpret_cast<float4*>(krow) = make_float4(key[0], key[1], key[2], key[3]);
                        } else if constexpr (NC == 2) {
                            *reinterpret_cast<float2*>(krow) = make_float2(key[0], key[1]);
                        } else {
#pragma unroll
                            for (int c = 0; c < NC; ++c) krow[c] = key[c];
                        }
                    }
                };
                switch (nC) {
                    case 1: pairs(IntC<1>{}); break;
                    case 2: pairs(IntC<2>{}); break;
                    case 3: pairs(IntC<3>{}); break;
                    default: pairs(IntC<4>{}); break;
                }
                __syncwarp();
                // entries in increasing order until they count k triples (at most 64 rounds; a
                // finite entry counts at least one triple; +inf: fewer than k valid triples)
                for (int need = k;;) {
                    const unsigned mb = __reduce_min_sync(kFull, __float_as_uint(m0));
                    tau0 = __uint_as_float(mb);
                    if (mb >= 0x7f800000u) break;
                    const int src = __ffs(__ballot_sync(kFull, __float_as_uint(m0) == mb)) - 1;
                    need -= __shfl_sync(kFull, c0, src);
                    if (need <= 0) break;
                    const bool me = lane == src;  // the lane whose smallest was taken
                    m0 = me ? m1 : m0;
                    c0 = me ? c1 : c0;
                    m1 = me ? kInf : m1;
                    c1 = me ? 0 : c1;
                }

                // ---- candidates: the triples whose minimum does not exceed tau0 (every point
                // of the top-k belongs to one), four per lane and 128 per step. Their ranks
                // are compacted in place to the front of the key array: a slot written in
                // block b lies in blocks <= b, whose keys every lane has read before the
                // ballot.
                int n_cand = 0;
                for (int b = 0; b < n_blk; ++b) {
                    const int t0 = (b << 7) + 4 * lane;  // this lane's four triples
                    const float4 kv = *reinterpret_cast<const float4*>(&w.key[t0]);
                    const unsigned m = (kv.x <= tau0 ? 1u : 0u) | (kv.y <= tau0 ? 2u : 0u) |
                                       (kv.z <= tau0 ? 4u : 0u) | (kv.w <= tau0 ? 8u : 0u);
                    if (__ballot_sync(kFull, m != 0u) == 0u) continue;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const unsigned bj = __ballot_sync(kFull, (m >> j) & 1u);
                        if ((m >> j) & 1u) w.key[n_cand + __popc(bj & below)] = __int_as_float(t0 + j);
                        n_cand += __popc(bj);
                    }
                }
                __syncwarp();

                // ---- selection: candidate triples 32 at a time, one per lane; each lane walks
                // its triple's grid sizes in increasing cost. The first batch starts from an
                // empty list, so its points, extracted in increasing cost, are appended at
                // list positions 0, 1, ... (a point that comes out of index order among equal
                // costs is inserted at its place instead); later batches merge into the list.
                for (int c0 = 0; c0 < n_cand; c0 += 32) {
                    const bool has = c0 + lane < n_cand;
                    int B = 0, base = 0;
                    float X = 0.0f;
                    if (has) {
                        const int tri = __float_as_int(w.key[c0 + lane]);
                        const int t_r = small_div(tri, rcp_uc);
                        const int uc_r = tri - t_r * nUC;
                        const int u_r = small_div(uc_r, rcp_c);
                        const int c = uc_r - u_r * nC;
                        const int4 ti = w.tinfo[t_r];
                        B = min(block_limit(t_r, ti, u_r), w.gs[c]);
                        X = __fmul_rn(__fmaf_rn(w.cm[u_r], ct.hide[B * ti.x], w.cnm[u_r]), __int_as_float(ti.y));
                        base = t_r * g_stride + uc_r;
                    }
                    if (c0 > 0) {
                        merge(has, B, X, base);
                        continue;
                    }
                    int rg = 0;
                    float hc = kInf;
                    int hi = 0x7fffffff;
                    auto advance = [&]() {
                        if (g_dense) {  // every axis grid size present: rank = position
                            if (rg < x.n_g) {
                                const int g = ct.perm[B - 1][rg++];
                                hc = __fmul_rn(X, ct.ipar[B - 1][g]);
                                hi = base + g * nUC;
                            } else {
                                hc = kInf;
                                hi = 0x7fffffff;
                            }
                            return;
                        }
                        hc = kInf;
                        hi = 0x7fffffff;
                        while (rg < x.n_g) {
                            const int g = ct.perm[B - 1][rg++];
                            if ((gm >> g) & 1u) {
                                hc = __fmul_rn(X, ct.ipar[B - 1][g]);
                                hi = base + __popc(gm & ((1u << g) - 1u)) * nUC;
                                break;
                            }
                        }
                    };
                    if (has) advance();
                    const bool relaxed = !ct.order_safe || __any_sync(kFull, has && !(X >= 0x1p-100f));
                    if (!relaxed) {
                        // every lane's walk is in (cost, index) order: the r-th extraction is the
                        // r-th best of the batch (points above tau0 cannot be among the top k)
                        for (int r = 0; r < k;) {
                            const unsigned mc = __reduce_min_sync(kFull, __float_as_uint(hc));
                            const float mcf = __uint_as_float(mc);
                            if (mc >= 0x7f800000u || mcf > tau0) break;
                            const bool tie = hc == mcf;
                            if (g_dense) {
                                // every lane's next head, straight-line (B and the position are
                                // clamped into range for lanes without one)
                                const int Bv = max(B, 1) - 1;
                                const int g = ct.perm[Bv][min(rg, x.n_g - 1)];
                                const bool more = rg < x.n_g;
                                const float nc = more ? __fmul_rn(X, ct.ipar[Bv][g]) : kInf;
                                const int ni = more ? base + g * nUC : 0x7fffffff;
                                // Heads of the smallest cost whose index is below every equal-cost
                                // next head are the next points in (cost, index) order, all of them
                                // (each walk is in that order). Where their indices rise with the
                                // lane, as they mostly do (candidates are in triple order), the
                                // first m go to list positions r.. at once through shared memory.
                                const unsigned bound =
                                    __reduce_min_sync(kFull, tie && nc == mcf ? (unsigned)ni : 0xffffffffu);
                                const bool elig = tie && (unsigned)hi < bound;
                                const unsigned before = __ballot_sync(kFull, elig) & below;
                                const int hprev = __shfl_sync(kFull, hi, before ? 31 - __clz(before) : lane);
                                if (__all_sync(kFull, !elig || !before || hprev < hi)) {
                                    const int m = min(__popc(__ballot_sync(kFull, elig)), k - r);
                                    const int rank = __popc(before);
                                    const bool take = elig && rank < m;
                                    // w.iparmin is free during the selection: [j] cost, [16 + j] index
                                    if (take) {
                                        w.iparmin[rank] = hc;
                                        w.iparmin[16 + rank] = __int_as_float(hi);
                                    }
                                    __syncwarp();
                                    if (lane >= r && lane < r + m) {
                                        lc = w.iparmin[lane - r];
                                        li = __float_as_int(w.iparmin[16 + lane - r]);
                                    }
                                    __syncwarp();
                                    hc = take ? nc : hc;
                                    hi = take ? ni : hi;
                                    rg += take ? 1 : 0;
                                    r += m;
                                    continue;
                                }
                                // indices out of lane order: one point, the lowest index
                                const unsigned mi = __reduce_min_sync(kFull, tie ? (unsigned)hi : 0xffffffffu);
                                lc = lane == r ? mcf : lc;
                                li = lane == r ? (int)mi : li;
                                const bool win = tie && hi == (int)mi;
                                hc = win ? nc : hc;
                                hi = win ? ni : hi;
                                rg += win ? 1 : 0;
                                ++r;
                                continue;
                            }
                            const unsigned mi = __reduce_min_sync(kFull, tie ? (unsigned)hi : 0xffffffffu);
                            lc = lane == r ? mcf : lc;
                            li = lane == r ? (int)mi : li;
                            if (tie && hi == (int)mi) advance();
                            ++r;
                        }
                        tau_c = __shfl_sync(kFull, lc, k - 1);
                        tau_i = __shfl_sync(kFull, li, k - 1);
                        continue;
                    }
                    int cnt = 0;  // list entries so far; (prev_c, prev_i) is the largest
                    float prev_c = 0.0f;
                    int prev_i = -1;
                    for (;;) {
                        const unsigned mc = __reduce_min_sync(kFull, __float_as_uint(hc));
                        const float mcf = __uint_as_float(mc);
                        if (mc >= 0x7f800000u || mcf > tau0 || mcf > tau_c) break;
                        const unsigned mi = __reduce_min_sync(kFull, hc == mcf ? (unsigned)hi : 0xffffffffu);
                        if (cnt == k && !relaxed && !key_less(mcf, (int)mi, tau_c, tau_i)) break;
                        if (cnt < k && (cnt == 0 || key_less(prev_c, prev_i, mcf, (int)mi))) {
                            if (lane == cnt) {  // in order: append
                                lc = mcf;
                                li = (int)mi;
                            }
                            prev_c = mcf;
                            prev_i = (int)mi;
                            if (++cnt == k) {
                                tau_c = __shfl_sync(kFull, lc, k - 1);
                                tau_i = __shfl_sync(kFull, li, k - 1);
                            }
                        } else if (key_less(mcf, (int)mi, tau_c, tau_i)) {
                            // out of index order among equal costs: insert at its place
                            warp_list_insert(lc, li, tau_c, tau_i, mcf, (int)mi, k, lane);
                            if (cnt < k && ++cnt == k) {
                                tau_c = __shfl_sync(kFull, lc, k - 1);
                                tau_i = __shfl_sync(kFull, li, k - 1);
                            }
                        }
                        if (hc == mcf && hi == (int)mi) advance();
                    }
                }
            } else {
                // ---- emitting pass: every point's B*, W* and cost is written; lanes walk
                // (T, U, C) triples, the t rank advancing by 32 / nUC per step.
                const float* ipar_rows = g_dense ? &ct.ipar[0][0] : &w.iparc[0][0];
                const int t0 = lane / nUC, uc0 = lane - (lane / nUC) * nUC;
                const int dq = 32 / nUC, dr = 32 - (32 / nUC) * nUC;
                const int n_iter = (nT * nUC + 31) >> 5;
                const int64_t off = pt_off[kid];
                int t_r = t0, uc_r = uc0;
                for (int it = 0; it < n_iter; ++it) {
                    bool any = false;
                    float X = 0.0f;
                    int B = 0, base = 0;
                    if (t_r < nT) {
                        const float4 ucv = w.uc[uc_r];
                        const int ur = __float_as_int(ucv.z);
                        const int4 ti = w.tinfo[t_r];
                        B = min((int)w.gwr[t_r][ur], __float_as_int(ucv.w));
                        const int W = B * ti.x;
                        X = __fmul_rn(__fmaf_rn(ucv.y, ct.hide[W], ucv.x), __int_as_float(ti.y));
                        base = t_r * g_stride + uc_r;
                        if (B > 0) {
                            const float* row = ipar_rows + (B - 1) * kIparStride;
                            any = __fmul_rn(X, w.iparmin[B]) <= tau_c;
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                if (j < nG) {
                                    const int64_t at = off + base + j * nUC;
                                    if (pt_b) pt_b[at] = B;
                                    if (pt_w) pt_w[at] = W;
                                    if (pt_c) pt_c[at] = __fmul_rn(X, row[j]);
                                }
                            }
                        } else {
                            for (int j = 0; j < nG; ++j) {
                                const int64_t at = off + base + j * nUC;
                                if (pt_b) pt_b[at] = 0;
                                if (pt_w) pt_w[at] = 0;
                                if (pt_c) pt_c[at] = kInf;
                            }
                        }
                        t_r += dq;
                        uc_r += dr;
                        if (uc_r >= nUC) {
                            uc_r -= nUC;
                            ++t_r;
                        }
                    }
                    if (__ballot_sync(kFull, any) == 0u) continue;
                    merge(any, B, X, base);
                }
            }

            if (lane < k) {
                topk_idx[kid * k + lane] = li;
                topk_cost[kid * k + lane] = lc;
            }
        } while (false);
        __syncwarp();  // the warp's tables are rewritten for the next descriptor
        kid = nk;
        v = v_next;
    }
}

// ---- thread-per-kernel schedule ---------------------------------------------
//
// One thread evaluates one kernel descriptor: per-unroll tables in shared
// memory (one column per thread), per-carveout limits packed in a register,
// then a bound pre-pass and the main pass over (T, U, C) triples with every
// grid size's cost computed. The thread keeps a sorted register list of its k
// best (cost, index); no warp collectives are involved, so kernels of any
// space size run without per-kernel warp overhead.

constexpr int kThreadsT = 128;

template <int KMAX>
__device__ __forceinline__ void tlist_insert(float (&lc)[KMAX], int (&li)[KMAX], float c, int i)
{
#pragma unroll
    for (int j = KMAX - 1; j > 0; --j) {
        const bool shift = key_less(c, i, lc[j - 1], li[j - 1]);
        const bool here = !shift && key_less(c, i, lc[j], li[j]);
        const float nc = shift ? lc[j - 1] : (here ? c : lc[j]);
        const int ni = shift ? li[j - 1] : (here ? i : li[j]);
        lc[j] = nc;
        li[j] = ni;
    }
    if (key_less(c, i, lc[0], li[0])) {
        lc[0] = c;
        li[0] = i;
    }
}

template <int KMAX, typename V>
__device__ __forceinline__ V list_kth(const V (&l)[KMAX], int k)
{
    // Select chain (not l[k - 1], which would force the list into local memory).
    V t = l[KMAX - 1];
#pragma unroll
    for (int j = KMAX - 2; j >= 0; --j) t = (j >= k - 1) ? l[j] : t;
    return t;
}

// Sorted insert of a value into an ascending list, dropping the largest.
template <int KMAX>
__device__ __forceinline__ void value_insert(float (&l)[KMAX], float v)
{
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
        const float lo = fminf(l[j], v);
        v = fmaxf(l[j], v);
        l[j] = lo;
    }
}

template <int KMAX>
__global__ void __maxnreg__(KMAX > 8 ? 128 : 96)
    tune_eval_thread_kernel(const __grid_constant__ EvalParams p, const int4* __restrict__ descs,
                            int32_t* __restrict__ topk_idx, float* __restrict__ topk_cost,
                            int* __restrict__ status)
{
    __shared__ CtaTables ct;
    __shared__ float4 utab[8][kThreadsT];  // per unroll position: C_nm, C_m, R, warps | wbmax << 8
    const tune_arch& a = p.a[0];
    build_cta_tables(p, a, ct);
    __syncthreads();

    const tune_axes& x = p.x;
    const float kInf = __int_as_float(0x7f800000);
    const int k = p.k;
    const int tid = threadIdx.x;
    const uint32_t g_all = (1u << x.n_g) - 1u;

    for (int64_t kid = (int64_t)blockIdx.x * kThreadsT + tid; kid < p.n_kernels;
         kid += (int64_t)gridDim.x * kThreadsT) {
        int4 vw[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) vw[q] = __ldg(descs + kid * 4 + q);
        Desc kd;
        unpack(vw, kd);
        const uint32_t tm = kd.tm, gm = kd.gm, um = kd.um, cm = kd.cm;
        const bool bad = desc_bad(kd, x);
        const int nT = __popc(tm), nG = __popc(gm), nU = __popc(um), nC = __popc(cm);
        if (bad || nT * nG * nU * nC == 0) {
            if (bad) atomicOr(status, tune::kStatusInvalid);
            for (int j = 0; j < k; ++j) {
                topk_idx[kid * k + j] = -1;
                topk_cost[kid * k + j] = kInf;
            }
            continue;
        }
        const int nUC = nU * nC;
        const int g_stride = nG * nUC;
        const bool g_dense = gm == g_all;

        // ---- per-unroll and per-carveout tables
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if ((um >> u) & 1u) {
                const int U = x.u[u];
                const int R = kd.r0 + 4 * (U - 1);
                float cnm, cmv;
                unit_costs(kd.n, kd.d, U, ct.rcp, a.work_scale, cnm, cmv);
                int warps, wbmax;
                reg_params(a, R, warps, wbmax);
                utab[u][tid] = make_float4(cnm, cmv, __int_as_float(R),
                                           __int_as_float(warps | (min(wbmax, 255) << 8)));
            }
        }
        uint32_t gsp = 0;  // G_S per carveout position, one byte each
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if ((cm >> c) & 1u) gsp |= (uint32_t)min(smem_blocks(a, kd.s0, x.c[c]), 255) << (8 * c);

        // ---- loop nest over the triples in canonical (T, U, C) order; body(B, W, X, base)
        auto for_triples = [&](auto&& body) {
            int t_r = 0;
            for (uint32_t tb = tm; tb; tb &= tb - 1u, ++t_r) {
                const int tp = __ffs(tb) - 1;
                const int wb = ct.wb[tp], gw = ct.gw[tp];
                const float ln = ct.lane[tp];
                int u_r = 0;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (!((um >> u) & 1u)) continue;
                    const float4 ut = utab[u][tid];
                    const int wr = __float_as_int(ut.w);
                    const int bu = min(gw, reg_blocks(a, ct, __float_as_int(ut.z), wb, tp, wr & 0xff, wr >> 8));
                    int c_r = 0;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        if (!((cm >> c) & 1u)) continue;
                        const int B = min(bu, (int)((gsp >> (8 * c)) & 0xffu));
                        if (B > 0) {
                            const int W = B * wb;
                            const float X = __fmul_rn(__fmaf_rn(ut.y, ct.hide[W], ut.x), ln);
                            body(B, X, t_r * g_stride + u_r * nC + c_r);
                        }
                        ++c_r;
                    }
                    ++u_r;
                }
            }
        };

        // ---- pre-pass: tau0 = k-th smallest triple minimum (k distinct triples each
        // own a point of cost <= tau0, so the k-th best point is <= tau0).
        float tk[KMAX];
#pragma unroll
        for (int j = 0; j < KMAX; ++j) tk[j] = kInf;
        float tau0 = kInf;
        for_triples([&](int B, float X, int) {
            float mn;
            if (g_dense) {
                mn = ct.iparmin[B - 1];
            } else {
                mn = kInf;
                for (uint32_t gb = gm; gb; gb &= gb - 1u) mn = fminf(mn, ct.ipar[B - 1][__ffs(gb) - 1]);
            }
            const float m = __fmul_rn(X, mn);
            if (m < tau0) {
                value_insert<KMAX>(tk, m);
                tau0 = list_kth<KMAX>(tk, k);
            }
        });

        // ---- main pass: every point's cost, folded into its triple's minimum;
        // points that can still enter the list are inserted exactly.
        float lc[KMAX];
        int li[KMAX];
#pragma unroll
        for (int j = 0; j < KMAX; ++j) {
            lc[j] = kInf;
            li[j] = -1;
        }
        float thr_c = kInf;
        int thr_i = -1;
        for_triples([&](int B, float X, int base) {
            if (g_dense) {
                // the triple's cheapest point (a product by X > 0 keeps the order of ipar)
                const float cmin = __fmul_rn(X, ct.iparmin[B - 1]);
                if (cmin <= fminf(thr_c, tau0)) {
                    // grid sizes in increasing cost: the order of ipar(B*, G) over G
#pragma unroll 1
                    for (int r = 0; r < x.n_g; ++r) {
                        const int g = ct.perm[B - 1][r];
                        const float cg = __fmul_rn(X, ct.ipar[B - 1][g]);
                        if (cg > fminf(thr_c, tau0)) break;
                        const int idx = base + g * nUC;
                        if (key_less(cg, idx, thr_c, thr_i)) {
                            tlist_insert<KMAX>(lc, li, cg, idx);
                            thr_c = list_kth<KMAX>(lc, k);
                            thr_i = list_kth<KMAX>(li, k);
                        }
                    }
                }
            } else {
                int g_r = 0;
                for (uint32_t gb = gm; gb; gb &= gb - 1u, ++g_r) {
                    const float cg = __fmul_rn(X, ct.ipar[B - 1][__ffs(gb) - 1]);
                    if (cg <= fminf(thr_c, tau0)) {
                        const int idx = base + g_r * nUC;
                        if (key_less(cg, idx, thr_c, thr_i)) {
                            tlist_insert<KMAX>(lc, li, cg, idx);
                            thr_c = list_kth<KMAX>(lc, k);
                            thr_i = list_kth<KMAX>(li, k);
                        }
                    }
                }
            }
        });
#pragma unroll
        for (int j = 0; j < KMAX; ++j) {
            if (j < k) {
                topk_idx[kid * k + j] = li[j];
                topk_cost[kid * k + j] = lc[j];
            }
        }
    }
}

template <int KMAX>
int launch_thread(const EvalParams& p, const tune_kernel_desc* descs, int32_t* ti, float* tc, int* status,
                  cudaStream_t s)
{
    auto kern = tune_eval_thread_kernel<KMAX>;
    static std::atomic<int> per_sm_cache[tune::kMaxDevices];
    int per_sm = 0;
    int rc = tune::blocks_per_sm(per_sm_cache, reinterpret_cast<const void*>(kern), kThreadsT, &per_sm);
    if (rc) return rc;
    const int sms = tune::device_sm_count();
    if (sms <= 0) return tune::fail(TUNE_ECUDA, "tune_eval: cannot query the SM count");
    const int64_t need = (p.n_kernels + kThreadsT - 1) / kThreadsT;
    const int64_t cap = (int64_t)sms * per_sm;
    const int grid = (int)(need < cap ? need : cap);
    EvalParams q = p;
    fill_host_tables(q);
    kern<<<grid, kThreadsT, 0, s>>>(q, reinterpret_cast<const int4*>(descs), ti, tc, status);
    TUNE_CUDA_TRY(cudaGetLastError(), "tune_eval: kernel launch");
    return TUNE_OK;
}

template <bool EMIT, bool MULTI>
int launch_rows(const EvalParams& p, const tune_kernel_desc* descs, int32_t* ti, float* tc, int32_t* pb,
                int32_t* pw, float* pc, const int64_t* po, int* status, cudaStream_t s, int ctas_per_sm,
                unsigned long long* queue)
{
    auto kern = tune_eval_kernel<EMIT, MULTI>;
    static std::atomic<int> per_sm_cache[tune::kMaxDevices];
    int per_sm = 0;
    int rc = tune::blocks_per_sm(per_sm_cache, reinterpret_cast<const void*>(kern), kThreads, &per_sm);
    if (rc) return rc;
    const int sms = tune::device_sm_count();
    if (sms <= 0) return tune::fail(TUNE_ECUDA, "tune_eval: cannot query the SM count");
    const int64_t need = (p.n_kernels + kWarps - 1) / kWarps;
    // a persistent grid shared by the architecture rows (blockIdx.y)
    int64_t cap = (int64_t)sms * (ctas_per_sm > 0 ? min(ctas_per_sm, per_sm) : per_sm) / p.n_arch;
    if (cap < 1) cap = 1;
    const int grid = (int)(need < cap ? need : cap);
    // By default the queue counters (one per row) follow the status word in the zeroed
    // workspace header.
    if (!queue) queue = reinterpret_cast<unsigned long long*>(status) + 1;
    EvalParams q = p;
    q.host_tables = 0;
    if (!MULTI) fill_host_tables(q);
    kern<<<dim3(grid, p.n_arch), kThreads, 0, s>>>(q, reinterpret_cast<const int4*>(descs), ti, tc, pb, pw, pc, po,
                                                  status, queue);
    TUNE_CUDA_TRY(cudaGetLastError(), "tune_eval: kernel launch");
    return TUNE_OK;
}

template <bool EMIT>
int launch(const EvalParams& p, const tune_kernel_desc* descs, int32_t* ti, float* tc, int32_t* pb,
           int32_t* pw, float* pc, const int64_t* po, int* status, cudaStream_t s, int ctas_per_sm = 0,
           unsigned long long* queue = nullptr)
{
    return p.n_arch > 1 ? launch_rows<EMIT, true>(p, descs, ti, tc, pb, pw, pc, po, status, s, ctas_per_sm, queue)
                        : launch_rows<EMIT, false>(p, descs, ti, tc, pb, pw, pc, po, status, s, ctas_per_sm, queue);
}

int validate(const tune_arch* a, const tune_axes* x, int32_t k)
{
    if (k < 1 || k > 16) return tune::fail(TUNE_EINVAL, "k = %d outside [1, 16]", k);
    return tune::validate_inputs(a, x);
}

}  // namespace

namespace tune {

int validate_inputs(const tune_arch* a, const tune_axes* x)
{
    if (!a || !x) return fail(TUNE_EINVAL, "arch and axes must be non-NULL host pointers");
    if (a->warp_size != 32) return fail(TUNE_EINVAL, "warp_size must be 32");
    if (a->n_sm < 1 || a->max_threads_block < 1 || a->max_warps_sm < 1 || a->max_warps_sm > kMaxW ||
        a->max_blocks_sm < 1 || a->max_blocks_sm > kMaxB)
        return fail(TUNE_EINVAL, "arch: n_sm, max_threads_block, max_warps_sm (<=64) or "
                                 "max_blocks_sm (<=32) out of range");
    if (a->regs_sm < 1 || a->regs_block_max < 1 || a->regs_thread_max < 1 ||
        a->regs_thread_max > 65536 || a->reg_alloc_unit < 1 || a->reg_alloc_unit > 65536 ||
        a->warp_alloc_gran < 1 || (a->reg_alloc_mode != 0 && a->reg_alloc_mode != 1))
        return fail(TUNE_EINVAL, "arch: register fields out of range");
    if (a->smem_block_max < 0 || a->smem_block_max > (1 << 24) || a->smem_reserved_block < 0 ||
        a->smem_reserved_block > (1 << 24) || a->smem_alloc_unit < 1 || a->smem_alloc_unit > (1 << 20) ||
        a->n_smem_caps < 1 || a->n_smem_caps > 16)
        return fail(TUNE_EINVAL, "arch: shared-memory fields out of range");
    for (int i = 0; i < a->n_smem_caps; ++i)
        if (a->smem_caps[i] < 0 || (i > 0 && a->smem_caps[i] < a->smem_caps[i - 1]) ||
            a->smem_caps[i] > (1 << 24))
            return fail(TUNE_EINVAL, "arch: smem_caps must be ascending, in [0, 16 MB]");
    for (int c = 0; c < TUNE_NCLASS; ++c)
        if (!(a->ipc[c] >= 0x1p-16f) || !isfinite(a->ipc[c]))
            return fail(TUNE_EINVAL, "arch: ipc[%d] must be finite and >= 2^-16", c);
    if (a->w_sat < 1 || a->w_sat > (1 << 20) || a->work_scale < 1 || a->work_scale > (1 << 24))
        return fail(TUNE_EINVAL, "arch: w_sat or work_scale out of range");
    if (x->n_t < 1 || x->n_t > 32 || x->n_g < 1 || x->n_g > 16 || x->n_u < 1 || x->n_u > 8 ||
        x->n_c < 1 || x->n_c > 4)
        return fail(TUNE_EINVAL, "axes: lengths out of range");
    for (int i = 0; i < x->n_t; ++i)
        if (x->t[i] < 1 || x->t[i] > 4096) return fail(TUNE_EINVAL, "axes: t[%d] outside [1, 4096]", i);
    for (int i = 0; i < x->n_g; ++i) {
        if (x->g[i] < 1 || (int64_t)a->n_sm * x->g[i] >= (1 << 24) ||
            (int64_t)x->g[i] + (int64_t)a->n_sm * a->max_blocks_sm >= (1 << 24))
            return fail(TUNE_EINVAL, "axes: g[%d] must be >= 1 with n_sm * g < 2^24", i);
    }
    for (int i = 0; i < x->n_u; ++i)
        if (x->u[i] < 1 || x->u[i] > 64) return fail(TUNE_EINVAL, "axes: u[%d] outside [1, 64]", i);
    for (int i = 0; i < x->n_c; ++i)
        if (x->c[i] < 0 || x->c[i] > 100) return fail(TUNE_EINVAL, "axes: c[%d] outside [0, 100]", i);
    return TUNE_OK;
}

}  // namespace tune

extern "C" int tune_eval(const tune_arch* arch, const tune_axes* axes, const tune_kernel_desc* descs,
                         int64_t n_kernels, int32_t k, uint32_t flags, int32_t* topk_idx,
                         float* topk_cost, int32_t* pt_blocks, int32_t* pt_warps, float* pt_cost,
                         const int64_t* pt_offsets, void* workspace, size_t ws_bytes,
                         tune_stream_t stream)
{
    tune::clear_error();
    int rc = validate(arch, axes, k);
    if (rc) return rc;
    if (n_kernels < 0) return tune::fail(TUNE_EINVAL, "n_kernels < 0");
    if (!workspace) return tune::fail(TUNE_EINVAL, "workspace is NULL");
    if (ws_bytes < tune_workspace_bytes(TUNE_CALL_EVAL, n_kernels, k))
        return tune::fail(TUNE_ENOMEM, "workspace of %zu bytes is smaller than %zu", ws_bytes,
                          tune_workspace_bytes(TUNE_CALL_EVAL, n_kernels, k));
    if (n_kernels > 0 && (!descs || !topk_idx || !topk_cost))
        return tune::fail(TUNE_EINVAL, "descs, topk_idx and topk_cost must be non-NULL");
    if ((reinterpret_cast<uintptr_t>(descs) & 15) != 0)
        return tune::fail(TUNE_EINVAL, "descs must be 16-byte aligned");
    if (flags & ~(TUNE_EMIT_POINTS | TUNE_SCHED_WARP | TUNE_SCHED_THREAD | 0xff00u))
        return tune::fail(TUNE_EINVAL, "unknown flags 0x%x", flags);
    const int chunk_code = (int)((flags >> 8) & 0xfu);
    if (chunk_code > 15) return tune::fail(TUNE_EINVAL, "bad chunk code");
    const int chunk = chunk_code == 0 ? 0 : (1 << (chunk_code - 1));
    const int ctas_per_sm = (int)((flags >> 12) & 0xfu);
    const bool emit = (flags & TUNE_EMIT_POINTS) != 0;
    if (emit && !pt_offsets) return tune::fail(TUNE_EINVAL, "TUNE_EMIT_POINTS needs pt_offsets");
    if ((flags & TUNE_SCHED_WARP) && (flags & TUNE_SCHED_THREAD))
        return tune::fail(TUNE_EINVAL, "TUNE_SCHED_WARP and TUNE_SCHED_THREAD are exclusive");
    if (emit && (flags & TUNE_SCHED_THREAD))
        return tune::fail(TUNE_EINVAL, "TUNE_EMIT_POINTS runs on the warp schedule only");
    const bool thread_sched = (flags & TUNE_SCHED_THREAD) != 0;

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int* status = static_cast<int*>(workspace);
    TUNE_CUDA_TRY(cudaMemsetAsync(workspace, 0, tune::kWorkspaceHeader, s), "tune_eval: status reset");
    if (n_kernels == 0) return TUNE_OK;

    EvalParams p;
    p.a[0] = *arch;
    p.n_arch = 1;
    p.x = *axes;
    p.n_kernels = n_kernels;
    p.k = k;
    p.chunk = chunk;
    if (thread_sched)
        return k <= 8 ? launch_thread<8>(p, descs, topk_idx, topk_cost, status, s)
                      : launch_thread<16>(p, descs, topk_idx, topk_cost, status, s);
    return emit ? launch<true>(p, descs, topk_idx, topk_cost, pt_blocks, pt_warps, pt_cost, pt_offsets,
                               status, s, ctas_per_sm)
                : launch<false>(p, descs, topk_idx, topk_cost, nullptr, nullptr, nullptr, nullptr, status,
                                s, ctas_per_sm);
}

// ---------------------------------------------------------------------------
// tune_eval_noalloc: the same evaluation for callers that cannot hand the
// library a workspace. Some hosts own every byte of device memory (a serving
// runtime or a framework allocator that gives plugins no way to ask for a
// buffer), and some run under a device-memory budget fixed at start-up that
// must not grow afterwards; neither can call cudaMalloc on the library's
// behalf. This entry point keeps its scratch in the file-scope array below
// instead, which every GPU that loads the library holds until the process
// exits, and allocates nothing itself.
// ---------------------------------------------------------------------------

namespace {

constexpr size_t kNoallocScratchBytes = 4096;  // stated maximum scratch for one call

// Scratch of tune_eval_noalloc (status word and counters). Shared by every
// call on a device: calls that overlap on the GPU race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[tune::kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device, looked up once
// per device (host code must not use the symbol itself: on the host it names a
// stand-in object, not device memory).
int noalloc_scratch(void** out)
{
    int dev = 0;
    TUNE_CUDA_TRY(cudaGetDevice(&dev), "tune_eval_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= tune::kMaxDevices) return tune::fail(TUNE_EUNSUPPORTED, "device ordinal %d too large", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        TUNE_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch), "tune_eval_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return TUNE_OK;
}

}  // namespace

extern "C" int tune_eval_noalloc(const tune_arch* arch, const tune_axes* axes,
                                 const tune_kernel_desc* descs, int64_t n_kernels, int32_t k,
                                 uint32_t flags, int32_t* topk_idx, float* topk_cost,
                                 int32_t* pt_blocks, int32_t* pt_warps, float* pt_cost,
                                 const int64_t* pt_offsets, tune_stream_t stream)
{
    tune::clear_error();
    int rc = validate(arch, axes, k);
    if (rc) return rc;
    if (n_kernels < 0) return tune::fail(TUNE_EINVAL, "n_kernels < 0");
    const size_t need = tune_workspace_bytes(TUNE_CALL_EVAL, n_kernels, k);
    if (need > kNoallocScratchBytes)
        return tune::fail(TUNE_ENOMEM,
                          "tune_eval_noalloc: this call needs %zu bytes of scratch, more than the "
                          "%zu-byte static area; use tune_eval with a workspace",
                          need, kNoallocScratchBytes);
    if (n_kernels > 0 && (!descs || !topk_idx || !topk_cost))
        return tune::fail(TUNE_EINVAL, "descs, topk_idx and topk_cost must be non-NULL");
    if ((reinterpret_cast<uintptr_t>(descs) & 15) != 0)
        return tune::fail(TUNE_EINVAL, "descs must be 16-byte aligned");
    if (flags & ~TUNE_EMIT_POINTS) return tune::fail(TUNE_EINVAL, "unknown flags 0x%x", flags);
    const bool emit = (flags & TUNE_EMIT_POINTS) != 0;
    if (emit && !pt_offsets) return tune::fail(TUNE_EINVAL, "TUNE_EMIT_POINTS needs pt_offsets");

    void* scratch = nullptr;
    rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // The array keeps the previous call's contents: clear the status word and counters.
    TUNE_CUDA_TRY(cudaMemsetAsync(scratch, 0, tune::kWorkspaceHeader, s), "tune_eval_noalloc: scratch reset");
    if (n_kernels > 0) {
        EvalParams p;
        p.a[0] = *arch;
        p.n_arch = 1;
        p.x = *axes;
        p.n_kernels = n_kernels;
        p.k = k;
        p.chunk = 0;
        int* status = static_cast<int*>(scratch);
        rc = emit ? launch<true>(p, descs, topk_idx, topk_cost, pt_blocks, pt_warps, pt_cost, pt_offsets, status, s)
                  : launch<false>(p, descs, topk_idx, topk_cost, nullptr, nullptr, nullptr, nullptr, status, s);
        if (rc) return rc;
    }
    // Report what the kernel found: wait for the stream and read the status word.
    int st = 0;
    TUNE_CUDA_TRY(cudaMemcpyAsync(&st, scratch, sizeof(int), cudaMemcpyDeviceToHost, s),
                  "tune_eval_noalloc: status read");
    TUNE_CUDA_TRY(cudaStreamSynchronize(s), "tune_eval_noalloc: cudaStreamSynchronize");
    if (st & tune::kStatusTimeout) return tune::fail(TUNE_ETIMEOUT, "a bounded device-side wait gave up");
    if (st & tune::kStatusInvalid)
        return tune::fail(TUNE_EINVAL, "a descriptor was malformed (mask outside the axes, negative "
                                       "count, register or shared-memory field)");
    return TUNE_OK;
}

// ---------------------------------------------------------------------------
// tune_eval_archs: the same ranking for every kernel against several
// architecture rows in one launch (blockIdx.y = row).
// ---------------------------------------------------------------------------
extern "C" int tune_eval_archs(const tune_arch* archs, int32_t n_arch, const tune_axes* axes,
                               const tune_kernel_desc* descs, int64_t n_kernels, int32_t k, uint32_t flags,
                               int32_t* topk_idx, float* topk_cost, void* workspace, size_t ws_bytes,
                               tune_stream_t stream)
{
    tune::clear_error();
    if (!archs || n_arch < 1 || n_arch > kMaxArch)
        return tune::fail(TUNE_EINVAL, "n_arch = %d outside [1, %d] or archs NULL", n_arch, kMaxArch);
    for (int i = 0; i < n_arch; ++i) {
        int rc = validate(&archs[i], axes, k);
        if (rc) return rc;
    }
    if (n_kernels < 0) return tune::fail(TUNE_EINVAL, "n_kernels < 0");
    if (!workspace || ws_bytes < tune::kWorkspaceHeader)
        return tune::fail(TUNE_ENOMEM, "workspace smaller than %d bytes", tune::kWorkspaceHeader);
    if (n_kernels > 0 && (!descs || !topk_idx || !topk_cost))
        return tune::fail(TUNE_EINVAL, "descs, topk_idx and topk_cost must be non-NULL");
    if ((reinterpret_cast<uintptr_t>(descs) & 15) != 0)
        return tune::fail(TUNE_EINVAL, "descs must be 16-byte aligned");
    if (flags & ~(TUNE_SCHED_WARP | 0xff00u))
        return tune::fail(TUNE_EINVAL, "flags 0x%x: only TUNE_SCHED_WARP and its chunk/CTA fields", flags);
    const int chunk_code = (int)((flags >> 8) & 0xfu);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int* status = static_cast<int*>(workspace);
    TUNE_CUDA_TRY(cudaMemsetAsync(workspace, 0, tune::kWorkspaceHeader, s), "tune_eval_archs: status reset");
    if (n_kernels == 0) return TUNE_OK;
    EvalParams p;
    for (int i = 0; i < n_arch; ++i) p.a[i] = archs[i];
    p.n_arch = n_arch;
    p.x = *axes;
    p.n_kernels = n_kernels;
    p.k = k;
    p.chunk = chunk_code == 0 ? 0 : (1 << (chunk_code - 1));
    return launch<false>(p, descs, topk_idx, topk_cost, nullptr, nullptr, nullptr, nullptr, status, s,
                         (int)((flags >> 12) & 0xfu));
}

// ---------------------------------------------------------------------------
// Internal launcher for the library's other entry points (one architecture row, no
// emitted points): validates nothing beyond what tune_eval does.
// ---------------------------------------------------------------------------
namespace tune {

int eval_launch(const tune_arch* arch, const tune_axes* axes, const tune_kernel_desc* descs, int64_t n_kernels,
                int32_t k, uint32_t flags, int32_t* topk_idx, float* topk_cost, int* status,
                unsigned long long* queue, cudaStream_t s)
{
    int rc = validate(arch, axes, k);
    if (rc) return rc;
    if (flags & ~(TUNE_SCHED_WARP | 0xff00u))
        return fail(TUNE_EINVAL, "flags 0x%x: only TUNE_SCHED_WARP and its chunk/CTA fields", flags);
    const int chunk_code = (int)((flags >> 8) & 0xfu);
    EvalParams p;
    p.a[0] = *arch;
    p.n_arch = 1;
    p.x = *axes;
    p.n_kernels = n_kernels;
    p.k = k;
    p.chunk = chunk_code == 0 ? 0 : (1 << (chunk_code - 1));
    return launch<false>(p, descs, topk_idx, topk_cost, nullptr, nullptr, nullptr, nullptr, status, s,
                         (int)((flags >> 12) & 0xfu), queue);
}

}  // namespace tune
