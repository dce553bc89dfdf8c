// tune_search: random and Nelder-Mead simplex search over each kernel's tuning space,
// optionally restricted to a subset of its thread counts (the statically pruned space),
// with the analytic cost as the objective. The paper's autotuner explores the space
// left after static pruning with one of its search methods, exhaustive, random or
// Nelder-Mead simplex (Sections III-C and IV-C); here the objective is the static model itself,
// so a search costs no runs of the kernel.
//
// One thread per kernel descriptor: a search is a sequential chain of evaluations.
// A point is a rank vector (a0, a1, a2, a3) over the searched lists of thread counts,
// grid sizes, unroll factors and carveouts; its objective is the FP32 cost of
// point_cost() (+inf without a valid configuration) and points are ordered by
// (cost, canonical index), the canonical index being the point's index in the
// kernel's full space (as in tune_eval).
//
// Random search: evaluation j draws a_d = below(draw(4 j + d), n_d).
// Nelder-Mead: vertices are fixed-point rank vectors (8 fractional bits) rounded to
// the nearest rank and clamped to the list; reflection 1, expansion 2, contraction
// 1/2 (outside or inside), shrink 1/2 towards the best vertex, all in integer
// arithmetic with floor shifts; the search stops when the evaluation budget is spent
// or a shrink leaves every vertex on one point. Both report the best point seen.
#include <stdint.h>

#include "eval_common.cuh"
#include "tune_internal.h"

using namespace tune_dev;

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr int kThreadsS = 128;
constexpr int kQ = 8;  // fractional bits of the simplex coordinates

// SplitMix64 finaliser (Steele, Lea and Flood, 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Draw j of kernel i, mapped to [0, n): SplitMix64 output of the state
// mix64(seed) + (i 2^32 + j + 1) gamma, top 32 bits times n, shifted down 32.
__device__ __forceinline__ int draw_below(uint64_t key, int64_t i, uint32_t j, int n)
{
    const uint64_t x = mix64(key + ((uint64_t)i * 4294967296ull + (uint64_t)j + 1ull) * kGamma);
    return (int)(((x >> 32) * (uint64_t)n) >> 32);
}

__device__ __forceinline__ bool key_less(float c, int i, float c2, int i2)
{
    return c < c2 || (c == c2 && i < i2);
}

struct Space {
    uint32_t mask[4];  // searched positions per axis (thread counts possibly pruned)
    uint32_t tm;       // the kernel's full thread-count mask (canonical index)
    int n[4];          // list lengths
    int nG, nU, nC;    // full axis counts of the kernel's space
};

struct Searcher {
    const tune_arch& a;
    const tune_axes& x;
    const Desc& kd;
    const Space& sp;
    int budget;
    int evals = 0;
    float best_c = INFINITY;
    int best_i = -1;

    // Objective of a rank vector; records the best point seen.
    __device__ __forceinline__ void eval(const int (&r)[4], float& c, int& idx)
    {
        const int tp = __fns(sp.mask[0], 0, r[0] + 1), gp = __fns(sp.mask[1], 0, r[1] + 1);
        const int up = __fns(sp.mask[2], 0, r[2] + 1), cp = __fns(sp.mask[3], 0, r[3] + 1);
        int B, W;
        c = point_cost(a, kd, x.t[tp], x.g[gp], x.u[up], x.c[cp], B, W);
        if (!(c == c)) c = __int_as_float(0x7f800000);  // NaN ranks as +inf
        const int t_full = __popc(sp.tm & ((1u << tp) - 1u));
        idx = ((t_full * sp.nG + r[1]) * sp.nU + r[2]) * sp.nC + r[3];
        ++evals;
        if (key_less(c, idx, best_c, best_i)) {
            best_c = c;
            best_i = idx;
        }
    }

    // Fixed-point vertex -> nearest rank, clamped to the list.
    __device__ __forceinline__ void round_vertex(const int (&v)[4], int (&r)[4]) const
    {
#pragma unroll
        for (int d = 0; d < 4; ++d) r[d] = min(max((v[d] + (1 << (kQ - 1))) >> kQ, 0), sp.n[d] - 1);
    }

    __device__ __forceinline__ bool eval_vertex(const int (&v)[4], float& c, int& idx)
    {
        if (evals >= budget) return false;
        int r[4];
        round_vertex(v, r);
        eval(r, c, idx);
        return true;
    }

    __device__ void random(uint64_t key, int64_t kid)
    {
        for (int j = 0; j < budget; ++j) {
            int r[4];
#pragma unroll
            for (int d = 0; d < 4; ++d) r[d] = draw_below(key, kid, (uint32_t)(4 * j + d), sp.n[d]);
            float c;
            int idx;
            eval(r, c, idx);
        }
    }

    __device__ void nelder_mead(uint64_t key, int64_t kid)
    {
        int V[5][4];
        float Fc[5];
        int Fi[5];
        int x0[4];
#pragma unroll
        for (int d = 0; d < 4; ++d) x0[d] = draw_below(key, kid, (uint32_t)d, sp.n[d]) << kQ;
        // initial simplex: x0 and one step of max(1, n_d / 4) ranks along each axis
        // (backwards where forwards leaves the list)
#pragma unroll
        for (int j = 0; j < 5; ++j)
#pragma unroll
            for (int d = 0; d < 4; ++d) V[j][d] = x0[d];
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const int s = max(1, sp.n[d] >> 2) << kQ;
            V[d + 1][d] = x0[d] + s <= ((sp.n[d] - 1) << kQ) ? x0[d] + s : x0[d] - s;
        }
        for (int j = 0; j < 5; ++j)
            if (!eval_vertex(V[j], Fc[j], Fi[j])) return;
        for (;;) {
            // order: best b, second worst sw, worst w by (cost, index, vertex)
            int ord[5] = {0, 1, 2, 3, 4};
            for (int p = 1; p < 5; ++p) {  // insertion sort, stable
                const int v = ord[p];
                int q = p;
                while (q > 0 && key_less(Fc[v], Fi[v], Fc[ord[q - 1]], Fi[ord[q - 1]])) {
                    ord[q] = ord[q - 1];
                    --q;
                }
                ord[q] = v;
            }
            const int b = ord[0], sw = ord[3], w = ord[4];
            int c[4], xr[4];
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                c[d] = (V[ord[0]][d] + V[ord[1]][d] + V[ord[2]][d] + V[ord[3]][d]) >> 2;
                xr[d] = 2 * c[d] - V[w][d];
            }
            float fr;
            int ir;
            if (!eval_vertex(xr, fr, ir)) return;
            if (key_less(fr, ir, Fc[b], Fi[b])) {
                int xe[4];
#pragma unroll
                for (int d = 0; d < 4; ++d) xe[d] = 3 * c[d] - 2 * V[w][d];
                float fe;
                int ie;
                const bool have_e = eval_vertex(xe, fe, ie);
                const bool take_e = have_e && key_less(fe, ie, fr, ir);
#pragma unroll
                for (int d = 0; d < 4; ++d) V[w][d] = take_e ? xe[d] : xr[d];
                Fc[w] = take_e ? fe : fr;
                Fi[w] = take_e ? ie : ir;
                if (!have_e) return;
                continue;
            }
            if (key_less(fr, ir, Fc[sw], Fi[sw])) {
#pragma unroll
                for (int d = 0; d < 4; ++d) V[w][d] = xr[d];
                Fc[w] = fr;
                Fi[w] = ir;
                continue;
            }
            // contraction: outside if the reflection beats the worst, else inside
            const bool outside = key_less(fr, ir, Fc[w], Fi[w]);
            int xc[4];
#pragma unroll
            for (int d = 0; d < 4; ++d) xc[d] = c[d] + (((outside ? xr[d] : V[w][d]) - c[d]) >> 1);
            float fc;
            int ic;
            if (!eval_vertex(xc, fc, ic)) return;
            const float lim_c = outside ? fr : Fc[w];
            const int lim_i = outside ? ir : Fi[w];
            if (key_less(fc, ic, lim_c, lim_i)) {
#pragma unroll
                for (int d = 0; d < 4; ++d) V[w][d] = xc[d];
                Fc[w] = fc;
                Fi[w] = ic;
                continue;
            }
            // shrink towards the best vertex
            for (int j = 0; j < 5; ++j) {
                if (j == b) continue;
#pragma unroll
                for (int d = 0; d < 4; ++d) V[j][d] = V[b][d] + ((V[j][d] - V[b][d]) >> 1);
                if (!eval_vertex(V[j], Fc[j], Fi[j])) return;
            }
            bool same = true;
            int rb[4];
            round_vertex(V[b], rb);
            for (int j = 0; j < 5; ++j) {
                int rj[4];
                round_vertex(V[j], rj);
#pragma unroll
                for (int d = 0; d < 4; ++d) same = same && rj[d] == rb[d];
            }
            if (same) return;
        }
    }
};

__global__ void __launch_bounds__(kThreadsS)
    tune_search_kernel(const __grid_constant__ tune_arch a, const __grid_constant__ tune_axes x,
                       const int4* __restrict__ descs, int64_t n_kernels, int method, int budget, uint64_t key,
                       const uint32_t* __restrict__ t_keep, int32_t* __restrict__ best_idx,
                       float* __restrict__ best_cost, int32_t* __restrict__ evals, int* __restrict__ status)
{
    const int64_t kid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (kid >= n_kernels) return;
    int4 v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = __ldg(descs + kid * 4 + q);
    Desc kd;
    unpack(v, kd);
    Space sp;
    sp.tm = kd.tm;
    sp.mask[0] = kd.tm & (t_keep ? t_keep[kid] : 0xffffffffu);
    sp.mask[1] = kd.gm;
    sp.mask[2] = kd.um;
    sp.mask[3] = kd.cm;
#pragma unroll
    for (int d = 0; d < 4; ++d) sp.n[d] = __popc(sp.mask[d]);
    sp.nG = sp.n[1];
    sp.nU = sp.n[2];
    sp.nC = sp.n[3];
    const bool bad = desc_bad(kd, x);
    if (bad) atomicOr(status, tune::kStatusInvalid);
    Searcher s{a, x, kd, sp, budget};
    if (!bad && sp.n[0] > 0 && sp.n[1] > 0 && sp.n[2] > 0 && sp.n[3] > 0) {
        if (method == TUNE_SEARCH_RANDOM)
            s.random(key, kid);
        else
            s.nelder_mead(key, kid);
    }
    best_idx[kid] = s.best_i;
    best_cost[kid] = s.best_c;
    evals[kid] = s.evals;
}

}  // namespace

extern "C" int tune_search(const tune_arch* arch, const tune_axes* axes, const tune_kernel_desc* descs,
                           int64_t n_kernels, int32_t method, int32_t budget, uint64_t seed, const uint32_t* t_keep,
                           int32_t* best_idx, float* best_cost, int32_t* evals, void* workspace, size_t ws_bytes,
                           tune_stream_t stream)
{
    tune::clear_error();
    if (!arch || !axes) return tune::fail(TUNE_EINVAL, "arch and axes must be non-NULL host pointers");
    if (method != TUNE_SEARCH_RANDOM && method != TUNE_SEARCH_NELDER_MEAD)
        return tune::fail(TUNE_EINVAL, "method %d is neither TUNE_SEARCH_RANDOM nor TUNE_SEARCH_NELDER_MEAD", method);
    if (budget < 1 || budget > (1 << 20)) return tune::fail(TUNE_EINVAL, "budget %d outside [1, 2^20]", budget);
    if (n_kernels < 0) return tune::fail(TUNE_EINVAL, "n_kernels < 0");
    if (!workspace || ws_bytes < (size_t)tune::kWorkspaceHeader)
        return tune::fail(TUNE_ENOMEM, "workspace smaller than %d bytes", tune::kWorkspaceHeader);
    if (n_kernels > 0 && (!descs || !best_idx || !best_cost || !evals))
        return tune::fail(TUNE_EINVAL, "descs and outputs must be non-NULL");
    if ((reinterpret_cast<uintptr_t>(descs) & 15) != 0) return tune::fail(TUNE_EINVAL, "descs must be 16-byte aligned");
    int rc = tune::validate_inputs(arch, axes);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    TUNE_CUDA_TRY(cudaMemsetAsync(workspace, 0, tune::kWorkspaceHeader, s), "tune_search: status reset");
    if (n_kernels == 0) return TUNE_OK;
    // key = mix64(seed), computed on the host with the same finaliser
    uint64_t z = seed;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    const uint64_t key = z ^ (z >> 31);
    const int64_t blocks = (n_kernels + kThreadsS - 1) / kThreadsS;
    tune_search_kernel<<<(unsigned)blocks, kThreadsS, 0, s>>>(*arch, *axes, reinterpret_cast<const int4*>(descs),
                                                              n_kernels, method, budget, key, t_keep, best_idx,
                                                              best_cost, evals, static_cast<int*>(workspace));
    TUNE_CUDA_TRY(cudaGetLastError(), "tune_search: kernel launch");
    return TUNE_OK;
}
