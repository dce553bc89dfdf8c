// tune_suggest: the paper's static search-space pruning (Section III-C, "Static
// Search Analysis"; Section IV-C, Table "Suggested parameters to achieve
// theoretical occupancy"): per kernel, the thread counts T* of its space that
// reach the best theoretical occupancy occ* at its registers and shared memory,
// the register headroom R* and the largest shared memory S* that keep occ*, and
// the rule-based reduction (intensity > 4.0 -> the upper half of T*, else the
// lower half). T* is the set of thread counts whose warp limit alone allows the
// most resident warps, as in the table, where T* is the same for every kernel
// of an architecture. One thread per descriptor; integer occupancy arithmetic.
#include <stdint.h>

#include "eval_common.cuh"
#include "tune_internal.h"

using namespace tune_dev;

namespace {

// Blocks per SM at (T, R, S) and carveout 100 % (the largest capacity), Eqs. 1-5.
__device__ int blocks_at(const tune_arch& a, int T, int R, int S)
{
    const int wb = (T + 31) / 32;
    if (T > a.max_threads_block) return 0;
    const int gw = min(a.max_blocks_sm, a.max_warps_sm / wb);
    int gr;
    if (R > a.regs_thread_max) {
        gr = 0;
    } else if (R <= 0) {
        gr = a.max_blocks_sm;
    } else if (a.reg_alloc_mode == 0) {
        const int rpw = ceil_div(R * 32, a.reg_alloc_unit) * a.reg_alloc_unit;
        gr = rpw * wb > a.regs_block_max ? 0 : ((a.regs_sm / rpw) / a.warp_alloc_gran * a.warp_alloc_gran) / wb;
    } else {
        const long long rpb = (long long)ceil_div(R * 32 * wb, a.reg_alloc_unit) * a.reg_alloc_unit;
        gr = rpb > a.regs_block_max ? 0 : (int)(a.regs_sm / rpb);
    }
    return min(gw, min(gr, smem_blocks(a, S, 100)));
}

__global__ void suggest_kernel(const __grid_constant__ tune_arch a, const __grid_constant__ tune_axes x,
                               const int4* __restrict__ descs, int64_t n, uint32_t* t_star, float* occ_star,
                               int32_t* r_head, int32_t* s_star, uint32_t* t_rule, int* status)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int4 v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = __ldg(descs + i * 4 + q);
    Desc kd;
    unpack(v, kd);
    if (desc_bad(kd, x)) {
        atomicOr(status, tune::kStatusInvalid);
        t_star[i] = t_rule[i] = 0;
        occ_star[i] = 0.0f;
        r_head[i] = s_star[i] = -1;
        return;
    }
    // T*: the thread counts of the space whose warp limit alone allows the most
    // resident warps (the table's T* depends on the architecture only); occ*: the
    // best occupancy over T* at the kernel's registers r0 and shared memory s0.
    int best_t = 0;
    uint32_t star = 0;
    for (uint32_t tb = kd.tm; tb; tb &= tb - 1u) {
        const int tp = __ffs(tb) - 1, T = x.t[tp], wb = (T + 31) / 32;
        const int w = T > a.max_threads_block ? 0 : min(a.max_blocks_sm, a.max_warps_sm / wb) * wb;
        if (w > best_t) {
            best_t = w;
            star = 0;
        }
        if (w == best_t && w > 0) star |= 1u << tp;
    }
    int best_w = 0;
    for (uint32_t tb = star; tb; tb &= tb - 1u) {
        const int T = x.t[__ffs(tb) - 1];
        best_w = max(best_w, blocks_at(a, T, kd.r0, kd.s0) * ((T + 31) / 32));
    }
    t_star[i] = star;
    occ_star[i] = (float)best_w / (float)a.max_warps_sm;
    if (best_w == 0) {
        t_rule[i] = 0;
        r_head[i] = s_star[i] = -1;
        return;
    }
    // R*: more registers while some thread count of T* still reaches occ*
    int R = kd.r0;
    while (R + 1 <= a.regs_thread_max) {
        int w = 0;
        for (uint32_t tb = star; tb; tb &= tb - 1u) {
            const int T = x.t[__ffs(tb) - 1];
            w = max(w, blocks_at(a, T, R + 1, kd.s0) * ((T + 31) / 32));
        }
        if (w < best_w) break;
        ++R;
    }
    r_head[i] = R - kd.r0;
    // S*: the largest shared memory per block keeping B* at the smallest thread
    // count of T* that reaches occ*
    int T0 = 0, B0 = 0;
    for (uint32_t tb = star; tb && !T0; tb &= tb - 1u) {
        const int T = x.t[__ffs(tb) - 1], b = blocks_at(a, T, kd.r0, kd.s0);
        if (b * ((T + 31) / 32) == best_w) T0 = T, B0 = b;
    }
    int lo = kd.s0, hi = a.smem_block_max;  // blocks_at is non-increasing in S at carveout 100 %
    while (lo < hi) {
        const int mid = lo + (hi - lo + 1) / 2;
        if (blocks_at(a, T0, kd.r0, mid) >= B0) lo = mid;
        else hi = mid - 1;
    }
    s_star[i] = lo;
    // rule: intensity = (FP32 + FP64) / (GLDST + SLDST); > 4.0 keeps the upper half of T*
    const float flops = kd.n[CL_FP32] + kd.n[CL_FP64], mem = kd.n[CL_GLDST] + kd.n[CL_SLDST];
    const bool upper = flops > 4.0f * mem;
    const int cnt = __popc(star), keep = max(1, cnt / 2);
    uint32_t rule = 0;
    int seen = 0;
    for (uint32_t tb = star; tb; tb &= tb - 1u, ++seen) {
        const int tp = __ffs(tb) - 1;
        if (upper ? seen >= cnt - keep : seen < keep) rule |= 1u << tp;
    }
    t_rule[i] = rule;
}

}  // namespace

extern "C" int tune_suggest(const tune_arch* arch, const tune_axes* axes, const tune_kernel_desc* descs,
                            int64_t n_kernels, uint32_t* t_star, float* occ_star, int32_t* r_headroom,
                            int32_t* s_star, uint32_t* t_rule, void* workspace, size_t ws_bytes,
                            tune_stream_t stream)
{
    tune::clear_error();
    if (!arch || !axes || !workspace || ws_bytes < tune::kWorkspaceHeader || n_kernels < 0)
        return tune::fail(TUNE_EINVAL, "tune_suggest: bad arguments");
    if (n_kernels > 0 && (!descs || !t_star || !occ_star || !r_headroom || !s_star || !t_rule))
        return tune::fail(TUNE_EINVAL, "tune_suggest: NULL array");
    int rc = tune::validate_inputs(arch, axes);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    TUNE_CUDA_TRY(cudaMemsetAsync(workspace, 0, tune::kWorkspaceHeader, s), "tune_suggest: status reset");
    if (n_kernels == 0) return TUNE_OK;
    suggest_kernel<<<(unsigned)((n_kernels + 127) / 128), 128, 0, s>>>(
        *arch, *axes, reinterpret_cast<const int4*>(descs), n_kernels, t_star, occ_star, r_headroom, s_star, t_rule,
        static_cast<int*>(workspace));
    TUNE_CUDA_TRY(cudaGetLastError(), "tune_suggest: launch");
    return TUNE_OK;
}
