// Per-kernel occupancy and cost arithmetic shared by the evaluation kernels and
// the feature kernel (Eqs. 3-6 with the library's FP32 operation order).
#pragma once

#include <math.h>
#include <stdint.h>

#include "tune.h"

namespace tune_dev {

constexpr int kMaxW = 64;  // warps per SM supported by the tables

enum { CL_FP32 = 0, CL_FP64, CL_INT, CL_GLDST, CL_SLDST, CL_BRANCH, CL_SFU };

__host__ __device__ __forceinline__ int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Compensated (Neumaier) FP32 sum, explicit round-to-nearest operations.
template <int M>
__device__ __forceinline__ float neumaier(const float (&x)[M])
{
    float s = 0.0f, comp = 0.0f;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        float t = __fadd_rn(s, x[i]);
        if (fabsf(s) >= fabsf(x[i]))
            comp = __fadd_rn(comp, __fadd_rn(__fsub_rn(s, t), x[i]));
        else
            comp = __fadd_rn(comp, __fadd_rn(__fsub_rn(x[i], t), s));
        s = t;
    }
    return __fadd_rn(s, comp);
}

// ---- per-kernel arithmetic shared by both schedules -------------------------

// Per-unroll cost sums in FP32, fixed order (Eq. 6 with c_x = 1 / IPC_x):
// v_c = n'_c * rcp_c (n'_BRANCH = n_BRANCH / U), compensated sums over the
// non-memory classes (FP32, FP64, INT, BRANCH, SFU) and the memory classes
// (GLDST, SLDST), each scaled by (1 + d) * K.
__device__ __forceinline__ void unit_costs(const float (&n)[7], float d, int U, const float* rcp,
                                           int work_scale, float& cnm, float& cm)
{
    float vv[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) {
        const float nc = c == CL_BRANCH ? __fdiv_rn(n[c], (float)U) : n[c];
        vv[c] = __fmul_rn(nc, rcp[c]);
    }
    const float nm[5] = {vv[CL_FP32], vv[CL_FP64], vv[CL_INT], vv[CL_BRANCH], vv[CL_SFU]};
    const float mm[2] = {vv[CL_GLDST], vv[CL_SLDST]};
    const float dk = __fmul_rn(__fadd_rn(1.0f, d), (float)work_scale);
    cnm = __fmul_rn(neumaier(nm), dk);
    cm = __fmul_rn(neumaier(mm), dk);
}

// Per-warp register allocation (Eq. 4): registers per warp rounded to the
// allocation unit; warps the register file holds, rounded down to the warp
// allocation granularity and clamped to kMaxW; the largest W_B whose block
// fits the per-block register limit.
__host__ __device__ __forceinline__ void reg_params(const tune_arch& a, int R, int& warps, int& wbmax)
{
    warps = 0;
    wbmax = 0;
    if (a.reg_alloc_mode == 0 && R > 0 && R <= a.regs_thread_max) {
        const int rpw = ceil_div(R * 32, a.reg_alloc_unit) * a.reg_alloc_unit;
        wbmax = a.regs_block_max / rpw;
        const int w = (a.regs_sm / rpw) / a.warp_alloc_gran * a.warp_alloc_gran;
        warps = w < kMaxW ? w : kMaxW;
    }
}

// G_S (Eq. 5) for s0 bytes of shared memory per block at carveout C percent.
__device__ __forceinline__ int smem_blocks(const tune_arch& a, int s0, int C)
{
    if (s0 > a.smem_block_max) return 0;
    const int s_alloc = ceil_div(s0 + a.smem_reserved_block, a.smem_alloc_unit) * a.smem_alloc_unit;
    if (s_alloc == 0) return a.max_blocks_sm;
    const int max_cap = a.smem_caps[a.n_smem_caps - 1];
    for (int i = 0; i < a.n_smem_caps; ++i) {
        const int ci = a.smem_caps[i];
        if (100LL * ci >= (long long)C * max_cap && ci >= s_alloc) return ci / s_alloc;
    }
    return 0;
}

// Descriptor fields of kernel kid, read as four 16-byte words.
struct Desc {
    float n[7];
    int r0, s0;
    float d;
    uint32_t tm, gm, um, cm, top;
};

__device__ __forceinline__ void unpack(const int4 (&v)[4], Desc& k)
{
    k.n[0] = __int_as_float(v[0].x);
    k.n[1] = __int_as_float(v[0].y);
    k.n[2] = __int_as_float(v[0].z);
    k.n[3] = __int_as_float(v[0].w);
    k.n[4] = __int_as_float(v[1].x);
    k.n[5] = __int_as_float(v[1].y);
    k.n[6] = __int_as_float(v[1].z);
    k.r0 = v[1].w;
    k.s0 = v[2].x;
    k.d = __int_as_float(v[2].y);
    const uint32_t mlo = (uint32_t)v[2].z, mhi = (uint32_t)v[2].w;
    k.tm = mlo;
    k.gm = mhi & 0xffffu;
    k.um = (mhi >> 16) & 0xffu;
    k.cm = (mhi >> 24) & 0xfu;
    k.top = mhi >> 28;
}

// Largest instruction count a descriptor may carry (2^40). With the architecture
// row's bounds (IPC >= 2^-16, W_sat <= 2^20, K <= 2^24) and d <= 1, every cost of
// a valid point stays below 2^114, so no FP32 cost overflows or turns into NaN.
constexpr float kMaxCount = 0x1p40f;

// Malformed descriptor: mask outside the axes, or a field out of range (counts
// outside [0, 2^40] or not a number, d outside [0, 1], r0 outside [0, 2^24),
// s0 outside [0, 2^30)).
__device__ __forceinline__ bool desc_bad(const Desc& k, const tune_axes& x)
{
    const uint32_t t_ok = x.n_t == 32 ? 0xffffffffu : ((1u << x.n_t) - 1u);
    const uint32_t g_ok = (1u << x.n_g) - 1u, u_ok = (1u << x.n_u) - 1u, c_ok = (1u << x.n_c) - 1u;
    bool bad = k.top != 0 || (k.tm & ~t_ok) || (k.gm & ~g_ok) || (k.um & ~u_ok) || (k.cm & ~c_ok) ||
               k.r0 < 0 || k.r0 >= (1 << 24) || k.s0 < 0 || k.s0 >= (1 << 30) ||
               !(k.d >= 0.0f && k.d <= 1.0f);
#pragma unroll
    for (int c = 0; c < 7; ++c) bad = bad || !(k.n[c] >= 0.0f && k.n[c] <= kMaxCount);
    return bad;
}

// Occupancy (Eqs. 1-5) and FP32 cost (Eq. 6 with the launch-shape terms, in the
// library's fixed operation order) of one point (T, G, U, C): B* and W* are returned,
// the cost is +inf where B* = 0. The same arithmetic as the evaluation kernels' tables.
__device__ __forceinline__ float point_cost(const tune_arch& a, const Desc& kd, int T, int G, int U, int C, int& B,
                                            int& W)
{
    const int R = kd.r0 + 4 * (U - 1);
    const int wb = ceil_div(T, 32);
    const int gw = T <= a.max_threads_block ? min(a.max_blocks_sm, a.max_warps_sm / wb) : 0;
    int gr;
    if (R > a.regs_thread_max) {
        gr = 0;
    } else if (R <= 0) {
        gr = a.max_blocks_sm;
    } else if (a.reg_alloc_mode == 0) {
        int warps, wbmax;
        reg_params(a, R, warps, wbmax);
        gr = wb > wbmax ? 0 : warps / wb;
    } else {
        const long long rpb = (long long)ceil_div(R * 32 * wb, a.reg_alloc_unit) * a.reg_alloc_unit;
        gr = rpb > a.regs_block_max ? 0 : (int)(a.regs_sm / rpb);
    }
    B = min(gw, min(gr, smem_blocks(a, kd.s0, C)));
    W = B * wb;
    if (B <= 0) return __int_as_float(0x7f800000);
    float rcp[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) rcp[c] = __fdiv_rn(1.0f, a.ipc[c]);
    float cnm, cm;
    unit_costs(kd.n, kd.d, U, rcp, a.work_scale, cnm, cm);
    const float hide = fmaxf(1.0f, __fdiv_rn((float)a.w_sat, (float)W));
    const float lane = __fdiv_rn((float)(32 * wb), (float)T);
    const float X = __fmul_rn(__fmaf_rn(cm, hide, cnm), lane);
    const int slots = a.n_sm * B;
    const int waves = ceil_div(G, slots);
    return __fmul_rn(X, __fdiv_rn((float)(waves * slots), (float)(a.n_sm * G)));
}

}  // namespace tune_dev
