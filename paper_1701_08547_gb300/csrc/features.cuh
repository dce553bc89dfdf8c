// The surrogate's 48 input features of one tuning point, from the analyzer's
// internals (occupancy limits, cost terms) and the descriptor. Each feature is
// scaled by a fixed constant so that typical values are O(1).
//
//  0- 6  log2(n_c + 1) / 20 per class          7-13  n_c / (sum_c n_c + 1)
//  14    log2((n_FP32 + n_FP64 + 1) / (n_GLDST + n_SLDST + 1)) / 10   (intensity)
//  15    r0 / 255       16  s0 / 65536     17  d
//  18    log2 T / 10    19  W_B / 32       20  lane = 32 W_B / T
//  21    log2 G / 16    22  U / 8          23  carveout / 100
//  24    R / 255        25  registers per warp (per-warp allocation) / 8192
//  26-28 G_W, G_R, G_S / 32 (capped at 64)   29  B* / 32   30  W* / 64   31  W* / W_mp
//  32-34 1 where G_W, G_R, G_S equals B*
//  35    log2 waves / 10   36  par / n_SM   37  hide / 32
//  38-40 log2(cost + 1), log2(C_nm + 1), log2(C_m + 1), each / 40
//  41    log2(G T) / 26   42  capacity / 233472   43  block allocation / 65536
//  44    log2(n_BRANCH / U + 1) / 20
//  45-47 256 (f - bf16(f)) for f = features 38, 39, 40: what BF16 storage drops of the
//        three cost terms, so that f + f_45..47 / 256 carries them to about 2^-16 (the
//        cost feature alone resolves costs to only 5-11 % once stored in BF16)
#pragma once

#include <cuda_bf16.h>

#include "eval_common.cuh"

namespace tune_dev {

constexpr int kFeatures = 48;

__device__ __forceinline__ void point_features(const tune_arch& a, const Desc& kd, int T, int G, int U, int C,
                                               float* f)
{
    float rcp[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) rcp[c] = __fdiv_rn(1.0f, a.ipc[c]);
    float tot = 0.0f;
#pragma unroll
    for (int c = 0; c < 7; ++c) tot += kd.n[c];
#pragma unroll
    for (int c = 0; c < 7; ++c) {
        f[c] = log2f(kd.n[c] + 1.0f) / 20.0f;
        f[7 + c] = kd.n[c] / (tot + 1.0f);
    }
    f[14] = log2f((kd.n[CL_FP32] + kd.n[CL_FP64] + 1.0f) / (kd.n[CL_GLDST] + kd.n[CL_SLDST] + 1.0f)) / 10.0f;
    f[15] = (float)kd.r0 / 255.0f;
    f[16] = (float)kd.s0 / 65536.0f;
    f[17] = kd.d;

    const int R = kd.r0 + 4 * (U - 1);
    const int wb = (T + 31) / 32;
    const int gw = T <= a.max_threads_block ? min(a.max_blocks_sm, a.max_warps_sm / wb) : 0;
    int gr, rpw = 0;
    if (R > a.regs_thread_max) {
        gr = 0;
    } else if (R <= 0) {
        gr = a.max_blocks_sm;
    } else if (a.reg_alloc_mode == 0) {
        rpw = ceil_div(R * 32, a.reg_alloc_unit) * a.reg_alloc_unit;
        const int warps = (a.regs_sm / rpw) / a.warp_alloc_gran * a.warp_alloc_gran;
        gr = rpw * wb > a.regs_block_max ? 0 : warps / wb;
    } else {
        const long long rpb = (long long)ceil_div(R * 32 * wb, a.reg_alloc_unit) * a.reg_alloc_unit;
        gr = rpb > a.regs_block_max ? 0 : (int)(a.regs_sm / rpb);
    }
    const int gs = smem_blocks(a, kd.s0, C);
    int cap = 0, s_alloc = 0;
    if (kd.s0 <= a.smem_block_max) {
        s_alloc = ceil_div(kd.s0 + a.smem_reserved_block, a.smem_alloc_unit) * a.smem_alloc_unit;
        const int max_cap = a.smem_caps[a.n_smem_caps - 1];
        for (int i = 0; i < a.n_smem_caps; ++i) {
            const int ci = a.smem_caps[i];
            if (100LL * ci >= (long long)C * max_cap && ci >= s_alloc) {
                cap = ci;
                break;
            }
        }
    }
    const int B = min(gw, min(gr, gs));
    const int W = B * wb;

    f[18] = log2f((float)T) / 10.0f;
    f[19] = (float)wb / 32.0f;
    f[20] = __fdiv_rn((float)(32 * wb), (float)T);
    f[21] = log2f((float)G) / 16.0f;
    f[22] = (float)U / 8.0f;
    f[23] = (float)C / 100.0f;
    f[24] = (float)R / 255.0f;
    f[25] = (float)rpw / 8192.0f;
    f[26] = (float)min(gw, 64) / 32.0f;
    f[27] = (float)min(gr, 64) / 32.0f;
    f[28] = (float)min(gs, 64) / 32.0f;
    f[29] = (float)B / 32.0f;
    f[30] = (float)W / 64.0f;
    f[31] = (float)W / (float)a.max_warps_sm;
    f[32] = (B > 0 && gw == B) ? 1.0f : 0.0f;
    f[33] = (B > 0 && gr == B) ? 1.0f : 0.0f;
    f[34] = (B > 0 && gs == B) ? 1.0f : 0.0f;

    float cnm, cm;
    unit_costs(kd.n, kd.d, U, rcp, a.work_scale, cnm, cm);
    float waves = 0.0f, par = 0.0f, hide = 0.0f, cost = 0.0f;
    if (B > 0) {
        const int slots = a.n_sm * B;
        const int wv = ceil_div(G, slots);
        waves = (float)wv;
        par = __fdiv_rn((float)(a.n_sm * G), (float)(wv * slots));
        hide = fmaxf(1.0f, __fdiv_rn((float)a.w_sat, (float)W));
        const float X = __fmul_rn(__fmaf_rn(cm, hide, cnm), f[20]);
        cost = __fmul_rn(X, __fdiv_rn((float)(wv * slots), (float)(a.n_sm * G)));
    }
    f[35] = waves > 0.0f ? log2f(waves) / 10.0f : 0.0f;
    f[36] = par / (float)a.n_sm;
    f[37] = hide / 32.0f;
    f[38] = log2f(cost + 1.0f) / 40.0f;
    f[39] = log2f(cnm + 1.0f) / 40.0f;
    f[40] = log2f(cm + 1.0f) / 40.0f;
    f[41] = log2f((float)G * (float)T) / 26.0f;
    f[42] = (float)cap / 233472.0f;
    f[43] = (float)s_alloc / 65536.0f;
    f[44] = log2f(__fdiv_rn(kd.n[CL_BRANCH], (float)U) + 1.0f) / 20.0f;
#pragma unroll
    for (int j = 0; j < 3; ++j) f[45 + j] = (f[38 + j] - __bfloat162float(__float2bfloat16_rn(f[38 + j]))) * 256.0f;
}

// Canonical index -> axis positions of (T, G, U, C) for a descriptor's masks (carveout fastest).
__device__ __forceinline__ void decode_point(const Desc& kd, int p, int& tp, int& gp, int& up, int& cp)
{
    const int nG = __popc(kd.gm), nU = __popc(kd.um), nC = __popc(kd.cm);
    const int c_r = p % nC;
    p /= nC;
    const int u_r = p % nU;
    p /= nU;
    const int g_r = p % nG;
    const int t_r = p / nG;
    tp = __fns(kd.tm, 0, t_r + 1);
    gp = __fns(kd.gm, 0, g_r + 1);
    up = __fns(kd.um, 0, u_r + 1);
    cp = __fns(kd.cm, 0, c_r + 1);
}

}  // namespace tune_dev
