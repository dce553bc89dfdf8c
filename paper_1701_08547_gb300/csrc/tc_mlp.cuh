// Fused surrogate inference on tcgen05: one persistent CTA per SM pushes
// 128-row tiles of feature rows through whole ensemble members (four hidden
// layers and the head) without writing activations to global memory.
//
// Work unit = (tile of 128 rows, member). A CTA runs two units at a time, one
// per "chain": each chain owns an activation buffer in shared memory and a
// 256-column FP32 accumulator in tensor memory. Layer l of a unit is
//   MMA:      acc = act . W_l^T            (tcgen05.mma, operands in smem)
//   epilogue: act = q(gelu(acc * s + b))   (tcgen05.ld, CUDA cores, st.shared)
// and the MMA issuer alternates the chains layer by layer, so one chain's
// epilogue runs while the other chain's MMAs occupy the tensor cores.
//
// Roles (320 threads): warp 0 streams weights (and each unit's input rows)
// with TMA through a ring of 32 KB stages; warp 1 issues the MMAs; warps 2-5
// are chain 0's epilogue and warps 6-9 chain 1's (thread = accumulator row).
//
// Precision: layer 1 (K = 128) is BF16 x BF16 in both variants. The BF16
// variant keeps layers 2-4 in BF16; the FP8 variant stores the hidden
// activations and W2..W4 as E4M3 codes (per-row weight scales applied in the
// epilogue, unit activation scale) and runs layers 2-4 with kind::f8f6f4.
// The head reads BF16(h4) and sums in FP32.
//
// Every wait is bounded; on timeout the kernel sets status bit 2, stops
// issuing work, waits (bounded) for the copies and MMAs it issued, frees its
// tensor memory and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "gelu.cuh"
#include "tc_gemm.cuh"

namespace tcm {

constexpr int kRows = 128, kIn = 128, kWid = 256, kLayers = 4;
constexpr int kThreads = 320;
constexpr int kChunkA = kRows * 128;  // one 128-byte-wide K chunk of an activation tile
constexpr int kChunkW = kWid * 128;   // one 128-byte-wide K chunk of a weight matrix

template <bool FP8>
struct Cfg {
    static constexpr int act_bytes = FP8 ? kRows * kWid : kRows * kWid * 2;  // >= the BF16 input tile
    static constexpr int stages = FP8 ? 3 : 2;
    static constexpr int smem = 1024 + 2 * act_bytes + stages * kChunkW;
    // 128-byte K chunks per layer: layer 1 reads 128 BF16 inputs
    __host__ __device__ static constexpr int chunks(int l) { return l == 0 ? 2 : (FP8 ? 2 : 4); }
};
static_assert(Cfg<false>::smem <= 227 * 1024 - 1024 && Cfg<true>::smem <= 227 * 1024 - 1024, "shared memory");

struct Args {
    int n;                  // feature rows
    int members;
    long long units;        // ceil(n / 128) * members
    const float* master;    // FP32 parameters, member stride P
    long long P;
    long long off_b[kLayers];
    long long off_w5, off_b5;
    const float* wscale;    // FP8: [members][3][256] per-row scales of W2..W4
    float* pred;            // [members][n]
    int* status;
};

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            tc::sa(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(tc::sa(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int x, int y, int z, int w,
                                            uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];\n" ::"r"(tc::sa(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(tc::sa(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(tc::sa(b)) : "memory");
}

// Instruction descriptor: kind::f8f6f4, E4M3 A and B, FP32 D, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_e4m3(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// Bounded wait that also gives up when another role has aborted.
__device__ __forceinline__ bool wait_bar(uint64_t* b, uint32_t parity, int* status, volatile int* abort_flag)
{
    for (long long i = 0; i < tc::kSpin; ++i) {
        if (tc::mbar_try(b, parity)) return true;
        if (*abort_flag) return false;
    }
    *abort_flag = 1;
    atomicOr(status, 2);
    return false;
}

// Byte offset of 16-byte unit j (0..7) of row r in a 128-row, 128-byte-wide K chunk
// laid out as TMA writes it with 128-byte swizzle (8-row groups of 1024 bytes).
__device__ __forceinline__ uint32_t swz(int r, int j) { return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((j ^ (r & 7)) << 4)); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ uint32_t pack_e4m3(float a, float b, float c, float d)
{
    const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
    return lo | (hi << 16);
}

__device__ __forceinline__ void st_shared_v4(uint8_t* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(tc::sa(p)), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

// grid: min(SMs, units) persistent CTAs; CTA b runs units b, b + gridDim.x, ...;
// its j-th unit goes to chain j % 2. Unit u = (tile u / members, member u % members).
template <bool FP8>
__global__ void __launch_bounds__(kThreads, 1) mlp_infer_kernel(const __grid_constant__ CUtensorMap tx,
                                                                const __grid_constant__ CUtensorMap tw1,
                                                                const __grid_constant__ CUtensorMap tw,
                                                                const __grid_constant__ Args g)
{
    using C = Cfg<FP8>;
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t w_full[C::stages], w_empty[C::stages];
    __shared__ uint64_t x_full[2], act_free[2], acc_full[2], act_ready[2], drain;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* ring = smem + 2 * C::act_bytes;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long my_units = g.units > (long long)blockIdx.x ? (g.units - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    volatile int* abort_v = &abort_flag;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tc::sa(&tmem_base)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (threadIdx.x == 32) {
        for (int i = 0; i < C::stages; ++i) {
            tc::mbar_init(&w_full[i], 1);
            tc::mbar_init(&w_empty[i], 1);
        }
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(&x_full[s], 1);
            tc::mbar_init(&act_free[s], 1);
            tc::mbar_init(&acc_full[s], 1);
            tc::mbar_init(&act_ready[s], 128);
        }
        tc::mbar_init(&drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        abort_flag = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        // ---- producer: per unit pair, layer by layer, chain by chain (the MMA order) ----
        if (lane == 0) {
            long long seq = 0;              // weight chunks issued
            long long x_last[2] = {-1, -1};  // last unit whose input rows were requested, per chain
            bool ok = true;
            for (long long j = 0; j < my_units && ok; j += 2) {
                for (int l = 0; l < kLayers && ok; ++l) {
                    for (int s = 0; s < 2 && ok; ++s) {
                        const long long jj = j + s;
                        if (jj >= my_units) break;
                        const long long u = blockIdx.x + jj * gridDim.x;
                        const int tile = (int)(u / g.members), mem = (int)(u % g.members);
                        if (l == 0) {
                            // the chain's buffer is free once the unit two before finished its MMAs
                            if (jj >= 2 && !(ok = wait_bar(&act_free[s], (uint32_t)(((jj - 2) >> 1) & 1), g.status,
                                                           abort_v)))
                                break;
                            uint8_t* act = smem + s * C::act_bytes;
                            tc::mbar_expect_tx(&x_full[s], 2 * kChunkA);
                            tma_load_2d(act, &tx, 0, tile * kRows, &x_full[s]);
                            tma_load_2d(act + kChunkA, &tx, 64, tile * kRows, &x_full[s]);
                            x_last[s] = jj;
                        }
                        for (int c = 0; c < C::chunks(l); ++c, ++seq) {
                            const int st = (int)(seq % C::stages);
                            const long long use = seq / C::stages;
                            if (use > 0 && !(ok = wait_bar(&w_empty[st], (uint32_t)((use - 1) & 1), g.status,
                                                           abort_v)))
                                break;
                            tc::mbar_expect_tx(&w_full[st], kChunkW);
                            if (l == 0)
                                tc::tma_load_3d(ring + st * kChunkW, &tw1, c * 64, 0, mem, &w_full[st]);
                            else
                                tma_load_4d(ring + st * kChunkW, &tw, c * (FP8 ? 128 : 64), 0, l - 1, mem,
                                            &w_full[st]);
                        }
                    }
                }
            }
            if (!ok) {
                // let the copies that may still be in flight land before the CTA exits
                for (long long q = seq - C::stages; q < seq; ++q)
                    if (q >= 0)
                        tc::mbar_wait(&w_full[q % C::stages], (uint32_t)((q / C::stages) & 1), g.status);
                for (int s = 0; s < 2; ++s)
                    if (x_last[s] >= 0) tc::mbar_wait(&x_full[s], (uint32_t)((x_last[s] >> 1) & 1), g.status);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer ----
        if (lane == 0) {
            long long seq = 0;
            bool ok = true;
            for (long long j = 0; j < my_units && ok; j += 2) {
                for (int l = 0; l < kLayers && ok; ++l) {
                    for (int s = 0; s < 2 && ok; ++s) {
                        const long long jj = j + s;
                        if (jj >= my_units) break;
                        const long long k = jj >> 1;  // unit's ordinal in its chain
                        if (l == 0 && !(ok = wait_bar(&x_full[s], (uint32_t)(k & 1), g.status, abort_v))) break;
                        // the epilogue of the chain's previous layer has written act and drained acc
                        const long long ph = 4 * k + l - 1;
                        if (ph >= 0 && !(ok = wait_bar(&act_ready[s], (uint32_t)(ph & 1), g.status, abort_v)))
                            break;
                        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                        const uint8_t* act = smem + s * C::act_bytes;
                        const uint32_t d = tmem + (uint32_t)(s * kWid);
                        const bool f8 = FP8 && l > 0;
                        const uint32_t idesc = f8 ? idesc_e4m3(kRows, kWid) : tc::idesc_bf16(kRows, kWid);
                        for (int c = 0; c < C::chunks(l); ++c, ++seq) {
                            const int st = (int)(seq % C::stages);
                            if (!(ok = wait_bar(&w_full[st], (uint32_t)((seq / C::stages) & 1), g.status, abort_v)))
                                break;
                            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint64_t a = tc::sdesc(act + c * kChunkA + kk * 32);
                                const uint64_t b = tc::sdesc(ring + st * kChunkW + kk * 32);
                                if (f8)
                                    mma_e4m3(d, a, b, idesc, (c | kk) != 0);
                                else
                                    tc::mma_bf16(d, a, b, idesc, (c | kk) != 0);
                            }
                            tc::mma_commit(&w_empty[st]);
                        }
                        if (!ok) break;
                        tc::mma_commit(&acc_full[s]);
                        if (l == kLayers - 1) tc::mma_commit(&act_free[s]);
                    }
                }
            }
            tc::mma_commit(&drain);  // arrives when every MMA issued above has completed
            tc::mbar_wait(&drain, 0, g.status);
        }
    } else {
        // ---- epilogue: chain s, TMEM lane quarter q, one accumulator row per thread ----
        const int s = (warp - 2) >> 2, q = warp & 3;
        const int r = q * 32 + lane;  // row in the tile
        uint8_t* act = smem + s * C::act_bytes;
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(s * kWid);
        bool ok = true;
        for (long long jj = s; jj < my_units && ok; jj += 2) {
            const long long k = jj >> 1;
            const long long u = blockIdx.x + jj * gridDim.x;
            const int tile = (int)(u / g.members), mem = (int)(u % g.members);
            const float* prm = g.master + mem * g.P;
            float yh = 0.0f;
            for (int l = 0; l < kLayers; ++l) {
                if (!(ok = wait_bar(&acc_full[s], (uint32_t)((4 * k + l) & 1), g.status, abort_v))) break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const float* bias = prm + g.off_b[l];
                const float* scl = (FP8 && l > 0) ? g.wscale + ((long long)mem * 3 + (l - 1)) * kWid : nullptr;
                const float* w5 = prm + g.off_w5;
                for (int n0 = 0; n0 < kWid; n0 += 32) {
                    float v[32];
                    tc::tmem_ld32(taddr + (uint32_t)n0, v);
#pragma unroll
                    for (int i = 0; i < 32; i += 4) {
                        const float4 b4 = __ldg(reinterpret_cast<const float4*>(bias + n0 + i));
                        if (FP8 && l > 0) {
                            const float4 s4 = __ldg(reinterpret_cast<const float4*>(scl + n0 + i));
                            v[i] = fmaf(v[i], s4.x, b4.x);
                            v[i + 1] = fmaf(v[i + 1], s4.y, b4.y);
                            v[i + 2] = fmaf(v[i + 2], s4.z, b4.z);
                            v[i + 3] = fmaf(v[i + 3], s4.w, b4.w);
                        } else {
                            v[i] += b4.x;
                            v[i + 1] += b4.y;
                            v[i + 2] += b4.z;
                            v[i + 3] += b4.w;
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 32; ++i) v[i] = mlp::gelu(v[i]);
                    if (l == kLayers - 1) {
#pragma unroll
                        for (int i = 0; i < 32; i += 4) {
                            const float4 w4 = __ldg(reinterpret_cast<const float4*>(w5 + n0 + i));
                            yh = fmaf(w4.x, __bfloat162float(__float2bfloat16_rn(v[i])), yh);
                            yh = fmaf(w4.y, __bfloat162float(__float2bfloat16_rn(v[i + 1])), yh);
                            yh = fmaf(w4.z, __bfloat162float(__float2bfloat16_rn(v[i + 2])), yh);
                            yh = fmaf(w4.w, __bfloat162float(__float2bfloat16_rn(v[i + 3])), yh);
                        }
                    } else if (FP8) {
                        // columns n0..n0+31 = bytes n0%128.. of chunk n0/128: two 16-byte units
                        uint8_t* base = act + (n0 >> 7) * kChunkA;
                        const int j0 = (n0 & 127) >> 4;
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const float* x = v + 16 * h;
                            st_shared_v4(base + swz(r, j0 + h), pack_e4m3(x[0], x[1], x[2], x[3]),
                                         pack_e4m3(x[4], x[5], x[6], x[7]), pack_e4m3(x[8], x[9], x[10], x[11]),
                                         pack_e4m3(x[12], x[13], x[14], x[15]));
                        }
                    } else {
                        // columns n0..n0+31 = bytes 2 (n0%64).. of chunk n0/64: four 16-byte units
                        uint8_t* base = act + (n0 >> 6) * kChunkA;
                        const int j0 = (n0 & 63) >> 3;
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            const float* x = v + 8 * h;
                            st_shared_v4(base + swz(r, j0 + h), pack_bf16(x[0], x[1]), pack_bf16(x[2], x[3]),
                                         pack_bf16(x[4], x[5]), pack_bf16(x[6], x[7]));
                        }
                    }
                }
                if (l < kLayers - 1) asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                mbar_arrive(&act_ready[s]);
            }
            if (!ok) break;
            const int row = tile * kRows + r;
            if (row < g.n) g.pred[(long long)mem * g.n + row] = yh + prm[g.off_b5];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(512));
}

}  // namespace tcm
