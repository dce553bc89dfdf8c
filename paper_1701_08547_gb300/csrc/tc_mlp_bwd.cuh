// Fused input-gradient chain of surrogate training on tcgen05: one persistent CTA
// per SM pushes 128-row tiles of the head's gradient dZ4 back through layers 4, 3
// and 2 of a member without re-reading its own outputs from global memory:
//   dZ_{l-1} = (dZ_l W_l) * gelu'(Z_{l-1}),   l = 4, 3, 2,
// every dZ rounded to BF16 (the operand precision of the next product) and stored
// for the weight gradients: dZ3 and dZ2 leave from the chain's activation buffer,
// where they are the next product's A operand, with bulk tensor stores the MMA
// issuer starts before that product (and waits to have read before the epilogue
// may overwrite the buffer); dZ1 is stored by the epilogue threads. Work unit = (tile of 128 rows, member); stage j of a unit
// is the product with W_{4-j} followed by the epilogue that multiplies in gelu'(Z_{3-j})
// (FP16, kept by the training forward pass) and writes dZ_{3-j}.
//
// The structure is the inference kernel's (tc_mlp.cuh): warp 0 streams the unit's
// dZ4 rows and 32 KB K chunks of the weights with TMA, warp 1 issues the MMAs of two
// chains alternately, warps 2-17 run the epilogues (thread = accumulator row, four
// warps per TMEM lane quarter, one per 64-column quarter). The product's B operand is
// W_l with the contraction over its output index o, i.e. W_l as stored ([o][i], i
// contiguous) read MN-major: a 32 KB stage holds 64 rows o of W_l as four boxes of 64
// inputs (the MN-major 128-byte-swizzle atoms, 8 KB apart along N), from the same BF16
// copy the forward pass uses.
//
// Every wait is bounded; on timeout the kernel sets status bit 2, stops issuing
// work, waits (bounded) for the copies and MMAs it issued, frees its tensor memory
// and returns.
#pragma once

#include "tc_mlp.cuh"

namespace tcm {

constexpr int kBwdStages = kLayers - 1;  // products with W4, W3, W2

// MN-major B operand of a weight stage, 128-byte swizzle: leading byte offset = distance
// between the 64-input atoms along N (one 64-row box, 8 KB), stride byte offset = distance
// between 8-row groups along K (1 KB).
__device__ __forceinline__ uint64_t sdesc_w_mn(const void* p)
{
    const uint64_t addr = tc::sa(p);
    return ((addr >> 4) & 0x3fffull) | ((uint64_t)((64 * 128) >> 4) << 16) | ((1024ull >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

struct BwdArgs {
    int members;
    long long units;                  // rows / 128 * members (rows a multiple of 128: every unit's rows exist)
    const __half* g[kBwdStages];      // stage j: gelu'(Z_{3-j}), [members][act_stride], tiled (mlp::gprime_at)
    __nv_bfloat16* dz[kBwdStages];    // stage j: dZ_{3-j}, same layout
    int dz_coord[kBwdStages];         // stage j: the layer coordinate of dz[j] in the map tdzs
    long long act_stride;             // member stride of z and dz (elements); rows of 256
    int* status;
};


// grid: min(SMs, units) persistent CTAs; CTA b runs units b, b + gridDim.x, ...; its
// j-th unit goes to chain j % 2. Unit u = (tile u / members, member u % members).
// tdz: dZ4 as 8-byte elements {64, rows, members}, box {16, 128, 1};
// tw: W2..W4 as 8-byte elements {64 (inputs), 256 (outputs), 3, members}, box {16, 64, 1, 1};
// tdzs: the dZ buffers as 8-byte elements {64, rows, members, layers}, box {16, 128, 1, 1}.
__global__ void __maxnreg__(96) mlp_bwd_kernel(const __grid_constant__ CUtensorMap tdz,
                                               const __grid_constant__ CUtensorMap tw,
                                               const __grid_constant__ CUtensorMap tdzs,
                                               const __grid_constant__ BwdArgs g)
{
    using C = Cfg<false>;
    constexpr int kChunks = kWid * 2 / 128;  // 128-byte K chunks of a 256-wide BF16 operand
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

    pdl::grid_dep_enter();  // launched after the head backward in a training step
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
            tc::mbar_init(&act_ready[s], 32 * kEpiWarps);
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
        // ---- producer: per unit pair, stage by stage, chain by chain (the MMA order) ----
        if (lane == 0) {
            long long seq = 0;
            long long x_last[2] = {-1, -1};
            bool ok = true;
            for (long long j = 0; j < my_units && ok; j += 2) {
                for (int l = 0; l < kBwdStages && ok; ++l) {
                    for (int s = 0; s < 2 && ok; ++s) {
                        const long long jj = j + s;
                        if (jj >= my_units) break;
                        const long long u = blockIdx.x + jj * gridDim.x;
                        const int tile = (int)(u / g.members), mem = (int)(u % g.members);
                        if (l == 0) {
                            if (jj >= 2 && !(ok = wait_bar(&act_free[s], (uint32_t)(((jj - 2) >> 1) & 1), g.status,
                                                           abort_v)))
                                break;
                            uint8_t* act = smem + s * C::act_bytes;
                            tc::mbar_expect_tx(&x_full[s], kChunks * kChunkA);
                            for (int c = 0; c < kChunks; ++c)
                                tc::tma_load_3d(act + c * kChunkA, &tdz, c * 16, tile * kRows, mem, &x_full[s]);
                            x_last[s] = jj;
                        }
                        {
                            // the epilogue of this (unit, stage) reads a 64 KB tile of gelu'(Z):
                            // request it into L2 while the MMAs run
                            const char* gt = reinterpret_cast<const char*>(
                                g.g[l] + (long long)mem * g.act_stride + (long long)tile * kRows * kWid);
                            for (int q = 0; q < 2; ++q)
                                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(gt + q * 32768),
                                             "r"(32768)
                                             : "memory");
                        }
                        for (int c = 0; c < kChunks; ++c, ++seq) {
                            const int st = (int)(seq % C::stages);
                            const long long use = seq / C::stages;
                            if (use > 0 && !(ok = wait_bar(&w_empty[st], (uint32_t)((use - 1) & 1), g.status,
                                                           abort_v)))
                                break;
                            tc::mbar_expect_tx(&w_full[st], kChunkW);
                            // stage l multiplies by W_{4-l} (matrix 2 - l of W2..W4): rows o of K
                            // chunk c, four boxes of 64 inputs
                            for (int q = 0; q < kChunkW / (64 * 128); ++q)
                                tma_load_4d(ring + st * kChunkW + q * (64 * 128), &tw, q * 16, c * 64,
                                            kBwdStages - 1 - l, mem, &w_full[st]);
                        }
                    }
                }
            }
            if (!ok) {
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
            // A (the dZ rows) K-major, B (W as stored) MN-major
            const uint32_t idesc = tc::idesc_bf16(kRows, kWid) | (1u << 16);
            for (long long j = 0; j < my_units && ok; j += 2) {
                for (int l = 0; l < kBwdStages && ok; ++l) {
                    for (int s = 0; s < 2 && ok; ++s) {
                        const long long jj = j + s;
                        if (jj >= my_units) break;
                        const long long k = jj >> 1;
                        if (l == 0 && !(ok = wait_bar(&x_full[s], (uint32_t)(k & 1), g.status, abort_v))) break;
                        // the chain's previous epilogue has written act and drained acc
                        const long long ph = kBwdStages * k + l - 1;
                        if (ph >= 0 && !(ok = wait_bar(&act_ready[s], (uint32_t)(ph & 1), g.status, abort_v)))
                            break;
                        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                        const uint8_t* act = smem + s * C::act_bytes;
                        if (l > 0) {
                            // act holds the previous stage's dZ (this unit's rows): copied to global
                            // memory by the tensor-store unit while the MMAs below read it
                            const long long u = blockIdx.x + jj * gridDim.x;
                            const int tile = (int)(u / g.members), mem = (int)(u % g.members);
                            for (int c = 0; c < kChunks; ++c)
                                tma_store_4d(&tdzs, act + c * kChunkA, c * 16, tile * kRows, mem, g.dz_coord[l - 1]);
                            bulk_commit();
                        }
                        const uint32_t d = tmem + (uint32_t)(s * kWid);
                        for (int c = 0; c < kChunks; ++c, ++seq) {
                            const int st = (int)(seq % C::stages);
                            if (!(ok = wait_bar(&w_full[st], (uint32_t)((seq / C::stages) & 1), g.status, abort_v)))
                                break;
                            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint64_t a = tc::sdesc(act + c * kChunkA + kk * 32);
                                const uint64_t b = sdesc_w_mn(ring + st * kChunkW + kk * 2048);
                                tc::mma_bf16(d, a, b, idesc, (c | kk) != 0);
                            }
                            tc::mma_commit(&w_empty[st]);
                        }
                        if (l > 0) bulk_wait_read();  // the epilogue rewrites act after acc_full
                        if (!ok) break;
                        tc::mma_commit(&acc_full[s]);
                        if (l == kBwdStages - 1) tc::mma_commit(&act_free[s]);
                    }
                }
            }
            bulk_wait_all();
            tc::mma_commit(&drain);
            tc::mbar_wait(&drain, 0, g.status);
        }
    } else {
        // ---- epilogue: dZ = bf16(acc * gelu'(z)) to global memory and, before the last
        // stage, to the chain's activation buffer as the next product's A operand ----
        const int e = warp - 2, q = warp & 3, cq = e >> 2;
        const int r = q * 32 + lane;
        const int c_beg = cq * (kWid / 4);
        bool ok = true;
        for (long long j = 0; j < my_units && ok; j += 2) {
            for (int l = 0; l < kBwdStages && ok; ++l) {
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const long long jj = j + s;
                    if (jj >= my_units || !ok) break;
                    const long long k = jj >> 1;
                    const long long u = blockIdx.x + jj * gridDim.x;
                    const int tile = (int)(u / g.members), mem = (int)(u % g.members);
                    const int row = tile * kRows + r;
                    const long long arow = (long long)mem * g.act_stride + (long long)row * kWid;
                    const __half* gr = g.g[l] + (long long)mem * g.act_stride;  // tiled (mlp::gprime_at)
                    __nv_bfloat16* dzr = g.dz[l] + arow;
                    uint8_t* act = smem + s * C::act_bytes;
                    const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(s * kWid);
                    const bool last = l == kBwdStages - 1;
                    // gelu'(Z) of the thread's 64 columns (FP16, four 32-byte loads) is requested
                    // before the accumulator wait
                    uint32_t gw[kWid / 4 / 16][8];
#pragma unroll
                    for (int b = 0; b < kWid / 4 / 16; ++b) ld_global_v8u(gr + mlp::gprime_at(row, c_beg + 16 * b), gw[b]);
                    if (!(ok = wait_bar(&acc_full[s], (uint32_t)((kBwdStages * k + l) & 1), g.status, abort_v)))
                        break;
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
                    for (int b = 0; b < kWid / 4 / 16; ++b) {
                        const int n0 = c_beg + 16 * b;
                        float v[16];
                        tmem_ld16(taddr + (uint32_t)n0, v);
                        uint32_t w[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const float2 d = __half22float2(*reinterpret_cast<const __half2*>(&gw[b][i]));
                            w[i] = pack_bf16(v[2 * i] * d.x, v[2 * i + 1] * d.y);
                        }
                        if (last) {
                            st_global_v8(dzr + n0, w);
                        } else {
                            // 16 columns = two 16-byte units of K chunk n0 / 64
                            uint8_t* base = act + (n0 >> 6) * kChunkA;
                            const int j0 = (n0 & 63) >> 3;
                            st_shared_v4(base + swz(r, j0), w[0], w[1], w[2], w[3]);
                            st_shared_v4(base + swz(r, j0 + 1), w[4], w[5], w[6], w[7]);
                        }
                    }
                    if (!last) asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                    mbar_arrive(&act_ready[s]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(512));
}

}  // namespace tcm
