// Fused surrogate inference on tcgen05: one persistent CTA per SM pushes
// 128-row tiles of feature rows through whole ensemble members (four hidden
// layers and the head) without writing activations to global memory.
//
// Work unit = (tile of 128 rows, member). A CTA runs two units at a time, one
// per "chain": each chain owns an activation buffer in shared memory and a
// 256-column FP32 accumulator in tensor memory. Layer l of a unit is
//   MMA:      acc = act . W_l^T              (tcgen05.mma, operands in smem)
//   epilogue: act = q(2 gelu(acc * s + b))   (tcgen05.ld, CUDA cores, st.shared)
// and the MMA issuer alternates the chains layer by layer, so one chain's
// epilogue runs while the other chain's MMAs occupy the tensor cores.
//
// Roles (576 threads): warp 0 streams weights (and each unit's input rows)
// with TMA through a ring of 32 KB stages (all 256 output rows of a 128-byte
// K chunk; the tensor maps address 8-byte elements, the bytes and their
// 128-byte swizzle being the same for BF16 and E4M3 data); warp 1 issues the MMAs; warps 2-17
// run the epilogues of both chains in the MMA issue order (each layer's
// epilogue gets all sixteen warps): thread = accumulator row, four warps per
// TMEM lane quarter, one per 64-column quarter.
//
// The epilogue stores 2 gelu(z) = z (1 + tanh u), one operation fewer than
// gelu itself, and the next layer (or the head) takes half its accumulator.
// In BF16 this is exact: doubling commutes with rounding, so the results are
// those of storing gelu(z). The training variant keeps h = gelu(z) itself in
// act, because act is also the activations H1..H3 the backward pass reads: the
// MMA issuer copies each layer's act to global memory with bulk tensor stores
// while that layer's MMAs read it, and waits for the copy to have read act
// before the epilogue may overwrite it.
//
// Precision: layer 1 (K = 64) is BF16 x BF16 in both variants; GELU is
// evaluated in FP32. The BF16 variant keeps layers 2-4 in BF16; the FP8
// variant stores E4M3 codes of 2 h (activation scale 1/2) and W2..W4 as E4M3
// codes with one scale per matrix, and runs layers 2-4 with kind::f8f6f4.
// The head takes the FP32 values 2 h4 and sums in FP32.
//
// Every wait is bounded; on timeout the kernel sets status bit 2, stops
// issuing work, waits (bounded) for the copies and MMAs it issued, frees its
// tensor memory and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "gelu.cuh"
#include "pdl.cuh"
#include "tc_gemm.cuh"

namespace tcm {

constexpr int kRows = 128, kIn = 64, kWid = 256, kLayers = 4;
constexpr int kEpiWarps = 16;  // shared by the two chains
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr int kChunkA = kRows * 128;  // one 128-byte-wide K chunk of an activation tile
constexpr int kChunkW = kWid * 128;   // one 128-byte-wide K chunk of a weight matrix

template <bool FP8>
struct Cfg {
    static constexpr int act_bytes = FP8 ? kRows * kWid : kRows * kWid * 2;  // >= the BF16 input tile
    static constexpr int stages = FP8 ? 3 : 2;
    static constexpr int smem = 1024 + 2 * act_bytes + stages * kChunkW;
    // 128-byte K chunks per layer: layer 1 reads kIn BF16 inputs
    __host__ __device__ static constexpr int chunks(int l) { return l == 0 ? kIn * 2 / 128 : (FP8 ? 2 : 4); }
};
static_assert(Cfg<false>::smem <= 227 * 1024 - 1024 && Cfg<true>::smem <= 227 * 1024 - 1024, "shared memory");
static_assert(kIn % 64 == 0 && kIn <= kWid, "input rows are whole 128-byte K chunks");

struct Args {
    int n;                  // feature rows
    int members;
    long long units;        // ceil(n / 128) * members
    const float* master;    // FP32 parameters, member stride P
    long long P;
    long long off_b[kLayers];
    long long off_w5, off_b5;
    const float* wscale_half;  // FP8: [members][3][256] halves of the scales of W2..W4 (one per matrix, repeated per row)
    float* pred;            // [members][pred_stride]
    long long pred_stride;  // member stride of pred (n for inference)
    // training (BF16 only): per layer gelu'(z) of the pre-activations (FP16, in the tiled
    // layout of mlp::gprime_at) and the activations h = gelu(z) (BF16, rows of 256) of every
    // row < n, [members][act_stride]; null: not kept. The kernel stores H4 through h_out[3];
    // H1..H3 go through the tensor map `th` (the same rows, layer = its last coordinate).
    __half* g_out[kLayers];
    __nv_bfloat16* h_out[kLayers];
    long long act_stride;
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

// Bulk tensor store of one box from shared memory into the issuing thread's bulk group (all
// coordinates non-negative, x a multiple of 16 bytes).
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, const void* src, int x, int y, int z, int w)
{
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5}], [%1];\n" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(tc::sa(src)), "r"(x), "r"(y), "r"(z), "r"(w)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }

// The thread's committed bulk stores have read their shared-memory sources.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }

// The thread's committed bulk stores are complete.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

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

// 16 parameters (biases or head weights, read again by every unit): kept in L1 with priority.
__device__ __forceinline__ void ld16(const float* p, float (&x)[16])
{
#pragma unroll
    for (int i = 0; i < 16; i += 4) {
        float4 q;
        asm volatile("ld.global.nc.L1::evict_last.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                     : "=f"(q.x), "=f"(q.y), "=f"(q.z), "=f"(q.w)
                     : "l"(p + i));
        x[i] = q.x;
        x[i + 1] = q.y;
        x[i + 2] = q.z;
        x[i + 3] = q.w;
    }
}

// Packed FP32 pairs (two IEEE single-precision operations, round to nearest, per
// instruction): the same result in each lane as the scalar fmaf / multiply.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{\n .reg .b64 a, b, c, d;\n mov.b64 a, {%2, %3};\n mov.b64 b, {%4, %5};\n mov.b64 c, {%6, %7};\n"
        " fma.rn.f32x2 d, a, b, c;\n mov.b64 {%0, %1}, d;\n}\n"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

__device__ __forceinline__ float2 mul2(float2 a, float2 b)
{
    float2 d;
    asm("{\n .reg .b64 a, b, d;\n mov.b64 a, {%2, %3};\n mov.b64 b, {%4, %5};\n mul.rn.f32x2 d, a, b;\n"
        " mov.b64 {%0, %1}, d;\n}\n"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// 256-bit global store of eight 32-bit words (address 32-byte aligned), not kept in L1 (what the
// epilogues store is read by later launches only).
__device__ __forceinline__ void st_global_v8(void* p, const uint32_t (&w)[8])
{
    asm volatile("st.global.L1::no_allocate.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n" ::"l"(p), "r"(w[0]), "r"(w[1]),
                 "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                 : "memory");
}

// 256-bit global load of eight floats (address 32-byte aligned; data not written by this kernel).
__device__ __forceinline__ void ld_global_v8(const float* p, float* x)
{
    asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                 : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3]), "=f"(x[4]), "=f"(x[5]), "=f"(x[6]), "=f"(x[7])
                 : "l"(p));
}

// 256-bit global load of eight 32-bit words (address 32-byte aligned; data not written by this kernel).
__device__ __forceinline__ void ld_global_v8u(const void* p, uint32_t (&x)[8])
{
    asm volatile("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                 : "=r"(x[0]), "=r"(x[1]), "=r"(x[2]), "=r"(x[3]), "=r"(x[4]), "=r"(x[5]), "=r"(x[6]), "=r"(x[7])
                 : "l"(p));
}

// 16 consecutive accumulator columns of this thread's TMEM lane (row), then the wait.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// grid: min(SMs, units) persistent CTAs; CTA b runs units b, b + gridDim.x, ...;
// its j-th unit goes to chain j % 2. Unit u = (tile u / members, member u % members).
// 96 registers per thread: the 18 warps spread over the SM's four sub-partitions of 16,384
// registers, five on the fullest (5 x 32 x 96 = 15,360; at 104 the launch does not fit).
template <bool FP8, bool TRAIN = false>
__global__ void __maxnreg__(96) mlp_infer_kernel(const __grid_constant__ CUtensorMap tx,
                                                                const __grid_constant__ CUtensorMap tw1,
                                                                const __grid_constant__ CUtensorMap tw,
                                                                const __grid_constant__ CUtensorMap th,
                                                                const __grid_constant__ Args g)
{
    using C = Cfg<FP8>;
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t w_full[C::stages], w_empty[C::stages];
    __shared__ uint64_t x_full[2], act_free[2], acc_full[2], act_ready[2], head_bar[2], drain;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ float head_part[2][3][kRows];  // head sums of column quarters 1-3, per chain

    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* ring = smem + 2 * C::act_bytes;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long my_units = g.units > (long long)blockIdx.x ? (g.units - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    volatile int* abort_v = &abort_flag;

    pdl::grid_dep_enter();  // launched after the batch gather in a training step
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
            tc::mbar_init(&head_bar[s], 3 * kRows);
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
                            tc::mbar_expect_tx(&x_full[s], C::chunks(0) * kChunkA);
                            for (int c = 0; c < C::chunks(0); ++c)
                                tma_load_2d(act + c * kChunkA, &tx, c * 16, tile * kRows, &x_full[s]);
                            x_last[s] = jj;
                        }
                        for (int c = 0; c < C::chunks(l); ++c, ++seq) {
                            const int st = (int)(seq % C::stages);
                            const long long use = seq / C::stages;
                            if (use > 0 && !(ok = wait_bar(&w_empty[st], (uint32_t)((use - 1) & 1), g.status,
                                                           abort_v)))
                                break;
                            tc::mbar_expect_tx(&w_full[st], kChunkW);
                            // maps address 8-byte elements: 16 per 128-byte K chunk
                            if (l == 0)
                                tc::tma_load_3d(ring + st * kChunkW, &tw1, c * 16, 0, mem, &w_full[st]);
                            else
                                tma_load_4d(ring + st * kChunkW, &tw, c * 16, 0, l - 1, mem, &w_full[st]);
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
                        if (TRAIN && l > 0) {
                            // act holds H of layer l - 1 (BF16 h, rows of this unit's tile): copied to
                            // global memory by the tensor-store unit while the MMAs below read it
                            const long long u = blockIdx.x + jj * gridDim.x;
                            const int tile = (int)(u / g.members), mem = (int)(u % g.members);
                            for (int c = 0; c < kWid * 2 / 128; ++c)
                                tma_store_4d(&th, act + c * kChunkA, c * 16, tile * kRows, mem, l - 1);
                            bulk_commit();
                        }
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
                        if (TRAIN && l > 0) bulk_wait_read();  // the epilogue rewrites act after acc_full
                        if (!ok) break;
                        tc::mma_commit(&acc_full[s]);
                        if (l == kLayers - 1) tc::mma_commit(&act_free[s]);
                    }
                }
            }
            if (TRAIN) bulk_wait_all();
            tc::mma_commit(&drain);  // arrives when every MMA issued above has completed
            tc::mbar_wait(&drain, 0, g.status);
        }
    } else {
        // ---- epilogue: all sixteen warps serve the chains in the MMA issue order; warp =
        // (TMEM lane quarter q, column quarter cq), thread = accumulator row ----
        const int e = warp - 2, q = warp & 3, cq = e >> 2;
        const int r = q * 32 + lane;  // row in the tile
        const int c_beg = cq * (kWid / 4), c_end = c_beg + kWid / 4;
        bool ok = true;
        for (long long j = 0; j < my_units && ok; j += 2) {
            for (int l = 0; l < kLayers && ok; ++l) {
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const long long jj = j + s;
                    if (jj >= my_units || !ok) break;
                    const long long k = jj >> 1;
                    const long long u = blockIdx.x + jj * gridDim.x;
                    const int tile = (int)(u / g.members), mem = (int)(u % g.members);
                    const float* prm = g.master + mem * g.P;
                    uint8_t* act = smem + s * C::act_bytes;
                    const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(s * kWid);
                    if (!(ok = wait_bar(&acc_full[s], (uint32_t)((4 * k + l) & 1), g.status, abort_v))) break;
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const float* bias = prm + g.off_b[l];
                    // E4M3 layers: the accumulator times half the matrix's weight scale (one value per
                    // member and layer, so the epilogue keeps it in a register)
                    const float sv = (FP8 && l > 0) ? __ldg(g.wscale_half + ((long long)mem * 3 + (l - 1)) * kWid) : 0.0f;
                    const float* w5 = prm + g.off_w5;
                    // Layers 2-4 read 2 h (see the header), so their accumulator is halved here; in
                    // training act holds h itself (it is also the H the backward pass reads).
                    const float acc_mul = (l > 0 && !TRAIN) ? 0.5f : 1.0f;
                    const bool f8 = FP8 && l > 0, head = l == kLayers - 1;
                    float yh = 0.0f;
                    for (int n0 = c_beg; n0 < c_end; n0 += 16) {
                        // the block's parameters are requested before the accumulator wait so that
                        // their latency overlaps it
                        float bb[16], ww[16];
                        ld16(bias + n0, bb);
                        if (head) ld16(w5 + n0, ww);
                        float v[16];
                        tmem_ld16(taddr + (uint32_t)n0, v);
                        const long long arow = (long long)mem * g.act_stride + (long long)(tile * kRows + r) * kWid + n0;
                        // z = acc * s + b, then 2 gelu(z) = z (1 + tanh u), u = z (K C z^2 + K), in FP32:
                        // one multi-function-unit tanh per element, the rest on column pairs (packed
                        // FP32x2 operations, half the instructions of the scalar form).
                        uint32_t gd[8];
                        if (TRAIN) {
#pragma unroll
                            for (int i = 0; i < 16; i += 2) {
                                const float2 z = fma2(make_float2(v[i], v[i + 1]), f2(acc_mul), make_float2(bb[i], bb[i + 1]));
                                const float2 zz = mul2(z, z);
                                const float2 u = mul2(z, fma2(f2(mlp::kGeluK * mlp::kGeluC), zz, f2(mlp::kGeluK)));
                                const float2 t = make_float2(mlp::tanh_hw(u.x), mlp::tanh_hw(u.y));
                                // gelu'(z) = (1 + t) / 2 + z / 2 (1 - t^2) K (1 + 3 C z^2), kept in FP16 for
                                // the backward pass; with 1 - t^2 = (1 - t)(1 + t) and a = (1 + t) / 2 it is
                                // a + (z K (1 + 3 C z^2)) (1 - t) a, six packed operations per pair
                                const float2 a = fma2(t, f2(0.5f), f2(0.5f));
                                const float2 w = mul2(z, fma2(f2(3.0f * mlp::kGeluK * mlp::kGeluC), zz, f2(mlp::kGeluK)));
                                const float2 d = fma2(mul2(w, fma2(t, f2(-1.0f), f2(1.0f))), a, a);
                                // h itself (2 h halved, exact): act, H and the head all take h in training
                                const float2 hh = mul2(fma2(z, t, z), f2(0.5f));
                                v[i] = hh.x;
                                v[i + 1] = hh.y;
                                const __half2 d2 = __floats2half2_rn(d.x, d.y);
                                gd[i / 2] = *reinterpret_cast<const uint32_t*>(&d2);
                            }
                        } else {
#pragma unroll
                            for (int i = 0; i < 16; i += 2) {
                                const float2 z = fma2(make_float2(v[i], v[i + 1]), f2(f8 ? sv : acc_mul),
                                                      make_float2(bb[i], bb[i + 1]));
                                const float2 uu =
                                    mul2(z, fma2(f2(mlp::kGeluK * mlp::kGeluC), mul2(z, z), f2(mlp::kGeluK)));
                                const float2 t = make_float2(mlp::tanh_hw(uu.x), mlp::tanh_hw(uu.y));
                                const float2 h2 = fma2(z, t, z);
                                v[i] = h2.x;
                                v[i + 1] = h2.y;
                            }
                        }
                        if (TRAIN && !FP8 && g.g_out[l])  // tiled layout (mlp::gprime_at): one 1 KB run per warp
                            st_global_v8(g.g_out[l] + (long long)mem * g.act_stride + mlp::gprime_at(tile * kRows + r, n0), gd);
                        if (FP8 && !head) {
                            // E4M3 codes of 2 h: 16 columns = one 16-byte unit
                            uint32_t w[4];
#pragma unroll
                            for (int qd = 0; qd < 4; ++qd) w[qd] = pack_e4m3(v[4 * qd], v[4 * qd + 1], v[4 * qd + 2], v[4 * qd + 3]);
                            st_shared_v4(act + (n0 >> 7) * kChunkA + swz(r, (n0 & 127) >> 4), w[0], w[1], w[2], w[3]);
                            continue;
                        }
                        if (TRAIN && head && g.h_out[l]) {
                            // H4 has no act copy: stored from here (H1..H3 leave from act, see the MMA issuer)
                            uint32_t w[8];
#pragma unroll
                            for (int t = 0; t < 8; ++t) w[t] = pack_bf16(v[2 * t], v[2 * t + 1]);
                            st_global_v8(g.h_out[l] + arow, w);
                        }
                        if (head) {
                            // head on 2 h4 (h4 in training); the sum is halved with b5 added below
#pragma unroll
                            for (int i = 0; i < 16; ++i) yh = fmaf(ww[i], v[i], yh);
                        } else {
                            // BF16(2 h) (BF16(h) in training): 16 columns = two 16-byte units of chunk n0/64
                            uint8_t* base = act + (n0 >> 6) * kChunkA;
                            const int j0 = (n0 & 63) >> 3;
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const float* x = v + 8 * h;
                                st_shared_v4(base + swz(r, j0 + h), pack_bf16(x[0], x[1]), pack_bf16(x[2], x[3]),
                                             pack_bf16(x[4], x[5]), pack_bf16(x[6], x[7]));
                            }
                        }
                    }
                    if (!head) {
                        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                    } else if (cq > 0) {
                        // the other column quarters' head sums for quarter 0; a quarter can only
                        // overwrite its slot at the chain's next unit, after quarter 0 has
                        // arrived on that unit's act_ready
                        head_part[s][cq - 1][r] = yh;
                        mbar_arrive(&head_bar[s]);
                    }
                    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                    mbar_arrive(&act_ready[s]);
                    if (head && cq == 0) {
                        if (!(ok = wait_bar(&head_bar[s], (uint32_t)(k & 1), g.status, abort_v))) break;
                        const int row = tile * kRows + r;
                        const float sum = ((yh + head_part[s][0][r]) + head_part[s][1][r]) + head_part[s][2][r];
                        if (row < g.n)
                            g.pred[(long long)mem * g.pred_stride + row] = fmaf(sum, TRAIN ? 1.0f : 0.5f, prm[g.off_b5]);
                    }
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
