// Blackwell (sm_103a) tensor-core GEMM for the surrogate's forward layers:
// TMA loads 64-wide K chunks of A (128 rows) and B (N rows) with 128-byte
// swizzle into shared memory, one thread issues tcgen05.mma (kind::f16, BF16
// inputs, FP32 accumulator in tensor memory), tcgen05.commit signals an
// mbarrier, and four warps read the accumulator rows back with tcgen05.ld for
// a fused bias + GELU epilogue.
//
//   C[m][n] = sum_k A[m][k] * B[n][k]   (both operands K-major, BF16)
//   H[m][n] = bf16(gelu(C[m][n] + bias[n])), optionally G[m][n] = fp16(gelu'(C[m][n] + bias[n]))
//
// Every wait is bounded: on timeout the kernel records TUNE_ETIMEOUT's status
// bit, waits (bounded) for its own copies and MMAs, frees its tensor memory
// and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "gelu.cuh"

namespace tc {

constexpr int kThreads = 256;  // eight warps: two per TMEM lane quarter (column halves)
constexpr int BM = 128;        // rows per CTA (UMMA M)
constexpr int BK = 64;         // K elements per chunk (one 128-byte swizzle span)
constexpr long long kSpin = 1LL << 22;  // try_wait iterations before giving up
constexpr long long kSpinShort = 1LL << 10;  // the first wait of a launch with an injected fault

struct Args {
    int M, N, K;
    int batched_a;          // A has a member coordinate (else member 0 for all)
    const float* bias;      // [members][N] at member stride sBias
    long long sBias;
    __half* G;              // optional [members][M][N]: gelu' of the pre-activations (backward pass)
    long long sG;
    __nv_bfloat16* H;       // [members][M][N]
    long long sH;
    int* status;            // bit 2 (timeout) set on a wait that gives up
    int fault_skip_first;   // injected fault: chunk 0 is never loaded; its wait gives up after kSpinShort
};

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(sa(b)), "r"(n));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(sa(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(sa(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait; false (and the status bit) after `limit` unsuccessful polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* status, long long limit = kSpin)
{
    for (long long i = 0; i < limit; ++i)
        if (mbar_try(b, parity)) return true;
    atomicOr(status, 2);
    return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(sa(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(sa(bar))
        : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(const void* p)
{
    const uint64_t addr = sa(p);
    return ((addr >> 4) & 0x3fffull) | (1ull << 16) | ((1024ull >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor: kind::f16, BF16 A and B, FP32 D, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(sa(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

using mlp::gelu;

// grid: (M / 128, members). Dynamic shared memory: 1024 alignment slack + kStages x (16 KB + N x 128 B).
// N: a multiple of 64 in [64, 256] (two column halves of whole 32-column loads). K chunks pass through a
// ring of kStages stages so that two CTAs fit on an SM and one's epilogue overlaps the other's MMAs.
constexpr int kStages = 2;

__host__ __device__ constexpr int smem_bytes(int N) { return 1024 + kStages * (BM * BK * 2 + N * BK * 2); }

__global__ void __launch_bounds__(kThreads) gemm_fwd_kernel(const __grid_constant__ CUtensorMap ta,
                                                            const __grid_constant__ CUtensorMap tb,
                                                            const __grid_constant__ Args g)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bar_full[kStages];
    __shared__ uint64_t bar_done[kStages];
    __shared__ uint64_t bar_mma;
    __shared__ uint32_t tmem_base;
    __shared__ int ok_flag;

    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int n_chunks = g.K / BK;
    const uint32_t a_bytes = BM * BK * 2, b_bytes = (uint32_t)g.N * BK * 2;
    uint8_t* sA = smem;                      // kStages x 16 KB
    uint8_t* sB = smem + kStages * a_bytes;  // kStages x (N x 128 B)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM, member = blockIdx.y;
    const uint32_t n_cols = g.N <= 32 ? 32 : g.N <= 64 ? 64 : g.N <= 128 ? 128 : 256;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(sa(&tmem_base)),
                     "r"(n_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (threadIdx.x == 32) {
        for (int c = 0; c < kStages; ++c) {
            mbar_init(&bar_full[c], 1);
            mbar_init(&bar_done[c], 1);
        }
        mbar_init(&bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        ok_flag = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (threadIdx.x == 0) {
        auto load = [&](int c) {  // chunk c -> stage c % kStages
            const int st = c % kStages;
            mbar_expect_tx(&bar_full[st], a_bytes + b_bytes);
            tma_load_3d(sA + st * a_bytes, &ta, c * BK, m0, g.batched_a ? member : 0, &bar_full[st]);
            tma_load_3d(sB + st * b_bytes, &tb, c * BK, 0, member, &bar_full[st]);
        };
        // with an injected fault chunk 0 is never requested (nothing is in flight for it), so
        // its wait below runs out after kSpinShort polls and the CTA takes the timeout path
        const bool skip0 = g.fault_skip_first != 0;
        for (int c = 0; c < n_chunks && c < kStages; ++c)
            if (!(skip0 && c == 0)) load(c);
        const uint32_t idesc = idesc_bf16(BM, g.N);
        int loaded = n_chunks < kStages ? n_chunks : kStages;  // chunks 0 .. loaded-1 requested
        bool ok = true;
        for (int c = 0; c < n_chunks; ++c) {
            const int st = c % kStages;
            ok = mbar_wait(&bar_full[st], (c / kStages) & 1, g.status, skip0 && c == 0 ? kSpinShort : kSpin);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
                mma_bf16(tmem, sdesc(sA + st * a_bytes + kk * 32), sdesc(sB + st * b_bytes + kk * 32), idesc,
                         (c | kk) != 0);
            mma_commit(&bar_done[st]);
            // refill the stage of the previous chunk once its MMAs are done
            if (c >= 1 && c - 1 + kStages < n_chunks) {
                const int pc = c - 1, pst = pc % kStages;
                ok = mbar_wait(&bar_done[pst], (pc / kStages) & 1, g.status);
                if (!ok) break;
                load(pc + kStages);
                ++loaded;
            }
        }
        if (!ok) {
            ok_flag = 0;
            // let the copies already issued finish before the CTA exits
            for (int c = skip0 ? 1 : 0; c < loaded; ++c)
                mbar_wait(&bar_full[c % kStages], (c / kStages) & 1, g.status);
        }
        mma_commit(&bar_mma);  // arrives when the issued MMAs (if any) complete
    }
    // epilogue: thread = accumulator row (TMEM lane); warp w reads lane quarter w % 4 and
    // column half w / 4, 32 columns per load
    const bool done = mbar_wait(&bar_mma, 0, g.status);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (done && ok_flag) {
        const int quarter = warp & 3, half = warp >> 2;
        const int row = m0 + quarter * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
        const float* bias = g.bias + member * g.sBias;
        __nv_bfloat16* H = g.H + member * g.sH + (long long)row * g.N;
        __half* G = g.G ? g.G + member * g.sG : nullptr;  // tiled layout (mlp::gprime_at), N = 256
        const int c_beg = half * (g.N / 2), c_end = c_beg + g.N / 2;
        for (int c0 = c_beg; c0 < c_end; c0 += 32) {
            float v[32];
            tmem_ld32(lane_addr + c0, v);
#pragma unroll
            for (int i = 0; i < 32; i += 4) {
                const float4 b4 = __ldg(reinterpret_cast<const float4*>(bias + c0 + i));
                v[i] += b4.x;
                v[i + 1] += b4.y;
                v[i + 2] += b4.z;
                v[i + 3] += b4.w;
            }
            if (G) {
#pragma unroll
                for (int i = 0; i < 32; i += 8) {
                    uint4 pk;
                    uint32_t* q = reinterpret_cast<uint32_t*>(&pk);
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const __half2 d = __floats2half2_rn(mlp::gelu_grad(v[i + 2 * t]), mlp::gelu_grad(v[i + 2 * t + 1]));
                        q[t] = *reinterpret_cast<const uint32_t*>(&d);
                    }
                    *reinterpret_cast<uint4*>(G + mlp::gprime_at(row, c0 + i)) = pk;
                }
            }
#pragma unroll
            for (int i = 0; i < 32; i += 8) {
                __nv_bfloat162 h0 = __floats2bfloat162_rn(gelu(v[i]), gelu(v[i + 1]));
                __nv_bfloat162 h1 = __floats2bfloat162_rn(gelu(v[i + 2]), gelu(v[i + 3]));
                __nv_bfloat162 h2 = __floats2bfloat162_rn(gelu(v[i + 4]), gelu(v[i + 5]));
                __nv_bfloat162 h3 = __floats2bfloat162_rn(gelu(v[i + 6]), gelu(v[i + 7]));
                uint4 pk;
                pk.x = *reinterpret_cast<uint32_t*>(&h0);
                pk.y = *reinterpret_cast<uint32_t*>(&h1);
                pk.z = *reinterpret_cast<uint32_t*>(&h2);
                pk.w = *reinterpret_cast<uint32_t*>(&h3);
                *reinterpret_cast<uint4*>(H + c0 + i) = pk;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(n_cols));
}

}  // namespace tc
