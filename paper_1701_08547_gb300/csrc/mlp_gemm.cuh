// BF16 tensor-core GEMM for the surrogate MLP (CTA tile 128 x 128 x 32, 8 warps,
// cp.async double buffering, ldmatrix fragments, FP32 accumulation).
//
// C[m][n] = sum_k A(m, k) * B(k, n), batched over blockIdx.z (ensemble members).
// Operand layouts in global memory:
//   A: A_KM = false -> A[m * lda + k] (K contiguous); true -> A[k * lda + m] (M contiguous)
//   B: B_KN = false -> B[n * ldb + k] (K contiguous); true -> B[k * ldb + n] (N contiguous)
// Tiles are copied to shared memory in their global orientation; ldmatrix.trans
// produces the fragments of the transposed orientations. M, N multiples of 64 (a
// tile's rows past M or N are filled with zeros and not stored), K a multiple of 32,
// leading dimensions multiples of 8 elements.
#pragma once

#include "gelu.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace mlp {

constexpr int GBM = 128, GBN = 128, GBK = 32;
constexpr int kGemmThreads = 256;

enum Epilogue : int {
    EPI_BIAS_GELU = 0,  // z = acc + bias[n]; G[m][n] = fp16(gelu'(z)) (optional); H[m][n] = bf16(gelu(z))
    EPI_GELU_GRAD = 1,  // D[m][n] = bf16(acc * G[m][n])
    EPI_F32 = 2,        // F[m][n] = acc (fp32)
};

struct GemmArgs {
    const __nv_bfloat16* A;
    const __nv_bfloat16* B;
    int M, N, K, lda, ldb;
    long long sA, sB;  // per-batch strides (elements)
    // epilogue operands (per-batch strides in elements)
    const float* bias;
    long long sBias;
    __half* G;         // EPI_BIAS_GELU: gelu'(pre-activation) out (may be null); EPI_GELU_GRAD: its input;
                       // N = 256 columns in the tiled layout of gprime_at (ldc does not apply)
    long long sG;
    __nv_bfloat16* H;  // bf16 output
    long long sH;
    float* F;          // fp32 output
    long long sF;
    int ldc;           // leading dimension of H / F
    int k_split;       // split-K: blockIdx.z = batch * k_split + split; F gets [split] slices
    long long sSplit;  // stride between split slices of F
};


__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Shared-memory tile geometry (bf16 elements), padded by 8 elements per row so
// that the eight 16-byte rows of every ldmatrix fall in distinct banks.
template <bool KM>
struct Tile;
template <>
struct Tile<false> {  // [128 rows (m or n)][32 k]
    static constexpr int ROW = GBK + 8;
    static constexpr int ELEMS = GBM * ROW;
};
template <>
struct Tile<true> {  // [32 k][128 (m or n)]
    static constexpr int ROW = GBM + 8;
    static constexpr int ELEMS = GBK * ROW;
};

// Copy one 128 x 32 operand tile (global orientation kept) with 16-byte cp.async; rows
// (m or n) at or past lim are zero-filled instead of read.
template <bool KM>
__device__ __forceinline__ void load_tile(__nv_bfloat16* s, const __nv_bfloat16* g, int ld, int row0, int k0, int lim)
{
    const int t = threadIdx.x;
    if (!KM) {  // 128 rows x 32 k: 4 chunks of 8 per row -> 512 chunks
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int c = t + i * kGemmThreads;
            const int r = c >> 2, q = c & 3;
            __nv_bfloat16* d = s + r * Tile<false>::ROW + q * 8;
            if (row0 + r < lim)
                cp_async16(d, g + (long long)(row0 + r) * ld + k0 + q * 8);
            else
                *reinterpret_cast<uint4*>(d) = make_uint4(0u, 0u, 0u, 0u);
        }
    } else {  // 32 k x 128: 16 chunks per k row -> 512 chunks
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int c = t + i * kGemmThreads;
            const int r = c >> 4, q = c & 15;
            __nv_bfloat16* d = s + r * Tile<true>::ROW + q * 8;
            if (row0 + q * 8 < lim)
                cp_async16(d, g + (long long)(k0 + r) * ld + row0 + q * 8);
            else
                *reinterpret_cast<uint4*>(d) = make_uint4(0u, 0u, 0u, 0u);
        }
    }
}

// A fragment (16 x 16 at rows m0.., k k0..) for the warp.
template <bool KM>
__device__ __forceinline__ void frag_a(uint32_t (&a)[4], const __nv_bfloat16* s, int m0, int k0, int lane)
{
    const int q = lane >> 3, r = lane & 7;
    if (!KM) {
        // matrices: (m 0-7, k 0-7), (m 8-15, k 0-7), (m 0-7, k 8-15), (m 8-15, k 8-15)
        const int m = m0 + (q & 1) * 8 + r, k = k0 + (q >> 1) * 8;
        ldsm_x4(a, s + m * Tile<false>::ROW + k);
    } else {
        // stored [k][m]: matrix q covers m (q & 1) * 8.., k (q >> 1) * 8..; rows of the stored matrix are k
        const int k = k0 + (q >> 1) * 8 + r, m = m0 + (q & 1) * 8;
        ldsm_x4_t(a, s + k * Tile<true>::ROW + m);
    }
}

// B fragments for two n8 tiles (n0.. n0 + 15) at k k0..: b[0], b[1] for n0..n0+7; b[2], b[3] for n0+8..
template <bool KN>
__device__ __forceinline__ void frag_b(uint32_t (&b)[4], const __nv_bfloat16* s, int n0, int k0, int lane)
{
    const int q = lane >> 3, r = lane & 7;
    if (!KN) {
        // stored [n][k]: matrices (n 0-7, k 0-7), (n 0-7, k 8-15), (n 8-15, k 0-7), (n 8-15, k 8-15)
        const int n = n0 + (q >> 1) * 8 + r, k = k0 + (q & 1) * 8;
        ldsm_x4(b, s + n * Tile<false>::ROW + k);
    } else {
        // stored [k][n]: same four matrices, transposed on load
        const int k = k0 + (q & 1) * 8 + r, n = n0 + (q >> 1) * 8;
        ldsm_x4_t(b, s + k * Tile<true>::ROW + n);
    }
}

template <bool A_KM, bool B_KN, int EPI>
__global__ void __launch_bounds__(kGemmThreads) gemm_bf16_kernel(const __grid_constant__ GemmArgs g)
{
    __shared__ __align__(128) __nv_bfloat16 sA[2][Tile<A_KM>::ELEMS];
    __shared__ __align__(128) __nv_bfloat16 sB[2][Tile<B_KN>::ELEMS];

    const int batch = blockIdx.z / g.k_split, split = blockIdx.z % g.k_split;
    const int m_blk = blockIdx.y * GBM, n_blk = blockIdx.x * GBN;
    const int k_len = g.K / g.k_split, k_beg = split * k_len;
    const __nv_bfloat16* A = g.A + batch * g.sA;
    const __nv_bfloat16* B = g.B + batch * g.sB;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 2) * 64, wn = (warp & 3) * 32;  // 2 x 4 warps, 64 x 32 each

    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.0f;

    const int n_k = k_len / GBK;
    load_tile<A_KM>(sA[0], A, g.lda, m_blk, k_beg, g.M);
    load_tile<B_KN>(sB[0], B, g.ldb, n_blk, k_beg, g.N);
    cp_async_commit();
    for (int kt = 0; kt < n_k; ++kt) {
        const int cur = kt & 1;
        if (kt + 1 < n_k) {
            load_tile<A_KM>(sA[cur ^ 1], A, g.lda, m_blk, k_beg + (kt + 1) * GBK, g.M);
            load_tile<B_KN>(sB[cur ^ 1], B, g.ldb, n_blk, k_beg + (kt + 1) * GBK, g.N);
        }
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; kk += 16) {
            uint32_t af[4][4], bf[2][4];
#pragma unroll
            for (int i = 0; i < 4; ++i) frag_a<A_KM>(af[i], sA[cur], wm + i * 16, kk, lane);
#pragma unroll
            for (int j = 0; j < 2; ++j) frag_b<B_KN>(bf[j], sB[cur], wn + j * 16, kk, lane);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j >> 1][(j & 1) * 2], bf[j >> 1][(j & 1) * 2 + 1]);
        }
        __syncthreads();
    }
    cp_async_wait<0>();

    // Epilogue: thread holds rows (lane >> 2) and + 8, columns 2 * (lane & 3) + {0, 1} of each 16 x 8.
    const int gr = lane >> 2, gc = (lane & 3) * 2;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = m_blk + wm + i * 16 + gr + h * 8;
                const int n = n_blk + wn + j * 8 + gc;
                if (m >= g.M || n >= g.N) continue;  // zero-filled rows of a partial tile
                const float v0 = acc[i][j][2 * h], v1 = acc[i][j][2 * h + 1];
                const long long off = (long long)m * g.ldc + n;
                if (EPI == EPI_BIAS_GELU) {
                    const float z0 = v0 + g.bias[batch * g.sBias + n];
                    const float z1 = v1 + g.bias[batch * g.sBias + n + 1];
                    if (g.G)
                        *reinterpret_cast<__half2*>(g.G + batch * g.sG + gprime_at(m, n)) =
                            __floats2half2_rn(gelu_grad(z0), gelu_grad(z1));
                    *reinterpret_cast<__nv_bfloat162*>(g.H + batch * g.sH + off) =
                        __floats2bfloat162_rn(gelu(z0), gelu(z1));
                } else if (EPI == EPI_GELU_GRAD) {
                    const float2 d = __half22float2(*reinterpret_cast<const __half2*>(g.G + batch * g.sG + gprime_at(m, n)));
                    *reinterpret_cast<__nv_bfloat162*>(g.H + batch * g.sH + off) =
                        __floats2bfloat162_rn(v0 * d.x, v1 * d.y);
                } else {
                    *reinterpret_cast<float2*>(g.F + batch * g.sF + split * g.sSplit + off) = make_float2(v0, v1);
                }
            }
        }
    }
}

}  // namespace mlp
