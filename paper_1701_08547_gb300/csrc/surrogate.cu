// Learned surrogate of the static cost: an ensemble of MLPs
// (64 inputs = 48 features + zero padding -> 256 -> 256 -> 256 -> 256 -> 1, GELU in tanh form),
// BF16 weights and activations, FP32 accumulation, FP32 master weights, Adam,
// trained by this file's kernels (forward, backward, optimiser) on the GPU.
// Members are batched through the grouped GEMM (blockIdx.z = member).
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include "mlp_gemm.cuh"
#include "pdl.cuh"
#include "tc_gemm.cuh"
#include "tc_mlp.cuh"
#include "tc_mlp_bwd.cuh"
#include "tc_wgrad.cuh"
#include "tune_internal.h"

using mlp::GemmArgs;

namespace {

constexpr int IN = TUNE_SURROGATE_INPUTS;  // input width (48 features + zeros: one 128-byte BF16 row)
constexpr int WID = 256;    // hidden width
constexpr int NL = 4;       // hidden layers
constexpr int KSPLIT = 8;   // split-K for weight gradients over the batch

// Per-member parameter layout (floats): W1 [256 x 64], b1, W2..W4 [256 x 256], b2..b4, w5 [256], b5.
__host__ __device__ constexpr long long fan_in(int l) { return l == 0 ? IN : WID; }
__host__ __device__ constexpr long long OFF_W(int l) { return l == 0 ? 0 : WID * IN + WID + (l - 1) * 65792LL; }
__host__ __device__ constexpr long long OFF_B(int l) { return OFF_W(l) + WID * fan_in(l); }
constexpr long long OFF_W5 = 214016, OFF_B5 = 214272;
constexpr long long P_REAL = 214273;
constexpr long long P = 214336;  // padded per-member stride (a multiple of 64 floats)
// bf16 copies of W1..W4 per member
__host__ __device__ constexpr long long BOFF_W(int l) { return l == 0 ? 0 : WID * IN + (l - 1) * 65536LL; }
constexpr long long PB = 212992;
static_assert(IN == tcm::kIn, "the fused kernels' input width");
static_assert(OFF_B(3) == 213760 && OFF_W5 == OFF_B(3) + WID && OFF_B5 == OFF_W5 + WID && P_REAL == OFF_B5 + 1 &&
                  P >= P_REAL && P % 64 == 0 && BOFF_W(3) + 65536 == PB,
              "layout");

}  // namespace

struct tune_surrogate {
    int members = 0, batch = 0;
    float lr = 1e-3f, b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    int step = 0;
    float *master = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16* wbf = nullptr;
    __nv_bfloat16* xin = nullptr;       // [batch x IN]
    __half* G[NL] = {};                 // gelu' of each layer's pre-activations, FP16 [members][batch x WID], tiled (mlp::gprime_at)
    __nv_bfloat16* H[NL] = {};          // [members][batch x WID]
    __nv_bfloat16* dZ[NL] = {};         // [members][batch x WID]: dZ of layer l (fused chain) or ping-pong
    float *y = nullptr, *lbl = nullptr, *loss = nullptr;  // [members][batch], [batch], [members]
    // the training batch being processed: its layer-1 input rows (xb_rows of them; rows past it
    // read as zeros through the tensor maps) and labels: xin / lbl after a gather, or the
    // caller's own arrays (fused tcgen05 path, no permutation)
    const __nv_bfloat16* xb = nullptr;
    const float* lb = nullptr;
    int xb_rows = 0;
    float* part = nullptr;              // split-K partials: part_slices x [WID x WID]
    int part_slices = 0;                // at least members x KSPLIT and the SM count
    void* block = nullptr;              // the one device allocation
    int* status = nullptr;              // device status word (timeouts of bounded waits)
    int use_tc = 1;                     // forward layers on tcgen05 (1) or mma.sync (0)
    int fwd_mode = 1;                   // surrogate_forward: 0 layer by layer, 1 fused BF16, 2 fused FP8
    int bwd_mode = 1;                   // backward: 0 mma.sync GEMMs, 1 fused input gradients + tcgen05 dW
    uint8_t* w8 = nullptr;              // E4M3 codes of W2..W4 [members][3][256][256]
    float* wscale = nullptr;            // their scales [members][3][256] (one per matrix, repeated per row)
    float* wscale_half = nullptr;       // the scales halved (the fused epilogue's multipliers)
    bool fp8_stale = true;              // master weights changed since the last quantisation
};

namespace {

template <typename T>
T* carve(char*& p, size_t count)
{
    T* r = reinterpret_cast<T*>(p);
    p += (count * sizeof(T) + 255) & ~size_t(255);
    return r;
}

// A kernel's dynamic shared-memory limit, set once per device (the attribute belongs to the
// device's context; `done` keeps one bit per device ordinal below 64).
template <typename Kernel>
int smem_attr(Kernel kernel, int bytes, std::atomic<uint64_t>& done, const char* what)
{
    int dev = 0;
    TUNE_CUDA_TRY(cudaGetDevice(&dev), what);
    const uint64_t bit = dev >= 0 && dev < 64 ? (1ull << dev) : 0;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return TUNE_OK;
    TUNE_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes), what);
    done.fetch_or(bit, std::memory_order_release);
    return TUNE_OK;
}

// ---- small kernels ------------------------------------------------------------

// y[mem][i] = sum_j w5[j] * H4[mem][i][j] + b5   (one warp per row, eight columns per lane)
__global__ void head_fwd(const __nv_bfloat16* __restrict__ H4, const float* __restrict__ master, float* y,
                         int n, int batch)
{
    const int mem = blockIdx.y;
    const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= n) return;
    const float* w5 = master + mem * P + OFF_W5 + 8 * lane;
    const uint4 hv = reinterpret_cast<const uint4*>(H4 + (long long)mem * batch * WID + (long long)row * WID)[lane];
    const float4 wa = *reinterpret_cast<const float4*>(w5), wb = *reinterpret_cast<const float4*>(w5 + 4);
    const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&hv);
    const float w[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
    float s = 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float2 f = __bfloat1622float2(h2[q]);
        s = fmaf(w[2 * q], f.x, s);
        s = fmaf(w[2 * q + 1], f.y, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[(long long)mem * batch + row] = s + master[mem * P + OFF_B5];
}

// Column sums over rows in two stages (deterministic): stage 1 sums slices of
// kRowSlice rows into part[mem][slice][WID + 1]; stage 2 adds the slices.
constexpr int kRowSlice = 64;
constexpr int kRedWarps = 32;  // warps per block of the slice sums

// Loss gradient and head backward in one pass over a slice of srows rows (block = (slice,
// member), 256 threads: eight row groups of 32 threads, each thread eight columns with 16-byte
// accesses): dy[i] = 2 (y[i] - lbl[i]) / n for the n labelled rows (0 past them),
// dZ4[i][j] = bf16(dy[i] * w5[j] * G4[i][j]) with G4 = gelu'(Z4), and part[.][.][j] = sum over
// the slice of dy[i] H4[i][j] (j < 256), of dy[i] (j = 256) and of (y[i] - lbl[i])^2 (j = 257;
// rows of kHeadStride floats). Row group q takes rows i0 + q, i0 + q + 8, ...; its sums are
// added to the other groups' in group order.
constexpr int kHeadGroups = 8;
constexpr int kHeadStride = WID + 2;
__global__ void __launch_bounds__(256) head_bwd(const float* __restrict__ y, const float* __restrict__ lbl, int n,
                                                const float* __restrict__ master, const __half* __restrict__ G4,
                                                const __nv_bfloat16* __restrict__ H4, __nv_bfloat16* dZ, float* part,
                                                int rows, int batch, int slices, int srows)
{
    pdl::grid_dep_enter();  // a step of the training chain: wait for the launch before it
    __shared__ float red[kHeadGroups][kHeadStride];
    const int mem = blockIdx.y, sl = blockIdx.x;
    const int q = threadIdx.x >> 5, j = 8 * (threadIdx.x & 31);
    const float* yv = y + (long long)mem * batch;
    const float n_f = (float)n;
    const long long base = (long long)mem * batch * WID + j;
    float w[8];
    {
        const float4 a = *reinterpret_cast<const float4*>(master + mem * P + OFF_W5 + j);
        const float4 b = *reinterpret_cast<const float4*>(master + mem * P + OFF_W5 + j + 4);
        w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w; w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
    }
    float sh[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, sb = 0.0f, se = 0.0f;
    const int i0 = sl * srows, i1 = min(rows, i0 + srows);
#pragma unroll 2
    for (int i = i0 + q; i < i1; i += kHeadGroups) {
        float di = 0.0f;
        if (i < n) {
            const float e = yv[i] - lbl[i];
            di = 2.0f * e / n_f;
            se += e * e;
        }
        const long long o = base + (long long)i * WID;
        const uint4 gv = __ldg(reinterpret_cast<const uint4*>(G4 + (long long)mem * batch * WID + mlp::gprime_at(i, j)));
        const uint4 hv = __ldg(reinterpret_cast<const uint4*>(H4 + o));
        const uint32_t gw[4] = {gv.x, gv.y, gv.z, gv.w}, hw[4] = {hv.x, hv.y, hv.z, hv.w};
        uint32_t out[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float2 g = __half22float2(*reinterpret_cast<const __half2*>(&gw[t]));
            const float2 h = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&hw[t]));
            const __nv_bfloat162 z = __floats2bfloat162_rn(di * w[2 * t] * g.x, di * w[2 * t + 1] * g.y);
            out[t] = *reinterpret_cast<const uint32_t*>(&z);
            sh[2 * t] = fmaf(di, h.x, sh[2 * t]);
            sh[2 * t + 1] = fmaf(di, h.y, sh[2 * t + 1]);
        }
        *reinterpret_cast<uint4*>(dZ + o) = make_uint4(out[0], out[1], out[2], out[3]);
        sb += di;
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) red[q][j + c] = sh[c];
    if (j == 0) {
        red[q][WID] = sb;
        red[q][WID + 1] = se;
    }
    __syncthreads();
    float* o = part + ((long long)mem * slices + sl) * kHeadStride;
    for (int c = threadIdx.x; c < kHeadStride; c += blockDim.x) {
        float v = red[0][c];
#pragma unroll
        for (int g = 1; g < kHeadGroups; ++g) v += red[g][c];
        o[c] = v;
    }
}

// part[.][.][j] = sum over the slice of dZ[i][j] (four independent partial sums)
__global__ void bias_partial(const __nv_bfloat16* __restrict__ dZ, float* part, int rows, int batch, int slices)
{
    const int mem = blockIdx.y, sl = blockIdx.x, j = threadIdx.x;
    const __nv_bfloat16* d = dZ + (long long)mem * batch * WID;
    float s[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    const int i0 = sl * kRowSlice, i1 = min(rows, i0 + kRowSlice);
    int i = i0;
    for (; i + 4 <= i1; i += 4) {
#pragma unroll
        for (int q = 0; q < 4; ++q) s[q] += __bfloat162float(d[(long long)(i + q) * WID + j]);
    }
    for (; i < i1; ++i) s[0] += __bfloat162float(d[(long long)i * WID + j]);
    part[((long long)mem * slices + sl) * (WID + 1) + j] = (s[0] + s[1]) + (s[2] + s[3]);
}

// grad[mem * P + off + j] = sum over slices of part[mem][slice][j], j < cols (slice rows of
// `stride` floats); with `loss`, column cols is the slices' sum of squared errors and
// loss[mem] = that sum / n. Block = 32 columns x kRedWarps warps; warp w adds slices w,
// w + kRedWarps, ... in order, then the warps' partial sums are added in warp order
// (deterministic).
__global__ void slices_reduce(const float* __restrict__ part, float* grad, long long off, int cols, int slices,
                              int stride, float* loss, int n)
{
    pdl::grid_dep_enter();  // a step of the training chain: wait for the launch before it
    // block = 32 columns x kRedWarps warps; warp w adds slices w, w + kRedWarps, ..., then
    // the warps' sums are added in warp order
    const int mem = blockIdx.y, w = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + (threadIdx.x & 31);
    __shared__ float red[kRedWarps][32];
    const int ncol = cols + (loss ? 1 : 0);
    float s = 0.0f;
    if (j < ncol)
        for (int q = w; q < slices; q += kRedWarps) s += part[((long long)mem * slices + q) * stride + j];
    red[w][threadIdx.x & 31] = s;
    __syncthreads();
    if (w == 0 && j < ncol) {
        float t = red[0][threadIdx.x];
#pragma unroll
        for (int q = 1; q < kRedWarps; ++q) t += red[q][threadIdx.x];
        if (j < cols)
            grad[mem * P + off + j] = t;
        else
            loss[mem] = t / (float)n;
    }
}

// grad W[o][i] = sum over splits of part[split][o][i], added in split order; four
// consecutive elements per thread (member m's partials start at part + m * mstride,
// partial q at + q * qstride; both strides multiples of 4). With bpart, the grid has
// one more block (256 threads), which forms the bias gradient grad b[o] = sum over the
// brows rows of bpart[m][.][o], in row order.
__global__ void split_reduce(const float* __restrict__ part, float* grad, long long off_w, int cols, int splits,
                             long long mstride, long long qstride, const float* __restrict__ bpart = nullptr,
                             long long off_b = 0, int brows = 0)
{
    const int mem = blockIdx.y;
    if (bpart && blockIdx.x == gridDim.x - 1) {
        const float* b = bpart + (long long)mem * brows * WID + threadIdx.x;
        float s = 0.0f;
        for (int q0 = 0; q0 < brows; q0 += 16) {
            // up to 16 rows requested together, then added in row order
            float t[16];
#pragma unroll
            for (int q = 0; q < 16; ++q)
                if (q0 + q < brows) t[q] = __ldg(b + (long long)(q0 + q) * WID);
#pragma unroll
            for (int q = 0; q < 16; ++q)
                if (q0 + q < brows) s += t[q];
        }
        grad[mem * P + off_b + threadIdx.x] = s;
        return;
    }
    const int e = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (e >= WID * cols) return;
    const float* p = part + (long long)mem * mstride + e;
    float4 s = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int q0 = 0; q0 < splits; q0 += 16) {
        // up to 16 partials requested together, then added in split order
        float4 t[16];
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (q0 + q < splits) t[q] = __ldg(reinterpret_cast<const float4*>(p + (long long)(q0 + q) * qstride));
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (q0 + q < splits) {
                s.x += t[q].x;
                s.y += t[q].y;
                s.z += t[q].z;
                s.w += t[q].w;
            }
    }
    *reinterpret_cast<float4*>(grad + mem * P + off_w + e) = s;
}

// Adam on FP32 master weights, then the BF16 copies of W1..W4; four consecutive
// parameters per thread (every parameter segment starts at a multiple of 4, so a group
// lies in one segment; padding past the last parameter is left alone).
__global__ void adam_update(float* master, const float* grad, float* m, float* v, __nv_bfloat16* wbf, int members,
                            float lr, float b1, float b2, float eps, float c1, float c2)
{
    pdl::grid_dep_enter();  // a step of the training chain: wait for the launch before it
    const long long e = 4 * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
    if (e >= (long long)members * P) return;
    const long long p = e % P;
    if (p >= P_REAL) return;
    float4 g4 = *reinterpret_cast<const float4*>(grad + e);
    float4 m4 = *reinterpret_cast<const float4*>(m + e), v4 = *reinterpret_cast<const float4*>(v + e);
    float4 w4 = *reinterpret_cast<const float4*>(master + e);
    const float* gg = &g4.x;
    float* mm = &m4.x;
    float* vv = &v4.x;
    float* ww = &w4.x;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (p + k >= P_REAL) break;
        mm[k] = b1 * mm[k] + (1.0f - b1) * gg[k];
        vv[k] = b2 * vv[k] + (1.0f - b2) * gg[k] * gg[k];
        ww[k] = ww[k] - lr * (mm[k] / c1) / (sqrtf(vv[k] / c2) + eps);
    }
    *reinterpret_cast<float4*>(m + e) = m4;
    *reinterpret_cast<float4*>(v + e) = v4;
    *reinterpret_cast<float4*>(master + e) = w4;
    const long long mem = e / P;
    for (int l = 0; l < NL; ++l) {
        const long long len = WID * fan_in(l);
        if (p >= OFF_W(l) && p < OFF_W(l) + len) {
            __nv_bfloat162* dst = reinterpret_cast<__nv_bfloat162*>(wbf + mem * PB + BOFF_W(l) + (p - OFF_W(l)));
            dst[0] = __floats2bfloat162_rn(ww[0], ww[1]);
            dst[1] = __floats2bfloat162_rn(ww[2], ww[3]);
        }
    }
}

__global__ void cast_weights(const float* master, __nv_bfloat16* wbf, int members)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)members * PB) return;
    const long long mem = e / PB, q = e % PB;
    int l = NL - 1;
    while (l > 0 && q < BOFF_W(l)) --l;
    wbf[e] = __float2bfloat16_rn(master[mem * P + OFF_W(l) + (q - BOFF_W(l))]);
}

// Per-row E4M3 quantisation of W2..W4 (FP32, as the oracle mirrors it): s = max |w| / 448
// (1 for a zero row), code = E4M3(w / s), nearest-even, saturating. grid (256, 3, members) x 256.
__global__ void quantize_fp8(const float* __restrict__ master, uint8_t* w8, float* wscale, float* wscale_half)
{
    // block = one matrix W_l of one member; thread t = column t (coalesced row reads)
    const int l = blockIdx.x + 1, mem = blockIdx.y, t = threadIdx.x;
    const float* W = master + mem * P + OFF_W(l);
    __shared__ float red[WID / 32];
    float a = 0.0f;
    for (int r = 0; r < WID; ++r) a = fmaxf(a, fabsf(W[(long long)r * WID + t]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
    if ((t & 31) == 0) red[t >> 5] = a;
    __syncthreads();
    float amax = 0.0f;
#pragma unroll
    for (int i = 0; i < WID / 32; ++i) amax = fmaxf(amax, red[i]);
    const float sc = amax > 0.0f ? __fdiv_rn(amax, 448.0f) : 1.0f;
    const long long m0 = ((long long)mem * 3 + (l - 1)) * WID;
    for (int r = 0; r < WID; ++r)
        w8[(m0 + r) * WID + t] = __nv_cvt_float_to_fp8(__fdiv_rn(W[(long long)r * WID + t], sc), __NV_SATFINITE, __NV_E4M3);
    wscale[m0 + t] = sc;  // every row of the matrix carries the matrix's scale
    wscale_half[m0 + t] = 0.5f * sc;
}

// Batch gather: xin[r] = feats[order[r]], lbl[r] = labels[order[r]] (rows past n are zero).
__global__ void gather_batch(const __nv_bfloat16* __restrict__ feats, const float* __restrict__ labels,
                             const int32_t* __restrict__ order, int n, int batch, __nv_bfloat16* xin, float* lbl)
{
    pdl::grid_dep_enter();  // a step of the training chain: wait for the launch before it
    const int r = blockIdx.x;
    const int c = threadIdx.x;  // 64 threads x 2 elements
    const __nv_bfloat162 z = __floats2bfloat162_rn(0.0f, 0.0f);
    __nv_bfloat162 val = z;
    if (r < n) {
        const long long src = order ? order[r] : r;
        val = reinterpret_cast<const __nv_bfloat162*>(feats + src * IN)[c];
        if (c == 0) lbl[r] = labels[src];
    } else if (c == 0) {
        lbl[r] = 0.0f;
    }
    reinterpret_cast<__nv_bfloat162*>(xin + (long long)r * IN)[c] = val;
}

// The same gather with 16-byte accesses (feats 16-byte aligned): kRowU4 threads per row of
// IN BF16 values, 256 / kRowU4 rows per block of 256 threads.
constexpr int kRowU4 = IN * 2 / 16;
constexpr int kGatherRows = 256 / kRowU4;
__global__ void gather_batch16(const __nv_bfloat16* __restrict__ feats, const float* __restrict__ labels,
                               const int32_t* __restrict__ order, int n, int batch, __nv_bfloat16* xin, float* lbl)
{
    pdl::grid_dep_enter();  // a step of the training chain: wait for the launch before it
    const int r = blockIdx.x * kGatherRows + threadIdx.x / kRowU4, c = threadIdx.x % kRowU4;
    if (r >= batch) return;
    uint4 val = make_uint4(0u, 0u, 0u, 0u);
    float lab = 0.0f;
    if (r < n) {
        const long long src = order ? order[r] : r;
        val = __ldg(reinterpret_cast<const uint4*>(feats + src * IN) + c);
        if (c == 0) lab = labels[src];
    }
    reinterpret_cast<uint4*>(xin + (long long)r * IN)[c] = val;
    if (c == 0) lbl[r] = lab;
}

template <bool A_KM, bool B_KN, int EPI>
int gemm(const GemmArgs& g, int batches, cudaStream_t s)
{
    dim3 grid((g.N + mlp::GBN - 1) / mlp::GBN, (g.M + mlp::GBM - 1) / mlp::GBM, batches * g.k_split);
    mlp::gemm_bf16_kernel<A_KM, B_KN, EPI><<<grid, mlp::kGemmThreads, 0, s>>>(g);
    TUNE_CUDA_TRY(cudaGetLastError(), "surrogate: gemm launch");
    return TUNE_OK;
}

GemmArgs gargs()
{
    GemmArgs g;
    memset(&g, 0, sizeof(g));
    g.k_split = 1;
    return g;
}

// ---- tcgen05 forward layers -----------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 3-D BF16 map [batch][rows][K] (K contiguous), box 64 x box_rows x 1, 128-byte swizzle.
int make_map(CUtensorMap* map, const void* base, uint64_t K, uint64_t rows, uint64_t batch, uint64_t row_bytes,
             uint64_t batch_bytes, uint32_t box_rows)
{
    auto fn = encode_fn();
    if (!fn) return tune::fail(TUNE_ECUDA, "surrogate: cuTensorMapEncodeTiled unavailable");
    const cuuint64_t dims[3] = {K, rows, batch};
    const cuuint64_t strides[2] = {row_bytes, batch_bytes};
    const cuuint32_t box[3] = {64, box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return tune::fail(TUNE_ECUDA, "surrogate: cuTensorMapEncodeTiled failed (%d)", (int)r);
    return TUNE_OK;
}

// One forward layer for every member: H = gelu(A W^T + b) (and G = gelu'(A W^T + b)) with tcgen05.
int tc_layer(tune_surrogate* h, int l, int n_pad, cudaStream_t s, const __nv_bfloat16* x_in, int n_valid,
             bool store_z)
{
    const int kin = (int)fan_in(l);
    CUtensorMap ta, tb;
    int rc;
    if (l == 0)  // rows past n_valid read as zeros (TMA out-of-bounds fill)
        rc = make_map(&ta, x_in, IN, n_valid, 1, IN * 2, (uint64_t)n_pad * IN * 2, tc::BM);
    else
        rc = make_map(&ta, h->H[l - 1], WID, n_pad, h->members, WID * 2, (uint64_t)h->batch * WID * 2, tc::BM);
    if (rc) return rc;
    rc = make_map(&tb, h->wbf + BOFF_W(l), kin, WID, h->members, (uint64_t)kin * 2, (uint64_t)PB * 2, WID);
    if (rc) return rc;
    tc::Args g;
    g.M = n_pad;
    g.N = WID;
    g.K = kin;
    g.batched_a = l != 0;
    g.bias = h->master + OFF_B(l);
    g.sBias = P;
    g.G = store_z ? h->G[l] : nullptr;
    g.sG = (long long)h->batch * WID;
    g.H = h->H[l];
    g.sH = (long long)h->batch * WID;
    g.status = h->status;
    g.fault_skip_first = tune::take_fault(TUNE_FAULT_WAIT) ? 1 : 0;
    const int smem = tc::smem_bytes(WID);
    static std::atomic<uint64_t> attr{0};
    rc = smem_attr(tc::gemm_fwd_kernel, smem, attr, "surrogate: tc smem attribute");
    if (rc) return rc;
    tc::gemm_fwd_kernel<<<dim3(n_pad / tc::BM, h->members), tc::kThreads, smem, s>>>(ta, tb, g);
    TUNE_CUDA_TRY(cudaGetLastError(), "surrogate: tc gemm launch");
    return TUNE_OK;
}

// N-D map (N <= 4) with 128-byte swizzle; strides in bytes for dimensions 1..N-1.
int make_map_nd(CUtensorMap* map, CUtensorMapDataType dt, int rank, const void* base, const cuuint64_t* dims,
                const cuuint64_t* strides, const cuuint32_t* box)
{
    auto fn = encode_fn();
    if (!fn) return tune::fail(TUNE_ECUDA, "surrogate: cuTensorMapEncodeTiled unavailable");
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = fn(map, dt, rank, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return tune::fail(TUNE_ECUDA, "surrogate: cuTensorMapEncodeTiled failed (%d)", (int)r);
    return TUNE_OK;
}

int refresh_fp8(tune_surrogate* h, cudaStream_t s)
{
    if (!h->fp8_stale) return TUNE_OK;
    quantize_fp8<<<dim3(NL - 1, h->members), WID, 0, s>>>(h->master, h->w8, h->wscale, h->wscale_half);
    TUNE_CUDA_TRY(cudaGetLastError(), "surrogate: quantize launch");
    h->fp8_stale = false;
    return TUNE_OK;
}

template <bool FP8, bool TRAIN = false>
int launch_fused(const CUtensorMap& tx, const CUtensorMap& tw1, const CUtensorMap& tw, const CUtensorMap& th,
                 const tcm::Args& g, unsigned grid, cudaStream_t s)
{
    constexpr int smem = tcm::Cfg<FP8>::smem;
    static std::atomic<uint64_t> attr{0};
    const int rc = smem_attr(tcm::mlp_infer_kernel<FP8, TRAIN>, smem, attr, "surrogate: fused smem attribute");
    if (rc) return rc;
    if constexpr (TRAIN)  // a step of the training chain (pdl.cuh)
        TUNE_CUDA_TRY(pdl::launch_dep(tcm::mlp_infer_kernel<FP8, TRAIN>, dim3(grid), dim3(tcm::kThreads), smem, s, tx,
                                      tw1, tw, th, g),
                      "surrogate: fused launch");
    else
        tcm::mlp_infer_kernel<FP8, TRAIN><<<grid, tcm::kThreads, smem, s>>>(tx, tw1, tw, th, g);
    TUNE_CUDA_TRY(cudaGetLastError(), "surrogate: fused launch");
    return TUNE_OK;
}

// Whole-ensemble forward of n feature rows in one persistent launch (tc_mlp.cuh):
// pred[m][i] for every member; BF16 throughout, or layers 2-4 on E4M3 codes.
int fused_forward(tune_surrogate* h, const __nv_bfloat16* feats, int64_t n, float* pred, bool fp8, cudaStream_t s)
{
    if (n <= 0) return TUNE_OK;
    if (n > (1LL << 30)) return tune::fail(TUNE_EINVAL, "surrogate_forward: more than 2^30 rows");
    if (fp8) {
        int rc = refresh_fp8(h, s);
        if (rc) return rc;
    }
    // The tensor maps address 8-byte elements: TMA moves the same bytes with the same
    // 128-byte swizzle whatever the element type, in a quarter (BF16) or an eighth (E4M3)
    // of the element count. Dimension 0 and the boxes are in 8-byte units.
    CUtensorMap tx, tw1, tw;
    const auto u64 = CU_TENSOR_MAP_DATA_TYPE_UINT64;
    const cuuint64_t xd[2] = {IN * 2 / 8, (cuuint64_t)n}, xs[1] = {IN * 2};
    const cuuint32_t xb[2] = {16, tcm::kRows};
    int rc = make_map_nd(&tx, u64, 2, feats, xd, xs, xb);
    if (rc) return rc;
    const cuuint64_t d1[3] = {IN * 2 / 8, WID, (cuuint64_t)h->members}, s1[2] = {IN * 2, PB * 2};
    const cuuint32_t b1[3] = {16, WID, 1};
    rc = make_map_nd(&tw1, u64, 3, h->wbf, d1, s1, b1);
    if (rc) return rc;
    const cuuint32_t bw[4] = {16, WID, 1, 1};
    if (fp8) {
        const cuuint64_t dw[4] = {WID / 8, WID, NL - 1, (cuuint64_t)h->members};
        const cuuint64_t sw[3] = {WID, WID * WID, (NL - 1) * WID * WID};
        rc = make_map_nd(&tw, u64, 4, h->w8, dw, sw, bw);
    } else {
        const cuuint64_t dw[4] = {WID * 2 / 8, WID, NL - 1, (cuuint64_t)h->members};
        const cuuint64_t sw[3] = {WID * 2, WID * WID * 2, PB * 2};
        rc = make_map_nd(&tw, u64, 4, h->wbf + BOFF_W(1), dw, sw, bw);
    }
    if (rc) return rc;
    tcm::Args g;
    g.n = (int)n;
    g.members = h->members;
    g.units = (n + tcm::kRows - 1) / tcm::kRows * h->members;
    g.master = h->master;
    g.P = P;
    for (int l = 0; l < NL; ++l) g.off_b[l] = OFF_B(l);
    g.off_w5 = OFF_W5;
    g.off_b5 = OFF_B5;
    g.wscale_half = h->wscale_half;
    g.pred = pred;
    g.pred_stride = n;
    for (int l = 0; l < NL; ++l) {
        g.g_out[l] = nullptr;
        g.h_out[l] = nullptr;
    }
    g.act_stride = 0;
    g.status = h->status;
    const long long sms = tune::device_sm_count();
    const unsigned grid = (unsigned)(g.units < sms ? g.units : sms);
    // (the activation map is used by the training variant only)
    return fp8 ? launch_fused<true>(tx, tw1, tw, tx, g, grid, s) : launch_fused<false>(tx, tw1, tw, tx, g, grid, s);
}

// Training forward of rows [0, n_pad) of the current batch (h->xb) through the fused kernel
// (BF16), keeping every layer's gelu'(Z) (FP16) and activations H for the backward pass and the
// head outputs in h->y.
int fused_train_forward(tune_surrogate* h, int n_pad, cudaStream_t s)
{
    CUtensorMap tx, tw1, tw;
    const auto u64 = CU_TENSOR_MAP_DATA_TYPE_UINT64;
    const cuuint64_t xd[2] = {IN * 2 / 8, (cuuint64_t)h->xb_rows}, xs[1] = {IN * 2};
    const cuuint32_t xb[2] = {16, tcm::kRows};
    int rc = make_map_nd(&tx, u64, 2, h->xb, xd, xs, xb);
    if (rc) return rc;
    const cuuint64_t d1[3] = {IN * 2 / 8, WID, (cuuint64_t)h->members}, s1[2] = {IN * 2, PB * 2};
    const cuuint32_t b1[3] = {16, WID, 1};
    rc = make_map_nd(&tw1, u64, 3, h->wbf, d1, s1, b1);
    if (rc) return rc;
    const cuuint32_t bw[4] = {16, WID, 1, 1};
    const cuuint64_t dw[4] = {WID * 2 / 8, WID, NL - 1, (cuuint64_t)h->members};
    const cuuint64_t sw[3] = {WID * 2, WID * WID * 2, PB * 2};
    rc = make_map_nd(&tw, u64, 4, h->wbf + BOFF_W(1), dw, sw, bw);
    if (rc) return rc;
    // H of layers 1-3 as the kernel stores them from its activation buffer: 128-row boxes of one
    // 128-byte column chunk, dimension 3 = layer (the H buffers are carved at a constant stride)
    const long long hstride = (const char*)h->H[1] - (const char*)h->H[0];
    if ((const char*)h->H[2] - (const char*)h->H[1] != hstride || hstride <= 0 || hstride % 16)
        return tune::fail(TUNE_EINVAL, "surrogate: activation buffers are not evenly spaced");
    CUtensorMap th;
    const cuuint64_t hd[4] = {WID * 2 / 8, (cuuint64_t)n_pad, (cuuint64_t)h->members, NL - 1};
    const cuuint64_t hs[3] = {WID * 2, (cuuint64_t)h->batch * WID * 2, (cuuint64_t)hstride};
    const cuuint32_t hb[4] = {16, tcm::kRows, 1, 1};
    rc = make_map_nd(&th, u64, 4, h->H[0], hd, hs, hb);
    if (rc) return rc;
    tcm::Args g;
    g.n = n_pad;
    g.members = h->members;
    g.units = (long long)(n_pad / tcm::kRows) * h->members;
    g.master = h->master;
    g.P = P;
    for (int l = 0; l < NL; ++l) g.off_b[l] = OFF_B(l);
    g.off_w5 = OFF_W5;
    g.off_b5 = OFF_B5;
    g.wscale_half = h->wscale_half;
    g.pred = h->y;
    g.pred_stride = h->batch;
    for (int l = 0; l < NL; ++l) {
        g.g_out[l] = h->G[l];
        g.h_out[l] = h->H[l];
    }
    g.act_stride = (long long)h->batch * WID;
    g.status = h->status;
    const long long sms = tune::device_sm_count();
    const unsigned grid = (unsigned)(g.units < sms ? g.units : sms);
    return launch_fused<false, true>(tx, tw1, tw, th, g, grid, s);
}

// Input gradients of layers 4, 3 and 2 in one persistent launch (tc_mlp_bwd.cuh):
// dz[l - 1] = bf16((dz[l] W_l) * G[l - 1]) for l = 3, 2, 1 (0-based), rows [0, n_pad),
// G = gelu'(Z) as the forward pass kept it.
int fused_backward(tune_surrogate* h, int n_pad, __nv_bfloat16* const* dz, cudaStream_t s)
{
    if (n_pad % tcm::kRows) return tune::fail(TUNE_EINVAL, "surrogate: fused backward needs whole 128-row tiles");
    CUtensorMap tdz, tw;
    const auto u64 = CU_TENSOR_MAP_DATA_TYPE_UINT64;
    const cuuint64_t dd[3] = {WID * 2 / 8, (cuuint64_t)n_pad, (cuuint64_t)h->members};
    const cuuint64_t ds[2] = {WID * 2, (cuuint64_t)h->batch * WID * 2};
    const cuuint32_t db[3] = {16, tcm::kRows, 1};
    int rc = make_map_nd(&tdz, u64, 3, dz[NL - 1], dd, ds, db);
    if (rc) return rc;
    // W2..W4 as the forward pass reads them ([o][i] rows), 64 rows o per box: the kernel reads
    // them MN-major, no transposed copy
    const cuuint64_t dw[4] = {WID * 2 / 8, WID, NL - 1, (cuuint64_t)h->members};
    const cuuint64_t sw[3] = {WID * 2, WID * WID * 2, PB * 2};
    const cuuint32_t bw[4] = {16, 64, 1, 1};
    rc = make_map_nd(&tw, u64, 4, h->wbf + BOFF_W(1), dw, sw, bw);
    if (rc) return rc;
    // dZ1..dZ3 as the kernel stores dZ3 and dZ2 from its activation buffer: 128-row boxes of one
    // 128-byte column chunk, dimension 3 = layer (the buffers must be evenly spaced)
    const long long zstride = (const char*)dz[1] - (const char*)dz[0];
    if ((const char*)dz[2] - (const char*)dz[1] != zstride || zstride <= 0 || zstride % 16)
        return tune::fail(TUNE_EINVAL, "surrogate: gradient buffers are not evenly spaced");
    CUtensorMap tdzs;
    const cuuint64_t zd[4] = {WID * 2 / 8, (cuuint64_t)n_pad, (cuuint64_t)h->members, NL - 1};
    const cuuint64_t zs[3] = {WID * 2, (cuuint64_t)h->batch * WID * 2, (cuuint64_t)zstride};
    const cuuint32_t zb[4] = {16, tcm::kRows, 1, 1};
    rc = make_map_nd(&tdzs, u64, 4, dz[0], zd, zs, zb);
    if (rc) return rc;
    tcm::BwdArgs g;
    g.members = h->members;
    g.units = (long long)(n_pad / tcm::kRows) * h->members;
    for (int j = 0; j < tcm::kBwdStages; ++j) {
        g.g[j] = h->G[NL - 2 - j];
        g.dz[j] = dz[NL - 2 - j];
        g.dz_coord[j] = NL - 2 - j;
    }
    g.act_stride = (long long)h->batch * WID;
    g.status = h->status;
    constexpr int smem = tcm::Cfg<false>::smem;
    static std::atomic<uint64_t> attr{0};
    rc = smem_attr(tcm::mlp_bwd_kernel, smem, attr, "surrogate: fused backward smem attribute");
    if (rc) return rc;
    const long long sms = tune::device_sm_count();
    const unsigned grid = (unsigned)(g.units < sms ? g.units : sms);
    TUNE_CUDA_TRY(pdl::launch_dep(tcm::mlp_bwd_kernel, dim3(grid), dim3(tcm::kThreads), smem, s, tdz, tw, tdzs, g),
                  "surrogate: fused backward launch");
    return TUNE_OK;
}

// Weight and bias gradients of every layer on tcgen05 in one launch (tc_wgrad.cuh): one CTA
// per 128 x 64 gradient tile and member, both operands MN-major, the whole batch in one TMEM
// accumulator. dz[l]: dZ of layer l ([members][batch][256]).
int wgrad_tc(tune_surrogate* h, int n_pad, __nv_bfloat16* const* dz, cudaStream_t s)
{
    const int M = h->members;
    tcw::Maps maps;
    tcw::Args g;
    memset(&g, 0, sizeof(g));
    const auto u64 = CU_TENSOR_MAP_DATA_TYPE_UINT64;
    const cuuint32_t box[3] = {16, tcw::kChunkRows, 1};
    const cuuint64_t da[3] = {WID * 2 / 8, (cuuint64_t)n_pad, (cuuint64_t)M};
    const cuuint64_t sa[2] = {WID * 2, (cuuint64_t)h->batch * WID * 2};
    g.n_items = NL;
    for (int j = 0; j < NL; ++j) {
        const int l = NL - 1 - j;  // layers 4, 3, 2, 1
        int rc = make_map_nd(&maps.ta[j], u64, 3, dz[l], da, sa, box);
        if (rc) return rc;
        if (l == 0) {
            const cuuint64_t db[3] = {IN * 2 / 8, (cuuint64_t)h->xb_rows, 1};
            const cuuint64_t sb[2] = {IN * 2, (cuuint64_t)h->xb_rows * IN * 2};
            rc = make_map_nd(&maps.tb[j], u64, 3, h->xb, db, sb, box);
        } else {
            rc = make_map_nd(&maps.tb[j], u64, 3, h->H[l - 1], da, sa, box);
        }
        if (rc) return rc;
        g.kin[j] = (int)fan_in(l);
        g.b_batched[j] = l != 0;
        g.grad_w[j] = OFF_W(l);
        g.grad_b[j] = OFF_B(l);
    }
    g.grad_stride = P;
    g.chunks = n_pad / tcw::kChunkRows;
    g.grad = h->grad;
    g.status = h->status;
    static std::atomic<uint64_t> attr{0};
    const int rc = smem_attr(tcw::wgrad_kernel, tcw::kSmem, attr, "surrogate: weight-gradient smem attribute");
    if (rc) return rc;
    TUNE_CUDA_TRY(pdl::launch_dep(tcw::wgrad_kernel, dim3(tcw::tiles_per_member(g), M), dim3(tcw::kThreads), tcw::kSmem,
                                  s, maps, g),
                  "surrogate: weight-gradient launch");
    return TUNE_OK;
}

// Forward through all members for rows [0, n_pad) (n_pad a multiple of 128).
// x_in: layer-1 input rows (null: the current training batch; else the caller's features on the
// tcgen05 path);
// n_valid rows of it exist; store_z keeps gelu' of the pre-activations for a backward pass.
int forward(tune_surrogate* h, int n_pad, cudaStream_t s, const __nv_bfloat16* x_in = nullptr, int n_valid = -1,
            bool store_z = true)
{
    // training with tcgen05 and the fused forward selected: one launch for all layers and the
    // head over the current batch (h->xb)
    if (store_z && h->use_tc && h->fwd_mode == 1 && !x_in) return fused_train_forward(h, n_pad, s);
    if (!x_in) x_in = h->xin;
    if (n_valid < 0) n_valid = n_pad;
    for (int l = 0; l < NL; ++l) {
        if (h->use_tc) {
            int rc = tc_layer(h, l, n_pad, s, x_in, n_valid, store_z);
            if (rc) return rc;
            continue;
        }
        GemmArgs g = gargs();
        g.A = l == 0 ? h->xin : h->H[l - 1];
        g.sA = l == 0 ? 0 : (long long)h->batch * WID;
        g.lda = l == 0 ? IN : WID;
        g.B = h->wbf + BOFF_W(l);
        g.sB = PB;
        g.ldb = (int)fan_in(l);
        g.M = n_pad;
        g.N = WID;
        g.K = (int)fan_in(l);
        g.bias = h->master + OFF_B(l);
        g.sBias = P;
        g.G = h->G[l];
        g.sG = (long long)h->batch * WID;
        g.H = h->H[l];
        g.sH = (long long)h->batch * WID;
        g.ldc = WID;
        int rc = gemm<false, false, mlp::EPI_BIAS_GELU>(g, h->members, s);
        if (rc) return rc;
    }
    head_fwd<<<dim3((n_pad + 7) / 8, h->members), 256, 0, s>>>(h->H[NL - 1], h->master, h->y, n_pad, h->batch);
    TUNE_CUDA_TRY(cudaGetLastError(), "surrogate: head launch");
    return TUNE_OK;
}

// Backward for the current batch (h->xb / h->lb; n valid rows, n_pad rows computed); grads into h->grad.
// Weight gradient of layer l as a split-K mma.sync GEMM (mlp_gemm.cuh) and its reduction into grad.
int wgrad_mma(tune_surrogate* h, int l, int n_pad, const __nv_bfloat16* dz, cudaStream_t s)
{
    const int B = h->batch;
    const int kin = (int)fan_in(l);
    GemmArgs g = gargs();
    g.A = dz;
    g.sA = (long long)B * WID;
    g.lda = WID;
    g.B = l == 0 ? h->xin : h->H[l - 1];
    g.sB = l == 0 ? 0 : (long long)B * WID;
    g.ldb = kin;
    g.M = WID;
    g.N = kin;
    g.K = n_pad;
    g.F = h->part;
    g.sF = (long long)KSPLIT * WID * WID;
    g.ldc = kin;
    // split the batch (K) so every split is a multiple of 32 rows: n_pad / 32 is a multiple of 4
    int splits = KSPLIT;
    while ((n_pad / 32) % splits) splits >>= 1;
    g.k_split = splits;
    g.sSplit = (long long)WID * WID;
    const int rc = gemm<true, true, mlp::EPI_F32>(g, h->members, s);
    if (rc) return rc;
    split_reduce<<<dim3((WID * kin / 4 + 255) / 256, h->members), 256, 0, s>>>(
        h->part, h->grad, OFF_W(l), kin, splits, (long long)KSPLIT * WID * WID, (long long)WID * WID);
    TUNE_CUDA_TRY(cudaGetLastError(), "surrogate: split reduce launch");
    return TUNE_OK;
}

int backward(tune_surrogate* h, int n, int n_pad, cudaStream_t s)
{
    const int B = h->batch;
    const int slices = (n_pad + kRowSlice - 1) / kRowSlice;
    // dZ of layer l: a buffer per layer when the input-gradient chain runs fused, else two
    // buffers in turn (each is consumed by its weight gradient before it is overwritten)
    const bool fused = h->use_tc && h->bwd_mode == 1;
    __nv_bfloat16* dzl[NL];
    for (int l = 0; l < NL; ++l) dzl[l] = h->dZ[fused ? l : (l & 1)];
    // the loss gradient, the head's weight and bias gradients (slices, then their sum), the
    // loss and dZ4 in one pass and its reduction: steps of the training chain (pdl.cuh)
    // (64-row slices, longer where their partials would not fit the partial buffer)
    int hrows = 64;
    while ((long long)h->members * ((n_pad + hrows - 1) / hrows) * kHeadStride > (long long)h->part_slices * WID * WID)
        hrows *= 2;
    const int hslices = (n_pad + hrows - 1) / hrows;
    TUNE_CUDA_TRY(pdl::launch_dep(head_bwd, dim3(hslices, h->members), dim3(32 * kHeadGroups), 0, s, h->y, h->lb, n,
                                  h->master, h->G[NL - 1], h->H[NL - 1], dzl[NL - 1], h->part, n_pad, B, hslices, hrows),
                  "surrogate: head backward launch");
    TUNE_CUDA_TRY(pdl::launch_dep(slices_reduce, dim3((kHeadStride + 31) / 32, h->members), dim3(32 * kRedWarps), 0,
                                  s, h->part, h->grad, OFF_W5, WID + 1, hslices, kHeadStride, h->loss, n),
                  "surrogate: head backward launch");
    TUNE_CUDA_TRY(cudaGetLastError(), "surrogate: head backward launch");
    if (fused) {  // input gradients dZ3..dZ1, then every layer's weight and bias gradients
        int rc = fused_backward(h, n_pad, dzl, s);
        if (rc) return rc;
        return wgrad_tc(h, n_pad, dzl, s);
    }
    // mma.sync backward: per layer the weight gradient, the bias gradient and the input gradient
    for (int l = NL - 1; l >= 0; --l) {
        const __nv_bfloat16* dz = dzl[l];
        const int kin = (int)fan_in(l);
        // weight gradient: dW[o][i] = sum_r dZ[r][o] * Hprev[r][i]   (split over the batch)
        int rc = wgrad_mma(h, l, n_pad, dz, s);
        if (rc) return rc;
        bias_partial<<<dim3(slices, h->members), WID, 0, s>>>(dz, h->part, n_pad, B, slices);
        slices_reduce<<<dim3(WID / 32, h->members), 32 * kRedWarps, 0, s>>>(h->part, h->grad, OFF_B(l), WID, slices,
                                                                          WID + 1, nullptr, 0);
        TUNE_CUDA_TRY(cudaGetLastError(), "surrogate: reduce launch");
        if (l == 0) continue;
        // input gradient of layer l, times gelu' of layer l-1: dZ_{l-1} = (dZ_l W_l) * gelu'(Z_{l-1})
        GemmArgs d = gargs();
        d.A = dz;
        d.sA = (long long)B * WID;
        d.lda = WID;
        d.B = h->wbf + BOFF_W(l);
        d.sB = PB;
        d.ldb = kin;
        d.M = n_pad;
        d.N = kin;
        d.K = WID;
        d.G = h->G[l - 1];
        d.sG = (long long)B * WID;
        d.H = dzl[l - 1];
        d.sH = (long long)B * WID;
        d.ldc = WID;
        rc = gemm<false, true, mlp::EPI_GELU_GRAD>(d, h->members, s);
        if (rc) return rc;
    }
    return TUNE_OK;
}

int adam(tune_surrogate* h, cudaStream_t s)
{
    h->step += 1;
    const float c1 = 1.0f - powf(h->b1, (float)h->step), c2 = 1.0f - powf(h->b2, (float)h->step);
    const long long total = (long long)h->members * P;
    TUNE_CUDA_TRY(pdl::launch_dep(adam_update, dim3((unsigned)((total / 4 + 255) / 256)), dim3(256), 0, s, h->master,
                                  h->grad, h->m, h->v, h->wbf, h->members, h->lr, h->b1, h->b2, h->eps, c1, c2),
                  "surrogate: adam launch");
    h->fp8_stale = true;
    TUNE_CUDA_TRY(cudaGetLastError(), "surrogate: adam launch");
    return TUNE_OK;
}

int load_batch(tune_surrogate* h, const __nv_bfloat16* feats, const float* labels, const int32_t* order, int n,
               cudaStream_t s)
{
    if ((reinterpret_cast<uintptr_t>(feats) & 15) == 0)
        TUNE_CUDA_TRY(pdl::launch_dep(gather_batch16, dim3((h->batch + kGatherRows - 1) / kGatherRows), dim3(256), 0, s,
                                      feats, labels, order, n, h->batch, h->xin, h->lbl),
                      "surrogate: gather launch");
    else
        TUNE_CUDA_TRY(pdl::launch_dep(gather_batch, dim3(h->batch), dim3(IN / 2), 0, s, feats, labels, order, n,
                                      h->batch, h->xin, h->lbl),
                      "surrogate: gather launch");
    TUNE_CUDA_TRY(cudaGetLastError(), "surrogate: gather launch");
    h->xb = h->xin;
    h->lb = h->lbl;
    h->xb_rows = h->batch;
    return TUNE_OK;
}

// The caller's first n rows and labels as the training batch, without a gather: on the fused
// tcgen05 path, whose reads of the input rows go through tensor maps (rows past n read as
// zeros) and whose labels are read for the n labelled rows only; the arrays must be 16-byte
// (rows) and 4-byte (labels) aligned. Returns false where the gather is needed.
bool use_batch_in_place(tune_surrogate* h, const __nv_bfloat16* feats, const float* labels, int n)
{
    if (!(h->use_tc && h->fwd_mode == 1 && h->bwd_mode == 1)) return false;
    if ((reinterpret_cast<uintptr_t>(feats) & 15) || (reinterpret_cast<uintptr_t>(labels) & 3)) return false;
    h->xb = feats;
    h->lb = labels;
    h->xb_rows = n;
    return true;
}

}  // namespace

extern "C" {

int surrogate_param_count(void) { return (int)P; }

int surrogate_members(const tune_surrogate* h) { return h ? h->members : 0; }

int surrogate_set_option(tune_surrogate* h, int option, int value)
{
    tune::clear_error();
    if (!h) return tune::fail(TUNE_EINVAL, "surrogate_set_option: NULL handle");
    if (option == 0) {
        h->use_tc = value != 0;
        return TUNE_OK;
    }
    if (option == 1) {
        if (value < 0 || value > 2) return tune::fail(TUNE_EINVAL, "surrogate_set_option: forward mode outside 0..2");
        h->fwd_mode = value;
        return TUNE_OK;
    }
    if (option == 2) {
        if (value < 0 || value > 1) return tune::fail(TUNE_EINVAL, "surrogate_set_option: backward mode outside 0..1");
        h->bwd_mode = value;
        return TUNE_OK;
    }
    return tune::fail(TUNE_EINVAL, "surrogate_set_option: unknown option %d", option);
}

int surrogate_status(tune_surrogate* h)
{
    tune::clear_error();
    if (!h) return tune::fail(TUNE_EINVAL, "surrogate_status: NULL handle");
    int st = 0;
    TUNE_CUDA_TRY(cudaMemcpy(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost), "surrogate_status: copy");
    if (st) TUNE_CUDA_TRY(cudaMemset(h->status, 0, sizeof(int)), "surrogate_status: clear");
    if (st & 2) return tune::fail(TUNE_ETIMEOUT, "a bounded wait in a surrogate kernel gave up");
    return TUNE_OK;
}

int surrogate_create(tune_surrogate** out, const tune_surrogate_cfg* cfg)
{
    tune::clear_error();
    if (!out || !cfg) return tune::fail(TUNE_EINVAL, "surrogate_create: NULL argument");
    if (cfg->members < 1 || cfg->members > 16) return tune::fail(TUNE_EINVAL, "members outside [1, 16]");
    if (cfg->batch < 128 || cfg->batch % 128 || cfg->batch > (1 << 16))
        return tune::fail(TUNE_EINVAL, "batch must be a multiple of 128 in [128, 65536]");
    tune_surrogate* h = new tune_surrogate();
    h->members = cfg->members;
    h->batch = cfg->batch;
    h->lr = cfg->lr;
    h->b1 = cfg->beta1;
    h->b2 = cfg->beta2;
    h->eps = cfg->eps;
    const size_t M = (size_t)h->members, B = (size_t)h->batch;
    size_t bytes = 0;
    auto add = [&](size_t n) { bytes += (n + 255) & ~size_t(255); };
    for (int i = 0; i < 4; ++i) add(M * P * 4);
    add(M * PB * 2);
    add(B * IN * 2);
    for (int l = 0; l < NL; ++l) add(M * B * WID * 2);
    for (int l = 0; l < NL; ++l) add(M * B * WID * 2);
    for (int l = 0; l < NL; ++l) add(M * B * WID * 2);
    add(M * B * 4);
    add(B * 4);
    add(M * 4);
    const size_t part_slices = std::max<size_t>(M * KSPLIT, (size_t)tune::device_sm_count());
    add(part_slices * WID * WID * 4);
    add(256);
    add(M * (NL - 1) * WID * WID);
    add(M * (NL - 1) * WID * 4);
    add(M * (NL - 1) * WID * 4);
    cudaError_t e = cudaMalloc(&h->block, bytes);
    if (e != cudaSuccess) {
        delete h;
        return tune::cuda_fail(e, "surrogate_create: cudaMalloc");
    }
    cudaMemset(h->block, 0, bytes);
    char* p = static_cast<char*>(h->block);
    h->master = carve<float>(p, M * P);
    h->grad = carve<float>(p, M * P);
    h->m = carve<float>(p, M * P);
    h->v = carve<float>(p, M * P);
    h->wbf = carve<__nv_bfloat16>(p, M * PB);
    h->xin = carve<__nv_bfloat16>(p, B * IN);
    for (int l = 0; l < NL; ++l) h->G[l] = carve<__half>(p, M * B * WID);
    for (int l = 0; l < NL; ++l) h->H[l] = carve<__nv_bfloat16>(p, M * B * WID);
    for (int l = 0; l < NL; ++l) h->dZ[l] = carve<__nv_bfloat16>(p, M * B * WID);
    h->y = carve<float>(p, M * B);
    h->lbl = carve<float>(p, B);
    h->loss = carve<float>(p, M);
    h->part = carve<float>(p, part_slices * WID * WID);
    h->part_slices = (int)part_slices;
    h->status = carve<int>(p, 64);
    h->w8 = carve<uint8_t>(p, M * (NL - 1) * WID * WID);
    h->wscale = carve<float>(p, M * (NL - 1) * WID);
    h->wscale_half = carve<float>(p, M * (NL - 1) * WID);
    *out = h;
    return TUNE_OK;
}

void surrogate_free(tune_surrogate* h)
{
    if (!h) return;
    if (h->block) cudaFree(h->block);
    delete h;
}

int surrogate_set_params(tune_surrogate* h, const float* host, int64_t n)
{
    tune::clear_error();
    if (!h || !host || n != (int64_t)h->members * P) return tune::fail(TUNE_EINVAL, "surrogate_set_params: size");
    TUNE_CUDA_TRY(cudaMemcpy(h->master, host, n * sizeof(float), cudaMemcpyHostToDevice), "set_params: copy");
    TUNE_CUDA_TRY(cudaMemset(h->m, 0, n * sizeof(float)), "set_params: reset m");
    TUNE_CUDA_TRY(cudaMemset(h->v, 0, n * sizeof(float)), "set_params: reset v");
    h->step = 0;
    h->fp8_stale = true;
    const long long tot = (long long)h->members * PB;
    cast_weights<<<(unsigned)((tot + 255) / 256), 256>>>(h->master, h->wbf, h->members);
    TUNE_CUDA_TRY(cudaGetLastError(), "set_params: cast");
    TUNE_CUDA_TRY(cudaDeviceSynchronize(), "set_params: sync");
    return TUNE_OK;
}

int surrogate_get(tune_surrogate* h, int what, float* host, int64_t n)
{
    tune::clear_error();
    if (!h || !host) return tune::fail(TUNE_EINVAL, "surrogate_get: NULL argument");
    const float* src = what == 0 ? h->master : what == 1 ? h->grad : what == 2 ? h->m : what == 3 ? h->v : nullptr;
    int64_t cnt = (int64_t)h->members * P;
    if (what == 4) {
        src = h->loss;
        cnt = h->members;
    }
    if (what == 5) {
        src = h->y;
        cnt = (int64_t)h->members * h->batch;
    }
    if (what == 6 || what == 7) {  // E4M3 codes of W2..W4 (decoded), their row scales
        const int64_t rows = (int64_t)h->members * (NL - 1) * WID;
        if (n != (what == 6 ? rows * WID : rows)) return tune::fail(TUNE_EINVAL, "surrogate_get: bad size");
        int rc = refresh_fp8(h, 0);
        if (rc) return rc;
        TUNE_CUDA_TRY(cudaDeviceSynchronize(), "surrogate_get: sync");
        if (what == 7) {
            TUNE_CUDA_TRY(cudaMemcpy(host, h->wscale, n * sizeof(float), cudaMemcpyDeviceToHost), "surrogate_get: copy");
            return TUNE_OK;
        }
        std::vector<uint8_t> codes(n);
        TUNE_CUDA_TRY(cudaMemcpy(codes.data(), h->w8, n, cudaMemcpyDeviceToHost), "surrogate_get: copy");
        for (int64_t i = 0; i < n; ++i) {  // E4M3: sign, 4 exponent bits (bias 7), 3 mantissa bits
            const uint8_t b = codes[i];
            const int e = (b >> 3) & 15, m = b & 7;
            float v = e ? ldexpf(1.0f + m / 8.0f, e - 7) : ldexpf(m / 8.0f, -6);
            if (e == 15 && m == 7) v = NAN;
            host[i] = (b & 0x80) ? -v : v;
        }
        return TUNE_OK;
    }
    if (!src || n != cnt) return tune::fail(TUNE_EINVAL, "surrogate_get: bad selector or size");
    TUNE_CUDA_TRY(cudaDeviceSynchronize(), "surrogate_get: sync");
    TUNE_CUDA_TRY(cudaMemcpy(host, src, n * sizeof(float), cudaMemcpyDeviceToHost), "surrogate_get: copy");
    return TUNE_OK;
}

int surrogate_forward(tune_surrogate* h, const uint16_t* feats, int64_t n, float* pred, tune_stream_t stream)
{
    tune::clear_error();
    if (!h || (n > 0 && (!feats || !pred))) return tune::fail(TUNE_EINVAL, "surrogate_forward: NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const auto* f = reinterpret_cast<const __nv_bfloat16*>(feats);
    if (h->fwd_mode != 0) return fused_forward(h, f, n, pred, h->fwd_mode == 2, s);
    for (int64_t r0 = 0; r0 < n; r0 += h->batch) {
        const int nb = (int)((n - r0) < h->batch ? (n - r0) : h->batch);
        const int n_pad = (nb + 127) / 128 * 128;
        int rc;
        if (h->use_tc) {  // layer 1 reads the caller's rows directly; no gelu' kept
            rc = forward(h, n_pad, s, f + r0 * IN, nb, false);
        } else {
            rc = load_batch(h, f + r0 * IN, h->lbl /*unused labels*/, nullptr, nb, s);
            if (!rc) rc = forward(h, n_pad, s);
        }
        if (rc) return rc;
        for (int mem = 0; mem < h->members; ++mem)
            TUNE_CUDA_TRY(cudaMemcpyAsync(pred + mem * n + r0, h->y + (long long)mem * h->batch, nb * sizeof(float),
                                          cudaMemcpyDeviceToDevice, s),
                          "surrogate_forward: copy out");
    }
    return TUNE_OK;
}

int surrogate_train_step(tune_surrogate* h, const uint16_t* feats, const float* labels, int64_t n,
                         int32_t apply_update, tune_stream_t stream)
{
    tune::clear_error();
    if (!h || !feats || !labels || n < 1 || n > h->batch)
        return tune::fail(TUNE_EINVAL, "surrogate_train_step: need 1 <= n <= batch and non-NULL data");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int nb = (int)n, n_pad = (nb + 127) / 128 * 128;
    const auto* f = reinterpret_cast<const __nv_bfloat16*>(feats);
    int rc = use_batch_in_place(h, f, labels, nb) ? TUNE_OK : load_batch(h, f, labels, nullptr, nb, s);
    if (!rc) rc = forward(h, n_pad, s);
    if (!rc) rc = backward(h, nb, n_pad, s);
    if (!rc && apply_update) rc = adam(h, s);
    return rc;
}

int surrogate_train(tune_surrogate* h, const uint16_t* feats, const float* labels, int64_t n,
                    const int32_t* order, int32_t epochs, float* loss_trace, tune_stream_t stream)
{
    tune::clear_error();
    if (!h || !feats || !labels || !order || n < 1 || epochs < 1)
        return tune::fail(TUNE_EINVAL, "surrogate_train: bad arguments");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const auto* f = reinterpret_cast<const __nv_bfloat16*>(feats);
    const int64_t steps = (n + h->batch - 1) / h->batch;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int64_t st = 0; st < steps; ++st) {
            const int64_t r0 = st * h->batch;
            const int nb = (int)((n - r0) < h->batch ? (n - r0) : h->batch);
            const int n_pad = (nb + 127) / 128 * 128;
            int rc = load_batch(h, f, labels, order + (int64_t)ep * n + r0, nb, s);
            if (!rc) rc = forward(h, n_pad, s);
            if (!rc) rc = backward(h, nb, n_pad, s);
            if (!rc) rc = adam(h, s);
            if (rc) return rc;
            if (loss_trace)
                TUNE_CUDA_TRY(cudaMemcpyAsync(loss_trace + ((int64_t)ep * steps + st) * h->members, h->loss,
                                              h->members * sizeof(float), cudaMemcpyDeviceToDevice, s),
                              "surrogate_train: loss trace");
        }
    }
    return TUNE_OK;
}

}  // extern "C"
