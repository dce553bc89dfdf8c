// Surrogate features and ranking: per-point features (tune_features), and
// surrogate_infer — features of every point, ensemble forward, per-point mean
// and spread of the predicted runtime, per-kernel top-k by predicted runtime,
// and a per-kernel fallback to the analytic top-k where the members disagree.
#include <cuda_bf16.h>
#include <stdint.h>
#include <string.h>

#include "features.cuh"
#include "tune_internal.h"

using namespace tune_dev;

namespace {

constexpr int IN = TUNE_SURROGATE_INPUTS;  // feature row width (48 features + zeros)
constexpr int64_t kChunkPoints = 1 << 20;  // points per inference chunk

__device__ __forceinline__ void load_desc(const int4* descs, int64_t kid, Desc& kd)
{
    int4 v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = __ldg(descs + kid * 4 + q);
    unpack(v, kd);
}

__device__ __forceinline__ void write_row(__nv_bfloat16* row, const float* f)
{
    __nv_bfloat162* r2 = reinterpret_cast<__nv_bfloat162*>(row);
#pragma unroll
    for (int j = 0; j < kFeatures / 2; ++j) r2[j] = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
    const __nv_bfloat162 z = __floats2bfloat162_rn(0.0f, 0.0f);
#pragma unroll
    for (int j = kFeatures / 2; j < IN / 2; ++j) r2[j] = z;
}

// Features of listed samples (kernel id, canonical point index).
__global__ void features_samples(const __grid_constant__ tune_arch a, const __grid_constant__ tune_axes x,
                                 const int4* __restrict__ descs, const int64_t* __restrict__ skern,
                                 const int32_t* __restrict__ spoint, int64_t n, __nv_bfloat16* out, int* status)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Desc kd;
    load_desc(descs, skern[i], kd);
    const int size = __popc(kd.tm) * __popc(kd.gm) * __popc(kd.um) * __popc(kd.cm);
    float f[kFeatures];
    if (desc_bad(kd, x) || spoint[i] < 0 || spoint[i] >= size) {
        atomicOr(status, tune::kStatusInvalid);
        for (int j = 0; j < kFeatures; ++j) f[j] = 0.0f;
    } else {
        int tp, gp, up, cp;
        decode_point(kd, spoint[i], tp, gp, up, cp);
        point_features(a, kd, x.t[tp], x.g[gp], x.u[up], x.c[cp], f);
    }
    write_row(out + i * IN, f);
}

// Features of every point of kernels [k0, k1): one thread per point, row i of the chunk
// = global point p0 + i (p0 = pt_off[k0]); the point's kernel is found by a binary
// search over the offsets (the chunk's few offsets stay in L1).
__global__ void features_points(const __grid_constant__ tune_arch a, const __grid_constant__ tune_axes x,
                                const int4* __restrict__ descs, const int64_t* __restrict__ pt_off, int64_t k0,
                                int64_t k1, int64_t p0, int64_t np, __nv_bfloat16* out, int* status)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const int64_t gp_ = p0 + i;
    int64_t lo = k0, hi = k1;  // pt_off[lo] <= gp_ < pt_off[hi]
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (pt_off[mid] <= gp_)
            lo = mid;
        else
            hi = mid;
    }
    Desc kd;
    load_desc(descs, lo, kd);
    const int64_t p = gp_ - pt_off[lo];
    const int size = __popc(kd.tm) * __popc(kd.gm) * __popc(kd.um) * __popc(kd.cm);
    float f[kFeatures];
    if (desc_bad(kd, x) || p >= size) {
        atomicOr(status, tune::kStatusInvalid);
        for (int j = 0; j < kFeatures; ++j) f[j] = 0.0f;
    } else {
        int tp, gp, up, cp;
        decode_point(kd, (int)p, tp, gp, up, cp);
        point_features(a, kd, x.t[tp], x.g[gp], x.u[up], x.c[cp], f);
    }
    write_row(out + i * IN, f);
}

// Chunk-relative segment offsets: rel[j] = pt_off[k0 + j] - pt_off[k0], j = 0..nk.
__global__ void rebase_offsets(const int64_t* __restrict__ pt_off, int64_t k0, int64_t nk, int64_t* rel)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j <= nk) rel[j] = pt_off[k0 + j] - pt_off[k0];
}

// Per point: runtime estimate = mean over members of exp(prediction); spread = std / mean;
// invalid points (B* = 0: feature 29 is zero) get +inf.
__global__ void score_points(const float* __restrict__ pred, const __nv_bfloat16* __restrict__ feats, int64_t n,
                             int members, float* score, float* spread)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool valid = __bfloat162float(feats[i * IN + 29]) > 0.0f;
    float s = 0.0f, s2 = 0.0f;
    for (int m = 0; m < members; ++m) {
        const float r = expf(pred[(int64_t)m * n + i]);
        s += r;
        s2 += r * r;
    }
    const float mean = s / members;
    const float var = fmaxf(s2 / members - mean * mean, 0.0f);
    score[i] = valid ? mean : __int_as_float(0x7f800000);
    spread[i] = valid ? sqrtf(var) / mean : 0.0f;
}

// Per kernel: use the analytic top-k if any of the surrogate's top-k points has spread > thresh.
__global__ void apply_fallback(const int32_t* __restrict__ s_idx, const float* __restrict__ s_val,
                               const int32_t* __restrict__ a_idx, const float* __restrict__ a_val,
                               const float* __restrict__ spread, const int64_t* __restrict__ pt_off, int64_t k0,
                               int64_t nk, int k, float thresh, int32_t* out_idx, float* out_val, uint8_t* flag)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nk) return;
    const int64_t kid = k0 + j;
    const int64_t base = pt_off[kid] - pt_off[k0];
    bool fb = false;
    for (int r = 0; r < k; ++r) {
        const int p = s_idx[j * k + r];
        if (p >= 0 && spread[base + p] > thresh) fb = true;
    }
    flag[kid] = fb ? 1 : 0;
    for (int r = 0; r < k; ++r) {
        out_idx[kid * k + r] = fb ? a_idx[kid * k + r] : s_idx[j * k + r];
        out_val[kid * k + r] = fb ? a_val[kid * k + r] : s_val[j * k + r];
    }
}

int64_t align256(int64_t b) { return (b + 255) & ~int64_t(255); }

}  // namespace

extern "C" {

int tune_features(const tune_arch* arch, const tune_axes* axes, const tune_kernel_desc* descs,
                  const int64_t* sample_kernel, const int32_t* sample_point, int64_t n, uint16_t* feats,
                  void* workspace, size_t ws_bytes, tune_stream_t stream)
{
    tune::clear_error();
    if (!arch || !axes || !workspace || ws_bytes < tune::kWorkspaceHeader || n < 0)
        return tune::fail(TUNE_EINVAL, "tune_features: bad arguments");
    if (n > 0 && (!descs || !sample_kernel || !sample_point || !feats))
        return tune::fail(TUNE_EINVAL, "tune_features: NULL array");
    int rc = tune::validate_inputs(arch, axes);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    TUNE_CUDA_TRY(cudaMemsetAsync(workspace, 0, tune::kWorkspaceHeader, s), "tune_features: status reset");
    if (n == 0) return TUNE_OK;
    features_samples<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(
        *arch, *axes, reinterpret_cast<const int4*>(descs), sample_kernel, sample_point, n,
        reinterpret_cast<__nv_bfloat16*>(feats), static_cast<int*>(workspace));
    TUNE_CUDA_TRY(cudaGetLastError(), "tune_features: launch");
    return TUNE_OK;
}

}  // extern "C"

// surrogate_infer needs the handle's forward; declared in surrogate.cu.
extern "C" int surrogate_forward(tune_surrogate* h, const uint16_t* feats, int64_t n, float* pred,
                                 tune_stream_t stream);
extern "C" int surrogate_members(const tune_surrogate* h);

extern "C" size_t surrogate_infer_workspace_bytes(int members, int64_t n_kernels, int32_t k)
{
    int64_t b = 2 * tune::kWorkspaceHeader;           // status; header for the internal calls
    b += align256(kChunkPoints * IN * 2);              // features
    b += align256((int64_t)members * kChunkPoints * 4); // predictions
    b += 2 * align256(kChunkPoints * 4);                // score, spread
    b += align256((int64_t)(kChunkPoints / 64 + 2) * 8);  // chunk offsets (>= 64 points per kernel? sized below)
    b += 2 * align256(n_kernels * k * 4);               // analytic top-k
    b += 2 * align256(n_kernels * k * 4);               // surrogate top-k (per chunk, sized for all)
    b += align256((n_kernels + 1) * 8);                 // device offsets
    return (size_t)b;
}

extern "C" int surrogate_infer(tune_surrogate* h, const tune_arch* arch, const tune_axes* axes,
                               const tune_kernel_desc* descs, int64_t n_kernels, const int64_t* pt_offsets_host,
                               int32_t k, float thresh, int32_t* topk_idx, float* topk_score,
                               uint8_t* used_fallback, void* workspace, size_t ws_bytes, tune_stream_t stream)
{
    tune::clear_error();
    if (!h || !arch || !axes || !pt_offsets_host || k < 1 || k > 16 || n_kernels < 0)
        return tune::fail(TUNE_EINVAL, "surrogate_infer: bad arguments");
    const int members = surrogate_members(h);
    if (!workspace || ws_bytes < surrogate_infer_workspace_bytes(members, n_kernels, k))
        return tune::fail(TUNE_ENOMEM, "surrogate_infer: workspace smaller than surrogate_infer_workspace_bytes()");
    if (n_kernels == 0) return TUNE_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(workspace);
    int* status = reinterpret_cast<int*>(w);
    w += tune::kWorkspaceHeader;
    void* inner = w;  // workspace header of the tune_eval / tune_topk calls made here
    w += tune::kWorkspaceHeader;
    auto* feats = reinterpret_cast<__nv_bfloat16*>(w);
    w += align256(kChunkPoints * IN * 2);
    float* pred = reinterpret_cast<float*>(w);
    w += align256((int64_t)members * kChunkPoints * 4);
    float* score = reinterpret_cast<float*>(w);
    w += align256(kChunkPoints * 4);
    float* spread = reinterpret_cast<float*>(w);
    w += align256(kChunkPoints * 4);
    int64_t* coff = reinterpret_cast<int64_t*>(w);  // chunk-relative offsets, reused per chunk
    w += align256((int64_t)(kChunkPoints / 64 + 2) * 8);
    int32_t* a_idx = reinterpret_cast<int32_t*>(w);
    w += align256(n_kernels * k * 4);
    float* a_val = reinterpret_cast<float*>(w);
    w += align256(n_kernels * k * 4);
    int32_t* s_idx = reinterpret_cast<int32_t*>(w);
    w += align256(n_kernels * k * 4);
    float* s_val = reinterpret_cast<float*>(w);
    w += align256(n_kernels * k * 4);
    int64_t* d_off = reinterpret_cast<int64_t*>(w);

    TUNE_CUDA_TRY(cudaMemsetAsync(status, 0, tune::kWorkspaceHeader, s), "surrogate_infer: status reset");
    // Analytic top-k of every kernel (the fallback).
    int rc = tune_eval(arch, axes, descs, n_kernels, k, TUNE_SCHED_WARP, a_idx, a_val, nullptr, nullptr, nullptr,
                       nullptr, inner, tune::kWorkspaceHeader, stream);
    if (rc) return rc;
    TUNE_CUDA_TRY(cudaMemcpyAsync(d_off, pt_offsets_host, (n_kernels + 1) * 8, cudaMemcpyHostToDevice, s),
                  "surrogate_infer: offsets");
    int64_t k0 = 0;
    while (k0 < n_kernels) {
        // Chunk: as many whole kernels as fit kChunkPoints (and the offsets scratch).
        int64_t k1 = k0;
        while (k1 < n_kernels && pt_offsets_host[k1 + 1] - pt_offsets_host[k0] <= kChunkPoints &&
               k1 - k0 < kChunkPoints / 64)
            ++k1;
        if (k1 == k0) return tune::fail(TUNE_EINVAL, "surrogate_infer: a space larger than the chunk");
        const int64_t np = pt_offsets_host[k1] - pt_offsets_host[k0];
        const int64_t nk = k1 - k0;
        // Everything below is stream-ordered: the chunk buffers are reused without a host wait.
        rebase_offsets<<<(unsigned)((nk + 1 + 255) / 256), 256, 0, s>>>(d_off, k0, nk, coff);
        TUNE_CUDA_TRY(cudaGetLastError(), "surrogate_infer: offsets launch");
        if (np > 0) {
            features_points<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(
                *arch, *axes, reinterpret_cast<const int4*>(descs), d_off, k0, k1, pt_offsets_host[k0], np, feats,
                status);
            TUNE_CUDA_TRY(cudaGetLastError(), "surrogate_infer: features launch");
            rc = surrogate_forward(h, reinterpret_cast<const uint16_t*>(feats), np, pred, stream);
            if (rc) return rc;
            score_points<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(pred, feats, np, members, score, spread);
            TUNE_CUDA_TRY(cudaGetLastError(), "surrogate_infer: score launch");
        }
        rc = tune_topk(score, coff, nk, k, s_idx, s_val, inner, tune::kWorkspaceHeader, stream);
        if (rc) return rc;
        apply_fallback<<<(unsigned)((nk + 127) / 128), 128, 0, s>>>(s_idx, s_val, a_idx, a_val, spread, d_off, k0, nk,
                                                                   k, thresh, topk_idx, topk_score, used_fallback);
        TUNE_CUDA_TRY(cudaGetLastError(), "surrogate_infer: fallback launch");
        k0 = k1;
    }
    int st = 0;
    TUNE_CUDA_TRY(cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s), "surrogate_infer: status");
    TUNE_CUDA_TRY(cudaStreamSynchronize(s), "surrogate_infer: sync");
    if (st) return tune::fail(TUNE_EINVAL, "surrogate_infer: a descriptor was malformed");
    return TUNE_OK;
}
