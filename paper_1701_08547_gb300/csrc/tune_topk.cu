// tune_topk: segmented top-k over an external FP32 score array (HBM-bound).
//
// One warp per segment, CTAs of 8 warps striding over segments. Lanes read
// the segment with coalesced loads, four independent loads in flight per lane,
// and keep a sorted register list of their k best (score, index); each lane
// visits its elements in increasing index order, so a strict "<" keeps lower
// indices first among equal scores. A k-round warp merge over an
// order-preserving unsigned image of the scores emits the segment's top-k.
#include <stdint.h>

#include "tune_internal.h"

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr unsigned kFull = 0xffffffffu;

// Monotone map of non-NaN floats to unsigned integers (-inf smallest, +inf largest).
__device__ __forceinline__ unsigned order_key(float f)
{
    unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float key_value(unsigned k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

template <int KMAX>
__device__ __forceinline__ void insert(float (&lc)[KMAX], int (&li)[KMAX], float c, int i)
{
#pragma unroll
    for (int j = KMAX - 1; j > 0; --j) {
        bool shift = c < lc[j - 1];
        bool here = !shift && c < lc[j];
        float nc = shift ? lc[j - 1] : (here ? c : lc[j]);
        int ni = shift ? li[j - 1] : (here ? i : li[j]);
        lc[j] = nc;
        li[j] = ni;
    }
    if (c < lc[0]) {
        lc[0] = c;
        li[0] = i;
    }
}

template <int KMAX>
__device__ __forceinline__ float kth(const float (&lc)[KMAX], int k)
{
    // Select chain (not lc[k - 1], which would force the list into local memory).
    float t = lc[KMAX - 1];
#pragma unroll
    for (int j = KMAX - 2; j >= 0; --j) t = (j >= k - 1) ? lc[j] : t;
    return t;
}

template <int KMAX>
__device__ __forceinline__ void consider(float (&lc)[KMAX], int (&li)[KMAX], float& thr, int k, float v,
                                         int j)
{
    v = v + 0.0f;  // -0 -> +0: equal scores compare equal in the merge keys too
    if (v < thr) {  // false for NaN and for +inf
        insert<KMAX>(lc, li, v, j);
        thr = kth<KMAX>(lc, k);
    }
}

template <int KMAX>
__global__ void __launch_bounds__(kThreads)
    topk_segmented_kernel(const float* __restrict__ scores, const int64_t* __restrict__ off,
                          int64_t n_seg, int k, int32_t* __restrict__ out_i, float* __restrict__ out_s)
{
    const int lane = threadIdx.x & 31;
    const float kInf = __int_as_float(0x7f800000);
    for (int64_t s = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); s < n_seg;
         s += (int64_t)gridDim.x * kWarps) {
        const int64_t b = off[s];
        const int len = (int)(off[s + 1] - b);
        const float* seg = scores + b;
        float lc[KMAX];
        int li[KMAX];
#pragma unroll
        for (int j = 0; j < KMAX; ++j) {
            lc[j] = kInf;
            li[j] = -1;
        }
        float thr = kInf;
        int j = lane;
        for (; j + 96 < len; j += 128) {
            const float v0 = __ldcs(seg + j), v1 = __ldcs(seg + j + 32), v2 = __ldcs(seg + j + 64),
                        v3 = __ldcs(seg + j + 96);
            consider<KMAX>(lc, li, thr, k, v0, j);
            consider<KMAX>(lc, li, thr, k, v1, j + 32);
            consider<KMAX>(lc, li, thr, k, v2, j + 64);
            consider<KMAX>(lc, li, thr, k, v3, j + 96);
        }
        for (; j < len; j += 32) consider<KMAX>(lc, li, thr, k, __ldcs(seg + j), j);

        float oc = kInf;
        int oi = -1;
        for (int r = 0; r < k; ++r) {
            const unsigned hk = order_key(lc[0]);
            const unsigned mk = __reduce_min_sync(kFull, hk);
            if (mk >= order_key(kInf)) break;
            const unsigned cand = hk == mk ? (unsigned)li[0] : 0xffffffffu;
            const unsigned mi = __reduce_min_sync(kFull, cand);
            if (lane == r) {
                oc = key_value(mk);
                oi = (int)mi;
            }
            const bool win = hk == mk && (unsigned)li[0] == mi;
#pragma unroll
            for (int q = 0; q < KMAX - 1; ++q) {
                lc[q] = win ? lc[q + 1] : lc[q];
                li[q] = win ? li[q + 1] : li[q];
            }
            if (win) {
                lc[KMAX - 1] = kInf;
                li[KMAX - 1] = -1;
            }
        }
        if (lane < k) {
            out_i[s * k + lane] = oi;
            out_s[s * k + lane] = oc;
        }
    }
}

template <int KMAX>
int launch(const float* scores, const int64_t* off, int64_t n_seg, int k, int32_t* oi, float* os,
           cudaStream_t st)
{
    auto kern = topk_segmented_kernel<KMAX>;
    static int per_sm = 0;
    if (per_sm == 0) {
        TUNE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0),
                      "tune_topk: occupancy query");
        if (per_sm < 1) per_sm = 1;
    }
    const int sms = tune::device_sm_count();
    if (sms <= 0) return tune::fail(TUNE_ECUDA, "tune_topk: cannot query the SM count");
    const int64_t need = (n_seg + kWarps - 1) / kWarps;
    const int64_t cap = (int64_t)sms * per_sm;
    kern<<<(int)(need < cap ? need : cap), kThreads, 0, st>>>(scores, off, n_seg, k, oi, os);
    TUNE_CUDA_TRY(cudaGetLastError(), "tune_topk: kernel launch");
    return TUNE_OK;
}

}  // namespace

extern "C" int tune_topk(const float* scores, const int64_t* seg_offsets, int64_t n_seg, int32_t k,
                         int32_t* topk_idx, float* topk_score, void* workspace, size_t ws_bytes,
                         tune_stream_t stream)
{
    tune::clear_error();
    if (k < 1 || k > 16) return tune::fail(TUNE_EINVAL, "k = %d outside [1, 16]", k);
    if (n_seg < 0) return tune::fail(TUNE_EINVAL, "n_seg < 0");
    if (!workspace) return tune::fail(TUNE_EINVAL, "workspace is NULL");
    if (ws_bytes < tune_workspace_bytes(TUNE_CALL_TOPK, n_seg, k))
        return tune::fail(TUNE_ENOMEM, "workspace too small");
    if (n_seg > 0 && (!scores || !seg_offsets || !topk_idx || !topk_score))
        return tune::fail(TUNE_EINVAL, "scores, seg_offsets and outputs must be non-NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    TUNE_CUDA_TRY(cudaMemsetAsync(workspace, 0, tune::kWorkspaceHeader, s), "tune_topk: status reset");
    if (n_seg == 0) return TUNE_OK;
    return k <= 8 ? launch<8>(scores, seg_offsets, n_seg, k, topk_idx, topk_score, s)
                  : launch<16>(scores, seg_offsets, n_seg, k, topk_idx, topk_score, s);
}
