// tune_topk: segmented top-k over an external FP32 score array (HBM-bound).
//
// One warp per segment, CTAs of 8 warps striding over segments. Lanes read the
// segment with coalesced loads, eight independent loads in flight per lane.
// The warp keeps one exact top-k list (lane j = j-th best, as an
// order-preserving unsigned image of the score plus its index) and its k-th
// key; only when a block of 256 scores holds values at or below that key does
// the warp merge them, in increasing (value, index) order, into the list.
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

// Warp-wide top-k list: lane j < k holds the j-th best (order key, index), ascending.
__device__ __forceinline__ bool key_less(unsigned a, int ia, unsigned b, int ib)
{
    return a < b || (a == b && ia < ib);
}

__device__ __forceinline__ void list_insert(unsigned& lk, int& li, unsigned& tau_k, int& tau_i, unsigned k_new,
                                            int i_new, int k, int lane)
{
    const unsigned below = __ballot_sync(kFull, lane < k && key_less(lk, li, k_new, i_new));
    const int pos = __popc(below);
    const unsigned up_k = __shfl_up_sync(kFull, lk, 1);
    const int up_i = __shfl_up_sync(kFull, li, 1);
    if (lane < k) {
        if (lane == pos) {
            lk = k_new;
            li = i_new;
        } else if (lane > pos) {
            lk = up_k;
            li = up_i;
        }
    }
    tau_k = __shfl_sync(kFull, lk, k - 1);
    tau_i = __shfl_sync(kFull, li, k - 1);
}

constexpr int kLoads = 8;  // independent loads in flight per lane

__global__ void __launch_bounds__(kThreads)
    topk_segmented_kernel(const float* __restrict__ scores, const int64_t* __restrict__ off, int64_t n_seg, int k,
                          int32_t* __restrict__ out_i, float* __restrict__ out_s)
{
    const int lane = threadIdx.x & 31;
    const float kInf = __int_as_float(0x7f800000);
    const unsigned kInfKey = order_key(kInf);
    for (int64_t s = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); s < n_seg;
         s += (int64_t)gridDim.x * kWarps) {
        const int64_t b = off[s];
        const int len = (int)(off[s + 1] - b);
        const float* seg = scores + b;
        unsigned lk = kInfKey;  // list entry of this lane (lanes < k)
        int li = -1;
        unsigned tau_k = kInfKey;  // the list's k-th key: candidates must not exceed it
        int tau_i = -1;
        for (int base = 0; base < len; base += 32 * kLoads) {
            float v[kLoads];
#pragma unroll
            for (int q = 0; q < kLoads; ++q) {
                const int j = base + lane + 32 * q;
                v[q] = j < len ? __ldcs(seg + j) + 0.0f : __int_as_float(0x7fc00000);  // -0 -> +0; NaN pads
            }
            const float tau_v = key_value(tau_k);
            unsigned cm = 0;
#pragma unroll
            for (int q = 0; q < kLoads; ++q)
                if (v[q] <= tau_v && v[q] < kInf) cm |= 1u << q;  // false for NaN and +inf
            if (__ballot_sync(kFull, cm != 0u) == 0u) continue;
            // Merge this block's candidates in increasing (value, index) order.
            for (;;) {
                unsigned hk = 0xffffffffu;
                int hq = 0;
#pragma unroll
                for (int q = kLoads - 1; q >= 0; --q) {  // equal keys: the lower q (lower index) wins
                    const unsigned kq = order_key(v[q]);
                    if (((cm >> q) & 1u) && kq <= hk) {
                        hk = kq;
                        hq = q;
                    }
                }
                const unsigned mk = __reduce_min_sync(kFull, hk);
                if (mk == 0xffffffffu) break;
                const int my_i = base + lane + 32 * hq;
                const unsigned mi = __reduce_min_sync(kFull, hk == mk ? (unsigned)my_i : 0xffffffffu);
                if (!key_less(mk, (int)mi, tau_k, tau_i)) break;
                list_insert(lk, li, tau_k, tau_i, mk, (int)mi, k, lane);
                if (hk == mk && my_i == (int)mi) cm &= ~(1u << hq);
            }
        }
        if (lane < k) {
            out_i[s * k + lane] = li;
            out_s[s * k + lane] = lk == kInfKey ? kInf : key_value(lk);
        }
    }
}

int launch(const float* scores, const int64_t* off, int64_t n_seg, int k, int32_t* oi, float* os, cudaStream_t st)
{
    auto kern = topk_segmented_kernel;
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
    return launch(scores, seg_offsets, n_seg, k, topk_idx, topk_score, s);
}
