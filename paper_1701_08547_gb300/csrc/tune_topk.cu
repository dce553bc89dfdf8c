// tune_topk: segmented top-k over an external FP32 score array (HBM-bound).
//
// One warp per segment, CTAs of 8 warps striding over segments. Lanes read the
// segment's 16-byte-aligned body with coalesced float4 loads, the next batch in
// flight while the current one is filtered.
// The warp keeps one exact top-k list (lane j = j-th best, as an
// order-preserving unsigned image of the score plus its index) and its k-th
// key; only when a batch of 512 scores holds values at or below that key (one
// minimum per lane tells) does the warp merge them, a float4 group at a time and in
// increasing (value, index) order, into the list.
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

constexpr int kVec = 4;                 // 16-byte loads per lane per batch
constexpr int kBatchF4 = 32 * kVec;     // float4 words per warp batch (2 KB)
constexpr unsigned kNaNBits = 0x7fc00000u;

// Filter bound: a score can enter the list only if it is <= tau (ties are decided
// by index in the merge). While the list is not full, tau is +inf and every finite
// score qualifies; the bound is then the largest finite float, which also keeps
// +inf and NaN out (the comparison is false for NaN).
__device__ __forceinline__ float filter_bound(unsigned tau_k)
{
    const float t = key_value(tau_k);
    return t < __int_as_float(0x7f800000) ? t : __int_as_float(0x7f7fffff);
}

// Merges the candidates of one group (bit j of cm marks v[j]; index_of(j) is its
// index in the segment) into the warp list in increasing (key, index) order, until
// the smallest remaining candidate can no longer enter.
template <int N, typename IndexOf>
__device__ __forceinline__ void merge_batch(const float (&v)[N], unsigned cm, IndexOf index_of, unsigned& lk,
                                            int& li, unsigned& tau_k, int& tau_i, int k, int lane)
{
    for (;;) {
        unsigned hk = 0xffffffffu;
        int hq = 0;
#pragma unroll
        for (int q = N - 1; q >= 0; --q) {  // equal keys: the lower q (lower index) wins
            const unsigned kq = order_key(v[q] + 0.0f);  // -0 ranks as +0
            if (((cm >> q) & 1u) && kq <= hk) {
                hk = kq;
                hq = q;
            }
        }
        const unsigned mk = __reduce_min_sync(kFull, hk);
        if (mk == 0xffffffffu) break;
        const int my_i = index_of(hq);
        const unsigned mi = __reduce_min_sync(kFull, hk == mk ? (unsigned)my_i : 0xffffffffu);
        if (!key_less(mk, (int)mi, tau_k, tau_i)) break;
        list_insert(lk, li, tau_k, tau_i, mk, (int)mi, k, lane);
        if (hk == mk && my_i == (int)mi) cm &= ~(1u << hq);
    }
}

// One warp per segment. The segment's 16-byte-aligned body is read as float4
// words, kVec per lane per batch, and the next batch's loads are issued before
// the current batch is filtered, so each warp keeps up to 4 KB in flight; the
// (at most 3 + 3) unaligned head and tail scores are read with scalar loads.
__global__ void __launch_bounds__(kThreads)
    topk_segmented_kernel(const float* __restrict__ scores, const int64_t* __restrict__ off, int64_t n_seg, int k,
                          int32_t* __restrict__ out_i, float* __restrict__ out_s)
{
    const int lane = threadIdx.x & 31;
    const float kInf = __int_as_float(0x7f800000);
    const float kNaN = __int_as_float(kNaNBits);
    const unsigned kInfKey = order_key(kInf);
    const int64_t stride = (int64_t)gridDim.x * kWarps;
    int64_t s = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    int64_t nb = s < n_seg ? off[s] : 0, ne = s < n_seg ? off[s + 1] : 0;
    for (; s < n_seg; s += stride) {
        const int64_t b = nb;
        const int len = (int)(ne - b);
        if (s + stride < n_seg) {  // the next segment's bounds, ahead of this segment's work
            nb = off[s + stride];
            ne = off[s + stride + 1];
        }
        const float* seg = scores + b;
        // head: scores before the first 16-byte boundary; body: n4 float4 words; tail: the rest
        const int head = min((int)(((16u - ((unsigned)reinterpret_cast<uintptr_t>(seg) & 15u)) & 15u) >> 2), len);
        const int n4 = (len - head) >> 2;
        const int tail0 = head + 4 * n4;
        const float4* body = reinterpret_cast<const float4*>(seg + head);

        unsigned lk = kInfKey;  // list entry of this lane (lanes < k)
        int li = -1;
        unsigned tau_k = kInfKey;  // the list's k-th key
        int tau_i = -1;

        // head and tail together, one score per lane (lanes >= head take the tail)
        {
            const int j = lane < head ? lane : tail0 + (lane - head);
            float v[1];
            v[0] = (lane < head || j < len) ? __ldcs(seg + j) : kNaN;  // NaN pads
            const unsigned cm = v[0] <= filter_bound(tau_k) ? 1u : 0u;
            if (__ballot_sync(kFull, cm != 0u))
                merge_batch<1>(v, cm, [&](int) { return j; }, lk, li, tau_k, tau_i, k, lane);
        }

        auto load = [&](float4 (&w)[kVec], int f0) {
#pragma unroll
            for (int q = 0; q < kVec; ++q) {
                const int f = f0 + lane + 32 * q;
                w[q] = f < n4 ? __ldcs(body + f) : make_float4(kNaN, kNaN, kNaN, kNaN);
            }
        };
        float4 cur[kVec];
        load(cur, 0);
        for (int f0 = 0; f0 < n4; f0 += kBatchF4) {
            float4 nxt[kVec];
            load(nxt, f0 + kBatchF4);  // all-NaN (no loads) past the end
            float v[4 * kVec];
#pragma unroll
            for (int q = 0; q < kVec; ++q) {
                v[4 * q + 0] = cur[q].x;
                v[4 * q + 1] = cur[q].y;
                v[4 * q + 2] = cur[q].z;
                v[4 * q + 3] = cur[q].w;
            }
            // fast path: the lane's smallest score (fminf skips NaN) against the bound
            float mn = v[0];
#pragma unroll
            for (int j = 1; j < 4 * kVec; ++j) mn = fminf(mn, v[j]);
            const float tb = filter_bound(tau_k);
            if (__ballot_sync(kFull, mn <= tb) != 0u) {
                // merge one float4 group at a time (four values per lane), lowest indices first
                const int i0 = head + 4 * (f0 + lane);
#pragma unroll
                for (int q = 0; q < kVec; ++q) {
                    const float g[4] = {v[4 * q + 0], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]};
                    const float t = filter_bound(tau_k);
                    const unsigned cm = (g[0] <= t ? 1u : 0u) | (g[1] <= t ? 2u : 0u) | (g[2] <= t ? 4u : 0u) |
                                        (g[3] <= t ? 8u : 0u);
                    const unsigned who = __ballot_sync(kFull, cm != 0u);
                    if (who == 0u) continue;
                    const int iq = i0 + 128 * q;
                    // one lane with one candidate (the common case once the list has filled):
                    // insert it directly, without the reduction rounds of a merge
                    const int src = __ffs(who) - 1;
                    const unsigned cm_src = __shfl_sync(kFull, cm, src);
                    if ((who & (who - 1u)) == 0u && (cm_src & (cm_src - 1u)) == 0u) {
                        const int j = __ffs(cm_src) - 1;
                        const float gv = j == 0 ? g[0] : j == 1 ? g[1] : j == 2 ? g[2] : g[3];
                        const unsigned ck = __shfl_sync(kFull, order_key(gv + 0.0f), src);  // -0 ranks as +0
                        const int ci = __shfl_sync(kFull, iq + j, src);
                        if (key_less(ck, ci, tau_k, tau_i)) list_insert(lk, li, tau_k, tau_i, ck, ci, k, lane);
                        continue;
                    }
                    merge_batch<4>(g, cm, [&](int j) { return iq + j; }, lk, li, tau_k, tau_i, k, lane);
                }
            }
#pragma unroll
            for (int q = 0; q < kVec; ++q) cur[q] = nxt[q];
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
    static std::atomic<int> per_sm_cache[tune::kMaxDevices];
    int per_sm = 0;
    int rc = tune::blocks_per_sm(per_sm_cache, reinterpret_cast<const void*>(kern), kThreads, &per_sm);
    if (rc) return rc;
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
    if ((reinterpret_cast<uintptr_t>(scores) & 3) != 0)
        return tune::fail(TUNE_EINVAL, "scores must be 4-byte aligned");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    TUNE_CUDA_TRY(cudaMemsetAsync(workspace, 0, tune::kWorkspaceHeader, s), "tune_topk: status reset");
    if (n_seg == 0) return TUNE_OK;
    return launch(scores, seg_offsets, n_seg, k, topk_idx, topk_score, s);
}
