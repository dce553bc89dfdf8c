// tune_autotune: choose tune_eval's schedule for a workload by timing candidates
// on the caller's own descriptors (CUDA events on the caller's stream).
#include <cuda_runtime.h>

#include "tune_internal.h"

namespace {

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

}  // namespace

extern "C" int tune_autotune(const tune_arch* arch, const tune_axes* axes,
                             const tune_kernel_desc* descs, int64_t n_kernels, int32_t k,
                             int32_t reps, int32_t* topk_idx, float* topk_cost, void* workspace,
                             size_t ws_bytes, uint32_t* best_flags, float* best_ms,
                             tune_stream_t stream)
{
    tune::clear_error();
    if (!best_flags || !best_ms) return tune::fail(TUNE_EINVAL, "best_flags and best_ms must be non-NULL");
    if (reps < 1 || reps > 100) return tune::fail(TUNE_EINVAL, "reps = %d outside [1, 100]", reps);
    // Candidates: the warp schedule with a static stride or a work queue of
    // 1, 4, 16 or 64 descriptors per grab, at full residency or 2 / 3 CTAs per
    // SM; and the thread schedule.
    uint32_t cands[32];
    int nc = 0;
    const int chunks[] = {-1, 0, 2, 4, 6};
    const int ctas[] = {0, 2, 3};
    for (int c : chunks)
        for (int m : ctas)
            cands[nc++] = TUNE_SCHED_WARP | (c < 0 ? 0u : TUNE_SCHED_CHUNK(c)) | (m ? TUNE_SCHED_CTAS(m) : 0u);
    cands[nc++] = TUNE_SCHED_THREAD;

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    EventPair ev;
    TUNE_CUDA_TRY(cudaEventCreate(&ev.a), "tune_autotune: cudaEventCreate");
    TUNE_CUDA_TRY(cudaEventCreate(&ev.b), "tune_autotune: cudaEventCreate");
    float best = 3.0e38f;
    uint32_t best_f = cands[0];
    for (int i = 0; i < nc; ++i) {
        auto run = [&]() {
            return tune_eval(arch, axes, descs, n_kernels, k, cands[i], topk_idx, topk_cost, nullptr,
                             nullptr, nullptr, nullptr, workspace, ws_bytes, stream);
        };
        int rc = run();  // warm-up (also validates the arguments)
        if (rc) return rc;
        float t_min = 3.0e38f;
        for (int r = 0; r < reps; ++r) {
            TUNE_CUDA_TRY(cudaEventRecord(ev.a, s), "tune_autotune: cudaEventRecord");
            rc = run();
            if (rc) return rc;
            TUNE_CUDA_TRY(cudaEventRecord(ev.b, s), "tune_autotune: cudaEventRecord");
            TUNE_CUDA_TRY(cudaEventSynchronize(ev.b), "tune_autotune: cudaEventSynchronize");
            float ms = 0.0f;
            TUNE_CUDA_TRY(cudaEventElapsedTime(&ms, ev.a, ev.b), "tune_autotune: cudaEventElapsedTime");
            if (ms < t_min) t_min = ms;
        }
        if (t_min < best) {
            best = t_min;
            best_f = cands[i];
        }
    }
    // Leave the chosen schedule's results in the outputs.
    int rc = tune_eval(arch, axes, descs, n_kernels, k, best_f, topk_idx, topk_cost, nullptr, nullptr,
                       nullptr, nullptr, workspace, ws_bytes, stream);
    if (rc) return rc;
    TUNE_CUDA_TRY(cudaStreamSynchronize(s), "tune_autotune: cudaStreamSynchronize");
    *best_flags = best_f;
    *best_ms = best;
    return TUNE_OK;
}
