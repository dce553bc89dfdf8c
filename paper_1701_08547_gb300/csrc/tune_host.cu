// tune_eval_host: tune_eval with the descriptors and results in host memory; chunk i is
// copied in on one library stream, evaluated on the caller's stream and copied out on
// another while chunk i + 1 is copied in and evaluated (two device staging buffers).
// With TUNE_HOST_DIRECT and mapped pinned buffers, one launch reads and writes host
// memory in place over the host link (on Grace-Blackwell, NVLink-C2C), overlapping the
// transfers with the evaluation without staging copies or extra launches.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "tune_internal.h"

namespace {

int64_t align256(int64_t b) { return (b + 255) & ~int64_t(255); }

constexpr int kMaxDevices = 64;

struct HostPipe {
    cudaStream_t in = nullptr, out = nullptr;
    cudaEvent_t start = nullptr, done = nullptr, ev_in[2] = {}, ev_eval[2] = {}, ev_out[2] = {};
};

std::mutex g_pipe_mu;
HostPipe g_pipe[kMaxDevices];

int host_pipe(HostPipe** out)
{
    int dev = 0;
    TUNE_CUDA_TRY(cudaGetDevice(&dev), "tune_eval_host: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return tune::fail(TUNE_EUNSUPPORTED, "device ordinal %d too large", dev);
    std::lock_guard<std::mutex> lock(g_pipe_mu);
    HostPipe& p = g_pipe[dev];
    if (!p.in) {
        const unsigned f = cudaEventDisableTiming;
        TUNE_CUDA_TRY(cudaStreamCreateWithFlags(&p.in, cudaStreamNonBlocking), "tune_eval_host: stream");
        TUNE_CUDA_TRY(cudaStreamCreateWithFlags(&p.out, cudaStreamNonBlocking), "tune_eval_host: stream");
        TUNE_CUDA_TRY(cudaEventCreateWithFlags(&p.start, f), "tune_eval_host: event");
        TUNE_CUDA_TRY(cudaEventCreateWithFlags(&p.done, f), "tune_eval_host: event");
        for (int b = 0; b < 2; ++b) {
            TUNE_CUDA_TRY(cudaEventCreateWithFlags(&p.ev_in[b], f), "tune_eval_host: event");
            TUNE_CUDA_TRY(cudaEventCreateWithFlags(&p.ev_eval[b], f), "tune_eval_host: event");
            TUNE_CUDA_TRY(cudaEventCreateWithFlags(&p.ev_out[b], f), "tune_eval_host: event");
        }
    }
    *out = &p;
    return TUNE_OK;
}

}  // namespace

extern "C" size_t tune_eval_host_scratch_bytes(int64_t chunk, int32_t k)
{
    if (chunk < 1 || k < 1) return 0;
    return (size_t)(tune::kWorkspaceHeader + 2 * (align256(chunk * 64) + 2 * align256(chunk * k * 4)));
}

extern "C" int tune_eval_host(const tune_arch* arch, const tune_axes* axes, const tune_kernel_desc* host_descs,
                              int64_t n_kernels, int32_t k, uint32_t flags, int32_t* host_topk_idx,
                              float* host_topk_cost, int64_t chunk, void* dev_scratch, size_t scratch_bytes,
                              tune_stream_t stream)
{
    tune::clear_error();
    if (!arch || !axes) return tune::fail(TUNE_EINVAL, "arch and axes must be non-NULL host pointers");
    if (k < 1 || k > 16) return tune::fail(TUNE_EINVAL, "k = %d outside [1, 16]", k);
    if (n_kernels < 0) return tune::fail(TUNE_EINVAL, "n_kernels < 0");
    if (chunk < 1 || chunk > (1LL << 26)) return tune::fail(TUNE_EINVAL, "chunk %lld outside [1, 2^26]", (long long)chunk);
    // the direct mode uses only the status header of the scratch
    const size_t need = (flags & TUNE_HOST_DIRECT) ? tune::kWorkspaceHeader : tune_eval_host_scratch_bytes(chunk, k);
    if (!dev_scratch || scratch_bytes < need)
        return tune::fail(TUNE_ENOMEM, "scratch smaller than %zu bytes (tune_eval_host_scratch_bytes(chunk, k), or "
                                       "256 with TUNE_HOST_DIRECT)", need);
    if ((reinterpret_cast<uintptr_t>(dev_scratch) & 255) != 0)
        return tune::fail(TUNE_EINVAL, "dev_scratch must be 256-byte aligned");
    if (n_kernels > 0 && (!host_descs || !host_topk_idx || !host_topk_cost))
        return tune::fail(TUNE_EINVAL, "host_descs and outputs must be non-NULL");
    if (flags & ~(TUNE_SCHED_WARP | TUNE_HOST_DIRECT | 0xff00u))
        return tune::fail(TUNE_EINVAL, "flags 0x%x: only TUNE_SCHED_WARP with its chunk/CTA fields and TUNE_HOST_DIRECT",
                          flags);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (flags & TUNE_HOST_DIRECT) {
        // in place: every buffer must be pinned host memory the device can address
        const void* host[3] = {host_descs, host_topk_idx, host_topk_cost};
        void* dev[3] = {nullptr, nullptr, nullptr};
        for (int i = 0; i < 3 && n_kernels > 0; ++i) {
            cudaPointerAttributes at;
            TUNE_CUDA_TRY(cudaPointerGetAttributes(&at, host[i]), "tune_eval_host: cudaPointerGetAttributes");
            if (at.type != cudaMemoryTypeHost || !at.devicePointer)
                return tune::fail(TUNE_EINVAL, "TUNE_HOST_DIRECT: host buffer %d is not pinned, mapped memory", i);
            dev[i] = at.devicePointer;
        }
        int* status = static_cast<int*>(dev_scratch);
        unsigned long long* queue = reinterpret_cast<unsigned long long*>(dev_scratch) + 1;
        TUNE_CUDA_TRY(cudaMemsetAsync(dev_scratch, 0, tune::kWorkspaceHeader, s), "tune_eval_host: status reset");
        if (n_kernels == 0) return TUNE_OK;
        return tune::eval_launch(arch, axes, static_cast<const tune_kernel_desc*>(dev[0]), n_kernels, k,
                                 flags & ~TUNE_HOST_DIRECT, static_cast<int32_t*>(dev[1]), static_cast<float*>(dev[2]),
                                 status, queue, s);
    }
    HostPipe* hp = nullptr;
    int rc = host_pipe(&hp);
    if (rc) return rc;
    // scratch: header (status word, one queue counter per buffer), then per buffer the
    // descriptors, indices and costs of one chunk
    char* base = static_cast<char*>(dev_scratch);
    int* status = reinterpret_cast<int*>(base);
    unsigned long long* queues = reinterpret_cast<unsigned long long*>(base) + 1;
    char* bufs = base + tune::kWorkspaceHeader;
    const int64_t b_desc = align256(chunk * 64), b_out = align256(chunk * k * 4);
    auto buf_desc = [&](int b) { return reinterpret_cast<tune_kernel_desc*>(bufs + b * (b_desc + 2 * b_out)); };
    auto buf_idx = [&](int b) { return reinterpret_cast<int32_t*>(bufs + b * (b_desc + 2 * b_out) + b_desc); };
    auto buf_cost = [&](int b) { return reinterpret_cast<float*>(bufs + b * (b_desc + 2 * b_out) + b_desc + b_out); };

    TUNE_CUDA_TRY(cudaMemsetAsync(dev_scratch, 0, tune::kWorkspaceHeader, s), "tune_eval_host: status reset");
    TUNE_CUDA_TRY(cudaEventRecord(hp->start, s), "tune_eval_host: event");
    TUNE_CUDA_TRY(cudaStreamWaitEvent(hp->in, hp->start, 0), "tune_eval_host: wait");
    TUNE_CUDA_TRY(cudaStreamWaitEvent(hp->out, hp->start, 0), "tune_eval_host: wait");
    const int64_t n_chunks = (n_kernels + chunk - 1) / chunk;
    for (int64_t i = 0; i < n_chunks; ++i) {
        const int b = (int)(i & 1);
        const int64_t k0 = i * chunk, nk = std::min<int64_t>(chunk, n_kernels - k0);
        // buffer b is free once chunk i - 2 was evaluated (descriptors) and copied out (results)
        if (i >= 2) TUNE_CUDA_TRY(cudaStreamWaitEvent(hp->in, hp->ev_eval[b], 0), "tune_eval_host: wait");
        TUNE_CUDA_TRY(cudaMemcpyAsync(buf_desc(b), host_descs + k0, nk * 64, cudaMemcpyHostToDevice, hp->in),
                      "tune_eval_host: copy in");
        TUNE_CUDA_TRY(cudaEventRecord(hp->ev_in[b], hp->in), "tune_eval_host: event");
        TUNE_CUDA_TRY(cudaStreamWaitEvent(s, hp->ev_in[b], 0), "tune_eval_host: wait");
        if (i >= 2) TUNE_CUDA_TRY(cudaStreamWaitEvent(s, hp->ev_out[b], 0), "tune_eval_host: wait");
        TUNE_CUDA_TRY(cudaMemsetAsync(queues + b, 0, sizeof(unsigned long long), s), "tune_eval_host: queue reset");
        rc = tune::eval_launch(arch, axes, buf_desc(b), nk, k, flags, buf_idx(b), buf_cost(b), status, queues + b, s);
        if (rc) return rc;
        TUNE_CUDA_TRY(cudaEventRecord(hp->ev_eval[b], s), "tune_eval_host: event");
        TUNE_CUDA_TRY(cudaStreamWaitEvent(hp->out, hp->ev_eval[b], 0), "tune_eval_host: wait");
        TUNE_CUDA_TRY(cudaMemcpyAsync(host_topk_idx + k0 * k, buf_idx(b), nk * k * 4, cudaMemcpyDeviceToHost, hp->out),
                      "tune_eval_host: copy out");
        TUNE_CUDA_TRY(cudaMemcpyAsync(host_topk_cost + k0 * k, buf_cost(b), nk * k * 4, cudaMemcpyDeviceToHost, hp->out),
                      "tune_eval_host: copy out");
        TUNE_CUDA_TRY(cudaEventRecord(hp->ev_out[b], hp->out), "tune_eval_host: event");
    }
    // the caller's stream completes once every result is in host memory
    TUNE_CUDA_TRY(cudaEventRecord(hp->done, hp->out), "tune_eval_host: event");
    TUNE_CUDA_TRY(cudaStreamWaitEvent(s, hp->done, 0), "tune_eval_host: wait");
    return TUNE_OK;
}
