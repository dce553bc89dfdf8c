// C-ABI glue: error reporting, workspace sizing, status check, version.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "tune_internal.h"

namespace tune {

static thread_local char g_msg[512];

int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(TUNE_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

void clear_error() { g_msg[0] = 0; }

int device_sm_count()
{
    static std::atomic<int> cached[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
    int n = cached[dev].load(std::memory_order_relaxed);
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        cached[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

// Pending injected faults per kind (index = TUNE_FAULT_* value).
static std::atomic<int> g_faults[4];

bool take_fault(int kind)
{
    if (kind < 1 || kind > 3) return false;
    int n = g_faults[kind].load();
    while (n > 0)
        if (g_faults[kind].compare_exchange_weak(n, n - 1)) return true;
    return false;
}

int blocks_per_sm(std::atomic<int> (&cache)[kMaxDevices], const void* kern, int threads, int* out)
{
    int dev = 0;
    TUNE_CUDA_TRY(cudaGetDevice(&dev), "occupancy query: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(TUNE_EUNSUPPORTED, "device ordinal %d too large", dev);
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n == 0) {
        TUNE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, 0), "occupancy query");
        if (n < 1) n = 1;
        cache[dev].store(n, std::memory_order_relaxed);
    }
    *out = n;
    return TUNE_OK;
}

}  // namespace tune

extern "C" {

const char* tune_last_error(void) { return tune::g_msg; }

int tune_version(void) { return 100; }

int tune_inject_fault(int kind, int count)
{
    tune::clear_error();
    if (kind < TUNE_FAULT_COMPILE || kind > TUNE_FAULT_WAIT)
        return tune::fail(TUNE_EINVAL, "tune_inject_fault: unknown kind %d", kind);
    if (count < 0 || count > 1000000) return tune::fail(TUNE_EINVAL, "tune_inject_fault: count outside [0, 10^6]");
    tune::g_faults[kind].store(count);
    return TUNE_OK;
}

size_t tune_workspace_bytes(int call, int64_t n, int32_t k)
{
    (void)call;
    (void)n;
    (void)k;
    return tune::kWorkspaceHeader;
}

int tune_check(const void* workspace, tune_stream_t stream)
{
    tune::clear_error();
    if (!workspace) return tune::fail(TUNE_EINVAL, "tune_check: workspace is NULL");
    int status = 0;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    TUNE_CUDA_TRY(cudaMemcpyAsync(&status, workspace, sizeof(int), cudaMemcpyDeviceToHost, s),
                  "tune_check: cudaMemcpyAsync");
    TUNE_CUDA_TRY(cudaStreamSynchronize(s), "tune_check: cudaStreamSynchronize");
    if (status & tune::kStatusTimeout)
        return tune::fail(TUNE_ETIMEOUT, "a bounded device-side wait gave up");
    if (status & tune::kStatusInvalid)
        return tune::fail(TUNE_EINVAL, "a descriptor was malformed (mask outside the axes, "
                                       "negative count, register or shared-memory field)");
    return TUNE_OK;
}

}  // extern "C"
