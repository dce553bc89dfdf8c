// Internal helpers shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "tune.h"

namespace tune {

// Record an error message for tune_last_error() and return `code`.
int fail(int code, const char* fmt, ...);
// Map a CUDA error to TUNE_ECUDA with a message naming the call site.
int cuda_fail(cudaError_t e, const char* what);
// Clear the thread's last-error message.
void clear_error();

// Status word bits written by kernels into the first word of the workspace.
enum : int { kStatusInvalid = 1, kStatusTimeout = 2 };

// Workspace header: status word and counters, 256 bytes, zeroed per call.
constexpr size_t kWorkspaceHeader = 256;

// Number of SMs of the current device (cached per device).
int device_sm_count();

// Device ordinals the per-device caches cover.
constexpr int kMaxDevices = 64;

// Resident blocks per SM of `kern` launched with `threads` threads and no dynamic shared
// memory on the current device (at least 1): the occupancy query runs once per device and
// its answer is kept in cache[device] (one cache per kernel, shared by host threads).
int blocks_per_sm(std::atomic<int> (&cache)[kMaxDevices], const void* kern, int threads, int* out);

// Injected faults (tune_inject_fault): true, and one fewer pending, if a fault of this
// kind is pending.
bool take_fault(int kind);

// Host-side checks of an architecture row and tuning axes against the limits stated
// in tune.h (TUNE_EINVAL with a message, or TUNE_OK).
int validate_inputs(const tune_arch* arch, const tune_axes* axes);

// tune_eval's warp-schedule launch for one architecture row (flags: TUNE_SCHED_WARP
// with its chunk / CTA fields), with a caller-chosen status word and queue counter.
int eval_launch(const tune_arch* arch, const tune_axes* axes, const tune_kernel_desc* descs, int64_t n_kernels,
                int32_t k, uint32_t flags, int32_t* topk_idx, float* topk_cost, int* status,
                unsigned long long* queue, cudaStream_t s);

}  // namespace tune

#define TUNE_CUDA_TRY(call, what)                                         \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return ::tune::cuda_fail(e_, what);        \
    } while (0)
