// Programmatic dependent launch for the surrogate's training step.
//
// A training step is a chain of launches on one stream, each consuming the one
// before it. Launched with the programmatic-serialization attribute, a kernel
// may be scheduled while its predecessor is still running; its CTAs then park
// in grid_dep_wait() until the predecessor has completed and its memory
// operations are visible, so the launch latency between the two is hidden.
//
// Rules that keep this correct and free of deadlock:
//  * every kernel launched by launch_dep() calls grid_dep_wait() before any
//    global-memory access (read or write) and before allocating tensor memory;
//  * a kernel calls grid_dep_launch() only after its own grid_dep_wait(), so at
//    most one kernel waits ahead of the running one;
//  * in a kernel launched without the attribute both calls return at once.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace pdl {

__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// Both, in the order the rules above require.
__device__ __forceinline__ void grid_dep_enter()
{
    grid_dep_wait();
    grid_dep_launch();
}

// kern<<<grid, block, smem, s>>>(args...) with the programmatic-serialization attribute.
template <typename... KArgs, typename... Args>
cudaError_t launch_dep(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace pdl
