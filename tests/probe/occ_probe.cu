// Probe kernels for checking the sm_103 occupancy row against the CUDA
// occupancy API (test infrastructure). Each probe needs many live registers and
// is capped with __maxnreg__, so its register count is near the cap; the test
// reads the actual count with cudaFuncGetAttributes.
#include <cuda_runtime.h>

template <int R>
__global__ void __maxnreg__(R) probe(float* out, int n)
{
    extern __shared__ float dyn[];
    constexpr int A = 256;  // live values: more than any cap, so the cap decides the count
    float acc[A];
#pragma unroll
    for (int i = 0; i < A; ++i) acc[i] = out[(threadIdx.x + i) % 997];
    for (int it = 0; it < n; ++it) {
#pragma unroll
        for (int i = 0; i < A; ++i) acc[i] = acc[i] * acc[(i + 7) & (A - 1)] + 1.0f;
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < A; ++i) s += acc[i];
    if (n < 0) dyn[threadIdx.x] = s;
    out[threadIdx.x] = s;
}

typedef void (*kfn)(float*, int);
static const kfn kProbes[] = {probe<16>, probe<24>, probe<32>, probe<40>, probe<48>, probe<56>,
                              probe<64>, probe<72>, probe<96>, probe<128>, probe<168>, probe<255>};

extern "C" int probe_count(void) { return (int)(sizeof(kProbes) / sizeof(kProbes[0])); }

extern "C" int probe_regs(int i)
{
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, (const void*)kProbes[i]) != cudaSuccess) return -1;
    return a.numRegs;
}

extern "C" int probe_static_smem(int i)
{
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, (const void*)kProbes[i]) != cudaSuccess) return -1;
    return (int)a.sharedSizeBytes;
}

// Blocks per SM from the occupancy API, with the carveout preference set
// (carveout < 0 leaves the default) and dynamic shared memory opted in.
extern "C" int probe_occupancy(int i, int block, int dyn_smem, int carveout)
{
    const void* f = (const void*)kProbes[i];
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) != cudaSuccess)
        return -2;
    if (carveout >= 0 &&
        cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, carveout) != cudaSuccess)
        return -3;
    int nb = -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kProbes[i], block, (size_t)dyn_smem) != cudaSuccess)
        return -4;
    return nb;
}

extern "C" int probe_sm_count(void)
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}
