// tune_real_measure: the paper's benchmark kernels as tuning variants on this GPU —
// matVec2D (y = A x), ATAX (y = A^T (A x)) and BiCG (q = A p, s = A^T r), the
// dense linear-algebra kernels of its evaluation (Section IV-A, Table "Kernel specifications").
// A variant fixes the block size T, the grid size G, the unroll factor U of the
// inner loop and the shared-memory carveout C; each product is a grid-stride loop
// over output elements (one thread per row for A x, per column for A^T x), the
// inner loop over the matrix order unrolled U times. One module per U is compiled
// at run time (NVRTC, sm_103a) and cached per device.
#include <cuda_runtime.h>
#include <nvrtc.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "tune_internal.h"

namespace {

const char* kRealSource = R"(
extern "C" __global__ void rows(const float* __restrict__ A, const float* __restrict__ x, float* __restrict__ y, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float* a = A + (size_t)i * n;
        float s = 0.0f;
#pragma unroll UNROLL
        for (int j = 0; j < n; ++j) s = fmaf(a[j], x[j], s);
        y[i] = s;
    }
}
extern "C" __global__ void cols(const float* __restrict__ A, const float* __restrict__ x, float* __restrict__ y, int n)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        float s = 0.0f;
#pragma unroll UNROLL
        for (int i = 0; i < n; ++i) s = fmaf(A[(size_t)i * n + j], x[i], s);
        y[j] = s;
    }
}
)";

struct RealModule {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t rows = nullptr, cols = nullptr;
    int regs = 0;
};

std::mutex g_real_mu;
std::map<std::pair<int, int>, RealModule> g_real_mods;  // (device, unroll)

int real_module(int dev, int unroll, RealModule** out)
{
    std::lock_guard<std::mutex> lock(g_real_mu);
    if (tune::take_fault(TUNE_FAULT_COMPILE))
        return tune::fail(TUNE_ECOMPILE, "real kernel compile failed (injected fault)");
    auto key = std::make_pair(dev, unroll);
    auto it = g_real_mods.find(key);
    if (it != g_real_mods.end()) {
        *out = &it->second;
        return TUNE_OK;
    }
    std::string body = kRealSource;
    for (size_t p; (p = body.find("#pragma unroll UNROLL")) != std::string::npos;)
        body.replace(p, 21, "#pragma unroll " + std::to_string(unroll));
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, body.c_str(), "real.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
        return tune::fail(TUNE_ECOMPILE, "nvrtcCreateProgram failed");
    const char* opts[] = {"--gpu-architecture=sm_103a"};
    if (nvrtcCompileProgram(prog, 1, opts) != NVRTC_SUCCESS) {
        size_t n = 0;
        nvrtcGetProgramLogSize(prog, &n);
        std::string log(n, '\0');
        nvrtcGetProgramLog(prog, &log[0]);
        nvrtcDestroyProgram(&prog);
        return tune::fail(TUNE_ECOMPILE, "real kernel compile failed: %.300s", log.c_str());
    }
    size_t n = 0;
    nvrtcGetCUBINSize(prog, &n);
    std::vector<char> cubin(n);
    nvrtcGetCUBIN(prog, cubin.data());
    nvrtcDestroyProgram(&prog);
    RealModule m;
    TUNE_CUDA_TRY(cudaLibraryLoadData(&m.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0),
                  "tune_real_measure: cudaLibraryLoadData");
    TUNE_CUDA_TRY(cudaLibraryGetKernel(&m.rows, m.lib, "rows"), "tune_real_measure: cudaLibraryGetKernel");
    TUNE_CUDA_TRY(cudaLibraryGetKernel(&m.cols, m.lib, "cols"), "tune_real_measure: cudaLibraryGetKernel");
    cudaFuncAttributes fr, fc;
    TUNE_CUDA_TRY(cudaFuncGetAttributes(&fr, reinterpret_cast<const void*>(m.rows)), "tune_real_measure: attributes");
    TUNE_CUDA_TRY(cudaFuncGetAttributes(&fc, reinterpret_cast<const void*>(m.cols)), "tune_real_measure: attributes");
    m.regs = std::max(fr.numRegs, fc.numRegs);
    auto ins = g_real_mods.emplace(key, m);
    *out = &ins.first->second;
    return TUNE_OK;
}

// Deterministic operands: A[i][j] = ((7 i + 13 j) mod 17 - 8) / 8, v[j] = ((5 j + 3 w) mod 11 - 5) / 4
// for vector w (0: x or p, 1: r).
__global__ void init_matrix(float* A, int n)
{
    const size_t total = (size_t)n * n;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t i = e / n, j = e % n;
        A[e] = (float)((int)((7 * i + 13 * j) % 17) - 8) * 0.125f;
    }
}

__global__ void init_vector(float* v, int n, int w)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        v[j] = (float)((int)(((long long)5 * j + 3 * w) % 11) - 5) * 0.25f;
}

struct RealBufs {
    std::vector<void*> p;
    ~RealBufs()
    {
        for (auto x : p)
            if (x) cudaFree(x);
    }
};

}  // namespace

extern "C" int tune_real_measure(int32_t kernel, int32_t n, const int32_t* T, const int32_t* G, const int32_t* U,
                                 const int32_t* C, int32_t n_variants, int32_t reps, float* us, int32_t* regs,
                                 float* result, tune_stream_t stream)
{
    tune::clear_error();
    if (kernel < TUNE_REAL_MATVEC || kernel > TUNE_REAL_BICG || n < 1 || n > 16384 || n_variants < 0 || reps < 1 ||
        reps > 31 || (n_variants > 0 && (!T || !G || !U || !C || !us || !regs)))
        return tune::fail(TUNE_EINVAL, "tune_real_measure: bad arguments");
    for (int v = 0; v < n_variants; ++v)
        if (T[v] < 1 || T[v] > 1024 || G[v] < 1 || U[v] < 1 || U[v] > 64 || C[v] < 0 || C[v] > 100)
            return tune::fail(TUNE_EINVAL, "tune_real_measure: variant %d out of range", v);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0;
    TUNE_CUDA_TRY(cudaGetDevice(&dev), "tune_real_measure: cudaGetDevice");
    RealBufs b;
    b.p.assign(6, nullptr);  // A, x|p, r, out1, out2 (tmp for ATAX), spare
    float *A, *x, *r, *o1, *o2;
    TUNE_CUDA_TRY(cudaMalloc(&b.p[0], (size_t)n * n * sizeof(float)), "tune_real_measure: cudaMalloc");
    for (int i = 1; i < 5; ++i)
        TUNE_CUDA_TRY(cudaMalloc(&b.p[i], (size_t)n * sizeof(float)), "tune_real_measure: cudaMalloc");
    A = (float*)b.p[0];
    x = (float*)b.p[1];
    r = (float*)b.p[2];
    o1 = (float*)b.p[3];
    o2 = (float*)b.p[4];
    init_matrix<<<1024, 256, 0, s>>>(A, n);
    init_vector<<<64, 256, 0, s>>>(x, n, 0);
    init_vector<<<64, 256, 0, s>>>(r, n, 1);
    TUNE_CUDA_TRY(cudaGetLastError(), "tune_real_measure: init launch");
    std::vector<cudaEvent_t> ev(2 * reps);
    for (auto& e : ev) TUNE_CUDA_TRY(cudaEventCreate(&e), "tune_real_measure: cudaEventCreate");
    struct EvFree {
        std::vector<cudaEvent_t>& e;
        ~EvFree()
        {
            for (auto x : e) cudaEventDestroy(x);
        }
    } ev_free{ev};
    std::vector<float> t(reps);
    for (int v = 0; v < n_variants; ++v) {
        us[v] = __builtin_nanf("");
        regs[v] = 0;
        RealModule* mod = nullptr;
        int rc = real_module(dev, U[v], &mod);
        if (rc) return rc;
        regs[v] = mod->regs;
        const void* fr = reinterpret_cast<const void*>(mod->rows);
        const void* fc = reinterpret_cast<const void*>(mod->cols);
        if (cudaFuncSetAttribute(fr, cudaFuncAttributePreferredSharedMemoryCarveout, C[v]) != cudaSuccess ||
            cudaFuncSetAttribute(fc, cudaFuncAttributePreferredSharedMemoryCarveout, C[v]) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        // the kernel's launches: matVec2D y = A x; ATAX tmp = A x, y = A^T tmp; BiCG q = A p, s = A^T r
        void* a_rows[] = {&A, &x, &o1, &n};
        void* a_cols_atax[] = {&A, &o1, &o2, &n};
        void* a_cols_bicg[] = {&A, &r, &o2, &n};
        auto run = [&]() -> cudaError_t {
            cudaError_t e = cudaLaunchKernel(fr, dim3(G[v]), dim3(T[v]), a_rows, 0, s);
            if (e != cudaSuccess || kernel == TUNE_REAL_MATVEC) return e;
            return cudaLaunchKernel(fc, dim3(G[v]), dim3(T[v]), kernel == TUNE_REAL_ATAX ? a_cols_atax : a_cols_bicg,
                                    0, s);
        };
        // warm-up; a configuration the GPU cannot launch is reported as NaN
        if (run() != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        for (int q = 0; q < reps; ++q) {
            TUNE_CUDA_TRY(cudaEventRecord(ev[2 * q], s), "tune_real_measure: event");
            TUNE_CUDA_TRY(run(), "tune_real_measure: launch");
            TUNE_CUDA_TRY(cudaEventRecord(ev[2 * q + 1], s), "tune_real_measure: event");
        }
        TUNE_CUDA_TRY(cudaStreamSynchronize(s), "tune_real_measure: sync");
        for (int q = 0; q < reps; ++q) {
            TUNE_CUDA_TRY(cudaEventElapsedTime(&t[q], ev[2 * q], ev[2 * q + 1]), "tune_real_measure: elapsed");
            if (tune::take_fault(TUNE_FAULT_SLOW_REP)) t[q] += 1000.0f;  // injected: one second more
        }
        std::sort(t.begin(), t.end());
        us[v] = 1000.0f * t[reps / 2];
        if (v == 0 && result) {
            // matVec2D: y; ATAX: y (= A^T A x); BiCG: q then s
            if (kernel == TUNE_REAL_MATVEC) {
                TUNE_CUDA_TRY(cudaMemcpy(result, o1, (size_t)n * 4, cudaMemcpyDeviceToHost), "tune_real_measure: copy");
            } else if (kernel == TUNE_REAL_ATAX) {
                TUNE_CUDA_TRY(cudaMemcpy(result, o2, (size_t)n * 4, cudaMemcpyDeviceToHost), "tune_real_measure: copy");
            } else {
                TUNE_CUDA_TRY(cudaMemcpy(result, o1, (size_t)n * 4, cudaMemcpyDeviceToHost), "tune_real_measure: copy");
                TUNE_CUDA_TRY(cudaMemcpy(result + n, o2, (size_t)n * 4, cudaMemcpyDeviceToHost),
                              "tune_real_measure: copy");
            }
        }
    }
    TUNE_CUDA_TRY(cudaStreamSynchronize(s), "tune_real_measure: sync");
    return TUNE_OK;
}
