// tune_emit_measure: emit synthetic code variants for descriptors, compile them
// at run time (NVRTC, sm_103a), run each sampled tuning point on this GPU and
// time it — the labels of the learned surrogate.
//
// Every thread of a variant executes `items` work items (the same per-thread
// work at every launch configuration, as the static model assumes: its counts
// are per thread, and its cost is the time per unit of that work); per item it
// runs, for each instruction class, a dependent loop of round(n_c * scale)
// operations (FP32 FMA, FP64 FMA, integer LCG step, global load, shared
// load + store, data-dependent branch, SFU sine), unrolled U times; lanes
// below div_lanes repeat the FP32 loop (branch divergence d). NACC values
// are kept live across the item loop so that the register count follows the
// descriptor's r0. One module per (U, NACC) is compiled once per device.
#include <cuda_runtime.h>
#include <nvrtc.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "tune_internal.h"

namespace {

const char* kSource = R"(
// With TUNE_COUNT every thread also tallies the operations of each class it executes (one
// per iteration of that class's loop) and the warp's sums are added to counts[0..6].
#ifdef TUNE_COUNT
#define TALLY(c) (++tally[c])
#else
#define TALLY(c)
#endif
extern "C" __global__ void variant(const float* __restrict__ src, float* __restrict__ dst, int items,
                                   int n_fp32, int n_fp64, int n_int, int n_gld, int n_sld, int n_br,
                                   int n_sfu, int div_lanes, int smem_mask, unsigned long long* counts)
{
    extern __shared__ float sm[];
    const int lane = threadIdx.x & 31;
#ifdef TUNE_COUNT
    unsigned tally[7] = {0u, 0u, 0u, 0u, 0u, 0u, 0u};
#endif
    float keep[NACC];
#pragma unroll
    for (int i = 0; i < NACC; ++i) keep[i] = src[(threadIdx.x * 3 + i * 17) & 4095];
    float f = keep[0];
    double dd = (double)keep[NACC - 1];
    unsigned u = threadIdx.x * 2654435761u + blockIdx.x;
    if (smem_mask >= 0) {
        for (int i = threadIdx.x; i <= smem_mask; i += blockDim.x) sm[i] = (float)i;
        __syncthreads();
    }
    for (int item = 0; item < items; ++item) {
#pragma unroll
        for (int i = 0; i < NACC; ++i) asm volatile("" : "+f"(keep[i]));
#pragma unroll UNROLL
        for (int r = 0; r < n_fp32; ++r) {
            f = fmaf(f, 0.9999f, 0.5f);
            TALLY(0);
        }
#pragma unroll UNROLL
        for (int r = 0; r < n_fp64; ++r) {
            dd = fma(dd, 0.9999, 0.5);
            TALLY(1);
        }
#pragma unroll UNROLL
        for (int r = 0; r < n_int; ++r) {
            u = u * 1664525u + 1013904223u;
            TALLY(2);
        }
#pragma unroll UNROLL
        for (int r = 0; r < n_gld; ++r) {
            f += __ldg(src + ((u + (unsigned)r * 131u) & 1048575u));
            TALLY(3);
        }
#pragma unroll UNROLL
        for (int r = 0; r < n_sld; ++r) {
            const int w = (int)((threadIdx.x + (unsigned)r * 33u) & (unsigned)smem_mask);
            sm[w] = sm[w] * 0.5f + f;
            TALLY(4);
        }
#pragma unroll UNROLL
        for (int r = 0; r < n_br; ++r) {
            if ((u >> (r & 31)) & 1u) f += 1.0f;
            TALLY(5);
        }
#pragma unroll UNROLL
        for (int r = 0; r < n_sfu; ++r) {
            f = __sinf(f);
            TALLY(6);
        }
        if (lane < div_lanes) {
#pragma unroll UNROLL
            for (int r = 0; r < n_fp32; ++r) {
                f = fmaf(f, 1.0001f, 0.25f);
                TALLY(0);
            }
        }
    }
    float acc = f + (float)dd + (float)(u & 255u);
#pragma unroll
    for (int i = 0; i < NACC; ++i) acc += keep[i] * (float)(i + 1);
    dst[(blockIdx.x * blockDim.x + threadIdx.x) & 1048575] = acc;
#ifdef TUNE_COUNT
    const unsigned grp = __activemask();
#pragma unroll
    for (int c = 0; c < 7; ++c) {
        const unsigned v = __reduce_add_sync(grp, tally[c]);
        if (lane == __ffs(grp) - 1 && v) atomicAdd(counts + c, (unsigned long long)v);
    }
#endif
}
)";

struct Module {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
    int regs = 0;
    int static_smem = 0;
};

std::mutex g_mu;
std::map<std::tuple<int, int, int, int>, Module> g_mods;  // (device, unroll, nacc, counting)

int nacc_bucket(int r0)
{
    const int b[] = {8, 24, 40, 56, 72};
    int best = b[0];
    for (int v : b)
        if (std::abs(v + 16 - r0) < std::abs(best + 16 - r0)) best = v;
    return best;
}

int get_module(int dev, int unroll, int nacc, bool counting, Module** out)
{
    std::lock_guard<std::mutex> lock(g_mu);
    if (tune::take_fault(TUNE_FAULT_COMPILE))
        return tune::fail(TUNE_ECOMPILE, "variant compile failed (injected fault)");
    auto key = std::make_tuple(dev, unroll, nacc, counting ? 1 : 0);
    auto it = g_mods.find(key);
    if (it != g_mods.end()) {
        *out = &it->second;
        return TUNE_OK;
    }
    std::string src = std::string("#define NACC ") + std::to_string(nacc) + "\n";
    if (counting) src += "#define TUNE_COUNT 1\n";
    std::string body = kSource;
    for (size_t p; (p = body.find("#pragma unroll UNROLL")) != std::string::npos;)
        body.replace(p, 21, "#pragma unroll " + std::to_string(unroll));
    src += body;
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, src.c_str(), "variant.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
        return tune::fail(TUNE_ECOMPILE, "nvrtcCreateProgram failed");
    const char* opts[] = {"--gpu-architecture=sm_103a"};
    nvrtcResult r = nvrtcCompileProgram(prog, 1, opts);
    if (r != NVRTC_SUCCESS) {
        size_t n = 0;
        nvrtcGetProgramLogSize(prog, &n);
        std::string log(n, '\0');
        nvrtcGetProgramLog(prog, &log[0]);
        nvrtcDestroyProgram(&prog);
        return tune::fail(TUNE_ECOMPILE, "variant compile failed: %.300s", log.c_str());
    }
    size_t n = 0;
    nvrtcGetCUBINSize(prog, &n);
    std::vector<char> cubin(n);
    nvrtcGetCUBIN(prog, cubin.data());
    nvrtcDestroyProgram(&prog);
    Module m;
    TUNE_CUDA_TRY(cudaLibraryLoadData(&m.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0),
                  "tune_emit_measure: cudaLibraryLoadData");
    TUNE_CUDA_TRY(cudaLibraryGetKernel(&m.kern, m.lib, "variant"), "tune_emit_measure: cudaLibraryGetKernel");
    cudaFuncAttributes fa;
    TUNE_CUDA_TRY(cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(m.kern)),
                  "tune_emit_measure: cudaFuncGetAttributes");
    m.regs = fa.numRegs;
    m.static_smem = (int)fa.sharedSizeBytes;
    auto ins = g_mods.emplace(key, m);
    *out = &ins.first->second;
    return TUNE_OK;
}

struct Events {
    std::vector<cudaEvent_t> e;
    ~Events()
    {
        for (auto x : e) cudaEventDestroy(x);
    }
};

struct DevBuf {
    void* p = nullptr;
    ~DevBuf()
    {
        if (p) cudaFree(p);
    }
};

// One sample's variant: the decoded point, its module and the kernel arguments.
struct Launch {
    int T = 0, G = 0, U = 0, C = 0;
    Module* mod = nullptr;
    int n[7] = {0, 0, 0, 0, 0, 0, 0};  // operations per item and class (after scaling)
    int div_lanes = 0, smem_mask = -1, smem_bytes = 0;
};

// Decode sample i (canonical index -> (T, G, U, C), row-major over T, G, U, C restricted to the
// mask, C fastest), pick its module and compute the loop trip counts.
int prepare(const tune_axes* axes, const tune_kernel_desc* descs, int64_t n_kernels, int64_t i, int64_t kid,
            int32_t point, float count_scale, int dev, bool counting, Launch& L)
{
    if (kid < 0 || kid >= n_kernels) return tune::fail(TUNE_EINVAL, "sample %lld: kernel out of range", (long long)i);
    const tune_kernel_desc& d = descs[kid];
    const uint64_t m = d.space_mask;
    const uint32_t tm = (uint32_t)m, gm = (uint32_t)(m >> 32) & 0xffffu, um = (uint32_t)(m >> 48) & 0xffu,
                   cm = (uint32_t)(m >> 56) & 0xfu;
    const int nT = __builtin_popcount(tm), nG = __builtin_popcount(gm), nU = __builtin_popcount(um),
              nC = __builtin_popcount(cm);
    int p = point;
    if (p < 0 || p >= nT * nG * nU * nC) return tune::fail(TUNE_EINVAL, "sample %lld: point out of range", (long long)i);
    auto nth = [](uint32_t mask, int r) {
        for (int b = 0; b < 32; ++b)
            if ((mask >> b) & 1u)
                if (r-- == 0) return b;
        return -1;
    };
    const int c_r = p % nC;
    p /= nC;
    const int u_r = p % nU;
    p /= nU;
    const int g_r = p % nG, t_r = p / nG;
    L.T = axes->t[nth(tm, t_r)];
    L.G = axes->g[nth(gm, g_r)];
    L.U = axes->u[nth(um, u_r)];
    L.C = axes->c[nth(cm, c_r)];
    int rc = get_module(dev, L.U, nacc_bucket(d.r0), counting, &L.mod);
    if (rc) return rc;
    for (int c = 0; c < 7; ++c) L.n[c] = (int)(d.n[c] * count_scale + 0.5f);
    const int smem_words = d.s0 / 4;
    if (smem_words > 0) {
        int pw = 1;
        while (pw * 2 <= smem_words) pw *= 2;
        L.smem_mask = pw - 1;
    } else {
        L.n[4] = 0;  // no shared memory: no shared loads and stores
    }
    L.smem_bytes = d.s0;
    L.div_lanes = (int)(d.d * 32.0f + 0.5f);
    return TUNE_OK;
}

// Set the module's shared-memory attributes for carveout C; false if the GPU refuses them.
bool set_attributes(const Launch& L)
{
    const void* fn = reinterpret_cast<const void*>(L.mod->kern);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024 - L.mod->static_smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, L.C) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

}  // namespace

extern "C" int tune_emit_measure(const tune_axes* axes, const tune_kernel_desc* descs, int64_t n_kernels,
                                 const int32_t* sample_kernel, const int32_t* sample_point, int64_t n_samples,
                                 int32_t items, float count_scale, int32_t reps, float* us, int32_t* regs,
                                 int32_t* launched, tune_stream_t stream)
{
    tune::clear_error();
    if (!axes || !descs || !sample_kernel || !sample_point || !us || !regs || n_samples < 0 || items < 1 ||
        reps < 1 || reps > 31 || !(count_scale > 0.0f))
        return tune::fail(TUNE_EINVAL, "tune_emit_measure: bad arguments");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0;
    TUNE_CUDA_TRY(cudaGetDevice(&dev), "tune_emit_measure: cudaGetDevice");
    DevBuf src, dst;
    TUNE_CUDA_TRY(cudaMalloc(&src.p, (1 << 20) * sizeof(float)), "tune_emit_measure: cudaMalloc");
    TUNE_CUDA_TRY(cudaMalloc(&dst.p, (1 << 20) * sizeof(float)), "tune_emit_measure: cudaMalloc");
    {
        std::vector<float> h(1 << 20);
        for (size_t i = 0; i < h.size(); ++i) h[i] = 1.0f + (float)(i % 97) * 1e-3f;
        TUNE_CUDA_TRY(cudaMemcpy(src.p, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice),
                      "tune_emit_measure: init");
    }
    Events ev;
    ev.e.resize(2 * reps);
    for (auto& x : ev.e) TUNE_CUDA_TRY(cudaEventCreate(&x), "tune_emit_measure: cudaEventCreate");
    std::vector<float> t(reps);
    for (int64_t i = 0; i < n_samples; ++i) {
        us[i] = __builtin_nanf("");
        regs[i] = 0;
        Launch L;
        int rc = prepare(axes, descs, n_kernels, i, sample_kernel[i], sample_point[i], count_scale, dev, false, L);
        if (rc) return rc;
        if (launched) {
            launched[4 * i] = L.T;
            launched[4 * i + 1] = L.G;
            launched[4 * i + 2] = L.U;
            launched[4 * i + 3] = L.C;
        }
        regs[i] = L.mod->regs;
        if (!set_attributes(L)) continue;
        const void* fn = reinterpret_cast<const void*>(L.mod->kern);
        int T = L.T, G = L.G;
        unsigned long long* no_counts = nullptr;
        void* args[] = {&src.p, &dst.p, &items, &L.n[0], &L.n[1], &L.n[2], &L.n[3], &L.n[4], &L.n[5], &L.n[6],
                        &L.div_lanes, &L.smem_mask, &no_counts};
        // warm-up; a configuration the GPU cannot launch (too many registers or too much shared
        // memory for T) is skipped and reported as NaN
        if (cudaLaunchKernel(fn, dim3(G), dim3(T), args, (size_t)L.smem_bytes, s) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        for (int r = 0; r < reps; ++r) {
            TUNE_CUDA_TRY(cudaEventRecord(ev.e[2 * r], s), "tune_emit_measure: event");
            TUNE_CUDA_TRY(cudaLaunchKernel(fn, dim3(G), dim3(T), args, (size_t)L.smem_bytes, s),
                          "tune_emit_measure: launch");
            TUNE_CUDA_TRY(cudaEventRecord(ev.e[2 * r + 1], s), "tune_emit_measure: event");
        }
        TUNE_CUDA_TRY(cudaStreamSynchronize(s), "tune_emit_measure: sync");
        for (int r = 0; r < reps; ++r) {
            TUNE_CUDA_TRY(cudaEventElapsedTime(&t[r], ev.e[2 * r], ev.e[2 * r + 1]), "tune_emit_measure: elapsed");
            if (tune::take_fault(TUNE_FAULT_SLOW_REP)) t[r] += 1000.0f;  // injected: one second more
        }
        std::sort(t.begin(), t.end());
        us[i] = 1000.0f * t[reps / 2];
    }
    return TUNE_OK;
}

extern "C" int tune_emit_count(const tune_axes* axes, const tune_kernel_desc* descs, int64_t n_kernels,
                               const int32_t* sample_kernel, const int32_t* sample_point, int64_t n_samples,
                               int32_t items, float count_scale, uint64_t* counts, tune_stream_t stream)
{
    tune::clear_error();
    if (!axes || !descs || !sample_kernel || !sample_point || !counts || n_samples < 0 || items < 1 ||
        !(count_scale > 0.0f))
        return tune::fail(TUNE_EINVAL, "tune_emit_count: bad arguments");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0;
    TUNE_CUDA_TRY(cudaGetDevice(&dev), "tune_emit_count: cudaGetDevice");
    DevBuf src, dst, cnt;
    TUNE_CUDA_TRY(cudaMalloc(&src.p, (1 << 20) * sizeof(float)), "tune_emit_count: cudaMalloc");
    TUNE_CUDA_TRY(cudaMalloc(&dst.p, (1 << 20) * sizeof(float)), "tune_emit_count: cudaMalloc");
    TUNE_CUDA_TRY(cudaMalloc(&cnt.p, 7 * sizeof(unsigned long long)), "tune_emit_count: cudaMalloc");
    TUNE_CUDA_TRY(cudaMemsetAsync(src.p, 0, (1 << 20) * sizeof(float), s), "tune_emit_count: init");
    for (int64_t i = 0; i < n_samples; ++i) {
        for (int c = 0; c < 7; ++c) counts[7 * i + c] = UINT64_MAX;
        Launch L;
        int rc = prepare(axes, descs, n_kernels, i, sample_kernel[i], sample_point[i], count_scale, dev, true, L);
        if (rc) return rc;
        if (!set_attributes(L)) continue;
        TUNE_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, 7 * sizeof(unsigned long long), s), "tune_emit_count: reset");
        const void* fn = reinterpret_cast<const void*>(L.mod->kern);
        unsigned long long* c_dev = static_cast<unsigned long long*>(cnt.p);
        void* args[] = {&src.p, &dst.p, &items, &L.n[0], &L.n[1], &L.n[2], &L.n[3], &L.n[4], &L.n[5], &L.n[6],
                        &L.div_lanes, &L.smem_mask, &c_dev};
        if (cudaLaunchKernel(fn, dim3(L.G), dim3(L.T), args, (size_t)L.smem_bytes, s) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        TUNE_CUDA_TRY(cudaMemcpyAsync(counts + 7 * i, cnt.p, 7 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                      s),
                      "tune_emit_count: copy");
        TUNE_CUDA_TRY(cudaStreamSynchronize(s), "tune_emit_count: sync");
    }
    return TUNE_OK;
}
