// Weight and bias gradients of surrogate training on tcgen05:
//   dW_l[o][i] = sum over batch rows r of dZ_l[r][o] * Hprev[r][i],   db_l[o] = sum over r of dZ_l[r][o]
// (Hprev = the layer's input: the previous layer's activations, or the feature rows).
// The contraction runs over the batch, the index along which neither operand is
// contiguous, so both operands are fed to the MMA MN-major: TMA copies boxes of
// 64 rows x 64 BF16 columns with 128-byte swizzle, which is the MN-major swizzle
// atom (8 rows of K by 64 elements of M or N, 1 KB) repeated 8 times along K
// (1 KB apart) and, box by box, along M or N (8 KB apart).
//
// Grid (2 splits, members): CTA (2 s + h, m) sums a contiguous range of 64-row chunks
// for output rows o in [128 h, 128 h + 128) of member m and writes its FP32 partial
// [128][kin] into part[m][s] (the two halves of a split fill one [256][kin] slice);
// split_reduce adds the partials in split order (deterministic). The two halves of a
// split read the same Hprev rows at about the same time, so the second read is
// served from L2. The bias gradient comes from the same pass: the epilogue warps, idle
// until the last MMA, add up each stage's dZ columns from shared memory before the
// stage is released. Roles: warp 0 issues the TMA copies through a ring of four 48 KB
// stages, warp 1 issues the MMAs (one 128 x kin x 16 product per 16-row K step), warps
// 2-9 read the accumulator back (thread = output row, two warps per TMEM lane quarter,
// one per column half) and store the partial, row-contiguous through shared memory.
//
// Every wait is bounded; on timeout the kernel sets status bit 2, stops issuing work,
// waits (bounded) for the copies and MMAs it issued, frees its tensor memory and
// returns.
#pragma once

#include "tc_mlp.cuh"

namespace tcw {

constexpr int kChunkRows = 64;                 // batch rows (K) per stage
constexpr int kBox = kChunkRows * 128;         // one TMA box: 64 rows x 64 BF16 columns
constexpr int kStageA = 2 * kBox;              // dZ: the CTA's 128 output columns
constexpr int kStageB = 4 * kBox;              // Hprev: up to 256 input columns
constexpr int kStage = kStageA + kStageB;
constexpr int kStages = 4;
constexpr int kSmem = 1024 + kStages * kStage;
constexpr int kEpiWarps = 8;
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr int kBiasRows = 4;                   // row quarters of a chunk in the bias sums
static_assert(kSmem <= 227 * 1024, "shared memory");
static_assert(kEpiWarps * 32 * 33 * 4 <= kStages * kStage, "read-back tiles fit in the stage ring");

struct Args {
    int kin;          // input columns: 128 or 256
    int chunks;       // batch rows / 64
    int splits;       // CTA pairs per member; split s sums chunks [s chunks / splits, (s + 1) chunks / splits)
    float* part;      // [members][splits][256][kin]
    float* bpart;     // [members][splits][kBiasRows][256]: column sums of dZ over the split's rows
    int* status;
};

// MN-major operand, 128-byte swizzle: leading byte offset = distance between atoms
// adjacent in M or N (one box, 8 KB), stride byte offset = distance between atoms
// adjacent in K (8 rows of 128 bytes).
__device__ __forceinline__ uint64_t sdesc_mn(const void* p)
{
    const uint64_t addr = tc::sa(p);
    return ((addr >> 4) & 0x3fffull) | ((uint64_t)(kBox >> 4) << 16) | ((1024ull >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

// kind::f16 instruction descriptor with A and B MN-major.
__host__ __device__ constexpr uint32_t idesc_bf16_mn(int M, int N)
{
    return tc::idesc_bf16(M, N) | (1u << 15) | (1u << 16);
}

// ta: dZ as 8-byte elements {64, rows, members}, box {16, 64, 1};
// tb: Hprev as 8-byte elements {kin / 4, rows, members or 1}, box {16, 64, 1}; b_batched
// selects the member coordinate (0: one input shared by all members).
__global__ void __launch_bounds__(kThreads, 1) wgrad_kernel(const __grid_constant__ CUtensorMap ta,
                                                            const __grid_constant__ CUtensorMap tb,
                                                            const __grid_constant__ Args g, int b_batched)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full[kStages], empty[kStages], acc_full, drain;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int half = blockIdx.x & 1, split = blockIdx.x >> 1, mem = blockIdx.y;
    const int c_beg = (int)((long long)split * g.chunks / g.splits);
    const int c_end = (int)((long long)(split + 1) * g.chunks / g.splits);
    const int n = c_end - c_beg;
    const int nb = g.kin / 64;  // B boxes per stage
    volatile int* abort_v = &abort_flag;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tc::sa(&tmem_base)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (threadIdx.x == 32) {
        for (int i = 0; i < kStages; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1 + kEpiWarps);  // the MMAs' commit and each epilogue warp
        }
        tc::mbar_init(&acc_full, 1);
        tc::mbar_init(&drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        abort_flag = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        // ---- producer ----
        if (lane == 0) {
            int i = 0;
            bool ok = true;
            for (; i < n; ++i) {
                const int st = i % kStages, use = i / kStages;
                if (use > 0 && !(ok = tcm::wait_bar(&empty[st], (uint32_t)((use - 1) & 1), g.status, abort_v)))
                    break;
                uint8_t* a = smem + st * kStage;
                uint8_t* b = a + kStageA;
                const int r0 = (c_beg + i) * kChunkRows;
                tc::mbar_expect_tx(&full[st], (uint32_t)(kStageA + nb * kBox));
                for (int j = 0; j < 2; ++j) tc::tma_load_3d(a + j * kBox, &ta, (2 * half + j) * 16, r0, mem, &full[st]);
                for (int j = 0; j < nb; ++j)
                    tc::tma_load_3d(b + j * kBox, &tb, j * 16, r0, b_batched ? mem : 0, &full[st]);
            }
            if (!ok)  // let the copies in flight land before the CTA exits
                for (int q = i - kStages; q < i; ++q)
                    if (q >= 0) tc::mbar_wait(&full[q % kStages], (uint32_t)((q / kStages) & 1), g.status);
        }
    } else if (warp == 1) {
        // ---- MMA issuer ----
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_mn(128, g.kin);
            bool ok = true;
            for (int i = 0; i < n && ok; ++i) {
                const int st = i % kStages;
                if (!(ok = tcm::wait_bar(&full[st], (uint32_t)((i / kStages) & 1), g.status, abort_v))) break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint8_t* a = smem + st * kStage;
                const uint8_t* b = a + kStageA;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)  // 16 batch rows = two K atoms per step
                    tc::mma_bf16(tmem, sdesc_mn(a + kk * 2048), sdesc_mn(b + kk * 2048), idesc, (i | kk) != 0);
                tc::mma_commit(&empty[st]);
            }
            if (ok && n > 0) tc::mma_commit(&acc_full);
            tc::mma_commit(&drain);
            tc::mbar_wait(&drain, 0, g.status);
        }
    } else {
        // ---- epilogue warps, while the MMAs run: column sums of dZ (the bias gradient) from
        // each stage's two dZ boxes; thread et sums local columns c, c + 1 (c = 2 (et % 64))
        // over rows 16 (et / 64) .. + 15 of every chunk, then releases the stage with its warp ----
        const int et = threadIdx.x - 64;
        const int bc = 2 * (et & 63), rq = et >> 6;
        {
            float s0 = 0.0f, s1 = 0.0f;
            const int unit = (bc & 63) >> 3, byte = (bc & 7) * 2;
            for (int i = 0; i < n; ++i) {
                const int st = i % kStages;
                if (!tcm::wait_bar(&full[st], (uint32_t)((i / kStages) & 1), g.status, abort_v)) break;
                const uint8_t* box = smem + st * kStage + (bc >> 6) * kBox;
#pragma unroll 8
                for (int rr = 0; rr < kChunkRows / kBiasRows; ++rr) {
                    const int r = (kChunkRows / kBiasRows) * rq + rr;
                    // 128-byte swizzle: 16-byte unit u of row r sits at unit u ^ (r % 8)
                    const uint32_t w = *reinterpret_cast<const uint32_t*>(box + r * 128 + ((unit ^ (r & 7)) << 4) + byte);
                    s0 += __uint_as_float(w << 16);
                    s1 += __uint_as_float(w & 0xffff0000u);
                }
                __syncwarp();
                if (lane == 0) tcm::mbar_arrive(&empty[st]);
            }
            *reinterpret_cast<float2*>(g.bpart + (((long long)mem * g.splits + split) * kBiasRows + rq) * 256 +
                                       128 * half + bc) = make_float2(s0, s1);
        }
        // the accumulator read-back below reuses the stage ring: every epilogue warp has
        // finished reading it (all 256 epilogue threads reach this barrier once, on every path)
        asm volatile("bar.sync 1, %0;\n" ::"n"(32 * kEpiWarps) : "memory");
        // ---- then partial[o][c] for o = 128 half + 32 q + lane ----
        const int e = warp - 2, q = warp & 3, ch = e >> 2;
        const int ncol = g.kin / 2, col0 = ch * ncol;
        const int o0 = 128 * half + 32 * q;
        float* out = g.part + ((long long)mem * g.splits + split) * 256 * g.kin;
        if (n == 0) {  // an empty split (more splits than chunks) contributes zeros
            for (int c = col0; c < col0 + ncol; ++c) out[(long long)(o0 + lane) * g.kin + c] = 0.0f;
        } else if (tcm::wait_bar(&acc_full, 0, g.status, abort_v)) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            // Every MMA has completed, so the stage ring is free: each warp turns its 32 x 32
            // accumulator blocks around in a padded 32 x 33 tile there, so that every global
            // store writes 128 contiguous bytes of one output row.
            float* tile = reinterpret_cast<float*>(smem) + e * 32 * 33;
            for (int c = col0; c < col0 + ncol; c += 32) {
                float v[32];
                tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
#pragma unroll
                for (int t = 0; t < 32; ++t) tile[lane * 33 + t] = v[t];
                __syncwarp();
                float* dst = out + (long long)o0 * g.kin + c + lane;
#pragma unroll 8
                for (int rr = 0; rr < 32; ++rr) dst[(long long)rr * g.kin] = tile[rr * 33 + lane];
                __syncwarp();
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(256));
}

}  // namespace tcw
