// Weight and bias gradients of surrogate training on tcgen05, every layer in one launch:
//   dW_l[o][i] = sum over batch rows r of dZ_l[r][o] * Hprev_l[r][i],   db_l[o] = sum over r of dZ_l[r][o]
// (Hprev = the layer's input: the previous layer's activations, or the feature rows).
//
// Output-stationary: CTA (t, m) owns one 128 x 64 tile of member m's weight gradients
// (output rows o in [128 h, 128 h + 128) and input columns [64 c, 64 c + 64) of one layer)
// and runs the whole batch through one TMEM accumulator, so every gradient element is one
// MMA accumulation chain over the batch, written once, with no partial sums in memory.
// Tile t enumerates the layers in the order of Args::kin, each as (o half, column block);
// a member has 2 (64 / 64 + 3 x 256 / 64) = 26 tiles, all of the same cost.
//
// The contraction runs over the batch, the index along which neither operand is
// contiguous, so both operands are fed to the MMA MN-major: TMA copies boxes of
// 128 rows x 64 BF16 columns with 128-byte swizzle, which is the MN-major swizzle atom
// (8 rows of K by 64 elements of M or N, 1 KB) repeated 16 times along K (1 KB apart)
// and, box by box, along M (16 KB apart). A stage holds 128 batch rows: two dZ boxes
// (the tile's 128 output columns) and one Hprev box (its 64 input columns). The stages
// are that deep because the MMA issuer's fixed cost per stage (barrier wait, fences,
// commit: about 0.2 us) outweighed the eight 128 x 64 x 16 products of a 64-row stage.
//
// The bias gradient of the tiles with c = 0 comes from the same MMAs: their B operand is
// 80 columns wide, the tile's 64 Hprev columns and 16 columns of a constant all-ones
// block (a second MN atom, which the descriptor's leading byte offset points at), so
// accumulator columns 64-79 each hold sum over r of dZ[r][o].
//
// Roles (192 threads): warp 0 issues the TMA copies through a ring of four 48 KB
// stages, warp 1 issues the MMAs, warps 2-5 read the accumulator back (thread = output
// row, one warp per TMEM lane quarter) and store the gradient rows.
//
// Every wait is bounded; on timeout the kernel sets status bit 2, stops issuing work,
// waits (bounded) for the copies and MMAs it issued, frees its tensor memory and returns.
#pragma once

#include "tc_mlp.cuh"

namespace tcw {

constexpr int kChunkRows = 128;                // batch rows (K) per stage
constexpr int kBox = kChunkRows * 128;         // one TMA box: 128 rows x 64 BF16 columns
constexpr int kStageA = 2 * kBox;              // dZ: the tile's 128 output columns
constexpr int kStage = kStageA + kBox;         // and Hprev: its 64 input columns
constexpr int kStages = 4;
constexpr int kEpiWarps = 4;
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr int kOnes = kBox;                    // all-ones MN atom: 128 K rows x 64 BF16
constexpr int kSmem = 1024 + kStages * kStage + kOnes;
constexpr int kTileCols = 64;                  // input columns of a tile
constexpr int kBiasCols = 16;                  // accumulator columns of the bias sums
constexpr int kMaxItems = 4;                   // layers of one launch
constexpr int kTmemCols = 128;                 // the tile's accumulator and the bias columns
static_assert(kSmem <= 227 * 1024 - 256, "shared memory");

struct Args {
    int n_items;                     // layers of this launch
    int kin[kMaxItems];              // input columns of item j's layer: 64 or 256
    int b_batched[kMaxItems];        // Hprev has a member coordinate (0: one input for all members)
    long long grad_w[kMaxItems];     // offsets of dW and db of item j's layer in a member's gradient
    long long grad_b[kMaxItems];
    long long grad_stride;           // floats per member in grad
    int chunks;                      // batch rows / 128
    float* grad;
    int* status;
};

// ta[j]: item j's dZ as 8-byte elements {64, rows, members}, box {16, 128, 1};
// tb[j]: its Hprev as 8-byte elements {kin / 4, rows, members or 1}, box {16, 128, 1}.
struct Maps {
    CUtensorMap ta[kMaxItems];
    CUtensorMap tb[kMaxItems];
};

// Tiles of one member for the layers of `g` (2 x kin / 64 per layer).
__host__ __device__ inline int tiles_per_member(const Args& g)
{
    int t = 0;
    for (int j = 0; j < g.n_items; ++j) t += 2 * (g.kin[j] / kTileCols);
    return t;
}

// MN-major operand, 128-byte swizzle: leading byte offset = distance between atoms
// adjacent in M or N (one box, 16 KB), stride byte offset = distance between atoms
// adjacent in K (8 rows of 128 bytes).
__device__ __forceinline__ uint64_t sdesc_mn(const void* p, uint32_t lbo = kBox)
{
    const uint64_t addr = tc::sa(p);
    return ((addr >> 4) & 0x3fffull) | ((uint64_t)((lbo >> 4) & 0x3fffu) << 16) | ((1024ull >> 4) << 32) |
           (1ull << 46) | (2ull << 61);
}

// kind::f16 instruction descriptor with A and B MN-major.
__host__ __device__ constexpr uint32_t idesc_bf16_mn(int M, int N)
{
    return tc::idesc_bf16(M, N) | (1u << 15) | (1u << 16);
}

// grid: (tiles_per_member(g), members), one CTA per tile.
__global__ void __launch_bounds__(kThreads, 1) wgrad_kernel(const __grid_constant__ Maps maps,
                                                            const __grid_constant__ Args g)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full[kStages], empty[kStages], acc_full, drain;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* ones = smem + kStages * kStage;  // 1 KB aligned, after every stage
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mem = blockIdx.y;
    pdl::grid_dep_enter();  // launched after the input-gradient chain in a training step
    // tile -> (layer item j, output half, input column block)
    int j = 0, tt = blockIdx.x;
    while (j < g.n_items && tt >= 2 * (g.kin[j] / kTileCols)) {
        tt -= 2 * (g.kin[j] / kTileCols);
        ++j;
    }
    if (j >= g.n_items) return;  // past the last tile (the whole CTA leaves before any barrier)
    const int kin = g.kin[j], nb = kin / kTileCols;
    const int half = tt / nb, cb = tt - (tt / nb) * nb;
    const bool bias = cb == 0;  // this tile also forms the bias gradient of its 128 rows
    const int n = g.chunks;
    volatile int* abort_v = &abort_flag;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tc::sa(&tmem_base)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (threadIdx.x == 32) {
        for (int i = 0; i < kStages; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        tc::mbar_init(&acc_full, 1);
        tc::mbar_init(&drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        abort_flag = 0;
    }
    // the all-ones block (BF16 1.0 = 0x3f80), made visible to the tensor cores' proxy
    for (int i = threadIdx.x; i < kOnes / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(ones)[i] = 0x3f803f80u;
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        // ---- producer ----
        if (lane == 0 && n > 0) {
            int i = 0;
            bool ok = true;
            for (; i < n; ++i) {
                const int st = i % kStages, use = i / kStages;
                if (use > 0 && !(ok = tcm::wait_bar(&empty[st], (uint32_t)((use - 1) & 1), g.status, abort_v))) break;
                uint8_t* a = smem + st * kStage;
                const int r0 = i * kChunkRows;
                tc::mbar_expect_tx(&full[st], (uint32_t)kStage);
                for (int q = 0; q < 2; ++q)
                    tc::tma_load_3d(a + q * kBox, &maps.ta[j], (2 * half + q) * 16, r0, mem, &full[st]);
                tc::tma_load_3d(a + kStageA, &maps.tb[j], cb * 16, r0, g.b_batched[j] ? mem : 0, &full[st]);
            }
            if (!ok)  // let the copies in flight land before the CTA exits
                for (int q = i - kStages; q < i; ++q)
                    if (q >= 0) tc::mbar_wait(&full[q % kStages], (uint32_t)((q / kStages) & 1), g.status);
        }
    } else if (warp == 1) {
        // ---- MMA issuer ----
        if (lane == 0 && n > 0) {
            // bias tiles: N = 64 Hprev columns + 16 all-ones columns (the atom at ones)
            const uint32_t idesc = idesc_bf16_mn(128, bias ? kTileCols + kBiasCols : kTileCols);
            bool ok = true;
            for (int i = 0; i < n && ok; ++i) {
                const int st = i % kStages;
                if (!(ok = tcm::wait_bar(&full[st], (uint32_t)((i / kStages) & 1), g.status, abort_v))) break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint8_t* a = smem + st * kStage;
#pragma unroll
                for (int kk = 0; kk < kChunkRows / 16; ++kk)  // 16 batch rows = two K atoms per step
                    tc::mma_bf16(tmem, sdesc_mn(a + kk * 2048),
                                 sdesc_mn(a + kStageA + kk * 2048, (uint32_t)(ones - (a + kStageA))), idesc, (i | kk) != 0);
                tc::mma_commit(&empty[st]);
            }
            if (ok) tc::mma_commit(&acc_full);
            tc::mma_commit(&drain);  // arrives when every MMA issued above has completed
            tc::mbar_wait(&drain, 0, g.status);
        }
    } else {
        // ---- epilogue warps ----
        // the tile: thread = output row o (warp % 4 = its TMEM lane quarter)
        const int q = warp & 3;
        const int o = 128 * half + 32 * q + lane;
        float* grow = g.grad + (long long)mem * g.grad_stride + g.grad_w[j] + (long long)o * kin + cb * kTileCols;
        float* gb = g.grad + (long long)mem * g.grad_stride + g.grad_b[j] + o;
        if (n == 0) {
            for (int c = 0; c < kTileCols; c += 4) *reinterpret_cast<float4*>(grow + c) = make_float4(0.f, 0.f, 0.f, 0.f);
            if (bias) *gb = 0.0f;
        } else if (tcm::wait_bar(&acc_full, 0, g.status, abort_v)) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16);
#pragma unroll
            for (int c0 = 0; c0 < kTileCols; c0 += 32) {
                float v[32];
                tc::tmem_ld32(tb + (uint32_t)c0, v);
#pragma unroll
                for (int c = 0; c < 32; c += 4)
                    *reinterpret_cast<float4*>(grow + c0 + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
            }
            if (bias) {
                float v[16];
                tcm::tmem_ld16(tb + (uint32_t)kTileCols, v);
                *gb = v[0];
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
}

}  // namespace tcw
