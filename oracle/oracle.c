/*
 * CPU oracle for static occupancy + instruction-mix cost evaluation and
 * per-kernel top-k selection (Lim, Norris & Malony, "Autotuning GPU Kernels
 * via Static and Predictive Analysis", Section III).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the bench's
 * CPU-baseline leg load this library. The product path never calls it, and
 * it shares no code, header or table with the CUDA implementation: it reads
 * the same input records (descriptor bytes, architecture row, axes) and
 * nothing else.
 *
 * Plain and slow on purpose: every point is evaluated from scratch in
 * canonical order (threads, grid, unroll, carveout; carveout fastest), with
 * int64 occupancy arithmetic, an FP64 cost, an FP32 mirror of the cost in a
 * fixed operation order (so FP32 keys can be compared bit for bit), and a
 * full sort per kernel for the top-k. OpenMP splits work over kernels only.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no fast-math:
 * the FP32 mirror relies on IEEE round-to-nearest for every operation and
 * on no multiply-add contraction other than the explicit fmaf).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_NCLASS 7
enum { C_FP32 = 0, C_FP64, C_INT, C_GLDST, C_SLDST, C_BRANCH, C_SFU };

/* Architecture row (filled by the Python wrapper from the row dict). */
typedef struct {
    int64_t cc, n_sm, warp_size, max_threads_block, max_warps_sm, max_blocks_sm;
    int64_t regs_sm, regs_block_max, regs_thread_max, reg_alloc_unit, reg_alloc_mode,
        warp_alloc_gran;
    int64_t smem_block_max, smem_reserved_block, smem_alloc_unit, n_smem_caps;
    int64_t smem_caps[16];
    double ipc[OR_NCLASS];
    int64_t w_sat, work_scale;
} or_arch;

typedef struct {
    int64_t n_t, n_g, n_u, n_c;
    int64_t t[32], g[16], u[8], c[4];
} or_axes;

/* Occupancy of one (T, R, S, carveout) configuration. */
typedef struct {
    int64_t W_B, G_W, G_R, G_S, B, W, cap, valid;
} or_occ;

/* One kernel, decoded from its 64-byte descriptor record. */
typedef struct {
    double n[OR_NCLASS];
    float n32[OR_NCLASS];
    int64_t r0, s0;
    float d;
    uint64_t mask;
} or_kernel;

static int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
static int64_t round_up(int64_t a, int64_t u) { return ceil_div(a, u) * u; }
static int64_t round_down(int64_t a, int64_t u) { return (a / u) * u; }
static int64_t min2(int64_t a, int64_t b) { return a < b ? a : b; }

static void decode(const unsigned char* rec, or_kernel* k)
{
    int32_t i32;
    memcpy(k->n32, rec, 28);
    for (int c = 0; c < OR_NCLASS; ++c) k->n[c] = (double)k->n32[c];
    memcpy(&i32, rec + 28, 4);
    k->r0 = i32;
    memcpy(&i32, rec + 32, 4);
    k->s0 = i32;
    memcpy(&k->d, rec + 36, 4);
    memcpy(&k->mask, rec + 40, 8);
}

/* Eq. 3: blocks per SM limited by warps, G_W = min(B_mp, floor(W_mp / W_B)). */
static int64_t occ_G_W(const or_arch* a, int64_t W_B)
{
    return min2(a->max_blocks_sm, a->max_warps_sm / W_B);
}

/*
 * Eq. 4: blocks per SM limited by registers.
 * Case 1: R above the per-thread maximum -> 0. Case 3: R not given -> B_mp.
 * Case 2 (the printed product of ceilings is not dimensionally consistent;
 * read as the occupancy-calculator form with floors): per-warp allocation
 * rounds R*warp up to the allocation unit, the register file holds
 * floor(regs_sm / that) warps, rounded down to the warp allocation
 * granularity, shared by blocks of W_B warps; per-block allocation rounds
 * R*warp*W_B up to the unit. A block larger than the per-block register
 * maximum cannot launch (0).
 */
static int64_t occ_G_R(const or_arch* a, int64_t R, int64_t W_B)
{
    if (R > a->regs_thread_max) return 0;
    if (R <= 0) return a->max_blocks_sm;
    if (a->reg_alloc_mode == 0) {
        int64_t regs_per_warp = round_up(R * a->warp_size, a->reg_alloc_unit);
        if (regs_per_warp * W_B > a->regs_block_max) return 0;
        int64_t warps = round_down(a->regs_sm / regs_per_warp, a->warp_alloc_gran);
        return warps / W_B;
    } else {
        int64_t regs_per_block = round_up(R * a->warp_size * W_B, a->reg_alloc_unit);
        if (regs_per_block > a->regs_block_max) return 0;
        return a->regs_sm / regs_per_block;
    }
}

/*
 * Eq. 5: blocks per SM limited by shared memory.
 * Case 1: S above the per-block maximum -> 0. Case 3: no shared memory at
 * all (S plus the per-block reservation is 0) -> B_mp. Case 2 (the printed
 * ceiling is read as a floor; a ceiling would admit a block that does not
 * fit): per-block allocation = S + reserved, rounded up to the allocation
 * unit; the per-SM capacity is the smallest supported capacity that is at
 * least carveout% of the largest one and at least one block's allocation.
 */
static int64_t occ_G_S(const or_arch* a, int64_t S, int64_t carveout, int64_t* cap_out)
{
    *cap_out = 0;
    if (S > a->smem_block_max) return 0;
    int64_t S_alloc = round_up(S + a->smem_reserved_block, a->smem_alloc_unit);
    int64_t max_cap = a->smem_caps[a->n_smem_caps - 1];
    int64_t cap = -1;
    for (int64_t i = 0; i < a->n_smem_caps; ++i) {
        int64_t ci = a->smem_caps[i];
        if (100 * ci >= carveout * max_cap && ci >= S_alloc) {
            cap = ci;
            break;
        }
    }
    if (S_alloc == 0) {
        *cap_out = cap;
        return a->max_blocks_sm;
    }
    if (cap < 0) return 0;
    *cap_out = cap;
    return cap / S_alloc;
}

/* Eqs. 1-2: B* = min over the three limits; W* = B* x W_B; valid if B* >= 1. */
int or_occupancy(const or_arch* a, int64_t T, int64_t R, int64_t S, int64_t carveout, or_occ* o)
{
    memset(o, 0, sizeof(*o));
    if (T <= 0) return -1;
    o->W_B = ceil_div(T, a->warp_size);
    o->G_W = occ_G_W(a, o->W_B);
    o->G_R = occ_G_R(a, R, o->W_B);
    o->G_S = occ_G_S(a, S, carveout, &o->cap);
    int64_t B = min2(o->G_W, min2(o->G_R, o->G_S));
    if (T > a->max_threads_block) B = 0;
    o->B = B;
    o->W = B * o->W_B;
    o->valid = B >= 1;
    return 0;
}

/* Registers per thread at unroll U: r0 plus 4 per extra unroll step. */
static int64_t regs_at(int64_t r0, int64_t U) { return r0 + 4 * (U - 1); }

/*
 * Eq. 6 in FP64, with the launch-configuration terms of this library's
 * model: per-class cycles C_c = (1+d) * K * n'_c / IPC_c (n'_BRANCH =
 * n_BRANCH / U, the loop branch amortised by unrolling; c_x = 1/IPC as in
 * Eq. 6), non-memory and memory sums, then
 *   cost = (C_nm + C_m * hide) * lane / par,
 *   hide = max(1, W_sat / W*), lane = warp * W_B / T,
 *   par  = n_SM * G / (waves * slots), slots = n_SM * B*, waves = ceil(G / slots).
 */
double or_cost64(const or_arch* a, const double n[OR_NCLASS], double d, int64_t U, int64_t T,
                 int64_t G, int64_t B, int64_t W)
{
    double delta = 1.0 + d;
    double K = (double)a->work_scale;
    double C[OR_NCLASS];
    for (int c = 0; c < OR_NCLASS; ++c) {
        double nc = (c == C_BRANCH) ? n[c] / (double)U : n[c];
        C[c] = delta * K * nc / a->ipc[c];
    }
    double C_nm = C[C_FP32] + C[C_FP64] + C[C_INT] + C[C_BRANCH] + C[C_SFU];
    double C_m = C[C_GLDST] + C[C_SLDST];
    int64_t W_B = ceil_div(T, a->warp_size);
    int64_t slots = a->n_sm * B;
    int64_t waves = ceil_div(G, slots);
    double par = (double)(a->n_sm * G) / (double)(waves * slots);
    double hide = (double)a->w_sat / (double)W;
    if (hide < 1.0) hide = 1.0;
    double lane = (double)(a->warp_size * W_B) / (double)T;
    return (C_nm + C_m * hide) * lane / par;
}

/* Compensated (Neumaier) FP32 sum, terms in the given order. */
static float neumaier32(const float* x, int m)
{
    float s = 0.0f, comp = 0.0f;
    for (int i = 0; i < m; ++i) {
        float t = s + x[i];
        if (fabsf(s) >= fabsf(x[i]))
            comp += (s - t) + x[i];
        else
            comp += (x[i] - t) + s;
        s = t;
    }
    return s + comp;
}

/*
 * The same cost in FP32, every operation rounded to nearest in this order:
 *   rcp_c = 1 / IPC_c;  v_c = n'_c * rcp_c  (n'_BRANCH = n_BRANCH / U)
 *   S_nm = Neumaier(v_FP32, v_FP64, v_INT, v_BRANCH, v_SFU); S_m = Neumaier(v_GLDST, v_SLDST)
 *   dk = (1 + d) * K;  C_nm = S_nm * dk;  C_m = S_m * dk
 *   hide = max(1, W_sat / W*);  lane = (warp * W_B) / T
 *   X = fma(C_m, hide, C_nm) * lane;  ipar = (waves * slots) / (n_SM * G)
 *   cost32 = X * ipar
 */
float or_cost32(const or_arch* a, const float n[OR_NCLASS], float d, int64_t U, int64_t T, int64_t G,
                int64_t B, int64_t W)
{
    float v[OR_NCLASS];
    for (int c = 0; c < OR_NCLASS; ++c) {
        float rcp = 1.0f / (float)a->ipc[c];
        float nc = (c == C_BRANCH) ? n[c] / (float)U : n[c];
        v[c] = nc * rcp;
    }
    float nm[5] = {v[C_FP32], v[C_FP64], v[C_INT], v[C_BRANCH], v[C_SFU]};
    float mm[2] = {v[C_GLDST], v[C_SLDST]};
    float S_nm = neumaier32(nm, 5);
    float S_m = neumaier32(mm, 2);
    float dk = (1.0f + d) * (float)a->work_scale;
    float C_nm = S_nm * dk;
    float C_m = S_m * dk;
    float hide = (float)a->w_sat / (float)W;
    if (!(hide > 1.0f)) hide = 1.0f;
    int64_t W_B = ceil_div(T, a->warp_size);
    float lane = (float)(a->warp_size * W_B) / (float)T;
    float X = fmaf(C_m, hide, C_nm) * lane;
    int64_t slots = a->n_sm * B;
    int64_t waves = ceil_div(G, slots);
    float ipar = (float)(waves * slots) / (float)(a->n_sm * G);
    return X * ipar;
}

/* Positions of the set bits of an axis field, ascending. */
static int64_t set_positions(uint64_t mask, int shift, int width, int64_t n_axis, int64_t* pos)
{
    int64_t m = 0;
    for (int b = 0; b < width; ++b) {
        if ((mask >> (shift + b)) & 1u) {
            if (b >= n_axis) return -1;
            pos[m++] = b;
        }
    }
    return m;
}

typedef struct {
    float key;
    int32_t idx;
} or_pair;

static int cmp_pair(const void* pa, const void* pb)
{
    const or_pair* a = (const or_pair*)pa;
    const or_pair* b = (const or_pair*)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

/*
 * Field ranges of a well-formed descriptor (the library's record format): every
 * instruction count a number in [0, 2^40], the divergence fraction d in [0, 1],
 * r0 in [0, 2^24), s0 in [0, 2^30). With these bounds no cost of a valid point
 * can overflow; a descriptor outside them is malformed and gets no points.
 */
static int fields_ok(const or_kernel* k)
{
    for (int c = 0; c < OR_NCLASS; ++c)
        if (!(k->n32[c] >= 0.0f && k->n32[c] <= 1099511627776.0f)) return 0; /* 2^40; false for NaN */
    if (!(k->d >= 0.0f && k->d <= 1.0f)) return 0;
    return k->r0 >= 0 && k->r0 < (1 << 24) && k->s0 >= 0 && k->s0 < (1 << 30);
}

/* Space size of one descriptor, or -1 if its mask selects values beyond the axes. */
int64_t or_space_size(const or_axes* ax, const void* rec)
{
    or_kernel k;
    int64_t p[32];
    decode((const unsigned char*)rec, &k);
    if (k.mask >> 60) return -1;
    int64_t nt = set_positions(k.mask, 0, 32, ax->n_t, p);
    int64_t ng = set_positions(k.mask, 32, 16, ax->n_g, p);
    int64_t nu = set_positions(k.mask, 48, 8, ax->n_u, p);
    int64_t nc = set_positions(k.mask, 56, 4, ax->n_c, p);
    if (nt < 0 || ng < 0 || nu < 0 || nc < 0) return -1;
    return nt * ng * nu * nc;
}

/*
 * Evaluate every point of every kernel's space and select each kernel's
 * k best (lowest FP32 cost; equal costs -> lower canonical index; fewer
 * than k valid points -> pad with index -1, cost +inf).
 * Optional per-point outputs (any may be NULL) are written at
 * pt_off[kernel] + canonical index.
 * A malformed descriptor (mask outside the axes, or a field outside the
 * ranges of fields_ok) gets padding only and no per-point outputs.
 * Returns 0, or -1 if any descriptor was malformed.
 */
int or_eval(const or_arch* a, const or_axes* ax, const void* descs, int64_t n_kernels, int64_t k,
            int32_t* topk_idx, float* topk_cost, int32_t* pt_B, int32_t* pt_W, float* pt_c32,
            double* pt_c64, const int64_t* pt_off, int nthreads)
{
    int err = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        or_pair* buf = (or_pair*)malloc(sizeof(or_pair) * 16384);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 8)
#endif
        for (int64_t i = 0; i < n_kernels; ++i) {
            or_kernel kd;
            decode((const unsigned char*)descs + 64 * i, &kd);
            int64_t tp[32], gp[16], up[8], cp[4];
            int64_t nt = set_positions(kd.mask, 0, 32, ax->n_t, tp);
            int64_t ng = set_positions(kd.mask, 32, 16, ax->n_g, gp);
            int64_t nu = set_positions(kd.mask, 48, 8, ax->n_u, up);
            int64_t nc = set_positions(kd.mask, 56, 4, ax->n_c, cp);
            if ((kd.mask >> 60) || nt < 0 || ng < 0 || nu < 0 || nc < 0 || !fields_ok(&kd)) {
                err = -1;
                for (int64_t r = 0; r < k; ++r) {
                    topk_idx[i * k + r] = -1;
                    topk_cost[i * k + r] = INFINITY;
                }
                continue;
            }
            int64_t nvalid = 0, idx = 0;
            for (int64_t it = 0; it < nt; ++it)
                for (int64_t ig = 0; ig < ng; ++ig)
                    for (int64_t iu = 0; iu < nu; ++iu)
                        for (int64_t ic = 0; ic < nc; ++ic, ++idx) {
                            int64_t T = ax->t[tp[it]], G = ax->g[gp[ig]];
                            int64_t U = ax->u[up[iu]], C = ax->c[cp[ic]];
                            or_occ o;
                            or_occupancy(a, T, regs_at(kd.r0, U), kd.s0, C, &o);
                            float c32 = INFINITY;
                            double c64 = INFINITY;
                            if (o.valid) {
                                c64 = or_cost64(a, kd.n, (double)kd.d, U, T, G, o.B, o.W);
                                c32 = or_cost32(a, kd.n32, kd.d, U, T, G, o.B, o.W);
                                buf[nvalid].key = c32;
                                buf[nvalid].idx = (int32_t)idx;
                                ++nvalid;
                            }
                            if (pt_off) {
                                int64_t at = pt_off[i] + idx;
                                if (pt_B) pt_B[at] = (int32_t)o.B;
                                if (pt_W) pt_W[at] = (int32_t)o.W;
                                if (pt_c32) pt_c32[at] = c32;
                                if (pt_c64) pt_c64[at] = c64;
                            }
                        }
            qsort(buf, (size_t)nvalid, sizeof(or_pair), cmp_pair);
            for (int64_t r = 0; r < k; ++r) {
                if (r < nvalid) {
                    topk_idx[i * k + r] = buf[r].idx;
                    topk_cost[i * k + r] = buf[r].key;
                } else {
                    topk_idx[i * k + r] = -1;
                    topk_cost[i * k + r] = INFINITY;
                }
            }
        }
        free(buf);
    }
    return err;
}

/*
 * Segmented top-k over an external score array: for each segment
 * [off[s], off[s+1]), the k smallest finite scores, ties -> lower index
 * within the segment; +inf and NaN scores are not candidates; pad with
 * (-1, +inf).
 */
int or_topk(const float* scores, const int64_t* off, int64_t n_seg, int64_t k, int32_t* topk_idx,
            float* topk_val, int nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthreads)
#endif
    for (int64_t s = 0; s < n_seg; ++s) {
        int64_t len = off[s + 1] - off[s];
        or_pair* buf = (or_pair*)malloc(sizeof(or_pair) * (size_t)(len > 0 ? len : 1));
        int64_t m = 0;
        for (int64_t j = 0; j < len; ++j) {
            float v = scores[off[s] + j];
            if (v < INFINITY) { /* false for +inf and NaN */
                buf[m].key = v;
                buf[m].idx = (int32_t)j;
                ++m;
            }
        }
        qsort(buf, (size_t)m, sizeof(or_pair), cmp_pair);
        for (int64_t r = 0; r < k; ++r) {
            topk_idx[s * k + r] = r < m ? buf[r].idx : -1;
            topk_val[s * k + r] = r < m ? buf[r].key : INFINITY;
        }
        free(buf);
    }
    return 0;
}

/* Round to bfloat16 through float32 (round to nearest, ties to even), as a double. */
static double bf16_round(double x)
{
    float f = (float)x;
    uint32_t b;
    memcpy(&b, &f, 4);
    b = (b + 0x7fffu + ((b >> 16) & 1u)) & 0xffff0000u;
    memcpy(&f, &b, 4);
    return (double)f;
}

/*
 * The surrogate's 48 input features of one point (T, G, U, C) of a kernel,
 * in FP64: fixed scalings of the descriptor, the launch parameters and the
 * occupancy and cost terms above (list in the library's features header).
 */
int or_features(const or_arch* a, const void* rec, int64_t T, int64_t G, int64_t U, int64_t C, double* f)
{
    or_kernel k;
    decode((const unsigned char*)rec, &k);
    double tot = 0.0;
    for (int c = 0; c < OR_NCLASS; ++c) tot += k.n[c];
    for (int c = 0; c < OR_NCLASS; ++c) {
        f[c] = log2(k.n[c] + 1.0) / 20.0;
        f[7 + c] = k.n[c] / (tot + 1.0);
    }
    f[14] = log2((k.n[C_FP32] + k.n[C_FP64] + 1.0) / (k.n[C_GLDST] + k.n[C_SLDST] + 1.0)) / 10.0;
    f[15] = (double)k.r0 / 255.0;
    f[16] = (double)k.s0 / 65536.0;
    f[17] = (double)k.d;
    int64_t R = regs_at(k.r0, U);
    or_occ o;
    or_occupancy(a, T, R, k.s0, C, &o);
    int64_t rpw = 0;
    if (a->reg_alloc_mode == 0 && R > 0 && R <= a->regs_thread_max) rpw = round_up(R * a->warp_size, a->reg_alloc_unit);
    int64_t s_alloc = 0;
    if (k.s0 <= a->smem_block_max) s_alloc = round_up(k.s0 + a->smem_reserved_block, a->smem_alloc_unit);
    f[18] = log2((double)T) / 10.0;
    f[19] = (double)o.W_B / 32.0;
    f[20] = (double)(a->warp_size * o.W_B) / (double)T;
    f[21] = log2((double)G) / 16.0;
    f[22] = (double)U / 8.0;
    f[23] = (double)C / 100.0;
    f[24] = (double)R / 255.0;
    f[25] = (double)rpw / 8192.0;
    f[26] = (double)min2(o.G_W, 64) / 32.0;
    f[27] = (double)min2(o.G_R, 64) / 32.0;
    f[28] = (double)min2(o.G_S, 64) / 32.0;
    f[29] = (double)o.B / 32.0;
    f[30] = (double)o.W / 64.0;
    f[31] = (double)o.W / (double)a->max_warps_sm;
    f[32] = (o.B > 0 && o.G_W == o.B) ? 1.0 : 0.0;
    f[33] = (o.B > 0 && o.G_R == o.B) ? 1.0 : 0.0;
    f[34] = (o.B > 0 && o.G_S == o.B) ? 1.0 : 0.0;
    double delta = 1.0 + (double)k.d, K = (double)a->work_scale, Cc[OR_NCLASS];
    for (int c = 0; c < OR_NCLASS; ++c) Cc[c] = delta * K * ((c == C_BRANCH) ? k.n[c] / (double)U : k.n[c]) / a->ipc[c];
    double C_nm = Cc[C_FP32] + Cc[C_FP64] + Cc[C_INT] + Cc[C_BRANCH] + Cc[C_SFU];
    double C_m = Cc[C_GLDST] + Cc[C_SLDST];
    double waves = 0.0, par = 0.0, hide = 0.0, cost = 0.0;
    if (o.valid) {
        int64_t slots = a->n_sm * o.B;
        int64_t wv = ceil_div(G, slots);
        waves = (double)wv;
        par = (double)(a->n_sm * G) / (double)(wv * slots);
        hide = (double)a->w_sat / (double)o.W;
        if (hide < 1.0) hide = 1.0;
        cost = or_cost64(a, k.n, (double)k.d, U, T, G, o.B, o.W);
    }
    f[35] = waves > 0.0 ? log2(waves) / 10.0 : 0.0;
    f[36] = par / (double)a->n_sm;
    f[37] = hide / 32.0;
    f[38] = log2(cost + 1.0) / 40.0;
    f[39] = log2(C_nm + 1.0) / 40.0;
    f[40] = log2(C_m + 1.0) / 40.0;
    f[41] = log2((double)G * (double)T) / 26.0;
    f[42] = (double)o.cap / 233472.0;
    f[43] = (double)s_alloc / 65536.0;
    f[44] = log2(k.n[C_BRANCH] / (double)U + 1.0) / 20.0;
    /* what BF16 storage of the three cost features drops, scaled by 256 */
    for (int j = 0; j < 3; ++j) f[45 + j] = (f[38 + j] - bf16_round(f[38 + j])) * 256.0;
    return 0;
}
