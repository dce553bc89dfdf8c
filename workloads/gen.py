"""Seeded synthetic inputs: kernel descriptors and tuning-space masks.

Pure input generation. Nothing here evaluates occupancy or cost; the CUDA
path and the CPU oracle both take these arrays as inputs.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used counter-style: draw j of
kernel i is the SplitMix64 output for state  key + (64*i + j + 1) * GAMMA,
with key = mix64(seed). Any kernel's draws can therefore be produced alone,
which is how bounded samples of a large workload are taken.

Descriptor record (64 bytes, little endian), the input format of both sides:

    offset  type        field
    0       float32[7]  n[c]: static instruction counts per class
                        (FP32, FP64, INT, GLDST, SLDST, BRANCH, SFU)
    28      int32       r0: registers per thread at unroll 1
    32      int32       s0: shared memory bytes per block
    36      float32     d: branch-divergence fraction
    40      uint64      space_mask: which axis values belong to the space
    48      int32[4]    reserved, zero

Space mask bits: bits 0..31 select threads-per-block values t[0..31],
bits 32..47 grid sizes g[0..15], bits 48..55 unroll factors u[0..7],
bits 56..59 carveout percentages c[0..3]; bits 60..63 are zero.

Workloads (the tuning axes follow the Orio PerfTuning specification of the
paper's Fig. "Performance tuning specification": thread counts 32..1024 step
32, unroll factors, an L1/shared split; grid sizes are powers of two):

* "dense128"  : every kernel's space = 32 thread counts x unroll {1,2,4,8},
                grid 1024, carveout 100 %  (128 points).
* "dense"     : every kernel's space = all 32 x 16 x 8 x 4 = 16384 points.
* "uneven"    : per-kernel size drawn log-uniform in [64, 65536], clamped to
                16384, split over the four axes in proportion to their bit
                widths (5, 4, 3, 2) and filled with random distinct values.
"""

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)
DRAWS_PER_KERNEL = 64

DESC_DTYPE = np.dtype(
    {
        "names": ["n", "r0", "s0", "d", "space_mask", "reserved"],
        "formats": [("<f4", (7,)), "<i4", "<i4", "<f4", "<u8", ("<i4", (4,))],
        "offsets": [0, 28, 32, 36, 40, 48],
        "itemsize": 64,
    }
)

# Tuning axes (values selected by the space-mask bits).
AXES = {
    "t": [32 * (i + 1) for i in range(32)],          # threads per block
    "g": [1 << j for j in range(16)],                # grid size in blocks
    "u": [u + 1 for u in range(8)],                  # unroll factor
    "c": [0, 25, 50, 100],                           # shared-memory carveout %
}

T_SHIFT, G_SHIFT, U_SHIFT, C_SHIFT = 0, 32, 48, 56
T_BITS, G_BITS, U_BITS, C_BITS = 32, 16, 8, 4


def axes():
    """The default tuning axes as a dict of lists."""
    return {k: list(v) for k, v in AXES.items()}


def _mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
    return z ^ (z >> np.uint64(31))


def draws(seed, kernel_ids, j):
    """Draw number j (0..63) for each kernel in kernel_ids, as uint64."""
    key = _mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF))
    ids = np.asarray(kernel_ids, dtype=np.uint64)
    with np.errstate(over="ignore"):
        ctr = ids * np.uint64(DRAWS_PER_KERNEL) + np.uint64(j + 1)
        state = key + ctr * GAMMA
    return _mix64(state)


def _uint_below(x, n):
    """Map uint64 draws to integers in [0, n) by multiply-shift on the top 32 bits."""
    hi = (x >> np.uint64(32)).astype(np.uint64)
    return ((hi * np.uint64(n)) >> np.uint64(32)).astype(np.int64)


def _unit53(x):
    """Map uint64 draws to doubles in [0, 1) with 53 random bits."""
    return (x >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _unit24(x):
    """Map uint64 draws to float32-exact values in [0, 1) with 24 random bits."""
    return ((x >> np.uint64(40)).astype(np.float64) * (1.0 / 16777216.0))


def mask_bits(t_idx=(), g_idx=(), u_idx=(), c_idx=()):
    """Build one space mask from lists of axis positions."""
    m = 0
    for i in t_idx:
        m |= 1 << (T_SHIFT + i)
    for i in g_idx:
        m |= 1 << (G_SHIFT + i)
    for i in u_idx:
        m |= 1 << (U_SHIFT + i)
    for i in c_idx:
        m |= 1 << (C_SHIFT + i)
    return m


MASK_DENSE = mask_bits(range(32), range(16), range(8), range(4))
MASK_DENSE128 = mask_bits(range(32), [10], [0, 1, 3, 7], [3])


def _uneven_masks(seed, ids):
    """Per-kernel random subsets of the four axes (sizes log-uniform 64..65536, clamped)."""
    n = len(ids)
    lo, hi = np.log2(64.0), np.log2(65536.0)
    log_s = lo + (hi - lo) * _unit53(draws(seed, ids, 10))
    log_s = np.minimum(log_s, 14.0)
    masks = np.zeros(n, dtype=np.uint64)
    caps = [(T_SHIFT, T_BITS, 5), (G_SHIFT, G_BITS, 4), (U_SHIFT, U_BITS, 3), (C_SHIFT, C_BITS, 2)]
    j = 11
    for shift, width, bits in caps:
        size = np.rint(np.exp2(log_s * bits / 14.0)).astype(np.int64)
        size = np.clip(size, 1, width)
        # Partial Fisher-Yates over the axis positions, one draw per swap.
        perm = np.tile(np.arange(width, dtype=np.int64), (n, 1))
        rows = np.arange(n)
        for s in range(width):
            r = _uint_below(draws(seed, ids, j + s), width - s) + s
            a = perm[rows, s].copy()
            perm[rows, s] = perm[rows, r]
            perm[rows, r] = a
        j += width
        take = np.arange(width)[None, :] < size[:, None]
        bit = np.left_shift(np.uint64(1), (perm + shift).astype(np.uint64))
        masks |= np.bitwise_or.reduce(np.where(take, bit, np.uint64(0)), axis=1)
    return masks


def descriptors(n_kernels, seed, space="dense", first=0):
    """Generate kernel descriptors first .. first+n_kernels-1 of a seeded workload.

    Counts are log-uniform in [1e2, 1e6] and rounded to integers (exact in
    float32); r0 is uniform in [16, 96]; s0 uniform in [0, 49152] bytes; d is
    uniform in [0, 0.5) with 24 random bits (exact in float32).
    """
    ids = np.arange(first, first + n_kernels, dtype=np.uint64)
    out = np.zeros(n_kernels, dtype=DESC_DTYPE)
    lo, hi = np.log(1e2), np.log(1e6)
    for c in range(7):
        u = _unit53(draws(seed, ids, c))
        out["n"][:, c] = np.rint(np.exp(lo + (hi - lo) * u)).astype(np.float32)
    out["r0"] = 16 + _uint_below(draws(seed, ids, 7), 81)
    out["s0"] = _uint_below(draws(seed, ids, 8), 49153)
    out["d"] = (0.5 * _unit24(draws(seed, ids, 9))).astype(np.float32)
    if space == "dense":
        out["space_mask"] = np.uint64(MASK_DENSE)
    elif space == "dense128":
        out["space_mask"] = np.uint64(MASK_DENSE128)
    elif space == "uneven":
        out["space_mask"] = _uneven_masks(seed, ids)
    else:
        raise ValueError(f"unknown space {space!r}")
    return out


def space_sizes(descs):
    """Number of points in each descriptor's space (product of per-axis popcounts)."""
    m = np.asarray(descs["space_mask"], dtype=np.uint64)

    def pop(shift, width):
        v = (m >> np.uint64(shift)) & np.uint64((1 << width) - 1)
        c = np.zeros(len(m), dtype=np.int64)
        for b in range(width):
            c += ((v >> np.uint64(b)) & np.uint64(1)).astype(np.int64)
        return c

    return pop(T_SHIFT, T_BITS) * pop(G_SHIFT, G_BITS) * pop(U_SHIFT, U_BITS) * pop(C_SHIFT, C_BITS)


def point_offsets(descs):
    """Exclusive prefix sum of space sizes (int64, length n+1)."""
    sizes = space_sizes(descs)
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    return off


def scores(n, seed, lo=1.0, hi=1e6):
    """Synthetic positive float32 scores, log-uniform in [lo, hi] (24 random bits each)."""
    ids = np.arange(n, dtype=np.uint64)
    u = _unit24(draws(seed, ids, 0))
    return np.exp(np.log(lo) + (np.log(hi) - np.log(lo)) * u).astype(np.float32)
