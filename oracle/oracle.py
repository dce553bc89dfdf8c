"""ctypes wrapper around the plain C oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
bench's CPU-baseline leg, never by the product package. It shares no code
with the CUDA implementation; both read the same input arrays.
"""

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", "-std=c11"]


def build(force=False):
    """Compile the oracle with gcc (idempotent)."""
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, SRC, "-o", tmp, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class Arch(C.Structure):
    _fields_ = [(f, C.c_int64) for f in (
        "cc", "n_sm", "warp_size", "max_threads_block", "max_warps_sm", "max_blocks_sm",
        "regs_sm", "regs_block_max", "regs_thread_max", "reg_alloc_unit", "reg_alloc_mode",
        "warp_alloc_gran", "smem_block_max", "smem_reserved_block", "smem_alloc_unit",
        "n_smem_caps")] + [("smem_caps", C.c_int64 * 16), ("ipc", C.c_double * 7),
                           ("w_sat", C.c_int64), ("work_scale", C.c_int64)]


class Axes(C.Structure):
    _fields_ = [("n_t", C.c_int64), ("n_g", C.c_int64), ("n_u", C.c_int64), ("n_c", C.c_int64),
                ("t", C.c_int64 * 32), ("g", C.c_int64 * 16), ("u", C.c_int64 * 8),
                ("c", C.c_int64 * 4)]


class Occ(C.Structure):
    _fields_ = [(f, C.c_int64) for f in ("W_B", "G_W", "G_R", "G_S", "B", "W", "cap", "valid")]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER
        L.or_occupancy.argtypes = [P(Arch), C.c_int64, C.c_int64, C.c_int64, C.c_int64, P(Occ)]
        L.or_occupancy.restype = C.c_int
        L.or_cost64.argtypes = [P(Arch), P(C.c_double), C.c_double, C.c_int64, C.c_int64,
                                C.c_int64, C.c_int64, C.c_int64]
        L.or_cost64.restype = C.c_double
        L.or_cost32.argtypes = [P(Arch), P(C.c_float), C.c_float, C.c_int64, C.c_int64,
                                C.c_int64, C.c_int64, C.c_int64]
        L.or_cost32.restype = C.c_float
        L.or_space_size.argtypes = [P(Axes), C.c_void_p]
        L.or_space_size.restype = C.c_int64
        L.or_eval.argtypes = [P(Arch), P(Axes), C.c_void_p, C.c_int64, C.c_int64,
                              C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                              C.c_void_p, C.c_void_p, C.c_int]
        L.or_eval.restype = C.c_int
        L.or_topk.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p,
                              C.c_void_p, C.c_int]
        L.or_topk.restype = C.c_int
        L.or_features.argtypes = [P(Arch), C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int64,
                                  P(C.c_double)]
        L.or_features.restype = C.c_int
        _lib = L
    return _lib


def make_arch(row):
    a = Arch()
    for f, _ in Arch._fields_:
        if f in ("smem_caps", "ipc"):
            continue
        if f == "n_smem_caps":
            a.n_smem_caps = len(row["smem_caps"])
        else:
            setattr(a, f, int(row[f]))
    for i, v in enumerate(row["smem_caps"]):
        a.smem_caps[i] = int(v)
    for i, v in enumerate(row["ipc"]):
        a.ipc[i] = float(v)
    return a


def make_axes(ax):
    a = Axes()
    a.n_t, a.n_g, a.n_u, a.n_c = len(ax["t"]), len(ax["g"]), len(ax["u"]), len(ax["c"])
    for name in ("t", "g", "u", "c"):
        arr = getattr(a, name)
        for i, v in enumerate(ax[name]):
            arr[i] = int(v)
    return a


def _ptr(x):
    return None if x is None else x.ctypes.data


def occupancy(row, T, R, S, carveout=100):
    """Occupancy of one configuration: dict with W_B, G_W, G_R, G_S, B, W, cap, valid."""
    o = Occ()
    a = make_arch(row)
    lib().or_occupancy(C.byref(a), int(T), int(R), int(S), int(carveout), C.byref(o))
    return {f: getattr(o, f) for f, _ in Occ._fields_}


def cost64(row, n, d, U, T, G, B, W):
    a = make_arch(row)
    nn = (C.c_double * 7)(*[float(x) for x in n])
    return lib().or_cost64(C.byref(a), nn, float(d), int(U), int(T), int(G), int(B), int(W))


def cost32(row, n, d, U, T, G, B, W):
    a = make_arch(row)
    nn = (C.c_float * 7)(*[float(x) for x in n])
    return lib().or_cost32(C.byref(a), nn, float(np.float32(d)), int(U), int(T), int(G), int(B),
                           int(W))


def space_size(axes, desc):
    a = make_axes(axes)
    rec = np.ascontiguousarray(np.asarray(desc).reshape(1))
    return lib().or_space_size(C.byref(a), rec.ctypes.data)


def evaluate(row, axes, descs, k, emit=False, offsets=None, nthreads=0, strict=True):
    """Evaluate all points and select each kernel's top-k.

    Returns dict(idx=int32[n,k], cost=float32[n,k]) and, with emit=True,
    per-point arrays B, W (int32), cost32 (float32), cost64 (float64) laid
    out at offsets[kernel] + canonical index (offsets: int64[n+1]).
    Malformed descriptors (mask outside the axes, counts outside [0, 2^40],
    d outside [0, 1], r0 or s0 out of range) get padding; with strict=True
    they raise ValueError, otherwise out["malformed"] is True.
    """
    descs = np.ascontiguousarray(descs)
    n = len(descs)
    idx = np.empty((n, k), dtype=np.int32)
    cost = np.empty((n, k), dtype=np.float32)
    out = {"idx": idx, "cost": cost}
    pB = pW = p32 = p64 = None
    if emit:
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        total = int(offsets[-1])
        pB = np.empty(total, dtype=np.int32)
        pW = np.empty(total, dtype=np.int32)
        p32 = np.empty(total, dtype=np.float32)
        p64 = np.empty(total, dtype=np.float64)
        out.update(B=pB, W=pW, cost32=p32, cost64=p64)
    a = make_arch(row)
    ax = make_axes(axes)
    rc = lib().or_eval(C.byref(a), C.byref(ax), descs.ctypes.data, n, int(k), idx.ctypes.data,
                       cost.ctypes.data, _ptr(pB), _ptr(pW), _ptr(p32), _ptr(p64),
                       _ptr(offsets) if emit else None, int(nthreads))
    if rc != 0 and strict:
        raise ValueError("oracle: malformed descriptor (mask outside the axes or a field out of range)")
    out["malformed"] = rc != 0
    return out


def topk(scores, offsets, k, nthreads=0):
    """Segmented top-k (smallest finite scores, ties -> lower index)."""
    scores = np.ascontiguousarray(scores, dtype=np.float32)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    n_seg = len(offsets) - 1
    idx = np.empty((n_seg, k), dtype=np.int32)
    val = np.empty((n_seg, k), dtype=np.float32)
    lib().or_topk(scores.ctypes.data, offsets.ctypes.data, n_seg, int(k), idx.ctypes.data,
                  val.ctypes.data, int(nthreads))
    return {"idx": idx, "cost": val}


def features(row, desc, T, G, U, carveout):
    """The surrogate's 48 features of one point, FP64 (numpy array)."""
    import numpy as np

    a = make_arch(row)
    rec = np.ascontiguousarray(np.asarray(desc).reshape(1))
    out = (C.c_double * 48)()
    lib().or_features(C.byref(a), rec.ctypes.data, int(T), int(G), int(U), int(carveout), out)
    return np.array(out[:], dtype=np.float64)


def decode_point(desc, axes, i):
    """Canonical index -> (T, G, U, carveout) of a descriptor's space (carveout fastest)."""
    m = int(desc["space_mask"])
    pos = lambda sh, w: [b for b in range(w) if (m >> (sh + b)) & 1]
    tp, gp, up, cp = pos(0, 32), pos(32, 16), pos(48, 8), pos(56, 4)
    i, ic = divmod(int(i), len(cp))
    i, iu = divmod(i, len(up))
    it, ig = divmod(i, len(gp))
    return axes["t"][tp[it]], axes["g"][gp[ig]], axes["u"][up[iu]], axes["c"][cp[ic]]


def threads_available():
    return os.cpu_count() or 1
