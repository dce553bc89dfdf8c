"""ctypes binding to libtune.so: the C-ABI entry points with the same names.

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels. PyTorch supplies device memory and the stream. If
the library has not been built, loading fails with an error; there is no
other code path.
"""

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtune.so")

TUNE_OK, TUNE_EINVAL, TUNE_ENOMEM, TUNE_ECUDA, TUNE_ETIMEOUT, TUNE_ECOMPILE, TUNE_EUNSUPPORTED = (
    0, -1, -2, -3, -4, -5, -6)
TUNE_EMIT_POINTS = 0x1
TUNE_FAULT_COMPILE, TUNE_FAULT_SLOW_REP, TUNE_FAULT_WAIT = 1, 2, 3
TUNE_SCHED_WARP, TUNE_SCHED_THREAD = 0x10, 0x20
TUNE_HOST_DIRECT = 0x40
TUNE_SURROGATE_INPUTS = 64  # surrogate feature row width (48 features + zero padding)


def TUNE_SCHED_CHUNK(c):
    return (c + 1) << 8


def TUNE_SCHED_CTAS(m):
    return m << 12

TUNE_CALL_EVAL, TUNE_CALL_TOPK = 0, 1

ERROR_NAMES = {0: "TUNE_OK", -1: "TUNE_EINVAL", -2: "TUNE_ENOMEM", -3: "TUNE_ECUDA",
               -4: "TUNE_ETIMEOUT", -5: "TUNE_ECOMPILE", -6: "TUNE_EUNSUPPORTED"}


class TuneArch(C.Structure):
    _fields_ = [(f, C.c_int32) for f in (
        "cc", "n_sm", "warp_size", "max_threads_block", "max_warps_sm", "max_blocks_sm",
        "regs_sm", "regs_block_max", "regs_thread_max", "reg_alloc_unit", "reg_alloc_mode",
        "warp_alloc_gran", "smem_block_max", "smem_reserved_block", "smem_alloc_unit",
        "n_smem_caps")] + [("smem_caps", C.c_int32 * 16), ("ipc", C.c_float * 7),
                           ("w_sat", C.c_int32), ("work_scale", C.c_int32)]


class TuneAxes(C.Structure):
    _fields_ = [("n_t", C.c_int32), ("n_g", C.c_int32), ("n_u", C.c_int32), ("n_c", C.c_int32),
                ("t", C.c_int32 * 32), ("g", C.c_int32 * 16), ("u", C.c_int32 * 8),
                ("c", C.c_int32 * 4)]


class TuneError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load():
    """Load libtune.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"{LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    L = C.CDLL(LIB_PATH)
    vp, i64, i32, u32, sz = C.c_void_p, C.c_int64, C.c_int32, C.c_uint32, C.c_size_t
    L.tune_eval.argtypes = [C.POINTER(TuneArch), C.POINTER(TuneAxes), vp, i64, i32, u32, vp, vp,
                            vp, vp, vp, vp, vp, sz, vp]
    L.tune_eval.restype = C.c_int
    L.tune_eval_archs.argtypes = [C.POINTER(TuneArch), i32, C.POINTER(TuneAxes), vp, i64, i32, u32, vp, vp, vp, sz,
                                  vp]
    L.tune_eval_archs.restype = C.c_int
    L.tune_topk.argtypes = [vp, vp, i64, i32, vp, vp, vp, sz, vp]
    L.tune_topk.restype = C.c_int
    L.tune_workspace_bytes.argtypes = [C.c_int, i64, i32]
    L.tune_workspace_bytes.restype = sz
    L.tune_check.argtypes = [vp, vp]
    L.tune_check.restype = C.c_int
    L.tune_last_error.argtypes = []
    L.tune_last_error.restype = C.c_char_p
    L.tune_version.argtypes = []
    L.tune_version.restype = C.c_int
    L.tune_autotune.argtypes = [C.POINTER(TuneArch), C.POINTER(TuneAxes), vp, i64, i32, i32, vp, vp,
                                vp, sz, C.POINTER(C.c_uint32), C.POINTER(C.c_float), vp]
    L.tune_autotune.restype = C.c_int
    L.tune_features.argtypes = [C.POINTER(TuneArch), C.POINTER(TuneAxes), vp, vp, vp, i64, vp, vp, sz, vp]
    L.tune_features.restype = C.c_int
    L.tune_suggest.argtypes = [C.POINTER(TuneArch), C.POINTER(TuneAxes), vp, i64, vp, vp, vp, vp, vp, vp, sz, vp]
    L.tune_suggest.restype = C.c_int
    L.tune_search.argtypes = [C.POINTER(TuneArch), C.POINTER(TuneAxes), vp, i64, i32, i32, C.c_uint64, vp, vp, vp,
                              vp, vp, sz, vp]
    L.tune_search.restype = C.c_int
    L.tune_real_measure.argtypes = [i32, i32, vp, vp, vp, vp, i32, i32, vp, vp, vp, vp]
    L.tune_real_measure.restype = C.c_int
    L.tune_eval_host_scratch_bytes.argtypes = [i64, i32]
    L.tune_eval_host_scratch_bytes.restype = sz
    L.tune_eval_host.argtypes = [C.POINTER(TuneArch), C.POINTER(TuneAxes), vp, i64, i32, u32, vp, vp, i64, vp, sz, vp]
    L.tune_eval_host.restype = C.c_int
    L.tune_inject_fault.argtypes = [C.c_int, C.c_int]
    L.tune_inject_fault.restype = C.c_int
    _lib = L
    return L


TUNE_SEARCH_RANDOM, TUNE_SEARCH_NELDER_MEAD = 1, 2
TUNE_REAL_MATVEC, TUNE_REAL_ATAX, TUNE_REAL_BICG = 0, 1, 2


def make_arch(row):
    """Marshal an architecture-row dict into the C struct."""
    a = TuneArch()
    for f, _ in TuneArch._fields_:
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
    """Marshal an axes dict {t, g, u, c: lists} into the C struct."""
    a = TuneAxes()
    a.n_t, a.n_g, a.n_u, a.n_c = len(ax["t"]), len(ax["g"]), len(ax["u"]), len(ax["c"])
    for name in ("t", "g", "u", "c"):
        arr = getattr(a, name)
        for i, v in enumerate(ax[name]):
            arr[i] = int(v)
    return a


def check(rc):
    if rc != TUNE_OK:
        raise TuneError(rc, load().tune_last_error().decode())
    return rc


def load_noalloc():
    """The library with tune_eval_noalloc's signature declared (see include/tune.h)."""
    L = load()
    if not getattr(L, "_noalloc_declared", False):
        vp, i64, i32, u32 = C.c_void_p, C.c_int64, C.c_int32, C.c_uint32
        L.tune_eval_noalloc.argtypes = [C.POINTER(TuneArch), C.POINTER(TuneAxes), vp, i64, i32, u32,
                                        vp, vp, vp, vp, vp, vp, vp]
        L.tune_eval_noalloc.restype = C.c_int
        L._noalloc_declared = True
    return L
