"""Binding for the surrogate MLP ensemble calls of libtune.so (argument marshalling only)."""

import ctypes as C

from . import native


class Cfg(C.Structure):
    _fields_ = [("members", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float)]


def _lib():
    L = native.load()
    if not getattr(L, "_surrogate_declared", False):
        vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
        L.surrogate_create.argtypes = [C.POINTER(C.c_void_p), C.POINTER(Cfg)]
        L.surrogate_create.restype = C.c_int
        L.surrogate_free.argtypes = [vp]
        L.surrogate_free.restype = None
        L.surrogate_param_count.argtypes = []
        L.surrogate_param_count.restype = C.c_int
        L.surrogate_set_params.argtypes = [vp, vp, i64]
        L.surrogate_set_params.restype = C.c_int
        L.surrogate_get.argtypes = [vp, C.c_int, vp, i64]
        L.surrogate_get.restype = C.c_int
        L.surrogate_forward.argtypes = [vp, vp, i64, vp, vp]
        L.surrogate_forward.restype = C.c_int
        L.surrogate_train_step.argtypes = [vp, vp, vp, i64, i32, vp]
        L.surrogate_train_step.restype = C.c_int
        L.surrogate_train.argtypes = [vp, vp, vp, i64, vp, i32, vp, vp]
        L.surrogate_train.restype = C.c_int
        L.surrogate_infer.argtypes = [vp, C.POINTER(native.TuneArch), C.POINTER(native.TuneAxes), vp, i64, vp,
                                      i32, C.c_float, vp, vp, vp, vp, C.c_size_t, vp]
        L.surrogate_infer.restype = C.c_int
        L.surrogate_infer_workspace_bytes.argtypes = [C.c_int, i64, i32]
        L.surrogate_infer_workspace_bytes.restype = C.c_size_t
        L.surrogate_set_option.argtypes = [vp, C.c_int, C.c_int]
        L.surrogate_set_option.restype = C.c_int
        L.surrogate_status.argtypes = [vp]
        L.surrogate_status.restype = C.c_int
        L._surrogate_declared = True
    return L


def _stream(stream):
    import torch

    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


class Surrogate:
    """A handle to an MLP ensemble living on the GPU."""

    GET_PARAMS, GET_GRADS, GET_M, GET_V, GET_LOSS, GET_PRED, GET_FP8_CODES, GET_FP8_SCALES = range(8)
    FWD_LAYERED, FWD_FUSED_BF16, FWD_FUSED_FP8 = range(3)
    BWD_LAYERED, BWD_FUSED = range(2)

    def __init__(self, members=5, batch=8192, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.L = _lib()
        self.members, self.batch = members, batch
        cfg = Cfg(members, batch, lr, beta1, beta2, eps)
        h = C.c_void_p()
        native.check(self.L.surrogate_create(C.byref(h), C.byref(cfg)))
        self.h = h
        self.P = self.L.surrogate_param_count()

    def close(self):
        if self.h:
            self.L.surrogate_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, option, value):
        native.check(self.L.surrogate_set_option(self.h, int(option), int(value)))

    def use_tcgen05(self, on=True):
        """Forward layers on tcgen05 tensor cores (default) or on mma.sync."""
        self.set_option(0, 1 if on else 0)

    def set_forward_mode(self, mode):
        """forward()/infer(): layer by layer (0), one fused launch in BF16 (1, the default),
        or fused with layers 2-4 on E4M3 codes (2)."""
        self.set_option(1, mode)

    def set_backward_mode(self, mode):
        """Backward pass: one mma.sync GEMM per input and weight gradient (0), or the fused
        tcgen05 input-gradient chain and tcgen05 weight gradients (1, the default; needs
        the tcgen05 option)."""
        self.set_option(2, mode)

    def check(self):
        native.check(self.L.surrogate_status(self.h))

    def set_params(self, flat):
        import numpy as np

        a = np.ascontiguousarray(flat, dtype=np.float32)
        native.check(self.L.surrogate_set_params(self.h, a.ctypes.data, a.size))

    def get(self, what):
        import numpy as np

        n = {4: self.members, 5: self.members * self.batch, 6: self.members * 3 * 256 * 256,
             7: self.members * 3 * 256}.get(what, self.members * self.P)
        out = np.empty(n, dtype=np.float32)
        native.check(self.L.surrogate_get(self.h, what, out.ctypes.data, n))
        return out

    def forward(self, feats, pred=None, stream=None):
        """feats: device bfloat16 [n, 64]; returns device float32 [members, n]."""
        import torch

        n = feats.shape[0]
        if pred is None:
            pred = torch.empty((self.members, n), dtype=torch.float32, device=feats.device)
        native.check(self.L.surrogate_forward(self.h, C.c_void_p(feats.data_ptr()), n,
                                              C.c_void_p(pred.data_ptr()), _stream(stream)))
        return pred

    def train_step(self, feats, labels, apply_update=True, stream=None):
        n = feats.shape[0]
        native.check(self.L.surrogate_train_step(self.h, C.c_void_p(feats.data_ptr()),
                                                 C.c_void_p(labels.data_ptr()), n, int(apply_update),
                                                 _stream(stream)))

    def train(self, feats, labels, order, epochs, loss_trace=None, stream=None):
        n = feats.shape[0]
        lt = None if loss_trace is None else C.c_void_p(loss_trace.data_ptr())
        native.check(self.L.surrogate_train(self.h, C.c_void_p(feats.data_ptr()),
                                            C.c_void_p(labels.data_ptr()), n,
                                            C.c_void_p(order.data_ptr()), int(epochs), lt,
                                            _stream(stream)))

    def infer(self, arch, axes, descs, pt_offsets, k, thresh=0.1, stream=None):
        """Rank every point of every kernel by predicted runtime with analytic fallback.
        descs: device descriptor tensor; pt_offsets: numpy int64 [n + 1].
        Returns (topk_idx, topk_score, used_fallback) device tensors."""
        import numpy as np
        import torch

        n = descs.numel() * descs.element_size() // 64
        dev = descs.device
        off = np.ascontiguousarray(pt_offsets, dtype=np.int64)
        idx = torch.empty((n, k), dtype=torch.int32, device=dev)
        val = torch.empty((n, k), dtype=torch.float32, device=dev)
        fb = torch.empty(n, dtype=torch.uint8, device=dev)
        nbytes = self.L.surrogate_infer_workspace_bytes(self.members, n, k)
        ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        a, x = native.make_arch(arch), native.make_axes(axes)
        native.check(self.L.surrogate_infer(self.h, C.byref(a), C.byref(x), C.c_void_p(descs.data_ptr()), n,
                                            off.ctypes.data, int(k), float(thresh), C.c_void_p(idx.data_ptr()),
                                            C.c_void_p(val.data_ptr()), C.c_void_p(fb.data_ptr()),
                                            C.c_void_p(ws.data_ptr()), nbytes, _stream(stream)))
        return idx, val, fb
