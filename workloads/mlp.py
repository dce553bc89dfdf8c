"""Parameter format and seeded initial weights of the surrogate MLP ensemble.

Pure data: the flat per-member layout (the same one include/tune.h documents)
and Gaussian initial weights drawn with numpy's PCG64 from a per-member seed
(weights N(0, 1/fan_in), biases 0; the zero-padded inputs 48..63 get zero
weights). Both the CUDA path and the oracle take these arrays as inputs.
"""

import numpy as np

IN, WID, FEATURES = 64, 256, 48  # 48 features zero-padded to 64 inputs (one 128-byte row)
LAYERS = [(IN, WID), (WID, WID), (WID, WID), (WID, WID)]
OFF_W = [0, 16640, 82432, 148224]
OFF_B = [16384, 82176, 147968, 213760]
OFF_W5, OFF_B5 = 214016, 214272
P = 214336  # floats per member (padded)


def init_params(members, seeds=None):
    """float32 [members * P] initial master weights; member m uses seed seeds[m] (default 5 + m)."""
    seeds = seeds or [5 + m for m in range(members)]
    out = np.zeros((members, P), dtype=np.float32)
    for m in range(members):
        rng = np.random.Generator(np.random.PCG64(seeds[m]))
        for l, (fin, fout) in enumerate(LAYERS):
            w = rng.standard_normal((fout, fin)) / np.sqrt(FEATURES if l == 0 else fin)
            if l == 0:
                w[:, FEATURES:] = 0.0
            out[m, OFF_W[l]:OFF_W[l] + fout * fin] = w.astype(np.float32).ravel()
        out[m, OFF_W5:OFF_W5 + WID] = (rng.standard_normal(WID) / np.sqrt(WID)).astype(np.float32)
    return out.ravel()


def unpack(flat, members):
    """Views {W1..W4, b1..b4, w5, b5} per member from a flat parameter array."""
    a = np.asarray(flat).reshape(members, P)
    res = []
    for m in range(members):
        d = {}
        for l, (fin, fout) in enumerate(LAYERS):
            d[f"W{l + 1}"] = a[m, OFF_W[l]:OFF_W[l] + fout * fin].reshape(fout, fin)
            d[f"b{l + 1}"] = a[m, OFF_B[l]:OFF_B[l] + fout]
        d["w5"] = a[m, OFF_W5:OFF_W5 + WID]
        d["b5"] = a[m, OFF_B5:OFF_B5 + 1]
        res.append(d)
    return res
