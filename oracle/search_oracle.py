"""Search over a kernel's tuning space with the static cost as the objective: random
search and Nelder-Mead simplex, the bounded-time methods the paper names for exploring
the space left after static pruning (Section III-C lists the autotuner's search
methods; Section IV-C recommends exhaustive search where it is affordable and random
or Nelder-Mead search where the tuning time must be capped).

TEST INFRASTRUCTURE ONLY: imported by the tests and the bench, never by the product
package. Plain Python over the C oracle's per-point FP32 costs (oracle.evaluate with
emit=True); shares no code with the CUDA path.

The paper does not define either method's details; the reading used here (and by
the library, whose results must match bit for bit):
* a point is a rank vector (a0, a1, a2, a3) over the searched lists of thread
  counts (the kernel's, optionally intersected with a kept set), grid sizes,
  unroll factors and carveouts; objective = the FP32 cost (+inf without a valid
  configuration); points are ordered by (cost, canonical index in the full space);
* draws: SplitMix64 (Steele, Lea and Flood, 2014) used counter-style, draw j of
  kernel i = mix64(mix64(seed) + (i 2^32 + j + 1) gamma) mod 2^64, mapped to
  [0, n) as ((x >> 32) n) >> 32;
* random search: evaluation j takes rank d from draw 4 j + d;
* Nelder-Mead: five vertices with 8 fractional bits, rounded as floor(v + 1/2) and
  clamped to the list; start from draws 0..3; vertex d + 1 steps max(1, n_d // 4)
  ranks along axis d (backwards if forwards leaves the list); vertices ordered by
  (cost, index, vertex number); centroid of the best four = sum >> 2; reflection
  2c - w; expansion 3c - 2w if the reflection beats the best (the better of the
  two replaces w); else the reflection replaces w if it beats the second worst;
  else contraction c + ((r - c) >> 1) if r beats w, otherwise c + ((w - c) >> 1),
  accepted if it beats the better of r and w (resp. w); else shrink every other
  vertex halfway to the best, v = b + ((v - b) >> 1), evaluating each. Every
  evaluation counts against the budget; the search ends when the budget is spent
  or a shrink leaves all vertices on one point. Result: the best point seen.
"""

import math

import numpy as np

from oracle import oracle as O

M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
Q = 8  # fractional bits of the simplex coordinates


def mix64(z):
    """SplitMix64 output function on a 64-bit state."""
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def draw_below(key, i, j, n):
    x = mix64(key + ((i << 32) + j + 1) * GAMMA)
    return ((x >> 32) * n) >> 32


def _positions(mask, width):
    return [b for b in range(width) if (mask >> b) & 1]


def _less(a, b):
    """(cost, index) keys; costs compare as floats (+inf equal to +inf)."""
    return a[0] < b[0] or (a[0] == b[0] and a[1] < b[1])


class _Kernel:
    def __init__(self, desc, costs, t_keep):
        m = int(desc["space_mask"])
        self.tm = m & 0xFFFFFFFF
        gm, um, cm = (m >> 32) & 0xFFFF, (m >> 48) & 0xFF, (m >> 56) & 0xF
        keep = self.tm if t_keep is None else self.tm & int(t_keep)
        self.lists = [_positions(keep, 32), _positions(gm, 16), _positions(um, 8), _positions(cm, 4)]
        self.n = [len(x) for x in self.lists]
        self.nG, self.nU, self.nC = self.n[1], self.n[2], self.n[3]
        self.costs = costs
        self.evals = 0
        self.best = (math.inf, -1)

    def index(self, r):
        tp = self.lists[0][r[0]]
        t_full = bin(self.tm & ((1 << tp) - 1)).count("1")
        return ((t_full * self.nG + r[1]) * self.nU + r[2]) * self.nC + r[3]

    def f(self, r):
        idx = self.index(r)
        c = float(self.costs[idx])
        if c != c:
            c = math.inf
        self.evals += 1
        key = (c, idx)
        if _less(key, self.best):
            self.best = key
        return key

    def rnd(self, v):
        return [min(max((v[d] + (1 << (Q - 1))) >> Q, 0), self.n[d] - 1) for d in range(4)]


def _random(kn, key, i, budget):
    for j in range(budget):
        kn.f([draw_below(key, i, 4 * j + d, kn.n[d]) for d in range(4)])


def _nelder_mead(kn, key, i, budget):
    def fv(v):
        if kn.evals >= budget:
            return None
        return kn.f(kn.rnd(v))

    x0 = [draw_below(key, i, d, kn.n[d]) << Q for d in range(4)]
    V = [list(x0) for _ in range(5)]
    for d in range(4):
        s = max(1, kn.n[d] >> 2) << Q
        V[d + 1][d] = x0[d] + s if x0[d] + s <= (kn.n[d] - 1) << Q else x0[d] - s
    F = []
    for j in range(5):
        k = fv(V[j])
        if k is None:
            return
        F.append(k)
    while True:
        order = sorted(range(5), key=lambda j: (F[j][0], F[j][1], j))
        b, sw, w = order[0], order[3], order[4]
        c = [(V[order[0]][d] + V[order[1]][d] + V[order[2]][d] + V[order[3]][d]) >> 2 for d in range(4)]
        xr = [2 * c[d] - V[w][d] for d in range(4)]
        fr = fv(xr)
        if fr is None:
            return
        if _less(fr, F[b]):
            xe = [3 * c[d] - 2 * V[w][d] for d in range(4)]
            fe = fv(xe)
            if fe is not None and _less(fe, fr):
                V[w], F[w] = xe, fe
            else:
                V[w], F[w] = xr, fr
            if fe is None:
                return
            continue
        if _less(fr, F[sw]):
            V[w], F[w] = xr, fr
            continue
        outside = _less(fr, F[w])
        src = xr if outside else V[w]
        xc = [c[d] + ((src[d] - c[d]) >> 1) for d in range(4)]
        fc = fv(xc)
        if fc is None:
            return
        if _less(fc, fr if outside else F[w]):
            V[w], F[w] = xc, fc
            continue
        for j in range(5):
            if j == b:
                continue
            V[j] = [V[b][d] + ((V[j][d] - V[b][d]) >> 1) for d in range(4)]
            k = fv(V[j])
            if k is None:
                return
            F[j] = k
        rb = kn.rnd(V[b])
        if all(kn.rnd(V[j]) == rb for j in range(5)):
            return


def search(row, axes, descs, method, budget, seed, t_keep=None, offsets=None, costs=None):
    """Best point per kernel: dict(idx=int32[n], cost=float32[n], evals=int32[n]).

    method: "random" or "nelder_mead"; t_keep: optional uint32[n] thread-count masks.
    costs/offsets: per-point FP32 costs from oracle.evaluate(emit=True) (computed here
    when not given).
    """
    descs = np.ascontiguousarray(descs)
    n = len(descs)
    if costs is None:
        from workloads import gen

        offsets = gen.point_offsets(descs)
        costs = O.evaluate(row, axes, descs, 1, emit=True, offsets=offsets)["cost32"]
    key = mix64(int(seed))
    out_i = np.full(n, -1, np.int32)
    out_c = np.full(n, np.inf, np.float32)
    out_e = np.zeros(n, np.int32)
    run = {"random": _random, "nelder_mead": _nelder_mead}[method]
    for i in range(n):
        kn = _Kernel(descs[i], costs[int(offsets[i]):int(offsets[i + 1])],
                     None if t_keep is None else t_keep[i])
        if min(kn.n) > 0:
            run(kn, key, i, budget)
        out_i[i], out_c[i], out_e[i] = kn.best[1], np.float32(kn.best[0]), kn.evals
    return {"idx": out_i, "cost": out_c, "evals": out_e}
