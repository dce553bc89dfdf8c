"""Oracle of the paper's static search-space pruning (Section III-C, Section IV-C
Table "Suggested parameters to achieve theoretical occupancy").

TEST INFRASTRUCTURE ONLY. Built on the C oracle's occupancy (Eqs. 1-5); no code
shared with the CUDA path. At the kernel's registers r0, shared memory s0 and the
largest shared-memory capacity (carveout 100 %):
  T*  = thread counts of the kernel's space whose warp limit alone (Eq. 1 with the
        block limit) allows the most resident warps -- the table's T* is the same
        for every kernel of an architecture; occ* = max over T* of W*(T, r0, s0) / W_mp;
  R*  = registers that can be added while max over T* of W* stays occ*;
  S*  = the largest shared memory per block keeping B* at the smallest T of T*
        reaching occ*
        (found by bisection: B* does not rise with S at a fixed capacity);
  rule: intensity (FP32 + FP64) / (GLDST + SLDST) > 4.0 keeps the upper
        floor(|T*|/2) (at least 1) thread counts of T*, else the lower ones.
"""

from oracle import oracle as O


def suggest(row, axes, desc):
    m = int(desc["space_mask"])
    tpos = [b for b in range(32) if (m >> b) & 1]
    r0, s0 = int(desc["r0"]), int(desc["s0"])

    def W(T, R, S):
        return O.occupancy(row, T, R, S, 100)["W"]

    def warp_only(T):
        if T > row["max_threads_block"]:
            return 0
        wb = -(-T // 32)
        return min(row["max_blocks_sm"], row["max_warps_sm"] // wb) * wb

    top = max((warp_only(axes["t"][p]) for p in tpos), default=0)
    star = [p for p in tpos if top > 0 and warp_only(axes["t"][p]) == top]
    ws = {p: W(axes["t"][p], r0, s0) for p in star}
    best = max(ws.values(), default=0)
    out = {"t_star": sum(1 << p for p in star), "occ_star": best / row["max_warps_sm"]}
    if best == 0:
        out.update(r_headroom=-1, s_star=-1, t_rule=0)
        return out
    R = r0
    while R + 1 <= row["regs_thread_max"] and max(W(axes["t"][p], R + 1, s0) for p in star) >= best:
        R += 1
    out["r_headroom"] = R - r0
    T0 = axes["t"][next(p for p in star if ws[p] == best)]
    B0 = O.occupancy(row, T0, r0, s0, 100)["B"]
    lo, hi = s0, row["smem_block_max"]
    while lo < hi:
        mid = lo + (hi - lo + 1) // 2
        if O.occupancy(row, T0, r0, mid, 100)["B"] >= B0:
            lo = mid
        else:
            hi = mid - 1
    out["s_star"] = lo
    n = [float(x) for x in desc["n"]]
    upper = (n[0] + n[1]) > 4.0 * (n[3] + n[4])
    keep = max(1, len(star) // 2)
    chosen = star[-keep:] if upper else star[:keep]
    out["t_rule"] = sum(1 << p for p in chosen)
    return out
