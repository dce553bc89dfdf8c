"""Descriptor field ranges and the no-overflow bound of the cost (CPU oracle).

Convention (the library's input format; the paper's counts are per-thread
instruction counts of real kernels, far below these limits): a well-formed
descriptor has every instruction count in [0, 2^40], the divergence fraction d
in [0, 1], r0 in [0, 2^24) and s0 in [0, 2^30); architecture rows have
IPC >= 2^-16, W_sat <= 2^20 and K <= 2^24. Within these ranges every term of
Eq. 6 with the launch-shape factors is bounded:
  C_c = (1 + d) K n'_c / IPC_c <= 2 * 2^24 * 2^40 * 2^16 = 2^81 per class,
  C_nm + C_m hide <= 5 * 2^81 + 2 * 2^81 * 2^20 < 2^103,
  lane = 32 W_B / T <= 32, ipar = waves slots / (n_SM G) < 1 / n_SM + B* / G <= 33,
so every cost is below 2^103 * 32 * 33 < 2^114: no valid point's FP32 cost
overflows, and +inf always means "no valid configuration". A descriptor outside
the ranges is malformed: it gets padding (-1, +inf) and the call reports it.
"""

import numpy as np

from workloads import archs, gen

TWO40 = np.float32(2.0 ** 40)


def extreme_arch():
    a = archs.arch("sm_103")
    a["ipc"] = [2.0 ** -16] * 7
    a["w_sat"] = 1 << 20
    a["work_scale"] = 1 << 24
    return a


def extreme_axes():
    return {"t": [1, 7, 32, 33, 1024], "g": [1, 2, 3, 1000, 32768], "u": [1, 8], "c": [0, 100]}


def extreme_descs():
    d = np.zeros(4, dtype=gen.DESC_DTYPE)
    d["n"] = TWO40
    d["d"] = np.float32(1.0)
    d["r0"] = [16, 16, 200, 32]
    d["s0"] = [0, 200000, 0, 48 * 1024]  # the second: one block per SM at full carveout (W* = W_B)
    d["n"][3, :] = [TWO40, 0, 1, TWO40, 0, 3, 0]
    d["space_mask"] = np.uint64(gen.mask_bits(range(5), range(5), range(2), range(2)))
    return d


def test_costs_at_the_field_bounds_are_finite(oracle):
    """Counts 2^40, d = 1, the extreme architecture row, T = 1 (lane 32) and G = 1 (ipar = B*):
    every valid point has a finite FP32 cost below 2^114 that agrees with FP64 to 1e-5,
    and the largest cost comes within a factor 2^14 of that bound."""
    a, ax, d = extreme_arch(), extreme_axes(), extreme_descs()
    off = gen.point_offsets(d)
    o = oracle.evaluate(a, ax, d, 5, emit=True, offsets=off)
    assert not o["malformed"]
    ok = o["B"] > 0
    assert ok.sum() > 100
    c32, c64 = o["cost32"][ok], o["cost64"][ok]
    assert np.all(np.isfinite(c32)) and np.all(np.isfinite(c64))
    assert c64.max() < 2.0 ** 114 and c64.max() > 2.0 ** 100
    assert np.max(np.abs(c32 - c64) / c64) <= 1e-5
    assert np.all(np.isinf(o["cost32"][~ok]))
    assert np.all(o["idx"][:3] >= 0) and np.all(np.isfinite(o["cost"][:3]))


def test_out_of_range_fields_are_malformed(oracle):
    """Each field just past its range (and non-numbers) makes exactly that descriptor
    malformed: padding, an error from strict evaluation; the others are unaffected."""
    a, ax = archs.arch("sm_103"), gen.axes()
    base = gen.descriptors(1, 41, "dense128")[0]
    cases = []

    def add(**kw):
        r = base.copy()
        for f, v in kw.items():
            if f.startswith("n"):
                r["n"][int(f[1:])] = v
            else:
                r[f] = v
        cases.append(r)

    above = np.nextafter(TWO40, np.float32(np.inf))
    add(n0=above)
    add(n3=np.float32(1e36))
    add(n6=np.float32(np.inf))
    add(n1=np.float32(np.nan))
    add(n2=np.float32(-1.0))
    add(d=np.nextafter(np.float32(1.0), np.float32(2.0)))
    add(d=np.float32(np.nan))
    add(d=np.float32(-1e-30))
    add(r0=-1)
    add(s0=1 << 30)
    bad = len(cases)
    add(n0=TWO40)                 # the bounds themselves are fine
    add(d=np.float32(1.0))
    add(n4=np.float32(0.0), d=np.float32(-0.0))
    d = np.array(cases, dtype=gen.DESC_DTYPE)
    o = oracle.evaluate(a, ax, d, 4, strict=False)
    assert o["malformed"]
    assert np.all(o["idx"][:bad] == -1) and np.all(np.isinf(o["cost"][:bad]))
    assert np.all(o["idx"][bad:] >= 0)
    good = oracle.evaluate(a, ax, d[bad:], 4)
    assert not good["malformed"]
    assert np.array_equal(good["idx"], o["idx"][bad:])
    for i in range(bad):
        try:
            oracle.evaluate(a, ax, d[i:i + 1], 4)
        except ValueError:
            continue
        raise AssertionError(f"case {i} was not rejected")
