"""Host logic of the real-kernel workload: descriptors written from the loop structure
of matVec2D, ATAX and BiCG, and the tuning sub-space's canonical enumeration."""

import numpy as np

from paper_1701_08547_gb300 import realkernels as R
from workloads import gen


def test_descriptor_counts_follow_the_loops():
    ax = gen.axes()
    n = 1000
    mv = R.descriptor("matvec", n, 30, ax)[0]
    at = R.descriptor("atax", n, 30, ax)[0]
    # per output element: n FMAs, 2n + 1 loads and stores, n + 4 index operations, n loop branches
    assert list(mv["n"]) == [1000, 0, 1004, 2001, 0, 1000, 0]
    assert list(at["n"]) == [2 * v for v in mv["n"]]  # two products
    assert mv["r0"] == 30 and mv["s0"] == 0 and mv["d"] == 0


def test_sub_space_enumeration_is_canonical():
    ax = gen.axes()
    d = R.descriptor("bicg", 64, 24, ax)
    assert int(gen.space_sizes(d)[0]) == 32 * 4 * 4 * 2
    pts = R.points(ax)
    assert len(pts) == 1024
    from oracle import oracle as O

    for i in (0, 1, 7, 8, 31, 32, 500, 1023):
        T, G, U, C = O.decode_point(d[0], ax, i)
        assert tuple(pts[i]) == (T, G, U, C)
