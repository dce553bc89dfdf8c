"""Pin of the sm_103 architecture row: the oracle's occupancy (Eqs. 1-5 with
the row's limits, granularities, per-block reservation and carveout reading)
against NVIDIA's occupancy API, cudaOccupancyMaxActiveBlocksPerMultiprocessor,
on probe kernels with forced register counts, over block sizes, dynamic
shared memory and carveout preferences."""

import ctypes as C
import os
import subprocess

import pytest

from workloads import archs

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    out = tmp_path_factory.mktemp("probe") / "libocc_probe.so"
    subprocess.check_call(["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                           "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared",
                           os.path.join(HERE, "probe", "occ_probe.cu"), "-o", str(out)])
    lib = C.CDLL(str(out))
    for f in ("probe_count", "probe_regs", "probe_static_smem", "probe_occupancy", "probe_sm_count"):
        getattr(lib, f).restype = C.c_int
    return lib


def test_sm_count_matches_row(probe):
    assert probe.probe_sm_count() == archs.arch("sm_103")["n_sm"]


@pytest.mark.parametrize("carveout", [0, 25, 50, 100])
def test_occupancy_api_matches_oracle(probe, oracle, carveout):
    a = archs.arch("sm_103")
    mismatches = []
    checked = 0
    for i in range(probe.probe_count()):
        R = probe.probe_regs(i)
        s_static = probe.probe_static_smem(i)
        assert R > 0
        for T in (32, 64, 96, 128, 192, 256, 384, 512, 640, 768, 1024):
            for dyn in (0, 100, 1000, 4000, 9000, 20000, 49152, 70000, 120000, 200000, 231000):
                api = probe.probe_occupancy(i, T, dyn, carveout)
                assert api >= 0, api
                o = oracle.occupancy(a, T, R, s_static + dyn, carveout)
                checked += 1
                if api != o["B"]:
                    mismatches.append((R, T, dyn, carveout, api, o["B"]))
    assert checked > 1000
    assert not mismatches, f"{len(mismatches)} of {checked} differ, e.g. {mismatches[:12]}"
