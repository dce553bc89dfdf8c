"""C-ABI checks that need no GPU: the library loads and exports every symbol
include/*.h declares, the record layouts agree between the header, the
Python binding and the input generator, and host-side argument validation
rejects bad calls before any CUDA work."""

import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from conftest import ROOT
from workloads import archs, gen

HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]
DECL = re.compile(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*\b([a-z][a-z0-9_]*)\s*\(", re.M)


@pytest.fixture(scope="module")
def lib():
    from paper_1701_08547_gb300 import build, native

    build.build()
    return native.load()


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        names += [m for m in DECL.findall(text) if m not in ("if", "while", "for", "return", "sizeof")]
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for want in ("tune_eval", "tune_topk", "tune_workspace_bytes", "tune_check", "tune_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_record_layouts_match_header(tmp_path):
    """sizeof/offsetof from a C compile of include/tune.h equal the binding's ctypes
    structs and the generator's descriptor dtype."""
    from paper_1701_08547_gb300 import native

    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "tune.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\","
        "sizeof(tune_kernel_desc), offsetof(tune_kernel_desc, r0), offsetof(tune_kernel_desc, s0),"
        "offsetof(tune_kernel_desc, d), offsetof(tune_kernel_desc, space_mask),"
        "sizeof(tune_arch), offsetof(tune_arch, ipc), sizeof(tune_axes), offsetof(tune_axes, c));"
        "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    dt = gen.DESC_DTYPE
    assert vals[:5] == [64, dt.fields["r0"][1], dt.fields["s0"][1], dt.fields["d"][1],
                        dt.fields["space_mask"][1]]
    assert vals[5] == C.sizeof(native.TuneArch) and vals[6] == native.TuneArch.ipc.offset
    assert vals[7] == C.sizeof(native.TuneAxes) and vals[8] == native.TuneAxes.c.offset


def test_surrogate_layout_matches_header(lib):
    """The surrogate's input width and per-member parameter count agree between the header,
    the library, the binding and the parameter format the tests and the oracle use."""
    from paper_1701_08547_gb300 import native
    from workloads import mlp as L

    text = open(os.path.join(ROOT, "include", "tune.h")).read()
    width = int(re.search(r"#define TUNE_SURROGATE_INPUTS (\d+)", text).group(1))
    assert width == native.TUNE_SURROGATE_INPUTS == L.IN == 64
    assert lib.surrogate_param_count() == L.P
    text = re.sub(r"\n\s*\*\s*", " ", text)  # comment lines joined
    for name, val in (("W1", 0), ("b1", L.OFF_B[0]), ("W2", L.OFF_W[1]), ("b4", L.OFF_B[3]),
                      ("w5", L.OFF_W5), ("b5", L.OFF_B5)):
        assert re.search(rf"{name} (\[[^\]]*\] )?at {val}\b", text), name


def _call_eval(lib, arch_row, axes, k, ws=1 << 12, flags=0, descs=16):
    from paper_1701_08547_gb300 import native

    a = native.make_arch(arch_row)
    x = native.make_axes(axes)
    fake = C.c_void_p(16)  # never dereferenced: validation fails first
    return lib.tune_eval(C.byref(a), C.byref(x), C.c_void_p(descs), 1, k, flags, fake, fake, None,
                         None, None, None, fake, ws, None)


def test_host_validation_rejects_bad_arguments(lib):
    from paper_1701_08547_gb300 import native

    a = archs.arch("sm_103")
    ax = gen.axes()
    assert _call_eval(lib, a, ax, 0) == native.TUNE_EINVAL
    assert _call_eval(lib, a, ax, 17) == native.TUNE_EINVAL
    assert _call_eval(lib, a, ax, 5, ws=8) == native.TUNE_ENOMEM
    assert _call_eval(lib, a, ax, 5, flags=0x80) == native.TUNE_EINVAL
    assert _call_eval(lib, a, ax, 5, flags=native.TUNE_EMIT_POINTS) == native.TUNE_EINVAL  # no offsets
    assert _call_eval(lib, a, ax, 5, descs=24) == native.TUNE_EINVAL  # misaligned
    bad = dict(a, warp_size=16)
    assert _call_eval(lib, bad, ax, 5) == native.TUNE_EINVAL
    bad = dict(a, max_warps_sm=65)
    assert _call_eval(lib, bad, ax, 5) == native.TUNE_EINVAL
    bad = dict(a, smem_caps=[8192, 4096])
    assert _call_eval(lib, bad, ax, 5) == native.TUNE_EINVAL
    bad = dict(a, ipc=[0.0] + a["ipc"][1:])
    assert _call_eval(lib, bad, ax, 5) == native.TUNE_EINVAL
    big = dict(ax, g=[1 << 20])
    assert _call_eval(lib, a, big, 5) == native.TUNE_EINVAL
    low = dict(a, ipc=[2.0 ** -17] + a["ipc"][1:])  # below 2^-16: costs could overflow
    assert _call_eval(lib, low, ax, 5) == native.TUNE_EINVAL
    at = dict(a, ipc=[2.0 ** -16] + a["ipc"][1:])
    assert _call_eval(lib, at, ax, 5) != native.TUNE_EINVAL or "ipc" not in lib.tune_last_error().decode()
    assert "k = 0" in (lib.tune_last_error().decode() if _call_eval(lib, a, ax, 0) else "")


def test_topk_validation(lib):
    from paper_1701_08547_gb300 import native

    fake = C.c_void_p(16)
    assert lib.tune_topk(fake, fake, 1, 0, fake, fake, fake, 256, None) == native.TUNE_EINVAL
    assert lib.tune_topk(fake, fake, -1, 4, fake, fake, fake, 256, None) == native.TUNE_EINVAL
    assert lib.tune_topk(fake, fake, 1, 4, fake, fake, fake, 8, None) == native.TUNE_ENOMEM


def test_binding_fails_loudly_without_library(monkeypatch):
    from paper_1701_08547_gb300 import native

    monkeypatch.setattr(native, "_lib", None)
    monkeypatch.setattr(native, "LIB_PATH", "/nonexistent/libtune.so")
    with pytest.raises(RuntimeError, match="missing"):
        native.load()


def test_fault_injection_arguments(lib):
    """tune_inject_fault takes a known kind and a count in [0, 10^6]; setting and clearing
    pending faults involves no GPU."""
    from paper_1701_08547_gb300 import native

    assert lib.tune_inject_fault(0, 1) == native.TUNE_EINVAL
    assert lib.tune_inject_fault(4, 1) == native.TUNE_EINVAL
    assert lib.tune_inject_fault(native.TUNE_FAULT_COMPILE, -1) == native.TUNE_EINVAL
    for kind in (native.TUNE_FAULT_COMPILE, native.TUNE_FAULT_SLOW_REP, native.TUNE_FAULT_WAIT):
        assert lib.tune_inject_fault(kind, 3) == 0
        assert lib.tune_inject_fault(kind, 0) == 0
