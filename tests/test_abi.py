"""The C ABI without a GPU: libquadbox builds for sm_103a, loads, exports every
function include/quadbox.h declares, and validates arguments before any
device call."""
import ctypes
import os
import re

import pytest

from paper_2605_04844_gb300 import _native as N
from paper_2605_04844_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "quadbox.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qb_[a-z_0-9]+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    B.build()
    lib = N.load()
    decl = declared_functions()
    assert len(decl) >= 13
    for name in decl:
        assert hasattr(lib, name), f"{name} declared in quadbox.h but not exported"
    assert set(decl) == set(N.EXPORTED) | (set(decl) - set(N.EXPORTED))
    for name in N.EXPORTED:
        assert name in decl, f"binding declares {name} which the header does not"


def test_version_and_last_error():
    lib = N.load()
    assert b"sm_103a" in lib.qb_version()
    assert isinstance(lib.qb_last_error(), bytes)


def test_workspace_bytes_sizes():
    a = N.qb_frame_workspace_bytes(1000, 256, 256, 10_000)
    b = N.qb_frame_workspace_bytes(2000, 256, 256, 10_000)
    c = N.qb_frame_workspace_bytes(1000, 256, 256, 20_000)
    assert 0 < a < b and a < c
    assert a % 256 == 0
    assert N.qb_frame_workspace_bytes(-1, 256, 256, 10) == 0
    assert N.qb_frame_workspace_bytes(10, 0, 256, 10) == 0
    assert N.qb_frame_workspace_bytes(10, 256, 256, (1 << 30) + 1) == 0
    # 1M Gaussians, 1080p, 20M pairs fits comfortably in HBM
    big = N.qb_frame_workspace_bytes(1_000_000, 1920, 1080, 20_000_000)
    assert big < 2 * 1024 ** 3


def test_frame_init_rejects_bad_workspace_without_device_calls():
    lib = N.load()
    fr = N.QbFrame()
    st = lib.qb_frame_init(ctypes.byref(fr), 10, 64, 64, 100, None, 1 << 20, None)
    assert st == N.QB_ERR_INVALID_ARG
    st = lib.qb_frame_init(ctypes.byref(fr), 10, 64, 64, 100, ctypes.c_void_p(0x1001), 1 << 20, None)
    assert st == N.QB_ERR_INVALID_ARG and b"aligned" in lib.qb_last_error()
    need = N.qb_frame_workspace_bytes(10, 64, 64, 100)
    st = lib.qb_frame_init(ctypes.byref(fr), 10, 64, 64, 100, ctypes.c_void_p(0x100000), need - 1, None)
    assert st == N.QB_ERR_INVALID_ARG and b"too small" in lib.qb_last_error()


def test_stage_order_checked_without_device_calls():
    lib = N.load()
    fr = N.QbFrame()
    assert lib.qb_sort(ctypes.byref(fr), None) == N.QB_ERR_INVALID_ARG  # no workspace bound


def test_sort_scratch_bytes():
    assert N.qb_sort_scratch_bytes(0, 44, 8) > 0
    assert N.qb_sort_scratch_bytes(10 ** 6, 44, 11) > N.qb_sort_scratch_bytes(10 ** 6, 44, 8)
    assert N.qb_sort_scratch_bytes(10, 44, 7) == 0
    assert N.qb_sort_scratch_bytes(10, 44, 12) == 0
    assert N.qb_sort_scratch_bytes((1 << 30) + 1, 44, 8) == 0


def test_header_struct_sizes_match_binding():
    # qb_frame / qb_camera layouts as seen by a C compiler
    src = r"""
    #include <stdio.h>
    #include <stddef.h>
    #include "quadbox.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu %zu\n", sizeof(qb_frame), sizeof(qb_camera), sizeof(qb_scene),
             sizeof(qb_frame_arrays), offsetof(qb_frame, n_pairs), offsetof(qb_frame, sorted_in_alt));
      return 0; }
    """
    import subprocess
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "s")
        r = subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], capture_output=True, text=True)
        if r.returncode != 0:
            pytest.skip("no C compiler: " + r.stderr)
        out = subprocess.run([exe], capture_output=True, text=True).stdout.split()
    got = [int(x) for x in out]
    want = [ctypes.sizeof(N.QbFrame), ctypes.sizeof(N.QbCamera), ctypes.sizeof(N.QbScene),
            ctypes.sizeof(N.QbFrameArrays), N.QbFrame.n_pairs.offset, N.QbFrame.sorted_in_alt.offset]
    assert got == want
