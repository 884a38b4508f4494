"""The C ABI library: it loads without a GPU, exports every function that
include/cch.h declares, and the binding's structure layouts match the
header's (checked against a C compiler)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

import paper_1508_05488_gb300 as cch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cch.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cch_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("cch_hull", "cch_hull_batched", "cch_serve_create", "cch_serve_submit", "cch_serve_poll",
                 "cch_serve_release", "cch_serve_destroy", "cch_workspace_bytes", "cch_release_workspace",
                 "cch_status_string"):
        assert must in names, must


def test_library_exports_every_declared_function():
    if not os.path.exists(cch.LIB_PATH):
        pytest.skip("libcch.so not built")
    lib = ctypes.CDLL(cch.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_host_checks_without_gpu():
    if not os.path.exists(cch.LIB_PATH):
        pytest.skip("libcch.so not built")
    lib = cch.lib()
    for code in range(0, -10, -1):
        assert lib.cch_status_string(code)
    # argument checks that return before touching the device
    assert lib.cch_hull(None, 4, 7, None, None, None) == -2
    assert lib.cch_hull(None, -1, 2, None, None, None) == -1
    assert lib.cch_workspace_bytes(-1, 2) == 0
    lib.cch_hull_f32soa.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]
    assert lib.cch_hull_f32soa(None, None, -1, 16, 16, None) == -1          # n < 0
    assert lib.cch_hull_f32soa(None, 64, 4, 16, 16, None) == -1             # x missing
    assert lib.cch_hull_f32soa(66, 64, 4, 16, 16, None) == -1               # x not 4-byte aligned
    assert lib.cch_hull_f32soa(64, 64, 4, None, 16, None) == -1             # out_idx missing
    assert lib.cch_hull_f32soa(64, 64, (1 << 30) + 1, 16, 16, None) == -4   # above 2^30 points


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_struct_layouts_match_header(tmp_path):
    c = tmp_path / "lay.c"
    c.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "cch.h"\nint main(void){\n'
                 'printf("%zu %zu %zu %zu %zu\\n", sizeof(cch_serve_config), offsetof(cch_serve_config, num_streams),'
                 ' offsetof(cch_serve_config, dtype), sizeof(cch_done), offsetof(cch_done, latency_ms));\n'
                 'return 0;}\n')
    exe = tmp_path / "lay"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(cch.ServeConfig), cch.ServeConfig.num_streams.offset, cch.ServeConfig.dtype.offset,
            ctypes.sizeof(cch.Done), cch.Done.latency_ms.offset]
    assert got == want
