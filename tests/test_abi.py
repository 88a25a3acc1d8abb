"""The C-ABI library loads on a machine without a GPU, exports every function that
include/*.h declares, and the Python binding's struct layouts match the C ones."""
import ctypes
import glob
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_1507_02087_gb300", "libsp2.so")


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(sp2_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def built():
    if not os.path.exists(LIB):
        from paper_1507_02087_gb300 import build
        build.build()
    return LIB


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sp2_create", "sp2_run", "sp2_run_host", "sp2_get_info", "sp2_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    lib = ctypes.CDLL(built)   # loads without a GPU
    for n in declared_functions():
        assert hasattr(lib, n)


def test_status_strings_without_gpu(built):
    from paper_1507_02087_gb300 import sp2
    L = sp2.lib()
    assert L.sp2_status_string(0) == b"ok"
    assert L.sp2_status_string(3).startswith(b"non-finite")
    o = sp2.sp2_opts()
    L.sp2_default_opts(ctypes.byref(o))
    assert (o.max_iter, o.guard, o.qtilde) == (200, 1, 1.8)


def test_invalid_arguments_rejected_before_any_cuda_call(built):
    from paper_1507_02087_gb300 import sp2
    L = sp2.lib()
    h = ctypes.c_void_p()
    assert L.sp2_create(0, 0, 0, None, ctypes.byref(h)) == 1
    assert L.sp2_create(10, 11, 0, None, ctypes.byref(h)) == 1
    assert L.sp2_create(10, -1, 0, None, ctypes.byref(h)) == 1
    assert L.sp2_create(10, 5, 99, None, ctypes.byref(h)) == 7
    bad = sp2.sp2_opts(0, 1, 1.8)
    assert L.sp2_create(10, 5, 0, ctypes.byref(bad), ctypes.byref(h)) == 1
    assert h.value is None
    assert L.sp2_run(None, None, None, None) == 1
    assert L.sp2_get_info(None, None) == 1
    L.sp2_destroy(None)


def test_struct_layout_matches_c():
    from paper_1507_02087_gb300 import sp2
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "sp2.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(sp2_opts), offsetof(sp2_opts, qtilde),
         sizeof(sp2_info), offsetof(sp2_info, lambda_min), offsetof(sp2_info, loop_ms), offsetof(sp2_info, v),
         offsetof(sp2_info, trace), offsetof(sp2_info, p));
  return 0;
}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = list(map(int, subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()))
    py = [ctypes.sizeof(sp2.sp2_opts), sp2.sp2_opts.qtilde.offset, ctypes.sizeof(sp2.sp2_info),
          sp2.sp2_info.lambda_min.offset, sp2.sp2_info.loop_ms.offset, sp2.sp2_info.v.offset, sp2.sp2_info.trace.offset,
          sp2.sp2_info.p.offset]
    assert vals == py
