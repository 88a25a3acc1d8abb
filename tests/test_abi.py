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
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
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


def test_status_strings_and_defaults_without_gpu(built):
    from paper_1507_02087_gb300 import sp2
    L = sp2.lib()
    assert L.sp2_status_string(0) == b"ok"
    assert L.sp2_status_string(3).startswith(b"non-finite")
    o = sp2.sp2_opts()
    L.sp2_default_opts(ctypes.byref(o))
    assert (o.max_iter, o.guard, o.qtilde, o.corrections, o.refine_steps, o.refine_fp64, o.launch_mode,
            o.history, o.tile, o.norm) == (200, 1, 1.8, 1, 2, 0, 0, 0, 0, 0)


def test_invalid_arguments_rejected_before_any_cuda_call(built):
    from paper_1507_02087_gb300 import sp2
    L = sp2.lib()
    h = ctypes.c_void_p()
    assert L.sp2_create(0, 0, 0, None, ctypes.byref(h)) == 1
    assert L.sp2_create(10, 11, 0, None, ctypes.byref(h)) == 1
    assert L.sp2_create(10, -1, 0, None, ctypes.byref(h)) == 1
    assert L.sp2_create(10, 5, 99, None, ctypes.byref(h)) == 7
    for bad in (sp2.sp2_opts(0, 1, 1.8, 1, 2, 0, 0, 0, 0, 0),      # max_iter
                sp2.sp2_opts(10, 2, 1.8, 1, 2, 0, 0, 0, 0, 0),     # guard
                sp2.sp2_opts(10, 1, 0.0, 1, 2, 0, 0, 0, 0, 0),     # qtilde
                sp2.sp2_opts(10, 1, 1.8, 2, 2, 0, 0, 0, 0, 0),     # corrections
                sp2.sp2_opts(10, 1, 1.8, 1, 1, 0, 0, 0, 0, 0),     # refine_steps
                sp2.sp2_opts(10, 1, 1.8, 1, 2, 3, 0, 0, 0, 0),     # refine_fp64
                sp2.sp2_opts(10, 1, 1.8, 1, 2, 0, 5, 0, 0, 0),     # launch_mode
                sp2.sp2_opts(10, 1, 1.8, 1, 2, 0, 0, 3, 0, 0),     # history
                sp2.sp2_opts(10, 1, 1.8, 1, 2, 0, 0, 0, 3, 0),     # tile
                sp2.sp2_opts(10, 1, 1.8, 1, 2, 0, 0, 0, 0, 3)):    # norm
        assert L.sp2_create(10, 5, 1, ctypes.byref(bad), ctypes.byref(h)) == 1
        assert h.value is None
    # the spectral-norm stop (norm = 2) exists on the FP64 path and for single tensor-core
    # problems, not for tensor-core batches
    spec = sp2.sp2_opts(10, 1, 1.8, 1, 2, 0, 0, 0, 0, 2)
    Ns = (ctypes.c_int64 * 2)(10, 12)
    occ = (ctypes.c_int64 * 2)(5, 6)
    assert L.sp2_create_batch(2, Ns, occ, 1, ctypes.byref(spec), ctypes.byref(h)) == 7
    assert h.value is None
    assert L.sp2_run(None, None, None, None) == 1
    assert L.sp2_run_host(None, None, None, None) == 1
    assert L.sp2_get_info(None, None) == 1
    assert L.sp2_set_bounds(None, None) == 1
    assert L.sp2_test_set_perturbation(None, None, 0) == 1
    assert L.sp2_test_tc_gemm(None, 256, 1, 0, 0, 0, 0, None, None) == 1
    L.sp2_destroy(None)


def test_struct_layout_matches_c():
    from paper_1507_02087_gb300 import sp2
    fields_opts = ["max_iter", "guard", "qtilde", "corrections", "refine_steps", "refine_fp64", "launch_mode",
                   "history", "tile", "norm"]
    fields_info = ["status", "n_iter", "stop_reason", "hist_len", "lambda_min", "lambda_max", "loop_ms",
                   "v", "trace", "p", "tile"]
    prints = [f"offsetof(sp2_opts, {f})" for f in fields_opts] + ["sizeof(sp2_opts)"]
    prints += [f"offsetof(sp2_info, {f})" for f in fields_info] + ["sizeof(sp2_info)"]
    src = ("#include <stdio.h>\n#include <stddef.h>\n#include \"sp2.h\"\nint main(void) {\n" +
           "".join(f'  printf("%zu\\n", (size_t){p});\n' for p in prints) + "  return 0;\n}\n")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = list(map(int, subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()))
    py = [getattr(sp2.sp2_opts, f).offset for f in fields_opts] + [ctypes.sizeof(sp2.sp2_opts)]
    py += [getattr(sp2.sp2_info, f).offset for f in fields_info] + [ctypes.sizeof(sp2.sp2_info)]
    assert vals == py


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # no CPU fallback: without the built library the first call raises
    from paper_1507_02087_gb300 import sp2
    monkeypatch.setattr(sp2, "_lib", None)
    monkeypatch.setattr(sp2, "LIB_PATH", str(tmp_path / "libsp2.so"))
    with pytest.raises(RuntimeError, match="not built"):
        sp2.lib()
    with pytest.raises(RuntimeError):
        sp2.Purifier(64, 32, "fp64")


def test_binding_types_every_declared_function(built):
    # the ctypes binding sets argument types for every C-ABI function, so no call goes through
    # ctypes' default int conversion of pointers and 64-bit sizes
    from paper_1507_02087_gb300 import sp2
    L = sp2.lib()
    untyped = [n for n in declared_functions() if getattr(L, n).argtypes is None]
    assert not untyped, f"no argtypes in the binding: {untyped}"


LIB_DEBUG = os.path.join(ROOT, "paper_1507_02087_gb300", "libsp2_debug.so")


@pytest.fixture(scope="module")
def built_debug():
    if not os.path.exists(LIB_DEBUG):
        from paper_1507_02087_gb300 import build
        build.build(debug=True)
    return LIB_DEBUG


def test_debug_library_exports_the_same_boundary_and_says_so(built, built_debug):
    out = subprocess.run(["nm", "-D", "--defined-only", built_debug], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert not [n for n in declared_functions() if n not in exported]
    dbg = ctypes.CDLL(built_debug)
    rel = ctypes.CDLL(built)
    dbg.sp2_build_device_checks.restype = ctypes.c_int32
    rel.sp2_build_device_checks.restype = ctypes.c_int32
    assert dbg.sp2_build_device_checks() == 1 and rel.sp2_build_device_checks() == 0
    dbg.sp2_status_string.restype = ctypes.c_char_p
    assert dbg.sp2_status_string(8).startswith(b"device-side bounds")
