"""Build the in-tree C-ABI library `libsp2.so` from csrc/ with nvcc for sm_103a.

Each .cu file compiles to its own object in parallel, then nvcc links the shared
library next to this file.  Run as `python -m paper_1507_02087_gb300.build`.

`debug=True` builds the same sources with SP2_DEVICE_CHECKS=1 into `libsp2_debug.so`
(objects in `_build_debug`): kernels check the indices they compute from the device
state against their buffers and report SP2_ERR_BOUNDS instead of touching memory out
of range.  `build_all` compiles both flavours in one pool.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsp2.so")
OUT_DIR_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libsp2_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsp2.so")


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _flavour(debug: bool) -> tuple[str, str, list[str]]:
    if debug:
        return OUT_DIR_DEBUG, LIB_DEBUG, ["-DSP2_DEVICE_CHECKS=1"]
    return OUT_DIR, LIB, []


def _compile_one(src: str, out_dir: str, defs: list[str], extra: list[str], verbose: bool) -> str:
    obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *defs, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
    if verbose:
        sys.stderr.write(r.stderr)
    return obj


def _link(objs: list[str], lib: str) -> str:
    tmp = lib + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-Xcompiler", "-fPIC", *objs, "-o", tmp, "-lcuda"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def build_all(debug_flavours=(False, True), verbose: bool = False, ptxas_info: bool = False) -> list[str]:
    """Compile every source of every requested flavour in one thread pool, then link each."""
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    jobs = []
    for debug in debug_flavours:
        out_dir, lib, defs = _flavour(debug)
        os.makedirs(out_dir, exist_ok=True)
        jobs += [(debug, src, out_dir, defs) for src in sources()]
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        futs = [(debug, ex.submit(_compile_one, src, out_dir, defs, extra, verbose or ptxas_info))
                for debug, src, out_dir, defs in jobs]
        objs = {debug: [] for debug in debug_flavours}
        for debug, f in futs:
            objs[debug].append(f.result())
    return [_link(objs[debug], _flavour(debug)[1]) for debug in debug_flavours]


def build(verbose: bool = False, ptxas_info: bool = False, debug: bool = False) -> str:
    return build_all((debug,), verbose=verbose, ptxas_info=ptxas_info)[0]


if __name__ == "__main__":
    if "--debug" in sys.argv:
        print(build(verbose=True, ptxas_info="--ptxas" in sys.argv, debug=True))
    else:
        print(build(verbose=True, ptxas_info="--ptxas" in sys.argv))
