"""Build step of the CUDA library: nvcc, sm_103a only, in-tree.

Compiles every ``csrc/*.cu`` translation unit in parallel and links
``lib/libffg_gb300.so`` (CUDA runtime linked statically, so the library
loads without a toolkit on the library path).  Rebuilds only when a source
or header is newer than the library.  ``build(checked=True)`` makes the
bounds-checked variant ``lib/libffg_gb300_checked.so`` (-DFFG_CHECKED: every
index a kernel derives from caller data is checked before its access and a
failed check is counted instead of reading or writing out of bounds); it has
the same entry points and is loaded in place of the normal library when
``FFG_LIB=checked`` is set.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB_DIR = os.path.join(PKG, "lib")
LIB_PATH = os.path.join(LIB_DIR, "libffg_gb300.so")
CHECKED_LIB_PATH = os.path.join(LIB_DIR, "libffg_gb300_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the FFG library needs the CUDA toolkit to build")


def _inputs():
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    deps = srcs + glob.glob(os.path.join(CSRC, "*.cuh")) + [
        os.path.join(ROOT, "include", "ffg.h"), os.path.abspath(__file__)]
    return srcs, deps


def up_to_date(checked: bool = False) -> bool:
    lib = CHECKED_LIB_PATH if checked else LIB_PATH
    if not os.path.exists(lib):
        return False
    _, deps = _inputs()
    return os.path.getmtime(lib) >= max(os.path.getmtime(d) for d in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    lib = CHECKED_LIB_PATH if checked else LIB_PATH
    if not force and up_to_date(checked):
        return lib
    nvcc = _nvcc()
    srcs, _ = _inputs()
    obj_dir = os.path.join(BUILD, "checked") if checked else BUILD
    os.makedirs(obj_dir, exist_ok=True)
    os.makedirs(LIB_DIR, exist_ok=True)
    flags = NVCC_FLAGS + (["-DFFG_CHECKED"] if checked else [])

    def compile_one(src):
        obj = os.path.join(obj_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *ARCH, *flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose=True, checked="--checked" in sys.argv[1:]))
