"""Build the CUDA library (libhipermotif.so) in-tree with nvcc for sm_103a.

Sources are compiled in parallel, one translation unit per file, then linked
into a shared library with the CUDA runtime linked statically.  Output:
``paper_2507_04130_gb300/_build/libhipermotif.so``; ``build(check=True)``
makes the bounds-checked ``libhipermotif_check.so`` (HM_CHECK=1) beside it.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libhipermotif.so")
# the bounds-checked build (HM_CHECK=1): same sources, own objects
BUILD_CHECK = os.path.join(BUILD, "check")
LIB_CHECK = os.path.join(BUILD, "libhipermotif_check.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", f"-I{INCLUDE}", f"-I{CSRC}"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return cand


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, check: bool = False) -> str:
    """Compile every source for sm_103a and link the shared library; returns its path.

    check=True builds the bounds-checked library (HM_CHECK=1) instead.
    """
    lib, objdir = (LIB_CHECK, BUILD_CHECK) if check else (LIB, BUILD)
    if not force and not _stale(lib):
        return lib
    nvcc = _nvcc()
    os.makedirs(objdir, exist_ok=True)
    defs = ["-DHM_CHECK=1"] if check else []

    def compile_one(src: str) -> str:
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, *COMMON, *defs, "-c", src, "-o", obj]
        if src.endswith(".cu"):
            cmd.insert(1, "-lineinfo")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = f"{lib}.tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-Xcompiler", "-fPIC", *objs, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
