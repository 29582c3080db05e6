"""Build libtgf.so (sm_103a) in-tree with nvcc; translation units compile in parallel.

    python -m paper_2107_03747_gb300.build          # or build() from Python
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libtgf.so")

SOURCES = ["stage.cu", "stage_tiles.cu", "measure.cu", "pack.cu", "api.cu", "peak.cu", "measure_static.cu", "mc.cu", "sun.cu", "coupling.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


LIB_CHECK = os.path.join(PKG, "libtgf_check.so")
BUILD_CHECK = os.path.join(PKG, "_build_check")


def _compile(src: str, verbose_ptxas: bool, check: bool = False) -> str:
    obj = os.path.join(BUILD_CHECK if check else BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj, "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
           "-I", os.path.join(ROOT, "include")] + (["-DTGF_CHECK"] if check else [])
    if src.endswith(".cu"):
        cmd += ARCH + ["-lineinfo"]
        if verbose_ptxas:
            cmd += ["-Xptxas", "-v"]
    else:
        cmd += ["-x", "c++"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    if verbose_ptxas and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def build(verbose_ptxas: bool = False, force: bool = False, check: bool = False) -> str:
    """Compile every source and link libtgf.so (check=True: the self-checking libtgf_check.so,
    compiled with -DTGF_CHECK); returns the library path."""
    lib = LIB_CHECK if check else LIB
    os.makedirs(BUILD_CHECK if check else BUILD, exist_ok=True)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "tgf.h")]
    if not force and os.path.exists(lib):
        lib_t = os.path.getmtime(lib)
        if all(os.path.getmtime(d) <= lib_t for d in deps):
            return lib
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose_ptxas, check), SOURCES))
    tmp = lib + ".tmp"
    cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose_ptxas="-v" in sys.argv, force="-f" in sys.argv))
