"""Builds libhough.so in-tree with nvcc for sm_103a (one object per .cu, compiled in parallel).

The "phase" variant (_build_phase/libhough.so) defines HOUGH_PHASE_TIMERS: the fused kernel
then counts the cycles of each phase of an item (hough_phase_cycles); results are unchanged."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libhough.so")
VARIANTS = {None: (OUT_DIR, []), "phase": (os.path.join(PKG, "_build_phase"), ["-DHOUGH_PHASE_TIMERS"])}

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + [
        os.path.join(ROOT, "include", "hough.h")]


def lib_path(variant=None) -> str:
    return os.path.join(VARIANTS[variant][0], "libhough.so")


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=(), variant=None) -> str:
    """Compiles every .cu under csrc/ and links libhough.so (of `variant`); returns its path."""
    out_dir, defines = VARIANTS[variant]
    lib = lib_path(variant)
    if not force and not _stale(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    objs = []

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [NVCC, *ARCH, *FLAGS, *defines, *extra_flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, _sources()))
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys

    print(build(force=True, verbose=True, extra_flags=["-Xptxas", "-v"],
                variant="phase" if "--phase" in sys.argv[1:] else None))
