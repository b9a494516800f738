"""Builds libgr.so (the CUDA library behind the C ABI) in-tree with nvcc for
sm_103a. Translation units compile in parallel, then link into one shared
library next to this file."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJDIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgr.so")
LIB_CHECKED = os.path.join(HERE, "libgr_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-Wall", "--expt-relaxed-constexpr"] + ARCH
HOST_FLAGS = ["-O3", "-std=c++17", "-fPIC", "-Wall"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgr.so")
    return cand


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                  if f.endswith((".cu", ".cpp")))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return hs


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, extra=(), suffix=".o") -> str:
    obj = os.path.join(OBJDIR, os.path.basename(src) + suffix)
    if not _stale(obj, [src, __file__] + _headers()):
        return obj
    cmd = [_nvcc(), "-c", src, "-o", obj, "-I", INCLUDE, "-I", CSRC] + NVCC_FLAGS + list(extra)
    if src.endswith(".cpp"):
        cmd = ([_nvcc(), "-x", "cu", "-c", src, "-o", obj, "-I", INCLUDE, "-I", CSRC] +
               NVCC_FLAGS + list(extra))
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{res.stdout}\n{res.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile every translation unit under csrc/ and link libgr.so (or,
    with checked=True, the bounds-checked diagnostic libgr_checked.so)."""
    os.makedirs(OBJDIR, exist_ok=True)
    srcs = sources()
    if force:
        for f in os.listdir(OBJDIR):
            os.remove(os.path.join(OBJDIR, f))
    extra = ["-DGR_CHECKED"] if checked else []
    suffix = ".checked.o" if checked else ".o"
    target = LIB_CHECKED if checked else LIB
    with cf.ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        objs = list(ex.map(lambda f: _compile(f, extra, suffix), srcs))
    if force or _stale(target, objs):
        tmp = target + f".tmp{os.getpid()}"
        cmd = [_nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-lcudart_static", "-lpthread", "-ldl", "-lrt"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
        os.replace(tmp, target)
    if verbose:
        print("built", target)
    return target


if __name__ == "__main__":
    import sys
    build(verbose=True, checked="--checked" in sys.argv)
