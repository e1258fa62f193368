"""Builds the CUDA library liblco.so in-tree for sm_103a with nvcc.

Each .cu file under csrc/ is compiled to an object in parallel, then linked
into ``_lib/liblco.so`` against the shared CUDA runtime.  Nothing here needs
a GPU: nvcc cross-compiles on any host.
"""
from __future__ import annotations

import concurrent.futures as cf
import fcntl
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_lib")
SO_PATH = os.path.join(OUT_DIR, "liblco.so")

ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-pthread", "-DLCO_BUILD_ARCH=1030",
          "-I", INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr"]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblco.so")
    return cand


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h")) + [__file__]


def is_stale() -> bool:
    if not os.path.exists(SO_PATH):
        return True
    t = os.path.getmtime(SO_PATH)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    """Compile and link liblco.so; returns its path.  Raises on any failure."""
    os.makedirs(OUT_DIR, exist_ok=True)
    lock_path = os.path.join(OUT_DIR, ".build.lock")
    with open(lock_path, "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        if not force and not is_stale():
            return SO_PATH
        nvcc = _nvcc()
        flags = COMMON + ARCH_FLAGS + list(extra_flags or [])
        objs = []

        def compile_one(src):
            obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + ".o")
            cmd = [nvcc, "-c", src, "-o", obj] + flags
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
            if verbose and r.stderr:
                print(r.stderr)
            return obj

        with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
            objs = list(ex.map(compile_one, _sources()))
        tmp = SO_PATH + f".tmp{os.getpid()}"
        cuda_lib = "/usr/local/cuda/lib64"
        cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH_FLAGS + \
            ["-cudart", "shared", "-lpthread", "-Xlinker", f"-rpath,{cuda_lib}"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of liblco.so failed:\n{r.stderr}")
        os.replace(tmp, SO_PATH)
        for o in objs:
            try:
                os.remove(o)
            except OSError:
                pass
        return SO_PATH


if __name__ == "__main__":
    print(build(force=True, verbose=True))
