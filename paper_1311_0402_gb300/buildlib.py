"""Build step of libdpd.so: nvcc for sm_103a, one object per translation unit
(compiled in parallel), linked into a shared library next to this file."""
from __future__ import annotations

import glob
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdpd.so")
# the checked variant: the same sources with DPD_CHECKED, whose kernels test
# the indices they read from device memory and report a bad one through the
# device error word instead of using it
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libdpd_checked.so")
INCLUDE = os.path.join(ROOT, "include")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")) + [
        os.path.abspath(__file__)]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, extra=None, checked: bool = False) -> str:
    """Compile every CUDA translation unit for sm_103a and link libdpd.so
    (checked: libdpd_checked.so, with DPD_CHECKED)."""
    LIB_OUT = LIB_CHECKED if checked else LIB
    BUILD_DIR = BUILD_CHECKED if checked else BUILD
    if not force and up_to_date(LIB_OUT):
        return LIB_OUT
    os.makedirs(BUILD_DIR, exist_ok=True)
    extra = list(extra or []) + (["-DDPD_CHECKED"] if checked else [])

    def compile_one(src):
        obj = os.path.join(BUILD_DIR, os.path.basename(src) + ".o")
        cmd = [NVCC, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, flush=True)
        return obj

    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = LIB_OUT + ".tmp.%d" % os.getpid()
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB_OUT)
    return LIB_OUT


def build_all(force: bool = False, verbose: bool = False) -> None:
    """Both variants, compiled side by side."""
    with ThreadPoolExecutor(max_workers=2) as ex:
        list(ex.map(lambda c: build(force=force, verbose=verbose, checked=c), (False, True)))


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
