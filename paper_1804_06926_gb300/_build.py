"""In-tree build of the CUDA library ``libtc.so`` for sm_103a (GB300).

Every translation unit under ``csrc/`` is compiled by nvcc in parallel and
linked into one shared library that exports the C ABI of ``include/tc.h``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build", platform.machine())
LIB = os.path.join(HERE, "libtc.so")
STAMP = LIB + ".arch"
# The TC_DEBUG build: every count kernel checks its indexes and table invariants,
# raises a bit of the device check word (tc_check) and skips the bad access.
DEBUG_LIB = os.path.join(HERE, "libtc_debug.so")
SOURCES = ["tc_build.cu", "tc_count.cu", "tc_sort.cu", "tc_api.cu", "tc_serve.cu", "tc_noalloc.cu", "tc_metrics.cu", "tc_support.cu", "tc_labels.cu", "tc_fused.cu"]
HEADERS = [os.path.join(CSRC, "tc_internal.cuh"), os.path.join(ROOT, "include", "tc.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtc.so")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile and link libtc.so (or, with debug=True, libtc_debug.so)."""
    bdir = os.path.join(BUILD, "debug") if debug else BUILD
    lib = DEBUG_LIB if debug else LIB
    stamp = lib + ".arch"
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    flags = NVCC_FLAGS + (["-DTC_DEBUG=1"] if debug else [])
    objs, jobs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(bdir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + HEADERS):
            jobs.append([cc] + flags + ["-I", os.path.join(ROOT, "include"), "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(run, jobs))
    if force or jobs or _stale(lib, objs) or not arch_ok(stamp):
        tmp = lib + f".{os.getpid()}.tmp"
        run([cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"])
        os.replace(tmp, lib)
        write_stamp(stamp)
    return lib


def arch_ok(stamp: str) -> bool:
    """True when the library next to `stamp` was built on this machine type."""
    try:
        with open(stamp) as f:
            return f.read().strip() == platform.machine()
    except OSError:
        return False


def write_stamp(stamp: str) -> None:
    with open(stamp, "w") as f:
        f.write(platform.machine() + "\n")


if __name__ == "__main__":
    print(build(verbose=True))
