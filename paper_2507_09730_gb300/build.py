"""In-tree build of ``libfrw.so`` (the C-ABI library of include/frw.h) for sm_103a.

Two translation units compiled in parallel with nvcc, linked into a shared
library next to this file.  Host code is compiled without floating-point
contraction so that FP64 geometry decisions are plain IEEE operations.

``build(checked=True)`` makes ``libfrw_checked.so``, the same library compiled
with -DFRW_CHECKS: the kernels test every lattice coordinate, queue, list and
table index and record / batch offset before using it, and on a failed test set
an error bit (reported as FRW_EDEVICE) instead of touching memory out of range.
The binding loads it when the environment has FRW_CHECKED=1.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libfrw.so")
LIB_CHECKED = os.path.join(HERE, "libfrw_checked.so")
SOURCES = ["frw_kernels.cu", "frw_runtime.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-I" + INCLUDE, "-Xcompiler", "-fPIC,-ffp-contract=off",
         "--expt-relaxed-constexpr"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "frw.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    bdir = os.path.join(HERE, "_build", "checked" if checked else "release")
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc, *ARCH, *FLAGS, *(["-DFRW_CHECKS"] if checked else []), "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("nvcc failed: " + " ".join(cmd) + "\n" + out.decode(errors="replace"))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed: " + r.stdout.decode(errors="replace"))
    os.replace(tmp, lib)
    return lib


def build_all(force: bool = False) -> list:
    """Both libraries, compiled concurrently."""
    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(2) as ex:
        return list(ex.map(lambda c: build(force=force, checked=c), (False, True)))


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
