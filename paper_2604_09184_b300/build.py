"""Build libnb.so (the CUDA library behind include/nb.h) for sm_103a.

    python -m paper_2604_09184_b300.build          # writes paper_2604_09184_b300/libnb.so
    python -m paper_2604_09184_b300.build --debug  # libnb_debug.so: -DNB_DEBUG index checks

nvcc cross-compiles without a GPU. The library is built in-tree so that it
travels with the repository to the machine that runs it.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libnb.so")
LIB_DEBUG = os.path.join(HERE, "libnb_debug.so")
SOURCES = ["abi.cu", "kick.cu", "drift.cu", "encounter.cu", "energy.cu", "peaks.cu",
           "noalloc.cu", "batch.cu", "adjoint.cu", "mathcheck.cu", "shard.cu"]
HEADERS = [os.path.join(CSRC, h) for h in ("nb_internal.cuh", "bs.cuh", "kepler.cuh")] + [
    os.path.join(ROOT, "include", "nb.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-I" + os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def needs_build(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in SOURCES] + HEADERS
    return any(os.path.getmtime(f) > t for f in deps)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None,
          debug: bool = False) -> str:
    """Compile and link the library; debug=True builds libnb_debug.so with the
    NB_DEBUG index checks (the binding loads it when NB_DEBUG=1)."""
    lib = LIB_DEBUG if debug else LIB
    if not (force or needs_build(lib)):
        return lib
    # one build at a time (ranks of a multi-process launch share the tree)
    import fcntl
    with open(os.path.join(HERE, ".build.lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        if not (force or needs_build(lib)):
            return lib
        return _build_locked(lib, verbose, extra, debug)


def _build_locked(lib, verbose, extra, debug):
    extra = list(extra or []) + (["-DNB_DEBUG"] if debug else [])
    objdir = os.path.join(HERE, "_build_debug" if debug else "_build")
    os.makedirs(objdir, exist_ok=True)
    objs = []
    procs = []
    for src in SOURCES:
        obj = os.path.join(objdir, src.replace(".cu", ".o"))
        cmd = [_nvcc()] + ARCH + NVCC_FLAGS + (extra or []) + ["-c", os.path.join(CSRC, src),
                                                                "-o", obj]
        if verbose:
            print(" ".join(cmd))
        procs.append((subprocess.Popen(cmd), cmd))
        objs.append(obj)
    for p, cmd in procs:
        if p.wait() != 0:
            raise RuntimeError("nvcc failed: " + " ".join(cmd))
    tmp = lib + ".tmp.%d" % os.getpid()
    subprocess.run([_nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"], check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None,
                debug="--debug" in sys.argv))
