"""Build the CUDA library (libbbe.so) for sm_103a with nvcc, in-tree.

Each translation unit is compiled in parallel and linked into
``paper_2108_02419_gb300/_lib/libbbe.so``.  The rollout translation units are compiled with
``--fmad=false``: the rollout arithmetic is pinned to explicit round-to-nearest
intrinsics and nothing may be contracted behind its back.

``build(checked=True)`` makes the checked build, ``_lib/checked/libbbe.so``: the same sources
with ``BBE_CHECKED`` defined, so that the rollout kernels check their computed indices and record
a failed check in the batch status instead of accessing out of range (the stand-in for a memory
checker).  The binding loads it when ``BBE_LIB`` names it.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
SO = os.path.join(LIBDIR, "libbbe.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
          "-I", INCLUDE, "--expt-relaxed-constexpr"]
# translation unit -> extra flags
UNITS = {
    "bbe_capi.cu": ["--fmad=false"],
    "bbe_rollout.cu": ["--fmad=false"],
    "bbe_win.cu": ["--fmad=false"],
    "bbe_win_time.cu": ["--fmad=false"],
    "bbe_win_place.cu": ["--fmad=false"],
    "bbe_win_place_time.cu": ["--fmad=false"],
    "bbe_noalloc.cu": ["--fmad=false"],
    "bbe_trajectory.cu": ["--fmad=false"],
    "bbe_surrogate.cu": [],
}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbbe.so")


def _inputs_digest() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            if name.endswith((".cu", ".cuh", ".h")):
                with open(os.path.join(d, name), "rb") as f:
                    h.update(name.encode() + f.read())
    h.update(repr((ARCH, COMMON, UNITS)).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile and link libbbe.so (or the checked build) if any source changed. Returns the
    library path."""
    libdir = os.path.join(LIBDIR, "checked") if checked else LIBDIR
    so = os.path.join(libdir, "libbbe.so")
    flags = ["-DBBE_CHECKED=1"] if checked else []
    os.makedirs(libdir, exist_ok=True)
    digest = _inputs_digest() + ("+checked" if checked else "")
    stamp = os.path.join(libdir, "build.stamp")
    if not force and os.path.exists(so) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return so
    cc = nvcc()
    objs = []

    def compile_unit(item):
        name, extra = item
        obj = os.path.join(libdir, name.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *COMMON, *flags, *extra, "-c", os.path.join(CSRC, name), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{res.stdout}\n{res.stderr}")
        if verbose and res.stderr:
            print(res.stderr)
        return obj

    with ThreadPoolExecutor(len(UNITS)) as ex:
        objs = list(ex.map(compile_unit, UNITS.items()))
    tmp = so + f".tmp{os.getpid()}"
    res = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"],
                         capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, so)
    with open(stamp, "w") as f:
        f.write(digest)
    return so


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
