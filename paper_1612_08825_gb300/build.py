"""Build the fastttc CUDA library in-tree for sm_103a.

``python -m paper_1612_08825_gb300.build`` (or ``__graft_entry__.build()``) compiles
every ``csrc/*.cu`` in parallel with nvcc and links ``_lib/libfastttc.so``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT_DIR, "libfastttc.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "-I" + INCLUDE, "-I" + CSRC]
STAMP = os.path.join(OUT_DIR, "flags.txt")


def extra_flags() -> list:
    """FASTTTC_CHECK=1 in the environment builds the checked library: the TTC passes compare
    every frame read and pyramid store with the extent of their call and report one outside it
    in the records (FT_FLAG_BOUNDS) instead of making it."""
    return ["-DFT_CHECK=1"] if os.environ.get("FASTTTC_CHECK", "0") not in ("", "0") else []


def nvcc_path() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def needs_build() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(STAMP):
        return True
    with open(STAMP) as f:
        if f.read() != " ".join(extra_flags()):
            return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _deps())


def build_library(force: bool = False, verbose: bool = False) -> str:
    if not force and not needs_build():
        return LIB
    _compile_and_link(_sources(), extra_flags(), LIB, verbose)
    with open(STAMP, "w") as f:
        f.write(" ".join(extra_flags()))
    return LIB


def build_checked_ttc(verbose: bool = False) -> str:
    """The TTC part of the library (ttc.cu, api.cu) built with FT_CHECK, in-tree as
    _lib/libfastttc_ttc_checked.so: for tests of the checked build."""
    out = os.path.join(OUT_DIR, "libfastttc_ttc_checked.so")
    srcs = [os.path.join(CSRC, "ttc.cu"), os.path.join(CSRC, "ttc_fused.cu"), os.path.join(CSRC, "api.cu")]
    if os.path.exists(out) and all(os.path.getmtime(f) <= os.path.getmtime(out) for f in _deps()):
        return out
    _compile_and_link(srcs, ["-DFT_CHECK=1"], out, verbose)
    return out


def _compile_and_link(sources, flags, out, verbose):
    nvcc = nvcc_path()
    os.makedirs(OUT_DIR, exist_ok=True)
    objs = []
    cmds = []
    for src in sources:
        obj = os.path.join(OUT_DIR, os.path.basename(src) + f".{os.getpid()}.o")
        objs.append(obj)
        cmds.append([nvcc, *ARCH, *NVCC_FLAGS, *flags, "-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, file=sys.stderr)

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(cmds), os.cpu_count() or 1))) as ex:
        list(ex.map(run, cmds))
    tmp = out + f".{os.getpid()}.tmp"
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")
    run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lcufft", "-L" + cuda_lib,
         "-Xlinker", "-rpath=" + cuda_lib, "-lrt", "-ldl", "-lpthread"])
    os.replace(tmp, out)
    for o in objs:
        os.remove(o)


if __name__ == "__main__":
    print(build_library(force="--force" in sys.argv, verbose=True))
