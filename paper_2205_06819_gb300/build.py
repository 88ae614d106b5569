"""Builds libbang.so (the C-ABI CUDA library) in-tree for sm_103a.

Each .cu translation unit is compiled by nvcc in parallel, then linked into
``paper_2205_06819_gb300/libbang.so`` against the shared CUDA runtime.  A stamp of the
sources and flags skips the build when nothing changed.

``build(checked=True)`` (or ``python -m paper_2205_06819_gb300.build --checked``) builds
the checked library ``libbang_checked.so`` with -DBANG_CHECKED: every kernel checks the
indexes it computes and the entry points return BANG_E_BOUNDS instead of touching memory
out of range.  The binding loads it instead of libbang.so when BANG_CHECKED=1 is set in
the environment.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libbang.so")
LIB_CHECKED = os.path.join(HERE, "libbang_checked.so")
BUILD_DIR = os.path.join(HERE, "_build")
BUILD_DIR_CHECKED = os.path.join(HERE, "_build_checked")
CHECKED_FLAGS = ["-DBANG_CHECKED"]

SOURCES = ["bang_api.cu", "bang_forward.cu", "bang_adjoint.cu", "bang_plain.cu", "bang_fp64.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbang.so")


def _present_sources():
    return [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def _stamp(flags) -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(CSRC, name), "rb") as f:
                h.update(name.encode() + f.read())
    with open(os.path.join(ROOT, "include", "bang.h"), "rb") as f:
        h.update(f.read())
    h.update(" ".join(ARCH + flags).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    lib_path = LIB_CHECKED if checked else LIB
    build_dir = BUILD_DIR_CHECKED if checked else BUILD_DIR
    flags = FLAGS + (CHECKED_FLAGS if checked else [])
    stamp_path = lib_path + ".stamp"
    stamp = _stamp(flags)
    if not force and os.path.exists(lib_path) and os.path.exists(stamp_path):
        with open(stamp_path) as f:
            if f.read() == stamp:
                return lib_path
    os.makedirs(build_dir, exist_ok=True)
    cc = nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(build_dir, src.replace(".cu", ".o"))
        cmd = [cc] + ARCH + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj

    srcs = _present_sources()
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = [cc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path)
    with open(stamp_path, "w") as f:
        f.write(stamp)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
