"""Build the CUDA library in-tree: nvcc for sm_103a, one object per .cu file
compiled in parallel, linked into _build/libmgr_gb300.so.

Run as ``python -m paper_1904_05960_gb300.build`` or through
``__graft_entry__.build()``.  A build is reused only when the source hash
recorded beside it (and compiled into it, ``mgr_build_id``) equals the hash of
the current sources and flags.  The setup kernels are compiled with
``-fmad=false`` so that no multiply-add is contracted there: the setup's
integer outputs (C/F marks, strength graphs, sparsity patterns) depend on
separately rounded products and sums.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmgr_gb300.so")
STAMP = os.path.join(BUILD, "libmgr_gb300.build_id")
ROOT = os.path.dirname(HERE)

SOURCES = ["setup.cu", "apply.cu", "krylov.cu", "capi.cu", "noalloc.cu", "batched.cu"]
NO_FMAD = {"setup.cu"}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmgr_gb300")


def _flags(verbose=False):
    # host code: no contracted multiply-adds either (GCC contracts them by
    # default on Arm, and where it does depends on the surrounding code), so
    # the host Givens rotations and triangular solves of the single-system and
    # the batched FGMRES round identically on every machine
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-ffp-contract=off", "-I", os.path.join(ROOT, "include")]
    if verbose:
        common += ["-Xptxas", "-v"]
    return common


def source_hash():
    """First 16 hex digits of a SHA-256 over every CUDA source, the C header
    and the compiler flags: the identity of a build.  It is compiled into the
    library (mgr_build_id) and written beside it; build() rebuilds whenever
    the recorded hash differs, whatever the file times say."""
    h = hashlib.sha256()
    for f in sorted(os.listdir(CSRC)):
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read() + b"\0")
    with open(os.path.join(ROOT, "include", "mgr_gb300.h"), "rb") as fh:
        h.update(fh.read())
    flags = [f.replace(ROOT, "<root>") for f in _flags()]
    h.update(" ".join(flags + sorted(NO_FMAD)).encode())
    return h.hexdigest()[:16]


def built_hash():
    """Hash recorded by the last successful build, or None."""
    try:
        with open(STAMP) as f:
            return f.read().strip()
    except OSError:
        return None


def build(force=False, verbose=False):
    os.makedirs(BUILD, exist_ok=True)
    want = source_hash()
    if not force and os.path.exists(LIB) and built_hash() == want:
        return LIB
    cc = nvcc()
    common = _flags(verbose) + [f'-DMGR_BUILD_ID="{want}"']

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        flags = list(common)
        flags.append("-fmad=false" if src in NO_FMAD else "-fmad=true")
        cmd = [cc] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(STAMP + ".tmp", "w") as f:
        f.write(want + "\n")
    os.replace(STAMP + ".tmp", STAMP)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
