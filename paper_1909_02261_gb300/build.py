"""Builds libtenscol.so (sm_103a) in-tree with nvcc.

The translation units compile in parallel, one `-gencode` each, and link into
one shared library next to this file (``paper_1909_02261_gb300/lib``).  A
second library, libtenscol_bounds.so, links the same objects except the
one-hot kernels, compiled with TC_BOUNDS=1 (device-side index checks of the
class walk that report TC_ERR_DEVICE_BOUNDS).
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
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libtenscol.so")
LIB_BOUNDS = os.path.join(LIBDIR, "libtenscol_bounds.so")
SOURCES = ["tenscol.cu", "tc_onehot.cu", "tc_dense.cu", "tc_relaxed.cu", "tc_noalloc.cu", "tc_multi.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtenscol")


def _digest() -> str:
    h = hashlib.sha256()
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(f.encode())
            h.update(open(os.path.join(CSRC, f), "rb").read())
    h.update(open(os.path.join(INCLUDE, "tenscol.h"), "rb").read())
    h.update(" ".join(ARCH + FLAGS).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if stale) and return the path of libtenscol.so."""
    os.makedirs(LIBDIR, exist_ok=True)
    stamp = LIB + ".sha256"
    digest = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(LIB_BOUNDS) and os.path.exists(stamp) and \
            open(stamp).read().strip() == digest:
        return LIB
    nvcc = _nvcc()
    objdir = os.path.join(LIBDIR, "_obj")
    os.makedirs(objdir, exist_ok=True)

    def compile_one(job):
        src, tag, extra = job
        obj = os.path.join(objdir, src.replace(".cu", tag + ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}{tag}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    jobs = [(src, "", []) for src in SOURCES] + [("tc_onehot.cu", "_bounds", ["-DTC_BOUNDS=1"])]
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        objs = list(ex.map(compile_one, jobs))
    plain, bounds_obj = objs[:len(SOURCES)], objs[-1]
    with_bounds = [bounds_obj if src == "tc_onehot.cu" else o for src, o in zip(SOURCES, plain)]
    for target, inputs in ((LIB, plain), (LIB_BOUNDS, with_bounds)):
        tmp = target + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *inputs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, target)
    with open(stamp, "w") as f:
        f.write(digest)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
