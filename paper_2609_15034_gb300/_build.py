"""Build libfastpair.so for sm_103a with nvcc (in-tree, no cmake).

Each CUDA translation unit compiles in its own nvcc process (in parallel),
then one link step makes the shared library next to this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libfastpair.so")

SOURCES = ["fp_api.cu", "fp_decode.cu", "fp_var16.cu", "fp_var12.cu", "fp_var8.cu", "fp_var12f.cu", "fp_batch.cu",
           "fp_plain.cu", "fp_serve.cu", "fp_sidecar.cu", "fp_rows.cu",
           "fp_varpk.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--cudart", "shared",
              "-Xptxas", "-v", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


# Sources of the single-column decode (fp_decode and its kernels): DRAM
# traffic counters taken on one build stay valid while these and the build
# flags are unchanged.
DECODE_PATH = ["fp_api.cu", "fp_decode.cu", "fp_var16.cu", "fp_var12.cu", "fp_var8.cu", "fp_var12f.cu", "fp_varpk.cu",
               "fp_variants.cuh", "fp_decoder.cuh", "fp_internal.h", "fp_warp.cuh"]


def decode_path_digest() -> str:
    return _inputs_digest(DECODE_PATH)


def _inputs_digest(names=None) -> str:
    h = hashlib.sha256()
    for name in sorted(names if names is not None else os.listdir(CSRC)) + ["../../include/fastpair.h"]:
        path = os.path.normpath(os.path.join(CSRC, name))
        if os.path.isfile(path):
            h.update(name.encode())
            with open(path, "rb") as f:
                h.update(f.read())
    # flags without this checkout's absolute paths, so the digest names the
    # sources and options, not where they sit
    flags = [f.replace(INCLUDE, "<include>").replace(CSRC, "<csrc>") for f in ARCH + NVCC_FLAGS]
    h.update(" ".join(flags).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


def _compile(src: str) -> tuple[str, str]:
    obj = os.path.join(BUILD, src.replace(".cu", ".o"))
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if sources changed) and return the library path."""
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "stamp")
    digest = _inputs_digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return LIB
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(_compile, SOURCES))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    with open(os.path.join(BUILD, "ptxas.log"), "w") as f:
        for _, log in results:
            f.write(log)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "--cudart", "shared", "-o", tmp, *[o for o, _ in results]]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(digest)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
