"""Build the CUDA library in-tree: one nvcc process per translation unit, then one link.

sm_103a only.  -fmad=false keeps every floating-point expression rounded as written (the exact
decisions of the method depend on it); FP32 fused multiply-adds are written out explicitly.
-ftz=true flushes subnormal FP32 results to zero: on the FP32 transport path a photon count
below FLT_MIN (about 1e-38 of a box's source photons per step) becomes 0, so its share counts
as absorbed where it is, and the packet, which carries nothing, is not transported further.
FP64 arithmetic (the FP64 path, the chemistry, every exact decision) is not affected.
"""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libtraphic_rt.so")
SOURCES = ["rt_api.cu", "rt_knn.cu", "rt_scan.cu", "rt_transport.cu", "rt_chem.cu"]
HEADERS = ["rt_internal.cuh", "rt_knn.cuh"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-ftz=true", "-Xcompiler",
                "-fPIC,-ffp-contract=off", "-Xptxas", "-warn-spills"]


def _inputs_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    files.append(os.path.join(HERE, "..", "include", "traphic_rt.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _inputs_mtime():
        return LIB

    def compile_one(src):
        obj = os.path.join(OUT, src.replace(".cu", ".o"))
        cmd = [NVCC] + FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".{os.getpid()}.tmp"
    r = subprocess.run([NVCC] + ARCH + ["-shared", "-o", tmp] + objs, capture_output=True,
                       text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
