"""Compile the CUDA sources into the in-tree shared library ``libctd_painn.so`` (sm_103a).

Every translation unit is compiled in parallel with nvcc for ``compute_103a/sm_103a``; host
code is compiled without floating-point contraction so that the host-side cell inverse used by
the neighbour test rounds exactly as documented in include/painn.h.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libctd_painn.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["api.cu", "neighbors.cu", "scan.cu", "model_fp32.cu", "md.cu", "prof.cu", "noalloc.cu", "gemm_bf16.cu", "edge_tc.cu", "edge_mma.cu", "serve.cu", "domain.cu", "selftest.cu", "model_local.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
              "--expt-relaxed-constexpr", "-Xptxas", "-v"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the engine")
    return path


def _newer(a: str, deps) -> bool:
    if not os.path.exists(a):
        return True
    t = os.path.getmtime(a)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "painn.h"))
    objs, jobs = [], []
    for src in SOURCES:
        s = os.path.join(SRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _newer(o, [s, *headers, __file__]):
            jobs.append((s, o))

    def compile_one(job):
        s, o = job
        cmd = [nvcc(), *ARCH, *NVCC_FLAGS, "-c", s, "-o", o + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {s}:\n{r.stderr}")
        os.replace(o + ".tmp", o)
        return s, r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, max(1, len(jobs)))) as ex:
        for s, log in ex.map(compile_one, jobs):
            with open(os.path.join(BUILD, os.path.basename(s) + ".ptxas.txt"), "w") as fh:
                fh.write(log)
            if verbose:
                print(f"compiled {os.path.basename(s)}", file=sys.stderr)
    if force or jobs or _newer(OUT, objs):
        tmp = OUT + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
               "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
        subprocess.check_call(cmd)
        os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
