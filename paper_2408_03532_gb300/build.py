"""Build the CUDA library in-tree: paper_2408_03532_gb300/lib/libpft_gb300.so.

Every translation unit is compiled by its own nvcc (device code) or g++ (host
code) process in parallel for sm_103a only, then linked with nvcc -shared.
Host code is compiled with -ffp-contract=off so the x86_64 and aarch64 builds
round identically.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "lib")
LIB = os.path.join(OUT_DIR, "libpft_gb300.so")

CU_SOURCES = ["api.cu", "plan.cu", "fft.cu", "pie.cu", "pie_pft.cu", "pie_full.cu", "pie_lf.cu", "noalloc.cu", "pft_tc.cu", "pft_tc64.cu", "pft_tc_adj.cu", "pft_tc64_adj.cu", "pft_lf.cu"]
CPP_SOURCES = ["coeffs.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand) and shutil.which(cand) is None:
        raise RuntimeError("nvcc not found (set NVCC or put the CUDA toolkit on PATH)")
    return cand


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile (if needed) and return the path of the shared library."""
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "pft.h"))
    jobs, objs = [], []
    for src in CU_SOURCES + CPP_SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(OUT_DIR, src + ".o")
        objs.append(obj)
        if not force and not _stale(obj, [path] + headers):
            continue
        if src.endswith(".cu"):
            cmd = [nvcc, *ARCH, "-O3", "-std=c++17", "-lineinfo", "--extended-lambda",
                   "-Xcompiler", "-fPIC,-ffp-contract=off", "-c", path, "-o", obj]
        else:
            cmd = [os.environ.get("CXX", "g++"), "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off",
                   "-c", path, "-o", obj]
        jobs.append((src, cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    failed = []
    for src, cmd, proc in jobs:
        out, _ = proc.communicate()
        if verbose and out:
            sys.stdout.write(out)
        if proc.returncode != 0:
            failed.append((src, " ".join(cmd), out))
    if failed:
        msg = "\n\n".join(f"[{s}] {c}\n{o}" for s, c, o in failed)
        raise RuntimeError("CUDA library build failed:\n" + msg)
    if force or jobs or _stale(LIB, objs):
        cmd = [nvcc, *ARCH, "-shared", "--cudart", "shared", "-o", LIB, *objs]
        res = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        if res.returncode != 0:
            raise RuntimeError("link failed:\n" + " ".join(cmd) + "\n" + res.stdout)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
