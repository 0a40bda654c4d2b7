"""Builds libtnc.so in-tree: host C++ with g++, CUDA for sm_103a with nvcc, in parallel.

Objects go to paper_2504_09186_gb300/_build/, the library to paper_2504_09186_gb300/libtnc.so.
Rebuilds only what changed (any header change rebuilds everything).
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libtnc.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _cuda_home() -> str:
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "bin", "nvcc")):
            return cand
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    raise RuntimeError("nvcc not found (set CUDA_HOME)")


def _newest(paths) -> float:
    return max((os.path.getmtime(p) for p in paths), default=0.0)


def build(verbose: bool = False, jobs: int | None = None) -> str:
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(BUILD, exist_ok=True)
    headers = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + [
        os.path.join(ROOT, "include", "tnc.h")
    ]
    hdr_time = _newest(headers)
    stamp = os.path.join(BUILD, "defines.txt")
    defines = os.environ.get("TNC_NVCC_DEFINES", "")
    if not os.path.exists(stamp) or open(stamp).read() != defines:
        os.makedirs(BUILD, exist_ok=True)
        with open(stamp, "w") as f:
            f.write(defines)
    hdr_time = max(hdr_time, os.path.getmtime(stamp))
    inc = ["-I" + os.path.join(ROOT, "include"), "-I" + CSRC, "-I" + os.path.join(cuda, "include")]
    jobs_list = []
    objs = []
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cpp")) + glob.glob(os.path.join(CSRC, "*.cu"))):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(obj)
        if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), hdr_time, os.path.getmtime(__file__)):
            continue
        if src.endswith(".cu"):
            extra = os.environ.get("TNC_NVCC_DEFINES", "").split()
            cmd = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                   "-Xptxas", "-O3", *extra, *inc, "-c", src, "-o", obj]
        else:
            cmd = ["g++", "-O2", "-g", "-fPIC", "-std=c++17", "-Wall", "-Wno-unused-function", *inc, "-c", src, "-o", obj]
        jobs_list.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)

    if jobs_list:
        with ThreadPoolExecutor(max_workers=jobs or min(8, os.cpu_count() or 4)) as ex:
            list(ex.map(run, jobs_list))
    if jobs_list or not os.path.exists(LIB) or os.path.getmtime(LIB) < _newest(objs):
        cmd = [nvcc, ARCH, "-shared", "-o", LIB + ".tmp", *objs, "-L" + os.path.join(cuda, "lib64"), "-lcudart"]
        run(cmd)
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
