"""Build the native library libamr_gb300.so in-tree (sm_103a only).

Translation units are compiled in parallel with nvcc (CUDA) and g++ (host
planner), then linked into ``paper_0910_5547_gb300/_build/libamr_gb300.so``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libamr_gb300.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", CSRC, "-I", INCLUDE]
# FP32 bulk kernels: approximate single-precision divide and square root.
FP32_FLAGS = ["-prec-div=false", "-prec-sqrt=false"]

UNITS = [
    ("amr_api.cu", []),
    ("amr_noalloc.cu", []),
    ("peak_probe.cu", []),
    ("ops_f64_euler.cu", []),
    ("ops_f32_euler.cu", FP32_FLAGS),
    ("ops_f64_mhd.cu", []),
    ("ops_f32_mhd.cu", FP32_FLAGS),
]
HOST_UNITS = ["hierarchy.cpp"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _sources():
    out = []
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            if f.endswith((".cu", ".cuh", ".h", ".cpp")):
                out.append(os.path.join(d, f))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False, extra: list | None = None) -> str:
    """Compile every translation unit (in parallel) and link the shared library."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    for src, flags in UNITS:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *NVCC_COMMON, *flags, *(extra or []), "-c", os.path.join(CSRC, src), "-o", obj]
        jobs.append((cmd, obj))
    for src in HOST_UNITS:
        obj = os.path.join(BUILD, src.replace(".cpp", ".o"))
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", "-I", CSRC, "-I", INCLUDE, "-c", os.path.join(CSRC, src),
               "-o", obj]
        jobs.append((cmd, obj))

    def run(job):
        cmd, _ = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        for log in ex.map(run, jobs):
            if verbose and log.strip():
                print(log, file=sys.stderr)
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *[o for _, o in jobs], "-lcudart", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
