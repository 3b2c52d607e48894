"""Builds libcip.so (the sm_103a CUDA library) in-tree with nvcc.

Each translation unit compiles in parallel; the column-pass kernels are split
into one object per precision.  Usage:  python -m paper_2006_08303_gb300.build
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libcip.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

# (source, extra defines, object name)
UNITS = [
    ("abi.cu", [], "abi.o"),
    ("passA.cu", [], "passA.o"),
    ("colpass.cu", [], "colpass.o"),
    ("fft_kernels.cu", [], "fft_kernels.o"),
    ("factor.cu", [], "factor.o"),
    ("noalloc.cu", [], "noalloc.o"),
    ("colsplit.cu", [], "colsplit.o"),
    ("convdict.cu", [], "convdict.o"),
    ("convdict3d.cu", [], "convdict3d.o"),
    ("wavelet.cu", [], "wavelet.o"),
    ("serve.cu", [], "serve.o"),
]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags(extra_ptxas: bool = False):
    f = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", *ARCH]
    if extra_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _tuning_defines():
    # optional register-budget overrides, e.g. CIP_NVCC_DEFINES="-DPASSA_RT32=64 -DPASSB_RT=80"
    return [d for d in os.environ.get("CIP_NVCC_DEFINES", "").split() if d.startswith("-D")]


def _compile(unit, verbose: bool):
    src, defs, obj = unit
    cmd = [nvcc(), *_flags(verbose), *defs, *_tuning_defines(), "-c", os.path.join(CSRC, src),
           "-o", os.path.join(BUILD, obj)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return unit, r.returncode, r.stdout + r.stderr


def _stale() -> bool:
    if not os.path.exists(OUT):
        return True
    t = os.path.getmtime(OUT)
    for f in os.listdir(CSRC):
        if os.path.getmtime(os.path.join(CSRC, f)) > t:
            return True
    inc = os.path.join(os.path.dirname(HERE), "include", "cip.h")
    return os.path.exists(inc) and os.path.getmtime(inc) > t


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    """Compile and link libcip.so; returns its path.  Raises on any compiler error."""
    if not force and not _stale():
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    jobs = jobs or min(len(UNITS), os.cpu_count() or 1)
    logs = []
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        for unit, rc, log in ex.map(lambda u: _compile(u, verbose), UNITS):
            if rc != 0:
                raise RuntimeError(f"nvcc failed on {unit[0]} {unit[1]}:\n{log}")
            logs.append((unit[2], log))
    objs = [os.path.join(BUILD, u[2]) for u in UNITS]
    tmp = OUT + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}{r.stderr}")
    os.replace(tmp, OUT)
    if verbose:
        for name, log in logs:
            print(f"== {name}\n{log}")
    return OUT


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(OUT)
