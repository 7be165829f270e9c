"""Build liblabf.so (the CUDA engine behind include/labf.h) for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into a
shared library inside the package (``paper_2307_08006_gb300/_build``).
Cross-compiles without a GPU.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblabf.so")
# range-checked debug build (-DLA_CHECKS=1), objects in their own folder
BUILD_CHECKS = os.path.join(BUILD, "checks")
LIB_CHECKS = os.path.join(BUILD, "liblabf_checks.so")
SOURCES = ["labf_api.cu", "k_dyn.cu", "k_list.cu", "k_pairs.cu", "k_io.cu", "k_static.cu", "k_peak.cu"]
HEADERS = ["labf_internal.cuh", "labf_launch.h", "labf_dyn.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -ftz=true: FP32 denormals flush to zero (MD forces and positions never need
# them; rsqrtf then maps to a single special-function instruction)
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-ftz=true", "-Xcompiler", "-fPIC,-ffp-contract=off",
         "--expt-relaxed-constexpr", "-I", CSRC, "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(dep) > t for dep in deps)


def build(force: bool = False, verbose: bool = False, extra=(), checks: bool = False) -> str:
    """Compile the engine; checks=True builds the range-checked debug
    library (liblabf_checks.so, -DLA_CHECKS=1) instead."""
    odir, lib = (BUILD_CHECKS, LIB_CHECKS) if checks else (BUILD, LIB)
    extra = [*extra, "-DLA_CHECKS=1"] if checks else list(extra)
    os.makedirs(odir, exist_ok=True)
    nvcc = _nvcc()
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "labf.h")]
    objs, jobs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(odir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            jobs.append([nvcc, *ARCH, *FLAGS, *extra, "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(run, jobs))
    if force or jobs or not os.path.exists(lib):
        tmp = lib + f".tmp{os.getpid()}"
        run([nvcc, *ARCH, "-shared", "--cudart", "static", "-o", tmp, *objs])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [], checks="--checks" in sys.argv))
