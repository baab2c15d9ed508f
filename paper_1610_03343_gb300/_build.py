"""Build libmd.so (the C-ABI CUDA library) in-tree with nvcc for sm_103a.

Each translation unit under csrc/ is compiled in parallel, then linked into
paper_1610_03343_gb300/libmd.so with the CUDA runtime linked statically, so the library
needs only the driver at run time.  `-Xptxas -v` output (registers, spills, shared
memory) goes to _build/ptxas.log.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libmd.so")
SOURCES = ["force.cu", "neigh.cu", "md_api.cu", "md_server.cu", "md_static.cu", "hcacf.cu", "peak.cu",
           "md_domain.cu"]
# force.cu is compiled as four units (its fp64 kernels of single systems and of pools and its
# fp32 kernels through the force_part_*.cu wrappers, and the rest) so that its large sets of
# kernel instantiations compile in parallel
# (each unit leaves the other units' helpers unused: their "declared but never referenced"
# diagnostics, number 177, are silenced for these units)
_QUIET = ["-Xcudafe", "--diag_suppress=177"]
UNITS = [("force_part_fp64.cu", _QUIET, "force_part_fp64.o"), ("force_part_fp64_pool.cu", _QUIET, "force_part_fp64_pool.o"),
         ("force_part_fp32.cu", _QUIET, "force_part_fp32.o"), ("force.cu", ["-DMD_FORCE_PART=0"] + _QUIET, "force.o")] + \
        [(src, [], os.path.splitext(src)[0] + ".o") for src in SOURCES if src != "force.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    raise RuntimeError("nvcc not found")


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "md.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    common = [cc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-I", INCLUDE, "-I", CSRC, "-Xptxas", "-v"]

    def compile_one(unit):
        src, defs, name = unit
        obj = os.path.join(BUILD, name)
        cmd = common + defs + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src} {' '.join(defs)}:\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        results = list(ex.map(compile_one, UNITS))
    with open(os.path.join(BUILD, "ptxas.log"), "w") as f:
        for (obj, log), (src, defs, _) in zip(results, UNITS):
            f.write(f"==== {src} {' '.join(defs)}\n{log}\n")
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [cc, *ARCH, "-shared", "-cudart", "static", "-o", tmp] + [o for o, _ in results] + ["-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print(open(os.path.join(BUILD, "ptxas.log")).read())
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
