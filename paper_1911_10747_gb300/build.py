"""Build the CUDA library liblbm_gb300.so in-tree for sm_103a.

Seven translation units compiled in parallel by nvcc, then linked:
  csrc/lbm_fp64.cu     FP64 kernels, -fmad=false (plain rounding of each op)
  csrc/lbm_fp64fma.cu  the same FP64 kernels with FMA contraction
  csrc/lbm_fp32.cu     FP32 / FP16-storage kernels
  csrc/lbm_runtime.cu  host runtime and the C ABI of include/lbm.h
  csrc/lbm_static_diag.cu  the allocation-free diagnostics entry point
  csrc/lbm_server.cu   continuous-batching request loop (host code)
  csrc/lbm_peak.cu     FMA-throughput probe (the arithmetic rooflines' peak)
Host code is compiled with -ffp-contract=off so the FP64 constants derived
on the host round the same way on x86-64 and AArch64.
"""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "liblbm_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = {"lbm_fp64.cu": ["-fmad=false"], "lbm_fp64fma.cu": ["-fmad=true"], "lbm_fp32.cu": [], "lbm_runtime.cu": [],
         "lbm_static_diag.cu": ["-fmad=false"], "lbm_server.cu": [], "lbm_peak.cu": []}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))] + \
        [os.path.join(INCLUDE, "lbm.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    base = [nvcc(), "-std=c++17", "-O3", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
            "-I", INCLUDE, "-I", CSRC]
    procs = []
    objs = []
    for unit, extra in UNITS.items():
        obj = os.path.join(BUILD, unit.replace(".cu", ".o"))
        objs.append(obj)
        cmd = base + extra + ["-c", os.path.join(CSRC, unit), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((unit, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for unit, pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0:
            errors.append(f"{unit}:\n{out.decode(errors='replace')}")
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    tmp = LIB + ".tmp.%d" % os.getpid()
    subprocess.check_call([nvcc(), "-shared", *ARCH, "-o", tmp, *objs])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
