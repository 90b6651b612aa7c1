"""In-tree build of the CUDA library ``libfvlbm.so`` for sm_103a (GB300).

The host translation unit is compiled by g++ and the device one by nvcc, in parallel; nvcc
links them into one shared library under ``paper_1812_00394_gb300/_build/``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libfvlbm.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
SOURCES = ["fvlbm_host.cpp", "fvlbm_kernels.cu", "fvlbm_noalloc.cu", "fvlbm_peak.cu"]
HEADERS = ["fvlbm_internal.h", "fvlbm_dual.h", "fvlbm_adjoint.cuh", "fvlbm_adjoint_sst.cuh",
           "fvlbm_fused_fv.cuh"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libfvlbm")
    return cand


def _stamp() -> str:
    return os.path.join(BUILD, "config.txt")


def _config() -> str:
    return f"FVLBM_FUSED_BLOCK={os.environ.get('FVLBM_FUSED_BLOCK', '')}"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    try:
        with open(_stamp()) as fh:
            if fh.read() != _config():
                return True
    except OSError:
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.join(INCLUDE, "fvlbm.h"),
                                                                 os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


# Single-precision square root of the kernels within 1 ulp instead of correctly rounded
# (double is untouched).  Measured on the sweep: the SST update 16 % faster, the FP32 error
# against FP64 unchanged.  (Approximate division everywhere, or denormals flushed to zero,
# did raise the error on a 200k-cell SST airfoil: to 1.2e-4 and 3.0e-5 against 1.2e-5 after
# 1,000 steps; the stage algebra and the SST gradients take the fast quotient, see sdiv in the
# kernels.)
FP32_FLAGS = ["-prec-sqrt=false"]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libfvlbm.so if any source is newer than it; return its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", INCLUDE, "-I", CSRC]
    fb = os.environ.get("FVLBM_FUSED_BLOCK")   # optional build-time tuning of the fused block
    if fb:
        inc += [f"-DFVLBM_FUSED_BLOCK={int(fb)}"]
    host_o = os.path.join(BUILD, "fvlbm_host.o")
    dev_o = os.path.join(BUILD, "fvlbm_kernels.o")
    na_o = os.path.join(BUILD, "fvlbm_noalloc.o")
    pk_o = os.path.join(BUILD, "fvlbm_peak.o")
    cmds = [
        ["g++", "-O2", "-std=c++17", "-fPIC", "-fopenmp", *inc, "-c",
         os.path.join(CSRC, "fvlbm_host.cpp"), "-o", host_o],
        [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
         *FP32_FLAGS, *inc, "-c", os.path.join(CSRC, "fvlbm_kernels.cu"), "-o", dev_o],
        [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         *inc, "-c", os.path.join(CSRC, "fvlbm_noalloc.cu"), "-o", na_o],
        [nvcc, ARCH, "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
         *inc, "-c", os.path.join(CSRC, "fvlbm_peak.cu"), "-o", pk_o],
    ]
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
             for c in cmds]
    outs = [p.communicate()[0] for p in procs]
    for c, p, o in zip(cmds, procs, outs):
        if p.returncode != 0:
            raise RuntimeError(f"build failed: {' '.join(c)}\n{o}")
        if verbose and o:
            print(o, file=sys.stderr)
    with open(os.path.join(BUILD, "ptxas.log"), "w") as fh:
        fh.write(outs[1])
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc, ARCH, "-shared", "-Xcompiler", "-fopenmp", host_o, dev_o, na_o,
                           pk_o, "-o", tmp])
    os.replace(tmp, LIB)
    with open(_stamp(), "w") as fh:
        fh.write(_config())
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
