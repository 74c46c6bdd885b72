"""Builds the CUDA shared library liblbm_gb300.so in-tree (sm_103a only).

Each translation unit is compiled by nvcc in parallel, then linked with
nvcc -shared.  The output sits next to this file, where the Python binding
loads it.
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "liblbm_gb300.so")
# (source, object name, extra nvcc flags): the stream/collide unit is compiled
# once per population storage format (LBM_FP32 = 0, LBM_FP16_SHIFT = 1,
# LBM_BF16_SHIFT = 2) so that its many kernel instances build in parallel
UNITS = [("lbm_api.cu", "lbm_api", []), ("lbm_kernels.cu", "lbm_kernels", []),
         ("lbm_collide.cu", "lbm_collide_fp32", ["-DLBM_COLLIDE_STORAGE=0"]),
         ("lbm_collide.cu", "lbm_collide_fp16", ["-DLBM_COLLIDE_STORAGE=1"]),
         ("lbm_collide.cu", "lbm_collide_bf16", ["-DLBM_COLLIDE_STORAGE=2"]),
         ("lbm_poisson.cu", "lbm_poisson", []), ("lbm_spectral.cu", "lbm_spectral", []),
         ("lbm_start.cu", "lbm_start", []), ("lbm_nn.cu", "lbm_nn", []),
         ("lbm_noalloc.cu", "lbm_noalloc", [])]
SOURCES = sorted({u[0] for u in UNITS})
HEADERS = ["lbm_internal.cuh", "lbm_lattice.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I", os.path.join(ROOT, "include")]


def _nvcc():
    exe = shutil.which("nvcc")
    if exe is None:
        cand = "/usr/local/cuda/bin/nvcc"
        if os.path.exists(cand):
            exe = cand
    if exe is None:
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return exe


def _compile(nvcc, unit, verbose):
    src, name, extra = unit
    obj = os.path.join(BUILD, name + ".o")
    cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return obj, r.stderr


def build_library(verbose: bool = False, force: bool = False) -> str:
    """Compiles and links the library; returns its path."""
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(CSRC, h) for h in HEADERS] + \
        [os.path.join(ROOT, "include", "lbm.h"), os.path.abspath(__file__)]
    if not force and os.path.exists(LIB):
        lib_t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= lib_t for d in deps):
            return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        results = list(ex.map(lambda u: _compile(nvcc, u, verbose), UNITS))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    objs = [o for o, _ in results]
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_library(verbose="-v" in sys.argv, force=True))
