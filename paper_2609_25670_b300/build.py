"""Build step of the CUDA library: nvcc for sm_103a into liblbm.so beside this file."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = [os.path.join(HERE, "csrc", "lbm_api.cu")]
DEPS = SRC + [os.path.join(HERE, "csrc", n) for n in ("lbm_kernels.cuh", "lbm_common.cuh", "lbm_aux.cuh", "lbm_transport.cuh", "lbm_strip.cuh")] + \
    [os.path.join(ROOT, "include", "lbm.h")]
LIB = os.path.join(HERE, "liblbm.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
# No -split-compile: with the module split across threads the code of one
# kernel depended on how unrelated kernels were partitioned (the FP32 flow
# strip ran 4 % slower in one split than in another; a 16-bit strip spilled
# in one).  One optimiser pass over the whole module takes about five minutes.
FLAGS = ["-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
         "-Xcompiler", "-fPIC", "-shared", "--expt-relaxed-constexpr"]


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    """Compile the library if any source is newer than liblbm.so; return its path."""
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in DEPS):
            return LIB
    cmd = [NVCC] + FLAGS + (["-Xptxas", "-v"] if verbose_ptxas else []) + SRC + ["-o", LIB]
    subprocess.check_call(cmd)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose_ptxas="-v" in sys.argv)
    print(LIB)
