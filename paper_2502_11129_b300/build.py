"""Build the in-tree CUDA library (sm_103a) with nvcc.

    python -m paper_2502_11129_b300.build

The library is compiled for sm_103a only (B300).  It is placed next to this
file (``libb3sim.so``) so that it travels with the source tree.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

LIBS = {
    "libb3sim.so": (["b3sim.cu", "chain.cu"], ["step_kernel.cuh", "step_common.cuh", "free_body.cuh", "model_pack.h",
                                               "chain_kernel.cuh", "chain_layout.h"], "b3sim.h"),
    "libb3sur.so": (["b3sur.cu"], [], "b3sur.h"),
    "libb3cpu.so": (["b3cpu.cu"], ["step_common.cuh", "free_body.cuh", "model_pack.h"], "b3cpu.h"),
}


def _stale(out, srcs):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(s) > t for s in srcs)


def build(force: bool = False, verbose: bool = False) -> list[str]:
    built = []
    for lib, (srcs, deps, header) in LIBS.items():
        out = os.path.join(HERE, lib)
        paths = [os.path.join(CSRC, s) for s in srcs]
        dep_paths = paths + [os.path.join(CSRC, d) for d in deps] + [os.path.join(INCLUDE, header)]
        if not force and not _stale(out, dep_paths):
            continue
        cmd = [NVCC, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
               "-I" + INCLUDE, "-o", out, *paths]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        built.append(out)
    return built


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
