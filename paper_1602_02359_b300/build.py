"""Build step of the CUDA library (sm_103a), run in-tree.

    python -m paper_1602_02359_b300.build

Compiles csrc/fargo_api.cu (which includes every kernel) into
libfargo_b300.so next to this file with nvcc.  Host code is compiled without
floating-point contraction so that the FP64 geometry tables match a plain
IEEE evaluation.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC_DIR = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libfargo_b300.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def sources():
    out = []
    for d in (SRC_DIR, os.path.join(os.path.dirname(HERE), "include")):
        for f in sorted(os.listdir(d)):
            if f.endswith((".cu", ".cuh", ".h")):
                out.append(os.path.join(d, f))
    return out


def nvcc_cmd(out=LIB, extra=()):
    return ["nvcc", ARCH, "-O3", "-lineinfo", "-std=c++17", "--shared", "-Xcompiler", "-fPIC,-ffp-contract=off",
            "-o", out, os.path.join(SRC_DIR, "fargo_api.cu"), *extra]


def build(force=False, verbose=False):
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(s) <= t for s in sources()):
            return LIB
    tmp = LIB + ".tmp"
    cmd = nvcc_cmd(tmp, ("-Xptxas", "-v") if verbose else ())
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
