"""Build step of the CUDA library (sm_103a), run in-tree.

    python -m paper_1602_02359_b300.build

Compiles the translation units csrc/fargo_api.cu (single-instance entry
points), csrc/fargo_batch.cu (batched engine) and csrc/mlp.cu (surrogate
network) in parallel with nvcc, then links them into libfargo_b300.so next
to this file.  Host code is compiled
without floating-point contraction so that the FP64 geometry tables match a
plain IEEE evaluation.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

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


UNITS = ("fargo_api.cu", "fargo_batch.cu", "mlp.cu")
OBJ_DIR = os.path.join(HERE, "_build")
FLAGS = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off"]


def nvcc_cmd(unit, out, extra=()):
    """Compile command of one translation unit into an object file."""
    return ["nvcc", *FLAGS, "-c", "-o", out, os.path.join(SRC_DIR, unit), *extra]


def build(force=False, verbose=False):
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(s) <= t for s in sources()):
            return LIB
    os.makedirs(OBJ_DIR, exist_ok=True)
    objs = [os.path.join(OBJ_DIR, u.replace(".cu", ".o")) for u in UNITS]
    extra = ("-Xptxas", "-v") if verbose else ()
    with ThreadPoolExecutor(len(UNITS)) as ex:
        procs = list(ex.map(lambda a: subprocess.run(nvcc_cmd(*a, extra)), zip(UNITS, objs)))
    for u, p in zip(UNITS, procs):
        if p.returncode != 0:
            raise subprocess.CalledProcessError(p.returncode, f"nvcc {u}")
    tmp = LIB + ".tmp"
    subprocess.check_call(["nvcc", ARCH, "--shared", "-o", tmp, *objs])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
