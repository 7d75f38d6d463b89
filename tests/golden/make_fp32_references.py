"""Write the FP64 oracle states that the long FP32 parity runs are judged against.

    python tests/golden/make_fp32_references.py [--threads N] [c2] [c4]

c2: the 768 x 256 planet disk run to 10 orbits (t = 20 pi).
c4: the two smallest disks of the 256-disk sweep (seed 1602, members 156
    and 126, 384 x 128 and 393 x 131) run to 500 orbits.
Each file stores the active density and the two velocity components in
float32 (the comparisons are at 1e-5 .. 1e-3 relative, far above float32
rounding), the end time and the oracle's step count.  Only the oracle and
the seeded workloads are called: no value comes from the CUDA library.
"""
import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle            # noqa: E402
import workloads as W    # noqa: E402


def run(w, path, label):
    o = oracle.Oracle(w)
    st = w.copy().state
    t0 = time.time()
    t, n = o.run(st, 0.0, w.t_end)
    vy = st["vy"][w.gz:w.gz + w.nz, w.gy:w.gy + w.ny + 1]
    np.savez_compressed(path, rho=w.active(st["rho"]).astype(np.float32),
                        vx=w.active(st["vx"]).astype(np.float32), vy=vy.astype(np.float32),
                        t_end=np.float64(t), steps=np.int64(n))
    print(f"{label}: {n} steps to t = {t!r} in {time.time() - t0:.0f} s -> {os.path.basename(path)}", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count())
    ap.add_argument("which", nargs="*", default=["c2", "c4"])
    a = ap.parse_args()
    oracle.set_threads(a.threads)
    if "c2" in a.which:
        run(W.disk2d(), os.path.join(HERE, "disk2d_768x256_10orbits.npz"), "disk2d 768x256, 10 orbits")
    if "c4" in a.which:
        P = W.batch_params()
        for i in (156, 126):
            w = W.batch_instance(P[i])
            run(w, os.path.join(HERE, f"batch_member{i}_500orbits.npz"),
                f"sweep member {i} ({w.nx}x{w.ny}), 500 orbits")


if __name__ == "__main__":
    main()
