"""Benchmark of the B300 FARGO3D hydro step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl b300|reference]
                    [--workload disk3d|disk2d] [--no-cpu-baseline] [--no-e2e]

Default workload: the 3D spherical adiabatic planet disk, 1536 x 512 x 96
active cells, FP32 fields with FP64 islands (Courant step, v0, shift, planet
offset, sums).  A step is one full update of every active cell (flow chart
cells 2-12); the metric is cell-updates per second.  The state (about 2.6 GB
of fields plus 5 GB of scratch) is far larger than the 126 MB L2, so no L2
flush is needed between steps.  A secondary measurement runs the 2D
cylindrical planet disk (256 x 768) in FP64, flushing L2 before every timed
step (its 30 MB state would otherwise stay L2-resident).

Multi-GPU: the hot path does not shard; with N > 1 ranks (torchrun) every
rank advances its own replica and `value` is the total over ranks.

--impl reference times the plain FP64 CPU oracle on a bounded slab of the same
workload on the host cores (rank 0 only).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

# Algorithmic bytes per active cell of each kernel (FP32; FP64 doubles them):
# every field the kernel must read or write, once.  3D adiabatic step: state
# rho, e, vx, vy, vz; six momenta; six viscous stresses.
ALG_FIELDS_3D = {
    "cfl_screen": 5,        # read rho, e, vx, vy, vz
    "cfl_exact": 0,         # re-reads only the candidate rings (a few)
    "substep1": 5 + 3,      # read the state, write 3 velocities
    "artvisc": 5 + 4,       # read rho, e, 3 v; write 3 v, e
    "visc_tau": 4 + 6,      # read rho, 3 v; write 6 stresses
    "visc_apply": 10 + 3,   # read 6 stresses, rho, 3 v; write 3 v
    "transport_x": 5 + 8,   # read rho, e, 3 v; write rho, e, 6 momenta
    "transport_y": 9 + 8,   # read 8 quantities + v_y; write 8
    "transport_z": 9 + 8,
    "orbital": 8 + 8,       # read and write 8 quantities
    "newvel": 7 + 3,        # read rho, 6 momenta; write 3 v
}
# 2D isothermal step: state rho, vx, vy; four momenta; three stresses.
ALG_FIELDS_2D_ISO = {
    "cfl_screen": 3, "cfl_exact": 0, "substep1": 3 + 2, "artvisc": 3 + 2, "visc_tau": 3 + 3,
    "visc_apply": 6 + 2, "transport_x": 3 + 5, "transport_y": 6 + 5, "orbital": 5 + 5, "newvel": 5 + 2,
}

# DRAM bytes per active cell and launch measured by ncu (dram__bytes_read.sum
# + dram__bytes_write.sum) on the 1536 x 128 x 48 case of the 3D disk, FP32,
# with the kernel sources whose SHA-256 prefix is KERNEL_SRC_HASH (see
# profiles/disk3d_fp32_step_ncu.md).  Traffic grows in proportion to the
# cells, so a full launch is this figure times the cells; once the sources
# change the figures no longer apply and the bench reports null.
TRAFFIC_PER_CELL_3D = {"cfl_screen": 23.25, "substep1": 33.35, "artvisc": 36.51, "visc_tau": 36.62, "visc_apply": 54.64, "transport_x": 60.58, "transport_y": 64.64, "transport_z": 65.79, "orbital": 70.83, "newvel": 54.01}
KERNEL_SRC_HASH = "a7f09bbf09ba8ed5"


def kernel_source_hash():
    d = os.path.join(ROOT, "paper_1602_02359_b300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh")):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class Clocks:
    """nvidia-smi sampler (SM clock, max clock, throttle reasons) during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[1]))
                mx.append(float(s[2]))
                for n, v in zip(names, s[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except Exception:
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_workload(name):
    if name == "disk3d":
        w = W.disk3d()
        return w, "disk3d-sph-adiabatic-planet-1536x512x96", True
    if name == "disk2d":
        w = W.disk2d()
        return w, "disk2d-cyl-isothermal-planet-768x256", False
    if name == "disk3d-small":
        # profiling case: the same disk on 1536 x 128 x 48 cells (state still far above L2)
        w = W.disk3d(ny=128, nz=48)
        return w, "disk3d-sph-adiabatic-planet-1536x128x48", True
    raise SystemExit(f"unknown workload {name}")


def cpu_baseline(wname, budget_s=20.0):
    """The plain FP64 oracle on a bounded slab of the workload, host cores."""
    import oracle
    if wname == "disk3d":
        w = W.disk3d(slab=(200, 24, 36, 24))
        sample = "oracle on a 1536x24x24 slab of the 1536x512x96 disk (rows 200-223, planes 36-59), frozen ghosts"
    else:
        w = W.disk2d()
        sample = "oracle on the full 768x256 disk"
    o = oracle.Oracle(w)
    st = w.copy().state
    t = 0.0
    n = 0
    t0 = time.perf_counter()
    while True:
        t += o.step(st, t, w.t_end)
        n += 1
        el = time.perf_counter() - t0
        if el > budget_s or n >= 50:
            break
    return {"value": w.cells * n / el, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"{sample}; {n} steps in {el:.1f} s"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    wname = args.workload
    _, label, _ = make_workload_meta(wname)
    import oracle
    if wname == "disk3d":
        w = W.disk3d(slab=(200, 24, 36, 24))
        sample = "1536x24x24 slab of the 1536x512x96 disk per step"
    else:
        w = W.disk2d()
        sample = "full 768x256 disk per step"
    o = oracle.Oracle(w)
    st = w.copy().state
    t = 0.0
    for _ in range(args.warmup):
        t += o.step(st, t, w.t_end)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        t += o.step(st, t, w.t_end)
    el = time.perf_counter() - t0
    val = w.cells * args.steps / el
    line = {"metric": "cell-updates/s", "value": val, "unit": "cell-updates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": label, "sample": sample},
            "cpu_baseline": {"value": val, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def make_workload_meta(wname):
    if wname == "disk3d":
        return None, "disk3d-sph-adiabatic-planet-1536x512x96", True
    return None, "disk2d-cyl-isothermal-planet-768x256", False


def fp64_plain_disk2d(torch, fb, steps=50, warmup=5):
    """2D planet disk in FP64, L2 flushed before every timed step."""
    w = W.disk2d()
    stream = torch.cuda.Stream()
    c = fb.Fargo(w, fb.F64, stream=stream.cuda_stream)
    c.set_state(w.state)
    c.set_time(0.0, 1e30)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            c.step(want_dt=False)
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            c.step(want_dt=False)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
    _, _, _, err = c.scalars()
    c.close()
    ms = tot / steps
    return {"workload": "disk2d-cyl-isothermal-planet-768x256", "dtype": "f64",
            "value": w.cells / (ms * 1e-3), "unit": "cell-updates/s", "ms_per_step": ms,
            "l2": "flushed (512 MB write) before every timed step", "err": err}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--workload", default="disk3d", choices=["disk3d", "disk2d", "disk3d-small"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import paper_1602_02359_b300 as fb

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    w, label, fp32 = make_workload(args.workload)
    prec = fb.F32 if fp32 else fb.F64
    stream = torch.cuda.Stream()
    c = fb.Fargo(w, prec, stream=stream.cuda_stream)
    c.set_state(w.state)
    c.set_time(0.0, 1e30)
    nl = c.launches_per_step()
    esz = 4 if fp32 else 8

    # ---- warm-up, then the timed region (CUDA graph replays on `stream`)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            c.step(want_dt=False)
        torch.cuda.synchronize()
        clk = Clocks(dev)
        clk.start()
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            c.step(want_dt=False)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1) / args.steps
        clocks = clk.stop()
        # ---- per-kernel device time over the same number of steps (live roofline)
        per = {}
        for _ in range(args.steps):
            for name, t in c.profile_step():
                per.setdefault(name, []).append(t)
    t_dev, dt_last, nsteps, err = c.scalars()
    if err:
        raise SystemExit(f"device error {err} during the benchmark")

    ms_t = torch.tensor([ms], device="cuda")
    if ws > 1:
        torch.distributed.all_reduce(ms_t, op=torch.distributed.ReduceOp.MAX)
    ms_max = float(ms_t.item())
    value = w.cells * ws / (ms_max * 1e-3)

    # roofline of the dominant kernel
    hbm, peak_kind = peaks()
    avg = {k: sum(v) / len(v) for k, v in per.items()}
    top = max(avg, key=avg.get)
    table = ALG_FIELDS_3D if (w.nz > 1 and not w.iso) else ALG_FIELDS_2D_ISO
    alg_bytes = table.get(top, 0) * esz * w.cells
    achieved = alg_bytes / (avg[top] * 1e-3) / 1e9
    share = {k: round(v / sum(avg.values()), 4) for k, v in sorted(avg.items(), key=lambda x: -x[1])}
    per_kernel = {k: {"ms": round(v, 4), "alg_GBps": round(table.get(k, 0) * esz * w.cells / (v * 1e-3) / 1e9, 1)}
                  for k, v in sorted(avg.items(), key=lambda x: -x[1]) if k in table}
    traffic = None
    if (fp32 and w.nz > 1 and not w.iso and top in TRAFFIC_PER_CELL_3D
            and kernel_source_hash() == KERNEL_SRC_HASH):
        traffic = int(TRAFFIC_PER_CELL_3D[top] * w.cells)
    roofline = {"bound": "hbm", "kernel": top, "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "peak_kind": f"{peak_kind} copy bandwidth",
                "alg_bytes_per_launch": alg_bytes, "ms_per_launch": round(avg[top], 4), "traffic": traffic,
                "kernel_share": share, "per_kernel": per_kernel}

    # ---- end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        names = ["rho", "e", "vx", "vy", "vz"] if not w.iso else ["rho", "vx", "vy", "vz"]
        if w.nz == 1:
            names = [n for n in names if n != "vz"]
        hdt = torch.float32 if fp32 else torch.float64
        host = {n: torch.empty(w.shape, dtype=hdt, pin_memory=True) for n in names}
        for n in names:
            host[n].numpy()[...] = w.state[n]
        bytes_io = sum(h.numel() * h.element_size() for h in host.values())
        ksteps = max(3, min(args.steps, 10))
        with torch.cuda.stream(stream):
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            for _ in range(ksteps):
                for n in names:
                    c.set_field(n, host[n].numpy())
                c.step(want_dt=False)
                for n in names:
                    c.get_field(n, out=host[n].numpy())
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            barrier()
        e2e = {"value": w.cells * ws * ksteps / el, "unit": "cell-updates/s",
               "h2d_bytes_per_step": bytes_io, "d2h_bytes_per_step": bytes_io, "steps": ksteps,
               "note": "every step uploads the full state from pinned host memory and reads it back"}
    c.close()
    del c

    fp64 = None
    if rank == 0 and not args.no_fp64 and args.workload == "disk3d":
        with torch.cuda.device(dev):
            fp64 = fp64_plain_disk2d(torch, fb)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and ws == 1 and args.workload != "disk3d-small":
        cpu = cpu_baseline(args.workload)

    if rank == 0:
        line = {
            "metric": "cell-updates/s", "value": value, "unit": "cell-updates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if fp32 else "f64", "data": "synthetic",
            "config": {"workload": label, "cells": w.cells, "steps_advanced": int(nsteps),
                       "precision": "FP32 fields, FP64 dt/v0/shift/planet offset/sums" if fp32 else "FP64",
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "l2": "inputs larger than L2 (state %.1f GB)" % (w.cells * 21 * esz / 1e9),
                       "graph": True},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": nl * args.steps,
            "clocks": clocks,
        }
        if fp64 is not None:
            line["fp64_plain"] = fp64
            line["fp32_vs_fp64_plain"] = value / fp64["value"]
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
