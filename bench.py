"""Benchmark of the B300 FARGO3D hydro step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl b300|reference]
                    [--workload batch256|disk3d|disk2d|disk3d-small|batch-small|batch-medium]
                    [--no-cpu-baseline] [--no-e2e] [--no-fp64] [--no-single]

Default workload (batch256): the batched parameter sweep of 256 independent
2D cylindrical isothermal planet disks, Nr ~ U{128..512}, Nphi = 3 Nr,
q log-uniform [1e-5, 1e-3], h U[0.03, 0.07], nu log-uniform [1e-6, 1e-5]
(seed 1602), about 88 M active cells in total, FP32 fields with FP64 islands
(Courant step, v0, shift, planet offset), advanced by the batched engine:
one launch per phase over every disk, each disk with its own Courant step,
the step captured as a CUDA graph.  A step is one full update of every
active cell of every disk (flow chart cells 2-12); the metric is
cell-updates per second.  The sweep's run length (500 orbits, ~1e5 steps
per disk) only multiplies the step count: the cost of a step does not depend
on the state, so the bench times K steps from the initial state.  The state
(about 16 GB) is far larger than the 126 MB L2; no flush is needed.

Reported beside it: the same metric for the plain FP64 single-instance
step (the 768 x 256 disk, L2 flushed before every timed step) and their
ratio, and the single-instance FP32 step of the 3D spherical adiabatic
planet disk (1536 x 512 x 96) with its own roofline.

Multi-GPU: the hot path does not shard; with N > 1 ranks (torchrun) every
rank advances its own replica and `value` is the total over ranks.

--impl reference times the plain FP64 CPU oracle on a bounded sample of the
same workload on the host cores (rank 0 only).
"""
import argparse
import hashlib
import json
import math
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
TRAFFIC_PER_CELL_3D = {"cfl_screen": 21.53, "substep1": 33.01, "artvisc": 36.07, "visc_tau": 36.22, "visc_apply": 54.3, "transport_x": 56.23, "transport_y": 64.36, "transport_z": 65.51, "orbital": 57.46, "newvel": 41.23}
KERNEL_SRC_HASH = "815003752373fcff"

# The same for the batched step: DRAM bytes per active cell of every batched
# phase (all its launches of one step summed), measured on batch-medium (the
# first 32 disks of the 256-disk sweep, 1.6 GB of state), with the sources
# whose hash is BATCH_SRC_HASH (profiles/batch256_fp32_step_ncu.md).
TRAFFIC_PER_CELL_BATCH = {"cfl_screen": 12.96, "substep1": 18.67, "artvisc": 19.2, "visc_tau": 21.82, "visc_apply": 33.29, "transport_x": 24.43, "transport_y": 42.82, "orbital": 32.25, "newvel": 27.0}
BATCH_SRC_HASH = "4b76d5a7c7c5f691"


# DRAM bytes per launch of the direct-sum planet force on the 3D disk (ncu,
# full size, one pass: dram__bytes_read.sum + dram__bytes_write.sum, median of
# four launches), valid while kernels_planet.cuh keeps PFORCE_SRC_HASH
# (profiles/planet_force_disk3d_ncu.md).
PFORCE_TRAFFIC_3D = 302.91e6
PFORCE_SRC_HASH = "17d5c57fa4766b55"

# Sources of the single-instance step's kernels (the traffic table above
# applies to them only).
STEP_SOURCES = ("fargo_internal.cuh", "tma.cuh", "kernels_bc_cfl.cuh", "kernels_source.cuh",
                "kernels_transport.cuh", "context.cuh", "fargo_api.cu")


def kernel_source_hash(sources=STEP_SOURCES):
    d = os.path.join(ROOT, "paper_1602_02359_b300", "csrc")
    h = hashlib.sha256()
    for f in sources:
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


def bf16_peak():
    """Dense bf16 tensor peak (TFLOP/s): the burst figure for a kernel timed alone."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1800.0, "fallback"


def bench_surrogate(torch, reps=20):
    """The surrogate network kernels (tcgen05 products): ensemble inference
    latency for the 205 evaluation queries of the sweep, one training step
    (batch 256, 4 members), and forward throughput at a large batch against
    the bf16 tensor peak.  Seeded random weights and inputs; the timing does
    not depend on their values."""
    import paper_1602_02359_b300.mlp as fm
    from paper_1602_02359_b300.surrogate import Ensemble
    dims = W.mlp_dims()
    flop_per_sample = 2 * sum(a * b for a, b in zip(dims[:-1], dims[1:]))
    ens = Ensemble(k=4, seed=1602, max_batch=65536)
    g = torch.Generator(device="cpu").manual_seed(1602)
    xq = torch.rand(205, dims[0], generator=g).cuda()
    st = ens.stream

    def timed(fn, n):
        with torch.cuda.stream(st):
            for _ in range(3):
                fn()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(n):
                fn()
            e1.record(st)
            e1.synchronize()
        return e0.elapsed_time(e1) / n

    ms_query = timed(lambda: ens.predict(xq), reps)
    xb = torch.rand(256, dims[0], generator=g).cuda()
    tb = torch.rand(256, dims[-1], generator=g).cuda()
    ms_train = timed(lambda: [n.train_step(xb, tb) for n in ens.nets], reps)
    big = 65536
    xl = torch.rand(big, dims[0], generator=g).cuda()
    yl = torch.empty(big, dims[-1], device="cuda")
    ms_big = timed(lambda: ens.nets[0].forward(xl, yl), reps)
    for n in ens.nets:
        n.status()
    ens.close()
    peak, kind = bf16_peak()
    tflops = flop_per_sample * big / (ms_big * 1e-3) / 1e12
    return {"network": "x".join(map(str, dims)), "ensemble": 4,
            "query_205_ms": round(ms_query, 4), "train_step_4_members_batch256_ms": round(ms_train, 4),
            "forward_batch65536_ms": round(ms_big, 4),
            "roofline": {"bound": "tensor", "achieved": round(tflops, 1), "peak": peak, "unit": "TFLOP/s",
                         "frac": round(tflops / peak, 4), "peak_kind": f"{kind} bf16 dense (burst)",
                         "flop_per_sample": flop_per_sample}}


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


class Ranks:
    """Rank plumbing of a replicas run: one process per GPU under torchrun
    (NCCL, reductions on the GPU), each rank stepping its own copy of the
    workload; the tests drive the same code with gloo on the CPU.  There is
    no collective on the data path: only the barrier around the timed region
    and the reductions of the timings."""

    def __init__(self, torch, backend="nccl", device="cuda"):
        self.torch = torch
        self.ws, self.rank, self.local = dist_env()
        self.device = device
        if self.ws > 1:
            torch.distributed.init_process_group(backend)

    def barrier(self):
        if self.ws > 1:
            self.torch.distributed.barrier()

    def max(self, x):
        t = self.torch.tensor([float(x)], device=self.device, dtype=self.torch.float64)
        if self.ws > 1:
            self.torch.distributed.all_reduce(t, op=self.torch.distributed.ReduceOp.MAX)
        return float(t.item())

    def aggregate(self, cells, ms, e2e_rate=None):
        """Whole-job figures of weak scaling: every rank processed `cells`
        per step; the job's step time is the slowest rank's, so the rate is
        ranks x cells / max time; the end-to-end rate likewise from the
        slowest rank's end-to-end rate."""
        ms_max = self.max(ms)
        value = cells * self.ws / (ms_max * 1e-3)
        e2e = None if e2e_rate is None else self.ws / self.max(1.0 / e2e_rate)
        return value, ms_max, e2e

    def close(self):
        if self.ws > 1:
            self.torch.distributed.destroy_process_group()


BATCH_WORKLOADS = {"batch256": 256, "batch-small": 16, "batch-medium": 32}


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


def batch_label(n):
    return f"batch{n}-disk2d-cyl-isothermal-planet-Nr128..512-Nphi3Nr-seed1602"


def batch_params(wname):
    """Parameters of the sweep (batch-small: the first 16 draws at a quarter
    of the radial resolution; batch-medium: the first 32 disks of the 256-disk
    sweep at full resolution; both profiling cases still far above L2)."""
    n = BATCH_WORKLOADS[wname]
    ps = W.batch_params(n=n, seed=1602)
    if wname == "batch-medium":
        ps = W.batch_params(n=256, seed=1602)[:n]
    if wname == "batch-small":
        ps = [dict(p, ny=max(32, p["ny"] // 4), nx=3 * max(32, p["ny"] // 4)) for p in ps]
    return ps


def make_batch(fb, ps, stream):
    """One FP32 context per disk (state uploaded, host copy dropped), then
    the batch over all of them."""
    mem, cells = [], 0
    for p in ps:
        w = W.batch_instance(p)
        c = fb.Fargo(w, fb.F32)
        c.set_state(w.state)
        c.set_time(0.0, 1e30)
        w.state = None
        cells += w.cells
        mem.append(c)
    return mem, fb.FargoBatch(mem, stream=stream), cells


def oracle_steps(make, budget_s, max_steps=50):
    """Step oracle instances from make() (at most max_steps steps each)
    until budget_s seconds of stepping have passed; instance set-up is not
    timed.  Returns (cell-updates, seconds, steps, instances)."""
    import oracle
    cells = 0
    n = 0
    k = 0
    el = 0.0
    while True:
        w = make(k)
        k += 1
        o = oracle.Oracle(w)
        st = w.copy().state
        t = 0.0
        for _ in range(max_steps):
            t0 = time.perf_counter()
            t += o.step(st, t, w.t_end)
            el += time.perf_counter() - t0
            cells += w.cells
            n += 1
            if el > budget_s:
                return cells, el, n, k


def cpu_sample(wname):
    """(instance maker, description) of the bounded oracle sample of a workload."""
    if wname in BATCH_WORKLOADS:
        ps = batch_params(wname)
        return (lambda k: W.batch_instance(ps[k % len(ps)]),
                "oracle stepping disks of the sweep in order (member 0 first), full meshes")
    if wname in ("disk3d", "disk3d-small"):
        return (lambda k: W.disk3d(slab=(200, 24, 36, 24)),
                "oracle on a 1536x24x24 slab of the 1536x512x96 disk (rows 200-223, planes 36-59), frozen ghosts")
    return (lambda k: W.disk2d(), "oracle on the full 768x256 disk")


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_baseline(wname, budget_s=12.0):
    """The plain FP64 oracle on a bounded sample of the workload on the host
    cores: its loops over rings shared by OpenMP threads on every core (the
    reported value), and on one thread beside it (bit-identical results)."""
    import oracle
    make, sample = cpu_sample(wname)
    nproc = os.cpu_count() or 1
    oracle.set_threads(1)
    c1, e1, n1, k1 = oracle_steps(make, budget_s)
    oracle.set_threads(nproc)
    cn, en, nn, kn = oracle_steps(make, budget_s)
    oracle.set_threads(1)
    return {"value": cn / en, "unit": "cell-updates/s", "cores": nproc, "kind": "oracle",
            "threads": nproc, "cpu": cpu_model(), "nproc": nproc,
            "single_thread": {"value": c1 / e1, "cores": 1, "steps": n1, "s": round(e1, 1)},
            "sample": f"{sample}; {nn} steps of {kn} instance(s) in {en:.1f} s on {nproc} OpenMP threads"}


def workload_label(wname):
    if wname in BATCH_WORKLOADS:
        return batch_label(BATCH_WORKLOADS[wname])
    return {"disk3d": "disk3d-sph-adiabatic-planet-1536x512x96",
            "disk3d-small": "disk3d-sph-adiabatic-planet-1536x128x48"}.get(
        wname, "disk2d-cyl-isothermal-planet-768x256")


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    wname = args.workload
    make, sample = cpu_sample(wname)
    import oracle
    nproc = os.cpu_count() or 1
    oracle.set_threads(nproc)
    # each step: about one second of oracle work on the sample
    oracle_steps(make, 0.5 * args.warmup, max_steps=args.warmup)
    cells, el, n, k = oracle_steps(make, 1.0 * args.steps)
    val = cells / el
    line = {"metric": "cell-updates/s", "value": val, "unit": "cell-updates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_label(wname), "sample": sample,
                       "step": "about 1 s of oracle work on the sample per step"},
            "cpu_baseline": {"value": val, "unit": "cell-updates/s", "cores": nproc, "kind": "oracle",
                             "cpu": cpu_model(),
                             "sample": f"{sample}; {n} oracle steps of {k} instance(s) in {el:.1f} s "
                                       f"on {nproc} OpenMP threads"},
            "e2e": {"value": val, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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


# FP64 operations per active cell of one step of the 768 x 256 disk in FP64
# (ncu: smsp__sass_thread_inst_executed_op_{dadd,dmul}_pred_on.sum + 2 x
# ..._op_dfma_pred_on.sum over every launch of a step, divided by the
# cells), valid while the step's sources keep FP64_FLOPS_SRC_HASH
# (profiles/fp64_disk2d_step_ncu.md).
FP64_FLOPS_PER_CELL_2D = 1107.8
FP64_FLOPS_SRC_HASH = "815003752373fcff"


def fp64_roofline(fp64, alu):
    """Roofline of the FP64 step against the measured FP64 multiply-add peak:
    the per-cell kernels run about 400 FP64 operations per cell, so the FP64
    units, not memory, bound it."""
    flops = (FP64_FLOPS_PER_CELL_2D if FP64_FLOPS_SRC_HASH and kernel_source_hash() == FP64_FLOPS_SRC_HASH
             else None)
    peak = alu["fp64"] if alu else None
    out = {"bound": "alu", "unit": "TFLOP/s", "peak": round(peak, 3) if peak else None,
           "peak_kind": "measured FP64 multiply-add throughput (fargo_alu_peaks)",
           "flops_per_cell": flops, "achieved": None, "frac": None}
    if flops and peak:
        ach = flops * fp64["value"] / 1e12
        out.update({"achieved": round(ach, 3), "frac": round(ach / peak, 4)})
    return out


def sod_latency(torch, fb):
    """The 1D Sod tube in FP64 (512 cells, Y axis, t = 0.2): 512 cells are
    far too few to load the GPU, so what is reported is the latency of a
    step: the run to t = 0.2 through fargo_run_to (graph replays, device time
    polled every 64 steps), CUDA events around it, after one untimed run."""
    w = W.sod()
    stream = torch.cuda.Stream()
    c = fb.Fargo(w, fb.F64, stream=stream.cuda_stream)
    with torch.cuda.stream(stream):
        c.set_state(w.state)
        c.set_time(0.0, w.t_end)
        c.run_to(w.t_end, poll=64)
        c.set_state(w.state)
        c.set_time(0.0, w.t_end)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        n = c.run_to(w.t_end, poll=64)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
    t, _, _, err = c.scalars()
    nl = c.launches_per_step()
    c.close()
    return {"workload": "sod1d-cart-adiabatic-512-t0.2", "dtype": "f64", "steps": n, "t": t, "err": err,
            "ms_total": round(ms, 3), "us_per_step": round(1e3 * ms / n, 2), "launches_per_step": nl,
            "value": w.cells * n / (ms * 1e-3), "unit": "cell-updates/s",
            "bound": "launch latency (one CUDA graph of %d launches per step on 512 cells)" % nl}


def disk2d_fp32(torch, fb, dev, steps=200, warmup=10):
    """The 768 x 256 planet disk in FP32 (single context, CUDA graph).  Its
    state (about 17 MB) stays in the 126 MB L2 between steps, so the line is
    a cell-update rate; an HBM fraction would not mean anything here."""
    w = W.disk2d()
    stream = torch.cuda.Stream()
    c = fb.Fargo(w, fb.F32, stream=stream.cuda_stream)
    c.set_state(w.state)
    c.set_time(0.0, 1e30)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            c.step(want_dt=False)
        ms, clocks = timed_steps(torch, stream, lambda: c.step(want_dt=False), steps, dev, lambda: None)
    err = c.scalars()[3]
    c.close()
    return {"workload": "disk2d-cyl-isothermal-planet-768x256", "dtype": "f32", "value": w.cells / (ms * 1e-3),
            "unit": "cell-updates/s", "ms_per_step": round(ms, 4), "steps": steps, "err": err,
            "l2": "L2-resident (state about 17 MB), no flush", "clocks": clocks}


# Algorithmic bytes per cell of the edge kernel (cells 8a-8d): it reads
# rho, v_x, v_y, v_z, B_x, B_y, B_z and writes e_x, e_y, e_z and the three
# velocities after the tension once.
MHD_EDGE_FIELDS = 13


def mhd_box(torch, fb, dev, steps=20, warmup=5, dims=(256, 128, 128), w=None, label=None, fp64=True):
    """A 3D periodic MHD box (Sec. 3.5; 256 x 128 x 128 cells, random
    divergence-free field, eta = 1e-3, artificial viscosity) in FP32 and
    FP64: cell updates per second of the whole step, and the share and
    roofline of the MHD kernels from a kernel-by-kernel step (CUDA
    events).  The state (about 0.5 GB in FP32) is larger than L2.  w and
    label give another MHD workload (the shearing sheet with orbital
    advection of the field); fp64=False measures FP32 only."""
    if w is None:
        w = W.random_mhd_box(*dims, seed=1602, eta=1e-3)
        label = "mhd3d-cart-periodic-%dx%dx%d" % dims
    peak, kind = peaks()
    out = {"workload": label, "cells": w.cells, "hbm_peak_kind": kind}
    precs = ((fb.F32, "f32", 4), (fb.F64, "f64", 8)) if fp64 else ((fb.F32, "f32", 4),)
    for prec, name, esz in precs:
        stream = torch.cuda.Stream()
        c = fb.Fargo(w, prec, stream=stream.cuda_stream)
        c.set_state(w.state)
        c.set_time(0.0, 1e30)
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                c.step(want_dt=False)
            ms, clocks = timed_steps(torch, stream, lambda: c.step(want_dt=False), steps, dev, lambda: None)
            per = c.profile_step()
        err = c.scalars()[3]
        c.close()
        tot = sum(t for _, t in per)
        mk = {k: round(t, 4) for k, t in per if k.startswith("mhd_")}
        emf = mk.get("mhd_edges")
        ach = MHD_EDGE_FIELDS * esz * w.cells / (emf * 1e-3) / 1e9 if emf else None
        out[name] = {"value": w.cells / (ms * 1e-3), "unit": "cell-updates/s", "ms_per_step": round(ms, 4),
                     "steps": steps, "err": err, "clocks": clocks, "mhd_kernels_ms": mk,
                     "mhd_share_of_step": round(sum(mk.values()) / tot, 4) if tot > 0 else None,
                     "edge_kernel_roofline": {"kernel": "k_mhd_edges", "bound": "hbm" if esz == 4 else "alu",
                                              "achieved_GBps": round(ach, 1) if ach else None,
                                              "hbm_peak_GBps": peak,
                                              "hbm_frac": round(ach / peak, 4) if ach else None,
                                              "bytes_per_cell": MHD_EDGE_FIELDS * esz}}
    return out


def batch_fp32_error(mem, ps, picks):
    """FP32 error of sampled disks of the batch after the steps the bench
    gave them, against the FP64 oracle run from the same initial state for
    the same number of steps (relative L1 over the active cells: density and
    the cell-centred momentum density); outside every timed region."""
    import oracle
    from tests.gpu_util import momentum_density, rel_l1
    oracle.set_threads(os.cpu_count() or 1)
    out = []
    for i in picks:
        w = W.batch_instance(ps[i])
        m = mem[i]
        n = m.scalars()[2]
        st = w.copy().state
        oracle.Oracle(w).run(st, 0.0, w.t_end, max_steps=n)
        g = {k: v.astype(np.float64) for k, v in m.get_state().items()}
        out.append({"member": i, "mesh": f"{w.nx}x{w.ny}", "steps": int(n),
                    "rho": float(rel_l1(w.active(g["rho"]), w.active(st["rho"]))),
                    "momentum": float(rel_l1(momentum_density(w, g), momentum_density(w, st)))})
    oracle.set_threads(1)
    return out


# The method's minimum traffic per cell-update: read the state once for the
# Courant step, then read and write it once for the update (3 F b).
METHOD_FIELDS_3D_ADI, METHOD_FIELDS_2D_ISO = 5, 3


def roofline_of(per, cells, table, esz, traffic_tab=None, method_fields=None):
    """Roofline of the dominant kernel from per-launch device times (ms)."""
    hbm, peak_kind = peaks()
    avg = {k: sum(v) / len(v) for k, v in per.items()}
    top = max(avg, key=avg.get)
    alg_bytes = table.get(top, 0) * esz * cells
    achieved = alg_bytes / (avg[top] * 1e-3) / 1e9
    tot = sum(avg.values())
    share = {k: round(v / tot, 4) for k, v in sorted(avg.items(), key=lambda x: -x[1])}
    per_kernel = {k: {"ms": round(v, 4), "alg_GBps": round(table.get(k, 0) * esz * cells / (v * 1e-3) / 1e9, 1)}
                  for k, v in sorted(avg.items(), key=lambda x: -x[1]) if k in table}
    traffic = None
    if traffic_tab is not None and top in traffic_tab:
        traffic = int(traffic_tab[top] * cells)
    step_alg = sum(table.get(k, 0) for k in avg) * esz * cells
    extra = {}
    if method_fields:
        mb = 3 * method_fields * esz * cells
        extra = {"method_bytes_per_cell": 3 * method_fields * esz,
                 "method_GBps": round(mb / (tot * 1e-3) / 1e9, 1),
                 "method_frac": round(mb / (tot * 1e-3) / 1e9 / hbm, 4)}
    return {**extra, "bound": "hbm", "kernel": top, "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4), "peak_kind": f"{peak_kind} copy bandwidth (burst)",
            "alg_bytes_per_launch": alg_bytes, "ms_per_launch": round(avg[top], 4), "traffic": traffic,
            "step_alg_GBps": round(step_alg / (tot * 1e-3) / 1e9, 1),
            "step_frac": round(step_alg / (tot * 1e-3) / 1e9 / hbm, 4),
            "kernel_share": share, "per_kernel": per_kernel}


def add_step_times(per, launches):
    """Accumulate one profiled step: the device times of the launches of one
    kernel within the step are summed (the batched engine launches a ring
    kernel once per cell-chunk group), one entry per step and kernel."""
    step = {}
    for name, t in launches:
        step[name] = step.get(name, 0.0) + t
    for name, t in step.items():
        per.setdefault(name, []).append(t)


def timed_steps(torch, stream, step, n, dev, barrier):
    """Device time per step (ms) of n steps on `stream` with CUDA events,
    clocks sampled during the region."""
    clk = Clocks(dev)
    clk.start()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    return e0.elapsed_time(e1) / n, clk.stop()


def bench_single(args, torch, fb, wname, dev, barrier, e2e_on=True, steps=None):
    steps = steps or args.steps
    w, label, fp32 = make_workload(wname)
    prec = fb.F32 if fp32 else fb.F64
    esz = 4 if fp32 else 8
    stream = torch.cuda.Stream()
    c = fb.Fargo(w, prec, stream=stream.cuda_stream)
    c.set_state(w.state)
    c.set_time(0.0, 1e30)
    nl = c.launches_per_step()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            c.step(want_dt=False)
        # launch shapes picked by the context's autotuner (per-cell block
        # width, Y/Z sweep segments: timed on snapshots of the state, which it
        # leaves unchanged); the timed steps run with its choice, and the
        # step time with the hand-set shapes is reported beside it
        ms_default, _ = timed_steps(torch, stream, lambda: c.step(want_dt=False), 5, dev, lambda: None)
        t0 = time.perf_counter()
        pick = c.autotune(reps=3)
        tune = {"cell_block": pick[0], "seg_y": pick[1], "seg_z": pick[2], "ms_default": round(ms_default, 4),
                "s": round(time.perf_counter() - t0, 1),
                "how": "fargo_autotune: each candidate shape timed on snapshot-restored trial steps (CUDA events)"}
        for _ in range(2):
            c.step(want_dt=False)
        torch.cuda.synchronize()
        ms, clocks = timed_steps(torch, stream, lambda: c.step(want_dt=False), steps, dev, barrier)
        tune["ms_tuned"] = round(ms, 4)
        tune["gain"] = round(ms_default / ms - 1.0, 4) if ms > 0 else None
        per = {}
        for _ in range(steps):
            add_step_times(per, c.profile_step())
    _, _, nsteps, err = c.scalars()
    if err:
        raise SystemExit(f"device error {err} during the benchmark")
    pforce = planet_force_timing(torch, c, stream, w, esz, dev) if w.geom != W.CART and w.planet_q > 0 else None
    table = ALG_FIELDS_3D if (w.nz > 1 and not w.iso) else ALG_FIELDS_2D_ISO
    traffic_tab = (TRAFFIC_PER_CELL_3D if (fp32 and w.nz > 1 and not w.iso
                                           and kernel_source_hash() == KERNEL_SRC_HASH) else None)
    roof = roofline_of(per, w.cells, table, esz, traffic_tab,
                       METHOD_FIELDS_3D_ADI if (w.nz > 1 and not w.iso) else METHOD_FIELDS_2D_ISO)
    e2e = None
    if e2e_on:
        names = ["rho", "e", "vx", "vy", "vz"] if not w.iso else ["rho", "vx", "vy", "vz"]
        if w.nz == 1:
            names = [n for n in names if n != "vz"]
        hdt = torch.float32 if fp32 else torch.float64
        host = {n: torch.empty(w.shape, dtype=hdt, pin_memory=True) for n in names}
        for n in names:
            host[n].numpy()[...] = w.state[n]
        bytes_io = sum(h.numel() * h.element_size() for h in host.values())
        ksteps = max(3, min(steps, 10))
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
        e2e = {"value": w.cells * ksteps / el, "unit": "cell-updates/s",
               "h2d_bytes_per_step": bytes_io, "d2h_bytes_per_step": bytes_io, "steps": ksteps,
               "note": "every step uploads the full state from pinned host memory and reads it back"}
    c.close()
    return {"workload": label, "cells": w.cells, "fp32": fp32, "ms": ms, "clocks": clocks, "roofline": roof,
            "e2e": e2e, "launches": nl, "steps_advanced": int(nsteps),
            "state_gb": w.cells * 21 * esz / 1e9, "planet_force": pforce, "autotune": tune}


def planet_force_timing(torch, c, stream, w, esz, dev, reps=20):
    """Force of the gas on the planet on the workload's state after the timed
    steps, direct sum and BM08.  Device time per call from CUDA events on the
    context's stream around `reps` queued calls (fargo_planet_force_async:
    the table and the force kernels, results left on the device); and the
    time of the synchronous call a host integrator makes
    (fargo_planet_force: the same two launches, the 32-byte copy back and
    the synchronisation), host clock.  Algorithmic bytes: one read of the
    density per active cell (the BM08 ring mean re-reads a ring that is
    still in L1/L2)."""
    hbm, kind = peaks()
    rp = (w.planet_a, 0.0, 0.0)
    res = torch.empty(4, dtype=torch.float64, device=dev)
    full_3d = w.name == "disk3d" and w.cells == 1536 * 512 * 96 and esz == 4
    traffic = (PFORCE_TRAFFIC_3D if full_3d and kernel_source_hash(("kernels_planet.cuh",)) == PFORCE_SRC_HASH
               else None)
    out = {"bound": "hbm", "peak": hbm, "peak_kind": f"{kind} copy bandwidth (burst)", "unit": "GB/s",
           "alg_bytes_per_call": w.cells * esz, "launches_per_call": 2, "traffic_direct": traffic}
    for bm08 in (False, True):
        with torch.cuda.stream(stream):
            for _ in range(3):
                c.planet_force_async(rp, w.planet_eps, res.data_ptr(), bm08)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                c.planet_force_async(rp, w.planet_eps, res.data_ptr(), bm08)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                c.planet_force(rp, w.planet_eps, bm08)
            sync_ms = (time.perf_counter() - t0) * 1e3 / reps
        key = "bm08" if bm08 else "direct"
        gbs = w.cells * esz / (ms * 1e-3) / 1e9
        out[key] = {"ms": round(ms, 4), "achieved": round(gbs, 1), "frac": round(gbs / hbm, 4),
                    "sync_call_ms": round(sync_ms, 4)}
    return out


def bench_batch(args, torch, fb, wname, dev, barrier, e2e_on=True):
    ps = batch_params(wname)
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    mem, b, cells = make_batch(fb, ps, stream.cuda_stream)
    setup_s = time.perf_counter() - t0
    # launch shapes picked by the batch autotuner (per-cell grouping, sweep
    # segments: timed on snapshots of the state, which it leaves unchanged);
    # the timed steps run with its choice
    t0 = time.perf_counter()
    tcfg, ms_def, ms_tuned = b.autotune(reps=3)
    tune = {**tcfg, "ms_default": round(ms_def, 4), "ms_tuned": round(ms_tuned, 4),
            "gain": round(ms_def / ms_tuned - 1.0, 4) if ms_tuned > 0 else None,
            "s": round(time.perf_counter() - t0, 1),
            "how": "fargo_batch_autotune: each candidate shape timed over 3 steps of a snapshot (CUDA events)"}
    nl = b.launches_per_step()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            b.step(sync=False)
        b.status()
        ms, clocks = timed_steps(torch, stream, lambda: b.step(sync=False), args.steps, dev, barrier)
        per = {}
        for _ in range(args.steps):
            add_step_times(per, b.profile_step())
    running, _ = b.status()
    nsteps = [m.scalars()[2] for m in mem]
    btraffic = (TRAFFIC_PER_CELL_BATCH if BATCH_SRC_HASH and
                kernel_source_hash(STEP_SOURCES + ("fargo_batch.cu",)) == BATCH_SRC_HASH else None)
    roof = roofline_of(per, cells, ALG_FIELDS_2D_ISO, 4, btraffic, method_fields=METHOD_FIELDS_2D_ISO)
    e2e = None
    if e2e_on:
        # public API end to end: every step uploads each disk's active state
        # (rho, v_x, v_y) from pinned host memory and reads it back, each field
        # of all disks as one packed buffer (member order, active cells)
        names = ["rho", "vx", "vy"]
        host = {n: torch.empty(cells, dtype=torch.float32, pin_memory=True) for n in names}
        for n in names:
            b.get_field_packed(n, host[n])
        bytes_io = sum(h.numel() * h.element_size() for h in host.values())
        ksteps = max(3, min(args.steps, 6))
        with torch.cuda.stream(stream):
            torch.cuda.synchronize()
            barrier()
            t1 = time.perf_counter()
            for _ in range(ksteps):
                for n in names:
                    b.set_field_packed(n, host[n])      # queued on the batch's stream
                b.step(sync=False)
                for n in names:
                    b.get_field_packed(n, host[n])      # one copy per field; synchronises
                b.status()
            torch.cuda.synchronize()
            el = time.perf_counter() - t1
            barrier()
        e2e = {"value": cells * ksteps / el, "unit": "cell-updates/s",
               "h2d_bytes_per_step": bytes_io, "d2h_bytes_per_step": bytes_io, "steps": ksteps,
               "note": "every step uploads every disk's active rho, v_x, v_y from pinned host memory "
                       "(fargo_batch_set_field_packed: one copy per field for all disks plus a scatter "
                       "kernel, queued on the batch's stream), steps the batch and reads them back "
                       "(fargo_batch_get_field_packed: a gather kernel and one copy per field)"}
    b.status()
    picks = sorted(range(len(ps)), key=lambda i: (ps[i]["ny"], i))[:2]
    fp32_err = batch_fp32_error(mem, ps, picks)
    b.close()
    for m in mem:
        m.close()
    return {"workload": batch_label(len(ps)), "cells": cells, "members": len(ps), "ms": ms, "clocks": clocks,
            "fp32_error": fp32_err,
            "roofline": roof, "e2e": e2e, "launches": nl, "setup_s": round(setup_s, 1), "autotune": tune,
            "steps_advanced_min": int(min(nsteps)), "running": running,
            "state_gb": cells * 2 * 22 * 4 / 1e9}


def vorticity_rms_diff(w, v_a, v_b):
    """r.m.s. over the active mesh of the difference of the vertical
    vorticity (1/r) d(r v_phi)/dr of two azimuthal-velocity fields (inertial
    v_phi = v_x + Omega_f r, radial differences at the faces between rings),
    both evaluated in FP64 from the stored values."""
    import numpy as np
    r = W.centres(w.yf)[w.gy:w.gy + w.ny]
    rf = w.yf[w.gy + 1:w.gy + w.ny]

    def omz(v):
        vp = w.active(v).astype(np.float64)[0] + w.omega_f * r[:, None]
        rv = r[:, None] * vp
        return (rv[1:] - rv[:-1]) / (r[1:] - r[:-1])[:, None] / rf[:, None]

    d = omz(v_a) - omz(v_b)
    return float(np.sqrt(np.mean(d * d)))


def precision_study(torch, fb, orbits=8.0):
    """Single versus double precision on the laminar planet disk (Sec. 6):
    the 4000 x 2000 inviscid disk with an Earth-mass planet in the frame
    corotating with it, run in FP64 and in the FP32 path side by side; the
    specific torque on the planet every quarter orbit, and the r.m.s.
    differences of the azimuthal velocity and of the vorticity between the
    two runs at the start and at the end.  One JSON line."""
    import numpy as np
    w = W.laminar_disk(orbits=orbits)
    c64 = fb.Fargo(w, fb.F64)
    c32 = fb.Fargo(w, fb.F32)
    for c in (c64, c32):
        c.set_state(w.state)
        c.set_time(0.0, w.t_end)
    w.state = None

    def vdiff():
        v64, v32 = c64.get_field("vx"), c32.get_field("vx")
        d = w.active(v32).astype(np.float64) - w.active(v64)
        return float(np.sqrt(np.mean(d * d))), vorticity_rms_diff(w, v32, v64)

    s0, om0 = vdiff()
    rp = (w.planet_a, 0.0, 0.0)
    samples = []
    t0 = time.perf_counter()
    nq = int(round(4 * orbits))
    for k in range(1, nq + 1):
        t = 0.25 * k * 2 * math.pi
        c64.run_to(t, poll=512)
        c32.run_to(t, poll=512)
        a, b = c64.scalars(), c32.scalars()
        if a[3] or b[3]:
            raise SystemExit(f"device error {a[3]} / {b[3]} in the precision study")
        samples.append([round(0.25 * k, 4), c64.planet_force(rp, w.planet_eps)[3],
                        c32.planet_force(rp, w.planet_eps)[3], a[2], b[2]])
    wall = time.perf_counter() - t0
    s1, om1 = vdiff()
    h = np.array([x[:3] for x in samples])
    scale = float(np.max(np.abs(h[h[:, 0] <= 1.0, 1])))
    rel = np.abs(h[:, 2] - h[:, 1]) / scale
    print(json.dumps({
        "metric": "sp_dp_torque_study", "workload": f"laminar disk {w.nx} x {w.ny}, q = {w.planet_q}, h = 0.05, "
        f"r in [0.6, 1.4], corotating, inviscid", "orbits": orbits,
        "columns": ["orbits", "torque_fp64", "torque_fp32", "steps_fp64", "steps_fp32"], "samples": samples,
        "torque_scale_first_orbit": scale, "diff_over_scale": [round(float(x), 4) for x in rel],
        "rms_dvx_t0": s0, "rms_dvorticity_t0": om0, "rms_dvx_end": s1, "rms_dvorticity_end": om1,
        "dr": float(w.yf[w.gy + 1] - w.yf[w.gy]), "wall_s": round(wall, 1)}))
    c64.close()
    c32.close()


def vortex_study(torch, fb, orbits=10.0, resolutions=((1024, 256), (2048, 512))):
    """Orbital advection and vortensity (Sec. 6): the vortex in a Keplerian
    disk, with and without orbital advection, at each resolution, in FP64
    and in the FP32 path; the vortensity minimum every half orbit of the
    vortex, the steps taken and the device time.  One JSON line."""
    res = []
    for (nx, ny), prec in [(r, p) for r in resolutions for p in ("f64", "f32")]:
        for fargo in (True, False):
            w = W.keplerian_vortex(nx=nx, ny=ny, fargo=fargo, orbits=orbits)
            c = fb.Fargo(w, fb.F64 if prec == "f64" else fb.F32)
            c.set_state(w.state)
            c.set_time(0.0, w.t_end)
            hist = [[0.0, float(W.vortensity(w, w.state).min())]]
            t0 = time.perf_counter()
            for k in range(1, int(round(2 * orbits)) + 1):
                c.run_to(0.5 * k * 2 * math.pi, poll=2048)
                if c.scalars()[3]:
                    raise SystemExit(f"device error in the vortex study ({nx} x {ny}, fargo={fargo})")
                hist.append([0.5 * k, float(W.vortensity(w, c.get_state()).min())])
            wall = time.perf_counter() - t0
            res.append({"nx": nx, "ny": ny, "dtype": prec, "orbital_advection": fargo, "steps": c.scalars()[2],
                        "wall_s": round(wall, 2), "vortensity_min": hist})
            c.close()
    print(json.dumps({"metric": "vortensity_min_decay", "workload": "Keplerian vortex, M = 10, K = -1, "
                      "h = c_s/(2 Omega), r in [0.4, 2], adiabatic, inviscid", "orbits": orbits,
                      "runs": res}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--workload", default="batch256",
                    choices=["batch256", "batch-small", "batch-medium", "disk3d", "disk2d", "disk3d-small",
                             "precision-study", "vortex-study"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-single", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import paper_1602_02359_b300 as fb

    ws, rank, local = dist_env()
    torch.cuda.set_device(local if ws > 1 else 0)
    if args.workload in ("precision-study", "vortex-study"):
        if rank == 0:
            (precision_study if args.workload == "precision-study" else vortex_study)(torch, fb)
        return
    ranks = Ranks(torch)
    dev = torch.cuda.current_device()
    barrier = ranks.barrier

    batched = args.workload in BATCH_WORKLOADS
    if batched:
        r = bench_batch(args, torch, fb, args.workload, dev, barrier, e2e_on=not args.no_e2e)
    else:
        r = bench_single(args, torch, fb, args.workload, dev, barrier, e2e_on=not args.no_e2e)
    value, ms_max, e2e_rate = ranks.aggregate(r["cells"], r["ms"],
                                              r["e2e"]["value"] if r["e2e"] is not None else None)
    if r["e2e"] is not None:
        r["e2e"]["value"] = e2e_rate

    single = None
    if rank == 0 and batched and not args.no_single:
        s = bench_single(args, torch, fb, "disk3d", dev, lambda: None, e2e_on=False, steps=min(args.steps, 20))
        single = {"workload": s["workload"], "dtype": "f32", "value": s["cells"] / (s["ms"] * 1e-3),
                  "unit": "cell-updates/s", "ms_per_step": s["ms"],
                  "roofline": {k: s["roofline"].get(k) for k in ("kernel", "achieved", "peak", "unit", "frac",
                                                                 "step_alg_GBps", "step_frac", "method_GBps",
                                                                 "method_frac", "traffic")},
                  "per_kernel": s["roofline"]["per_kernel"], "clocks": s["clocks"],
                  "planet_force": s["planet_force"], "autotune": s["autotune"]}

    surrogate = None
    if rank == 0 and batched and not args.no_surrogate:
        surrogate = bench_surrogate(torch)

    fp64 = None
    if rank == 0 and not args.no_fp64 and args.workload in ("disk3d",) + tuple(BATCH_WORKLOADS):
        fp64 = fp64_plain_disk2d(torch, fb)
    alu = fb.alu_peaks(torch.cuda.current_stream().cuda_stream) if rank == 0 else None
    if fp64 is not None:
        fp64["roofline"] = fp64_roofline(fp64, alu)
    extra_lines = {}
    if rank == 0 and batched and not args.no_single:
        extra_lines["sod_fp64"] = sod_latency(torch, fb)
        extra_lines["disk2d_fp32"] = disk2d_fp32(torch, fb, dev)
        extra_lines["mhd3d"] = mhd_box(torch, fb, dev)
        # the Keplerian MHD shearing sheet with orbital advection of the field
        # (Sec. 3.6): 512 x 192 x 64 cells, about 0.4 GB of FP32 state
        sheet = W.mhd_shearing_sheet(512, 192, 64, amp=0.002, seed=1602, vamp=0.02, lx=2.0, ly=0.75, lz=0.25)
        extra_lines["mhd_sheet_fargo"] = mhd_box(torch, fb, dev, w=sheet, fp64=False,
                                                 label="mhd3d-cart-shearing-sheet-fargo-512x192x64")

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and ws == 1 and args.workload not in ("disk3d-small", "batch-small", "batch-medium"):
        cpu = cpu_baseline(args.workload)

    if rank == 0:
        cfg = {"workload": r["workload"], "cells": r["cells"],
               "precision": "FP32 fields, FP64 dt/v0/shift/planet offset" if (batched or r["fp32"]) else "FP64",
               "parallelism": "replicas" if ws > 1 else "single GPU",
               "l2": "inputs larger than L2 (state %.1f GB)" % r["state_gb"], "graph": True}
        if batched:
            cfg.update({"members": r["members"], "engine": "batched, one launch per phase over all members, "
                                                            "per-member Courant step",
                        "steps_advanced_min": r["steps_advanced_min"], "setup_s": r["setup_s"],
                        "autotune": r["autotune"],
                        "run_length": "500 orbits per disk in the sweep; the bench times per-step throughput"})
        else:
            cfg["steps_advanced"] = r["steps_advanced"]
            cfg["autotune"] = r["autotune"]
        line = {
            "metric": "cell-updates/s", "value": value, "unit": "cell-updates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if (batched or r["fp32"]) else "f64",
            "data": "synthetic", "config": cfg,
            "roofline": r["roofline"],
            "cpu_baseline": cpu,
            "e2e": r["e2e"],
            "gpu_launches": r["launches"] * args.steps,
            "clocks": r["clocks"],
        }
        if fp64 is not None:
            line["fp64_plain"] = fp64
            key = "fp32_batched_vs_fp64_plain" if batched else "fp32_vs_fp64_plain"
            line[key] = value / ws / fp64["value"]
        if single is not None:
            line["single_instance_fp32"] = single
        if r.get("planet_force") is not None:
            line["planet_force"] = r["planet_force"]
        if surrogate is not None:
            line["surrogate_kernels"] = surrogate
        if alu is not None:
            line["alu_peaks"] = {"fp64_tflops": round(alu["fp64"], 2), "fp32_tflops": round(alu["fp32"], 1),
                                 "fp32x2_tflops": round(alu["fp32x2"], 1),
                                 "how": "fargo_alu_peaks: independent multiply-add chains on every SM, "
                                        "best of 3 launches, CUDA events"}
        line.update(extra_lines)
        if batched and r.get("fp32_error"):
            line["fp32_error_vs_fp64_oracle"] = {
                "members": r["fp32_error"],
                "note": "sampled disks of the batch after the bench's steps, against the FP64 oracle from "
                        "the same initial state; the errors at the sweep's run lengths (1000 steps, 500 "
                        "orbits) are measured by tests/test_gpu_fp32_long.py"}
        print(json.dumps(line), flush=True)
    ranks.close()


if __name__ == "__main__":
    main()
