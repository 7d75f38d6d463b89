"""Learned surrogate of the batched disk sweep, with the solver as fallback.

The network maps (log10 q, h, log10 nu) and the initial surface density on
256 logarithmic radial bins to the azimuthally averaged Sigma / Sigma_0 that
the solver reaches after a fixed number of orbits, on the same bins.  The
paper has no counterpart: it is built on the batched engine, which produces
its training data, and the solver remains the judge of its error and the
fallback whenever the surrogate's reported error exceeds a threshold.

Pipeline:
  solve()      disks advanced by the batched engine to their end time; each
               disk's Sigma(r) is averaged over azimuth and resampled
               (linear in log r) onto the bins;
  Surrogate    a deep ensemble of K networks (kernels of include/fargo_mlp.h)
               trained with Adam on the mean-squared error; the reported
               error of a query is the ensemble's relative spread times a
               factor calibrated on held-out data;
  query()      surrogate answers, and a solver run for every query whose
               reported error is above the threshold.

python -m paper_1602_02359_b300.surrogate [--runs N] [--orbits O] ... runs
the whole pipeline and prints one JSON line of results.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

import workloads as W

from . import F32, F64, ACTIVE, Fargo, FargoBatch
from . import mlp as fm

SIGMA0 = 1e-3          # initial surface density normalisation of the disks
THRESHOLD = 0.05       # reported relative error above which the solver answers


def features(p, bins):
    """Input vector of one disk: log10 q, h, log10 nu, Sigma_0(bins)."""
    return np.concatenate([[math.log10(p["q"]), p["h"], math.log10(p["nu"])], SIGMA0 * bins ** -0.5])


def radial_profile(w, rho_active, bins):
    """Azimuthal mean of Sigma over the initial Sigma_0, at the bins."""
    sig = rho_active.reshape(w.ny, w.nx).astype(np.float64).mean(axis=1)
    rc = W.centres(np.asarray(w.yf))[w.gy:w.gy + w.ny]
    ratio = sig / (SIGMA0 * rc ** -0.5)
    return np.interp(np.log(bins), np.log(rc), ratio)


def solve(params, orbits, precision=F32, chunk=1024, stream=None):
    """Advance every disk of `params` to `orbits` orbits with the batched
    engine; returns (profiles [n, bins], solver seconds, cell updates)."""
    import torch
    bins = W.surrogate_bins()
    out = np.zeros((len(params), bins.size))
    secs = 0.0
    updates = 0
    for c0 in range(0, len(params), chunk):
        ps = params[c0:c0 + chunk]
        ws, mem = [], []
        for p in ps:
            w = W.batch_instance(p, orbits=orbits)
            c = Fargo(w, precision, stream=stream)
            c.set_state(w.state)
            c.set_time(0.0, w.t_end)
            w.state = None
            ws.append(w)
            mem.append(c)
        b = FargoBatch(mem, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.run(poll=256)
        torch.cuda.synchronize()
        secs += time.perf_counter() - t0
        for i, (w, c) in enumerate(zip(ws, mem)):
            t, _, n, err = c.scalars()
            if err:
                raise RuntimeError(f"solver error {err} on disk {c0 + i}")
            updates += n * w.cells
            out[c0 + i] = radial_profile(w, c.get_field("rho", region=ACTIVE), bins)
        b.close()
        for c in mem:
            c.close()
    return out, secs, updates


def _flat(params):
    """Parameter vector (W_0 row-major, b_0, W_1, b_1, ...) in FP32."""
    return np.concatenate([np.concatenate([Wl.ravel(), bl]) for Wl, bl in params]).astype(np.float32)


class Ensemble:
    """Deep ensemble of K perceptrons (seeds seed .. seed+K-1) trained on the
    same data in different orders; mean prediction and calibrated error."""

    def __init__(self, dims=None, k=4, seed=1602, max_batch=4096):
        import torch
        self.dims = dims or W.mlp_dims()
        self.k = k
        self.seed = seed
        self.max_batch = max_batch
        self.nets = []
        # one stream for the networks and every tensor operation around them
        self.stream = torch.cuda.Stream()
        for e in range(k):
            n = fm.Mlp(self.dims, max_batch, stream=self.stream.cuda_stream)
            n.set_params(_flat(W.mlp_init(self.dims, seed + e)))
            self.nets.append(n)
        self.calib = 1.0
        self.dev = torch.device("cuda")

    def close(self):
        for n in self.nets:
            n.close()

    def set_maps(self, X, Y):
        """Standardise every input feature and output bin over the training
        set (features without spread are switched off)."""
        mu = X.mean(axis=0)
        sd = X.std(axis=0)
        scale = np.where(sd > 1e-12 * np.maximum(np.abs(mu), 1e-300), 1.0 / np.where(sd > 0, sd, 1.0), 0.0)
        ym = Y.mean(axis=0)
        ys = np.maximum(Y.std(axis=0), 1e-6)
        for n in self.nets:
            n.set_input_map(mu, scale)
            n.set_output_map(ym, ys)

    def fit(self, X, Y, epochs=200, batch=256, lr=1e-3, lr_end=2e-5):
        """Adam on mini-batches with a cosine decay of the learning rate from
        lr to lr_end; returns [(epoch, mean training loss of member 0)]."""
        import torch
        self.set_maps(X, Y)
        with torch.cuda.stream(self.stream):
            return self._fit(X, Y, epochs, batch, lr, lr_end)

    def _fit(self, X, Y, epochs, batch, lr, lr_end):
        import torch
        Xd = torch.tensor(X, dtype=torch.float32, device=self.dev)
        Yd = torch.tensor(Y, dtype=torch.float32, device=self.dev)
        nb = max(1, len(X) // batch)
        xb = torch.empty(batch, X.shape[1], device=self.dev)
        yb = torch.empty(batch, Y.shape[1], device=self.dev)
        losses = torch.zeros(nb, device=self.dev)
        hist = []
        gens = [torch.Generator(device="cpu").manual_seed(self.seed + 97 * e) for e in range(self.k)]
        for ep in range(epochs):
            rate = lr_end + 0.5 * (lr - lr_end) * (1.0 + math.cos(math.pi * ep / max(1, epochs - 1)))
            for n in self.nets:
                n.set_optimizer(lr=rate)
            for e, n in enumerate(self.nets):
                perm = torch.randperm(len(X), generator=gens[e]).to(self.dev)
                for i in range(nb):
                    idx = perm[i * batch:(i + 1) * batch]
                    if idx.numel() < batch:
                        idx = torch.cat([idx, perm[:batch - idx.numel()]])
                    torch.index_select(Xd, 0, idx, out=xb)
                    torch.index_select(Yd, 0, idx, out=yb)
                    n.train_step(xb, yb, losses[i:i + 1] if e == 0 else None)
            if ep % 10 == 0 or ep == epochs - 1:
                hist.append((ep, float(losses.mean().item())))
        return hist

    def predict(self, X):
        """(mean [n, out], spread [n]) on the device, ready on the current stream."""
        import torch
        cur = torch.cuda.current_stream()
        self.stream.wait_stream(cur)
        with torch.cuda.stream(self.stream):
            out = self._predict(X)
        cur.wait_stream(self.stream)
        return out

    def _predict(self, X):
        import torch
        Xd = torch.as_tensor(X, dtype=torch.float32, device=self.dev).contiguous()
        n = Xd.shape[0]
        ys = torch.empty(self.k, n, self.dims[-1], device=self.dev)
        for e, net in enumerate(self.nets):
            net.forward(Xd, ys[e])
        mean = torch.empty(n, self.dims[-1], device=self.dev)
        spread = torch.empty(n, device=self.dev)
        fm.ensemble(ys, mean, spread, self.stream.cuda_stream)
        return mean, spread

    def calibrate(self, X, Y, quantile=0.9):
        """Factor c such that c * spread bounds the actual relative L2 error
        of `quantile` of the held-out samples."""
        mean, spread = self.predict(X)
        err = rel_err(mean.cpu().numpy(), Y)
        s = np.maximum(spread.cpu().numpy().astype(np.float64), 1e-12)
        self.calib = float(np.quantile(err / s, quantile))
        return self.calib

    def reported_error(self, spread):
        return self.calib * spread


def rel_err(pred, ref):
    """Relative L2 error of each profile."""
    pred = np.asarray(pred, dtype=np.float64)
    return np.linalg.norm(pred - ref, axis=1) / np.linalg.norm(ref, axis=1)


def query(ens, params, orbits, threshold=THRESHOLD, precision=F32):
    """Profiles for `params`: the surrogate's where its reported error is at
    most `threshold`, the solver's otherwise.  Returns (profiles, reported
    errors, mask of the solver answers)."""
    bins = W.surrogate_bins()
    X = np.stack([features(p, bins) for p in params])
    mean, spread = ens.predict(X)
    rep = ens.reported_error(spread.cpu().numpy().astype(np.float64))
    prof = mean.cpu().numpy().astype(np.float64)
    fall = rep > threshold
    if fall.any():
        sub = [p for p, f in zip(params, fall) if f]
        prof[fall] = solve(sub, orbits, precision=precision)[0]
    return prof, rep, fall


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--runs", type=int, default=4096)
    ap.add_argument("--orbits", type=float, default=50.0)
    ap.add_argument("--nr", type=int, nargs=2, default=(48, 96))
    ap.add_argument("--epochs", type=int, default=1000)
    ap.add_argument("--k", type=int, default=4)
    ap.add_argument("--seed", type=int, default=1602)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    torch.cuda.set_device(0)
    params = W.surrogate_params(args.runs, seed=args.seed, nr=tuple(args.nr))
    bins = W.surrogate_bins()
    X = np.stack([features(p, bins) for p in params])
    ntr = int(round(0.9 * args.runs))
    t0 = time.perf_counter()
    Y, solver_s, updates = solve(params[:ntr], args.orbits, precision=F32)
    gen_s = time.perf_counter() - t0
    # held-out split: the FP32 batched solver (calibration) and the FP64 solver (the judge)
    Yv32, _, _ = solve(params[ntr:], args.orbits, precision=F32)
    t1 = time.perf_counter()
    Yv64, solver64_s, updates64 = solve(params[ntr:], args.orbits, precision=F64)
    judge_s = time.perf_counter() - t1
    ens = Ensemble(k=args.k, seed=args.seed)
    t2 = time.perf_counter()
    hist = ens.fit(X[:ntr], Y, epochs=args.epochs, lr=2e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t2
    nval = args.runs - ntr
    half = nval // 2
    ens.calibrate(X[ntr:ntr + half], Yv32[:half])
    # evaluation on the second half of the held-out split, judged by the FP64 solver
    Xe, Ye = X[ntr + half:], Yv64[half:]
    for _ in range(3):
        ens.predict(Xe)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    reps = 20
    for _ in range(reps):
        mean, spread = ens.predict(Xe)
    torch.cuda.synchronize()
    infer_s = (time.perf_counter() - t3) / reps
    err = rel_err(mean.cpu().numpy(), Ye)
    rep = ens.reported_error(spread.cpu().numpy().astype(np.float64))
    fall = rep > THRESHOLD
    naive = rel_err(np.broadcast_to(Y.mean(axis=0), Ye.shape), Ye)
    fp32_vs_fp64 = rel_err(Yv32[half:], Ye)
    solver_per_disk = solver_s / ntr
    res = {
        "runs": args.runs, "train": ntr, "calibration": half, "evaluation": len(Xe),
        "orbits": args.orbits, "nr": list(args.nr), "ensemble": args.k, "epochs": args.epochs,
        "solver_fp32_s": round(solver_s, 2), "solver_fp32_cell_updates": int(updates),
        "solver_fp32_rate": updates / solver_s, "data_generation_s": round(gen_s, 2),
        "solver_fp64_judge_s": round(solver64_s, 2), "train_s": round(train_s, 2),
        "final_train_loss": hist[-1][1],
        "surrogate_rel_l2": {"median": float(np.median(err)), "p90": float(np.quantile(err, 0.9)),
                             "max": float(err.max()), "mean": float(err.mean())},
        "naive_mean_profile_rel_l2_median": float(np.median(naive)),
        "fp32_solver_vs_fp64_rel_l2_median": float(np.median(fp32_vs_fp64)),
        "calibration_factor": ens.calib,
        "fallback_fraction": float(fall.mean()),
        "accepted_rel_l2_max": float(err[~fall].max()) if (~fall).any() else None,
        "accepted_within_threshold": float((err[~fall] <= THRESHOLD).mean()) if (~fall).any() else None,
        "inference_s_per_query_batch": infer_s, "inference_batch": len(Xe),
        "inference_s_per_disk": infer_s / len(Xe),
        "solver_fp32_s_per_disk_batched": solver_per_disk,
        "speedup_vs_batched_solver": solver_per_disk / (infer_s / len(Xe)),
    }
    ens.close()
    line = json.dumps(res)
    print(line, flush=True)
    if args.out:
        with open(args.out, "w") as f:
            f.write(line + "\n")


if __name__ == "__main__":
    main()
