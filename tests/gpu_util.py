"""Helpers shared by the GPU parity tests."""
import numpy as np
import pytest

import oracle
import workloads as W


def have_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def make_ctx(w, prec=None, t=0.0, t_end=1e300):
    import paper_1602_02359_b300 as fb
    prec = fb.F64 if prec is None else prec
    c = fb.Fargo(w, prec)
    c.set_state(w.state)
    c.set_time(t, t_end)
    return c


def rel_linf(a, b):
    """max |a - b| / max |b| (norm-wise relative L-infinity)."""
    d = np.max(np.abs(np.asarray(a, dtype=np.float64) - b))
    s = np.max(np.abs(b))
    return d / s if s > 0 else d


def rel_l1(a, b):
    s = np.sum(np.abs(b))
    d = np.sum(np.abs(np.asarray(a, dtype=np.float64) - b))
    return d / s if s > 0 else d


def active_faces(w, name, a):
    """Active region plus the upper boundary face of the staggered component."""
    gz, gy = w.gz, w.gy
    if name == "vy" and w.ny > 1:
        return a[gz:gz + w.nz, gy:gy + w.ny + 1, :]
    if name == "vz" and w.nz > 1:
        return a[gz:gz + w.nz + 1, gy:gy + w.ny, :]
    return w.active(a)


def fields_of(w):
    f = ["rho", "vx"]
    if not w.iso:
        f.append("e")
    if w.ny > 1:
        f.append("vy")
    if w.nz > 1:
        f.append("vz")
    return f


def compare_state(w, gpu_state, ora_state, tol, norm=rel_linf):
    worst = {}
    for k in fields_of(w):
        a = active_faces(w, k, gpu_state[k].astype(np.float64))
        b = active_faces(w, k, ora_state[k])
        worst[k] = norm(a, b)
    bad = {k: v for k, v in worst.items() if not v <= tol}
    assert not bad, f"parity beyond {tol}: {worst}"
    return worst


def momentum_density(w, st):
    """Cell-centred momentum density rho (v_{-1/2} + v_{+1/2})/2 of every
    active direction, stacked (the zone-centred momentum of Eq. 19)."""
    rho = w.active(st["rho"]).astype(np.float64)
    out = []
    vx = w.active(st["vx"]).astype(np.float64)
    out.append(rho * 0.5 * (vx + np.roll(vx, -1, axis=2)))
    if w.ny > 1:
        vy = st["vy"][w.gz:w.gz + w.nz, w.gy:w.gy + w.ny + 1].astype(np.float64)
        out.append(rho * 0.5 * (vy[:, :-1] + vy[:, 1:]))
    if w.nz > 1:
        vz = st["vz"][w.gz:w.gz + w.nz + 1, w.gy:w.gy + w.ny].astype(np.float64)
        out.append(rho * 0.5 * (vz[:-1] + vz[1:]))
    return np.stack(out)


def record(name, **vals):
    """Report measured parity figures: printed (visible with pytest -s), and
    appended as one JSON line to the file named by the environment variable
    FARGO_PARITY_RECORD when it is set.  Never read by a test."""
    import json
    import os
    line = json.dumps({"case": name, **{k: float(v) for k, v in vals.items()}})
    print(line)
    path = os.environ.get("FARGO_PARITY_RECORD")
    if path:
        with open(path, "a") as f:
            f.write(line + "\n")
