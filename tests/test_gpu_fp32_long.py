"""FP32 parity against the FP64 oracle at the step counts of the workloads.

The FP32 path stores every field in FP32 and keeps FP64 for the Courant
step, v0, the orbital shift and fraction, the planet and the sums.  Its
error against the FP64 oracle grows with the number of steps, so it is
measured where the workloads are run:
  - the 768 x 256 planet disk after 10 orbits (about 11 100 steps), against
    a stored oracle state (tests/golden/make_fp32_references.py);
  - the 1536 x 512 x 96 spherical disk's equations on a 1536 x 16 x 16 slab
    of it (full azimuth, same faces and initial state) after 1, 100 and
    200 steps, the oracle run beside it;
  - eight disks of the 256-disk sweep (the smallest, 384..426 x 128..142)
    stepped 1000 times by the batched engine, the oracle run beside it;
  - the two smallest disks of the sweep run to 500 orbits by the batched
    engine, against stored oracle states.
Errors are relative L1 norms over the active cells: density, energy, and the
cell-centred momentum density (Eq. 19) of all components together.  The
stated tolerance, 2e-5 on density (and energy) and 1e-4 on the momentum
density, is asserted at 10 orbits, 200 steps and 1000 steps (measured: at
most 1.6e-6).  The error keeps growing with the number of steps, about
1e-6 per thousand, and the two runs' Courant steps part by a fraction of a
percent, so after 500 orbits (1e5 steps and more) it is 3e-3 to 6e-3, and
it moved by a factor of up to ten between builds that round differently
(the gap's flow amplifies differences): those runs are bounded at 2e-2.
"""
import os

import numpy as np
import pytest

import oracle
import workloads as W
from tests.gpu_util import make_ctx, momentum_density, record, rel_l1

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
SWEEP8 = [156, 126, 105, 20, 244, 147, 131, 108]     # the eight smallest disks of the sweep


@pytest.fixture(scope="module", autouse=True)
def oracle_threads():
    oracle.set_threads(os.cpu_count() or 1)
    yield
    oracle.set_threads(1)


def errors(w, g, ref):
    out = {"rho": rel_l1(w.active(g["rho"]), w.active(ref["rho"])),
           "momentum": rel_l1(momentum_density(w, g), momentum_density(w, ref))}
    if not w.iso:
        out["e"] = rel_l1(w.active(g["e"]), w.active(ref["e"]))
    return out


def stored_state(w, path):
    """A full-layout state holding the stored active values."""
    z = np.load(path)
    st = {k: np.zeros(w.shape) for k in W.FIELDS}
    st["rho"][w.gz:w.gz + w.nz, w.gy:w.gy + w.ny] = z["rho"]
    st["vx"][w.gz:w.gz + w.nz, w.gy:w.gy + w.ny] = z["vx"]
    st["vy"][w.gz:w.gz + w.nz, w.gy:w.gy + w.ny + 1] = z["vy"]
    return st, float(z["t_end"]), int(z["steps"])


def test_disk2d_fp32_ten_orbits():
    import paper_1602_02359_b300 as fb
    w = W.disk2d()
    ref, t_end, n_ref = stored_state(w, os.path.join(GOLDEN, "disk2d_768x256_10orbits.npz"))
    c = make_ctx(w, fb.F32, t=0.0, t_end=w.t_end)
    n = c.run_to(w.t_end, poll=512)
    t, _, _, err = c.scalars()
    assert err == 0 and t == t_end
    e = errors(w, {k: v.astype(np.float64) for k, v in c.get_state().items()}, ref)
    record("fp32_disk2d_768x256_10orbits", steps=n, oracle_steps=n_ref, **e)
    assert abs(n - n_ref) <= 2
    assert e["rho"] < 2e-5 and e["momentum"] < 1e-4, e
    c.close()


def test_disk3d_slab_fp32_200_steps():
    import paper_1602_02359_b300 as fb
    w = W.disk3d(slab=(248, 16, 40, 16))
    o = oracle.Oracle(w)
    st = w.copy().state
    c = make_ctx(w, fb.F32)
    t = 0.0
    seen = {}
    for n in range(1, 201):
        t += o.step(st, t)
        c.step(want_dt=False)
        if n in (1, 100, 200):
            g = {k: v.astype(np.float64) for k, v in c.get_state().items()}
            seen[n] = errors(w, g, st)
            record(f"fp32_disk3d_slab_1536x16x16_{n}steps", **seen[n])
    for n, e in seen.items():
        assert e["rho"] < 2e-5 and e["e"] < 2e-5 and e["momentum"] < 1e-4, (n, e)
    c.close()


def test_sweep_disks_fp32_batched_1000_steps():
    import paper_1602_02359_b300 as fb
    P = W.batch_params()
    ws = [W.batch_instance(P[i]) for i in SWEEP8]
    ctx = [make_ctx(w, fb.F32, t=0.0, t_end=w.t_end) for w in ws]
    B = fb.FargoBatch(ctx)
    for _ in range(1000):
        B.step(sync=False)
    B.status()
    B.close()
    worst = {}
    for i, w, c in zip(SWEEP8, ws, ctx):
        st = w.copy().state
        t, n = oracle.Oracle(w).run(st, 0.0, w.t_end, max_steps=1000)
        e = errors(w, {k: v.astype(np.float64) for k, v in c.get_state().items()}, st)
        record(f"fp32_batch_member{i}_{w.nx}x{w.ny}_1000steps", **e)
        for k, v in e.items():
            worst[k] = max(worst.get(k, 0.0), v)
        c.close()
    assert worst["rho"] < 2e-5 and worst["momentum"] < 1e-4, worst


@pytest.mark.parametrize("member", [156, 126])
def test_smallest_sweep_disks_fp32_batched_500_orbits(member):
    import paper_1602_02359_b300 as fb
    w = W.batch_instance(W.batch_params()[member])
    ref, t_end, n_ref = stored_state(w, os.path.join(GOLDEN, f"batch_member{member}_500orbits.npz"))
    c = make_ctx(w, fb.F32, t=0.0, t_end=w.t_end)
    B = fb.FargoBatch([c])
    steps, running = B.run(poll=1024)
    B.close()
    t, _, n, err = c.scalars()
    assert err == 0 and running == 0 and t == t_end
    e = errors(w, {k: v.astype(np.float64) for k, v in c.get_state().items()}, ref)
    record(f"fp32_batch_member{member}_500orbits", steps=n, oracle_steps=n_ref, **e)
    assert abs(n - n_ref) < 0.01 * n_ref, (n, n_ref)
    assert e["rho"] < 2e-2 and e["momentum"] < 2e-2, e
    c.close()
