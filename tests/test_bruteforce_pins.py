"""Pin of the C oracle against an independent brute-force restatement.

tests/bruteforce.py restates every sub-step of one update from the paper's
equations (Sec. 3.3, 3.4, App. A, App. B, Eqs. 12-18, 26-38) in a different
form: values sampled at positions of the staggered mesh, every derivative a
difference of two samples over their coordinate difference, metric factors
written term by term, geometry from the closed-form integrals of the metric.
Each sub-step of the oracle is compared with it from the same input state
on 8x8x8 and 8x6x4 meshes (plus 2D disks and a shearing sheet) in every
geometry, with a rotating frame and a planet: the updated fields agree to
1e-13 relative (L-infinity), and the increments they add, the part a wrong
term would change, to 1e-10 of their own size.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from tests import bruteforce as bf

TOL_FIELD = 1e-13
TOL_INCR = 1e-10

CASES = [
    ("cart-8x8x8", lambda: W.random_box(W.CART, 8, 8, 8, g=3, seed=101, nu=2e-2)),
    ("cart-8x6x4-iso", lambda: W.random_box(W.CART, 8, 6, 4, g=3, seed=102, iso=True, nu=2e-2)),
    ("cyl-8x8x8", lambda: W.random_box(W.CYL, 8, 8, 8, g=3, seed=103, nu=2e-2, omega_f=0.3)),
    ("cyl-8x6x4-iso", lambda: W.random_box(W.CYL, 8, 6, 4, g=3, seed=104, iso=True, nu=2e-2, omega_f=-0.2)),
    ("sph-8x8x8", lambda: W.random_box(W.SPH, 8, 8, 8, g=3, seed=105, nu=2e-2, omega_f=0.4)),
    ("sph-8x6x4-iso", lambda: W.random_box(W.SPH, 8, 6, 4, g=3, seed=106, iso=True, nu=2e-2, omega_f=0.1)),
    ("cyl-2d-iso", lambda: W.random_box(W.CYL, 8, 8, 1, g=3, seed=107, iso=True, nu=2e-2, omega_f=0.25)),
    ("sph-2d", lambda: W.random_box(W.SPH, 8, 8, 1, g=3, seed=108, nu=2e-2)),
    ("sheet-8x8", lambda: W.perturb(W.shearing_sheet(nx=8, ny=8, cs=0.3), seed=109, amp=0.05)),
]
IDS = [c[0] for c in CASES]
DT = 3e-3


def rel_linf(a, b):
    s = np.max(np.abs(b))
    return np.max(np.abs(a - b)) / s if s > 0 else np.max(np.abs(a - b))


def agree(w, before, got, want, names):
    """Fields within TOL_FIELD and their increments within TOL_INCR."""
    for n in names:
        g, x, b = got[n], want[n], before[n]
        assert rel_linf(g, x) <= TOL_FIELD, (n, rel_linf(g, x))
        dg, dx = g - b, x - b
        if np.max(np.abs(dx)) > 0:
            assert rel_linf(dg, dx) <= TOL_INCR, (n, rel_linf(dg, dx))
        else:
            assert np.max(np.abs(dg)) == 0.0, n


def velocity_names(w):
    out = ["vx"] if w.nx > 1 else []
    if w.ny > 1:
        out.append("vy")
    if w.nz > 1:
        out.append("vz")
    return out


def prepared(make):
    w = make()
    o = oracle.Oracle(w)
    st = w.copy().state
    o.bc_fill(st)
    return w, o, st


def copy(st):
    return {k: v.copy() for k, v in st.items()}


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_potential_and_courant_step(case):
    w, o, st = prepared(case[1])
    t = 0.37
    ph_o, ph_b = o.potential(t), bf.potential(w, t)
    assert rel_linf(ph_o, ph_b) <= 1e-14 or np.max(np.abs(ph_b)) == 0.0
    v0 = o.v0(st)
    assert np.array_equal(v0, bf.v0_of(w, st))
    rc, dt = o.cfl(st, v0)
    assert rc == 0
    assert abs(dt - bf.courant(w, st, v0)) <= 1e-14 * dt


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_source_substeps(case):
    w, o, st = prepared(case[1])
    vel = velocity_names(w)
    t = 0.21
    # sub-step 1 (its own potential on each side)
    a = copy(st)
    o.substep1(a, o.potential(t), DT)
    b = bf.substep1(w, st, bf.potential(w, t), DT)
    agree(w, st, a, b, vel)
    # artificial viscosity and its heating, from the post-sub-step-1 state
    s1 = a
    a = copy(s1)
    o.artificial_viscosity(a, DT)
    b = bf.artificial_viscosity(w, s1, DT)
    agree(w, s1, a, b, vel + ([] if w.iso else ["e"]))
    # compression heating
    s2 = a
    if not w.iso:
        a = copy(s2)
        o.compression_heating(a, DT)
        agree(w, s2, a, bf.compression_heating(w, s2, DT), ["e"])
    # viscous stresses and their update
    s3 = a
    a = copy(s3)
    o.viscosity(a, DT)
    agree(w, s3, a, bf.viscosity(w, s3, DT), vel)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_transport_substeps(case):
    w, o, st = prepared(case[1])
    names = bf.quantities(w)
    v0 = o.v0(st)
    # left and right momenta (Eqs. 16-17, Tab. momenta)
    pis = o.momenta(st)
    pb = bf.momenta(w, st)
    keys = ["xm", "xp", "ym", "yp", "zm", "zp"]
    for n, arr in zip(keys, pis):
        if n in names:
            assert rel_linf(arr, pb[n]) <= TOL_FIELD, n

    def as_q(s, p):
        return {"rho": s["rho"], "e": s["e"], **dict(zip(keys, p))}

    dt = 0.2 * DT if w.geom == W.CART else DT
    # residual X sweep
    before = as_q(st, pis)
    before = {k: v.copy() for k, v in before.items()}
    sa, pa = copy(st), [p.copy() for p in pis]
    o.transport_x(sa, pa, v0, dt)
    qb = bf.transport_x(w, st, pb, v0, dt)
    agree(w, before, as_q(sa, pa), qb, names)
    # Y and Z sweeps from the X sweep's output
    for axis in ("y", "z"):
        if (axis == "y" and w.ny == 1) or (axis == "z" and w.nz == 1):
            continue
        before = {k: v.copy() for k, v in as_q(sa, pa).items()}
        getattr(o, f"transport_{axis}")(sa, pa, dt)
        qb = getattr(bf, f"transport_{axis}")(w, st, before, dt)
        agree(w, before, as_q(sa, pa), qb, names)
    # uniform orbital step (integer shift + PPA fractional step)
    before = {k: v.copy() for k, v in as_q(sa, pa).items()}
    o.orbital_shift(sa, pa, v0, 7.0 * dt)
    qb = bf.orbital_shift(w, before, v0, 7.0 * dt)
    agree(w, before, as_q(sa, pa), qb, names)
    # new velocities (Eq. 18)
    q = {k: v.copy() for k, v in as_q(sa, pa).items()}
    vb = bf.new_velocities(w, sa, q)
    o.new_velocities(sa, pa)
    for n in velocity_names(w):
        assert rel_linf(sa[n], vb[n]) <= TOL_FIELD, n


def test_orbital_step_with_a_multi_cell_shift_and_both_signs():
    """A ring moved by several cells per step, forward and backward: the
    integer part and the PPA fraction agree with the restatement."""
    for sign in (1.0, -1.0):
        w = W.random_box(W.CYL, 16, 4, 1, g=3, seed=110, iso=True, nu=0.0)
        st = w.copy().state
        st["vx"] *= sign
        o = oracle.Oracle(w)
        o.bc_fill(st)
        v0 = o.v0(st)
        pis = o.momenta(st)
        keys = ["xm", "xp", "ym", "yp", "zm", "zp"]
        q = {"rho": st["rho"].copy(), "e": st["e"].copy(), **{k: p.copy() for k, p in zip(keys, pis)}}
        dt = 2.5
        m = bf.Mesh(w)
        X = [v0[0, j] * dt / (m.R(2 * j + 1, 1) * m.dx) for j in range(m.j0, m.j1)]
        assert min(abs(x) for x in X) > 1.5          # several cells per step
        o.orbital_shift(st, pis, v0, dt)
        qb = bf.orbital_shift(w, q, v0, dt)
        names = bf.quantities(w)
        got = {"rho": st["rho"], **dict(zip(keys, pis))}
        for n in names:
            assert rel_linf(got[n], qb[n]) <= TOL_FIELD, n


@pytest.mark.parametrize("case", CASES[:6], ids=IDS[:6])
def test_whole_step(case):
    """One full update in flow-chart order from the restated sub-steps
    against or_step (same Courant step)."""
    w, o, st = prepared(case[1])
    t = 0.05
    a = copy(st)
    dt = o.step(a, t)
    b = copy(st)
    v0 = bf.v0_of(w, b)
    assert abs(bf.courant(w, b, v0) - dt) <= 1e-14 * dt
    b = bf.substep1(w, b, bf.potential(w, t), dt)
    b = bf.artificial_viscosity(w, b, dt)
    b = bf.compression_heating(w, b, dt)
    b = bf.viscosity(w, b, dt)
    o.bc_fill(b)                                  # cell 9 (its own pins cover the fill)
    q = _transport(w, b, {"rho": b["rho"], "e": b["e"], **bf.momenta(w, b)}, v0, dt)
    b = bf.new_velocities(w, b, q)
    for n in ["rho"] + ([] if w.iso else ["e"]) + velocity_names(w):
        assert rel_linf(a[n], b[n]) <= 1e-12, (n, rel_linf(a[n], b[n]))


def _transport(w, st, q, v0, dt):
    pm = {k: v for k, v in q.items() if k not in ("rho", "e")}
    out = bf.transport_x(w, st, pm, v0, dt)
    full = {"rho": st["rho"].copy(), "e": st["e"].copy(), **{k: v.copy() for k, v in pm.items()}}
    full.update(out)
    out = bf.transport_y(w, st, full, dt)
    full.update(out)
    out = bf.transport_z(w, st, full, dt)
    full.update(out)
    out = bf.orbital_shift(w, full, v0, dt)
    full.update(out)
    return full
