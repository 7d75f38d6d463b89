"""Magnetohydrodynamics (Sec. 3.5, MOCCT on Cartesian meshes) through the C
ABI against the oracle: each MHD sub-step alone (the magnetic pressure of
cell 7a, the EMFs of cells 8a-8c, the tension of cell 8d, the constrained
transport of cell 10), full steps with their Courant steps, the divergence
constraint, the paper's current-sheet test and a linear Alfven wave.

Meshes span several blocks of azimuths with a ragged tail (300 = 256 +
44), 2D X-Y, X-Z and Y-Z planes and 3D boxes, periodic and walled.

Tolerances (FP64): sub-steps 1e-12 of each field's largest value (the
kernels contract multiply-adds, the oracle does not); ten full steps
1e-11; Courant steps 1e-12 relative.  FP32: 2e-5 (density) and 1e-4
(velocities, field) in relative L1 after twenty steps."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from tests.gpu_util import make_ctx, record, rel_l1

pytestmark = pytest.mark.gpu

GAS = ("rho", "e", "vx", "vy", "vz")


def face_region(w, k, a):
    """Active cells, plus the upper face of a component staggered along a
    present Y or Z."""
    gz, gy = w.gz, w.gy
    if k in ("vy", "by") and w.ny > 1:
        return a[gz:gz + w.nz, gy:gy + w.ny + 1, :]
    if k in ("vz", "bz") and w.nz > 1:
        return a[gz:gz + w.nz + 1, gy:gy + w.ny, :]
    return w.active(a)


def worst(w, g, o, keys, floor=None):
    """Largest difference of each field over its largest value (or over
    floor[k] when that is larger: a field of second order in a wave's
    amplitude is compared at the scale of the amplitude)."""
    out = {}
    for k in keys:
        a = face_region(w, k, np.asarray(g[k], dtype=np.float64))
        b = face_region(w, k, o[k])
        s = max(np.abs(b).max(), (floor or {}).get(k, 0.0), 1e-300)
        out[k] = float(np.abs(a - b).max() / s)
    return out


def boxes():
    return [
        ("xy", W.random_mhd_box(300, 20, 1, seed=1, eta=0.01)),
        ("xz", W.random_mhd_box(300, 1, 12, seed=2, eta=0.0)),
        ("yz", W.random_mhd_box(1, 24, 20, seed=3, eta=0.02)),
        ("xyz", W.random_mhd_box(300, 10, 6, seed=4, eta=0.01)),
        ("xyz-iso", W.random_mhd_box(40, 12, 8, seed=5, iso=True, eta=0.0, nu=1e-3)),
        ("xyz-reflect", W.random_mhd_box(300, 10, 6, seed=6, eta=0.01, bc=W.BC_REFLECT)),
        ("xy-zerograd", W.random_mhd_box(300, 20, 1, seed=7, eta=0.01, bc=W.BC_ZEROGRAD)),
    ]


def fresh(w, prec=None):
    c = make_ctx(w, prec)
    assert c.mhd
    return c


@pytest.mark.parametrize("name,w", boxes())
def test_mhd_substeps_match_oracle(name, w):
    o = oracle.Oracle(w)
    dt = 2e-3
    keys = GAS + W.MHD_FIELDS
    res = {}
    # each sub-step from the same filled state
    base = w.copy().state
    o.bc_fill(base)
    for phase in ("pressure", "emf", "tension", "ct"):
        st = {k: v.copy() for k, v in base.items()}
        c = fresh(w)
        c.debug_phase(0)
        if phase == "pressure":
            c.debug_phase(10, dt)
            o.mhd_pressure(st, dt)
            res[phase] = worst(w, c.get_state(), st, keys)
        elif phase == "emf":
            c.debug_phase(11, dt)
            E = o.mhd_emf(st, dt)
            g = {f"e{q}": c.get_aux(7 + q) for q in range(3)}
            res[phase] = {}
            for q in range(3):
                s = max(np.abs(E[q]).max(), 1e-300)
                res[phase][f"e{q}"] = float(np.abs(g[f"e{q}"] - E[q]).max() / s)
        elif phase == "tension":
            c.debug_phase(12, dt)
            o.mhd_tension(st, dt)
            res[phase] = worst(w, c.get_state(), st, keys)
        else:
            c.debug_phase(11, dt)
            E = o.mhd_emf(st, dt)
            c.debug_phase(13, dt)
            o.mhd_ct(st, E, dt)
            res[phase] = worst(w, c.get_state(), st, keys)
        c.close()
    for phase, r in res.items():
        record(f"mhd_{phase}_{name}", **r)
        assert max(r.values()) <= 1e-12, (phase, r)


@pytest.mark.parametrize("name,w", boxes())
def test_mhd_steps_match_oracle(name, w):
    o = oracle.Oracle(w)
    st = w.copy().state
    c = fresh(w)
    t = 0.0
    for n in range(10):
        dt_o = o.step(st, t)
        dt_g = c.step()
        assert abs(dt_g - dt_o) <= 1e-12 * dt_o, (n, dt_g, dt_o)
        t += dt_o
    r = worst(w, c.get_state(), st, GAS + W.MHD_FIELDS)
    record(f"mhd_steps_{name}", **r)
    assert max(r.values()) <= 1e-11, r
    c.close()


def test_mhd_divergence_stays_at_round_off_on_the_gpu():
    w = W.random_mhd_box(300, 10, 6, seed=7, eta=0.01)
    o = oracle.Oracle(w)
    c = fresh(w)
    st0 = w.copy().state
    dx, dy, dz = 1.0 / w.nx, w.yf[1] - w.yf[0], w.zf[1] - w.zf[0]
    scale = max(np.abs(st0[k]).max() for k in W.MHD_FIELDS) * max(dy * dz, dx * dz, dx * dy)
    for _ in range(40):
        c.step()
    g = c.get_state()
    d = np.abs(o.mhd_divb(g)).max()
    record("mhd_divb_40_steps", max_abs=d, scale=scale)
    assert d <= 1e-13 * scale
    assert max(np.abs(w.active(g[k] - st0[k])).max() for k in W.MHD_FIELDS) > 1e-3
    c.close()


def test_current_sheet_on_the_gpu():
    """Sec. 5.2's current sheet at its 512 cells to 30 t0: the GPU against
    the oracle step for step (1e-11) and against the erf."""
    w = W.current_sheet()
    o = oracle.Oracle(w)
    st = w.copy().state
    c = make_ctx(w, t=w.t0, t_end=30.0 * w.t0)
    t, n = w.t0, 0
    while t < 30.0 * w.t0 - 1e-15:
        dt_o = o.step(st, t, t_end=30.0 * w.t0)
        dt_g = c.step()
        assert abs(dt_g - dt_o) <= 1e-12 * dt_o
        t += dt_o
        n += 1
    g = c.get_state()
    zc = W.centres(w.zf)[w.gz:w.gz + w.nz]
    by = w.active(g["by"])[:, 0, 0]
    err = np.abs(by - W.current_sheet_profile(zc, t))
    r = worst(w, g, st, ("by", "rho", "e"))
    record("current_sheet_gpu", steps=n, max_err_erf=err.max(), mean_err_erf=err.mean(), vs_oracle=r["by"])
    assert r["by"] <= 1e-11 and err.max() < 2e-3
    c.close()


def test_alfven_wave_on_the_gpu():
    """One period of the linear Alfven wave on 64 x 4 cells: the oracle's
    run (1e-11; v_x, of second order in the amplitude, at the amplitude's
    scale) and its phase (within 0.003 rad)."""
    w = W.alfven_wave(nx=64)
    o = oracle.Oracle(w)
    st = w.copy().state
    c = make_ctx(w, t_end=1.0)
    t = 0.0
    while t < 1.0 - 1e-15:
        dt_o = o.step(st, t, t_end=1.0)
        c.step()
        t += dt_o
    g = c.get_state()
    # v_x and B_x's departures are second order in the amplitude 1e-3
    r = worst(w, g, st, GAS + W.MHD_FIELDS, floor={"vx": 1e-3, "bx": 1e-3})
    xc = W._mhd_coords(w)[0]
    vy = w.active(g["vy"])[0, 0]
    ph = math.atan2(np.mean(vy * np.cos(2 * math.pi * xc)), np.mean(vy * np.sin(2 * math.pi * xc)))
    record("alfven_wave_gpu", phase=ph, **r)
    assert max(r.values()) <= 1e-11 and abs(ph) < 0.003
    c.close()


def test_mhd_fp32_within_stated_tolerance():
    import paper_1602_02359_b300 as fb
    for w in (W.random_mhd_box(300, 10, 6, seed=8, eta=0.01), W.random_mhd_box(300, 20, 1, seed=9)):
        o = oracle.Oracle(w)
        st = w.copy().state
        c = fresh(w, fb.F32)
        t = 0.0
        for _ in range(20):
            t += o.step(st, t)
            c.step()
        g = c.get_state()
        e = {k: rel_l1(face_region(w, k, g[k].astype(np.float64)), face_region(w, k, st[k]))
             for k in ("rho", "vx", "vy") + W.MHD_FIELDS + (("vz",) if w.nz > 1 else ())}
        record(f"mhd_fp32_20_steps_{w.nz}", **e)
        assert e["rho"] < 2e-5 and max(e.values()) < 1e-4, e
        c.close()


def test_mhd_launch_shapes_and_graph_agree_bit_for_bit():
    w = W.random_mhd_box(300, 10, 6, seed=10, eta=0.01)
    out = []
    for bs, graph in ((256, True), (64, True), (256, False)):
        c = fresh(w)
        c.set_launch_shape(bs)
        c.use_graph(graph)
        for _ in range(5):
            c.step()
        out.append(c.get_state())
        c.close()
    for g in out[1:]:
        for k in GAS + W.MHD_FIELDS:
            assert np.array_equal(g[k], out[0][k]), k


def test_passive_field_leaves_the_gas_as_without_it():
    w = W.random_mhd_box(300, 20, 1, seed=11, passive=True)
    h = w.copy()
    h.mhd = False
    cm, ch = fresh(w), make_ctx(h)
    for _ in range(5):
        cm.step_fixed(2e-3)
        ch.step_fixed(2e-3)
    gm, gh = cm.get_state(), ch.get_state()
    for k in GAS:
        assert np.array_equal(gm[k], gh[k]), k
    cm.close()
    ch.close()


def test_mhd_rejected_where_it_does_not_apply():
    import paper_1602_02359_b300 as fb
    cyl = make_ctx(W.random_box(W.CYL, 16, 8, 1, seed=1))
    with pytest.raises(fb.FargoError):
        cyl.enable_mhd()
    disk = make_ctx(W.disk2d(nx=64, ny=16))
    with pytest.raises(fb.FargoError):
        disk.enable_mhd()
    box = make_ctx(W.random_box(W.CART, 16, 8, 1, seed=1, planet=False, fargo=False))
    with pytest.raises(fb.FargoError):
        box.get_field("bx")
    with pytest.raises(fb.FargoError):
        box.enable_mhd(eta=-1.0)
    box.enable_mhd()
    assert np.all(box.get_field("by") == 0.0)
    w = W.random_mhd_box(16, 8, 1, seed=1)
    m = fresh(w)
    with pytest.raises(fb.FargoError):
        fb.FargoBatch([m])
    for c in (cyl, disk, box, m):
        c.close()


def test_field_loop_on_the_gpu_matches_the_oracle_and_the_paper():
    """The loop test of Sec. 5.2 (128 x 64, Y-Z plane, periodic).  FP64 on
    the oracle's run for 100 steps (1e-12 on B and rho, measured 5e-14),
    and both precisions to t = 2 on the paper's magnetic energy 1.235e-7
    within 1 % (tests/golden) and on the oracle's (1e-6 in FP64, 5e-3 in
    FP32).  Step-by-step parity is not carried to
    t = 2: v_z stays near zero in this flow, and the upwind side of Eq. 45's
    estimates along Z follows the sign of a v_z of order 1e-12, which
    rounding flips; the flipped reconstructions then grow apart (1e-11
    relative on rho by step 300).  The energy, an integral, does not."""
    import paper_1602_02359_b300 as fb
    from tests.test_oracle_pins import read_golden
    g = read_golden("field_loop_paper.txt")
    w = W.field_loop()
    o = oracle.Oracle(w)
    st = w.copy().state
    c = make_ctx(w)
    t = 0.0
    for _ in range(100):
        dt_o = o.step(st, t)
        dt_g = c.step()
        assert abs(dt_g - dt_o) <= 1e-12 * dt_o
        t += dt_o
    r = worst(w, c.get_state(), st, ("rho",) + W.MHD_FIELDS)
    c.close()
    assert max(r.values()) <= 1e-12, r
    o.run(st, t, g["t"])
    res = {}
    for prec, name in ((fb.F64, "f64"), (fb.F32, "f32")):
        c = make_ctx(w, prec, t_end=g["t"])
        c.run_to(g["t"])
        gs = {k: np.asarray(v, dtype=np.float64) for k, v in c.get_state().items()}
        res[name] = W.magnetic_energy(w, gs)
        c.close()
    e_o = W.magnetic_energy(w, st)
    record("field_loop_t2", oracle=e_o, steps100_worst=max(r.values()), **res)
    for name, e in res.items():
        assert abs(e - g["magnetic_energy_t2"]) <= 0.01 * g["magnetic_energy_t2"], (name, e)
    # measured: FP64 2e-10 and FP32 1.5e-3 of the oracle's energy
    assert abs(res["f64"] - e_o) <= 1e-6 * e_o and abs(res["f32"] - e_o) <= 5e-3 * e_o, (res, e_o)


@pytest.mark.parametrize("name,w,steps", [
    ("orszag_tang_yz", W.orszag_tang(64), 40),
    ("orszag_tang_xy", W.orszag_tang(64, plane="xy"), 40),
    ("brio_wu", W.brio_wu(400), 60),
    ("rotor", W.mhd_rotor(64), 30),
    ("current_sheet_2d", W.current_sheet_2d(64), 30),
])
def test_papers_mhd_setups_match_oracle(name, w, steps):
    """The MHD tests of Sec. 5.2 at reduced resolution (Orszag-Tang in the
    printed Y-Z plane and laid in X-Y, Brio-Wu with reflecting walls, the
    rotor with reflecting walls, the 2D current sheet): FP64 steps on the
    oracle's (1e-11), and the divergence at round-off."""
    o = oracle.Oracle(w)
    st = w.copy().state
    c = fresh(w)
    t = 0.0
    for n in range(steps):
        dt_o = o.step(st, t)
        dt_g = c.step()
        assert abs(dt_g - dt_o) <= 1e-12 * dt_o, (n, dt_g, dt_o)
        t += dt_o
    g = c.get_state()
    r = worst(w, g, st, GAS + W.MHD_FIELDS)
    bmax = max(np.abs(st[k]).max() for k in W.MHD_FIELDS)
    d = float(np.abs(o.mhd_divb({k: np.asarray(v, dtype=np.float64) for k, v in g.items()})).max())
    record(f"mhd_setup_{name}", steps=steps, divb=d, **r)
    assert max(r.values()) <= 1e-11, r
    assert d <= 1e-13 * bmax
    c.close()
