"""The planetary integrator on the device (fargo_nbody_rk5_async,
fargo_planets_force_async, fargo_planets_advance_async) against the FP64
oracle of Sec. 3.7 (oracle/nbody.py and the oracle's planet force).

Tolerance: 1e-12 absolute on positions and velocities of order one after
50 steps (the device contracts products into fused multiply-adds and sums
the pull of the other planets in another rounding order)."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import nbody as NB
from tests.gpu_util import compare_state, make_ctx, record

pytestmark = pytest.mark.gpu


def planets(n, seed):
    """n planets on mildly eccentric, inclined orbits between r = 0.6 and 2."""
    rng = np.random.default_rng(seed)
    y = np.zeros((n, 6))
    a = np.sort(rng.uniform(0.6, 2.0, size=n))
    ph = rng.uniform(0, 2 * math.pi, size=n)
    for i in range(n):
        r = a[i]
        v = math.sqrt(1.0 / r) * (1.0 + 0.05 * rng.uniform(-1, 1))
        y[i] = [r * math.cos(ph[i]), r * math.sin(ph[i]), 0.02 * rng.uniform(-1, 1),
                -v * math.sin(ph[i]), v * math.cos(ph[i]), 0.01 * rng.uniform(-1, 1)]
    m = 10.0 ** rng.uniform(-5, -3, size=n)
    return y, m


def dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("n,indirect", [(1, True), (5, True), (5, False), (32, True)])
def test_rk5_matches_oracle(n, indirect):
    import torch
    import paper_1602_02359_b300 as fb
    y, m = planets(n, 10 + n)
    yd, md = dev(y), dev(m)
    h = 0.01
    for _ in range(50):
        fb.nbody_rk5_async(n, yd.data_ptr(), md.data_ptr(), 1.0, h, indirect=indirect)
        y = NB.nbody_step(y, m, 1.0, h, indirect=indirect)
    torch.cuda.synchronize()
    e = np.max(np.abs(yd.cpu().numpy() - y))
    record("nbody_rk5_vs_oracle", n=n, indirect=int(indirect), max_abs=e)
    assert e < 1e-12


def test_rk5_kick_and_step_on_the_device():
    """The gas kick less the star's, and h read from device memory."""
    import torch
    import paper_1602_02359_b300 as fb
    y, m = planets(4, 3)
    rng = np.random.default_rng(4)
    kick = rng.uniform(-1e-4, 1e-4, size=(4, 4))
    star = rng.uniform(-1e-5, 1e-5, size=4)
    yd, md, kd, sd, hd = dev(y), dev(m), dev(kick), dev(star), dev([0.02])
    fb.nbody_rk5_async(4, yd.data_ptr(), md.data_ptr(), 1.0, h=123.0, h_ptr=hd.data_ptr(), kick_ptr=kd.data_ptr(),
                       kick_stride=4, kick_star_ptr=sd.data_ptr())
    torch.cuda.synchronize()
    ref = NB.nbody_step(y, m, 1.0, 0.02, kick=kick[:, :3] - star[None, :3])
    assert np.max(np.abs(yd.cpu().numpy() - ref)) < 1e-14


def test_rk5_rejects_bad_arguments():
    import paper_1602_02359_b300 as fb
    y, m = planets(2, 1)
    yd, md = dev(np.zeros((33, 6))), dev(np.ones(33) * 1e-4)
    with pytest.raises(fb.FargoError):
        fb.nbody_rk5_async(33, yd.data_ptr(), md.data_ptr(), 1.0, 0.01)
    with pytest.raises(fb.FargoError):
        fb.nbody_rk5_async(0, yd.data_ptr(), md.data_ptr(), 1.0, 0.01)
    with pytest.raises(fb.FargoError):
        fb.nbody_rk5_async(2, yd.data_ptr() + 4, md.data_ptr(), 1.0, 0.01)
    with pytest.raises(fb.FargoError):
        fb.nbody_rk5_async(2, yd.data_ptr(), md.data_ptr(), 1.0, 0.01, kick_ptr=md.data_ptr(), kick_stride=2)


def lumpy_disk(seed):
    w = W.disk2d(nx=300, ny=70, q=1e-3)
    rng = np.random.default_rng(seed)
    w.state["rho"] *= 1.0 + 0.3 * rng.uniform(-1, 1, size=w.state["rho"].shape)
    return w


def test_planets_force_equals_single_planet_calls():
    import torch
    w = lumpy_disk(6)
    c = make_ctx(w)
    y, _ = planets(3, 7)
    yd = dev(y)
    out = torch.zeros(12, dtype=torch.float64, device="cuda")
    for bm08 in (False, True):
        c.planets_force_async(3, yd.data_ptr(), 6, 0.03, out.data_ptr(), bm08)
        single = [c.planet_force(tuple(y[i, :3]), 0.03, bm08) for i in range(3)]   # synchronises
        got = out.cpu().numpy().reshape(3, 4)
        assert np.array_equal(got, np.array(single)), (got, single)
    c.close()


@pytest.mark.parametrize("indirect,bm08", [(True, False), (True, True), (False, False)])
def test_planets_advance_matches_oracle(indirect, bm08):
    """After one hydrodynamical step: the gas force on each planet (and on
    the star) from the oracle on the stepped state, the kick and one
    Cash-Karp step by that step's dt, against the device chain."""
    import torch
    w = lumpy_disk(8)
    c = make_ctx(w)
    c.step()
    t, dt, _, err = c.scalars()
    assert err == 0 and dt > 0
    st = c.get_state()
    y, m = planets(3, 9)
    yd, md = dev(y), dev(m)
    c.planets_advance_async(3, yd.data_ptr(), md.data_ptr(), 0.03, bm08, indirect)
    torch.cuda.synchronize()
    o = oracle.Oracle(w)
    acc = np.array([o.planet_force(st, tuple(y[i, :3]), 0.03, bm08)[:3] for i in range(3)])
    if indirect:
        acc = acc - np.array(o.planet_force(st, (0.0, 0.0, 0.0), 0.0, False)[:3])[None, :]
    ref = NB.nbody_step(y, m, w.star_mass, dt, kick=acc, indirect=indirect)
    e = np.max(np.abs(yd.cpu().numpy() - ref))
    record("planets_advance_vs_oracle", indirect=int(indirect), bm08=int(bm08), max_abs=e)
    assert e < 1e-12
    c.close()


def test_planet_coupled_to_the_step_matches_oracle():
    """The step's planet read from the integrator's state on the device
    (fargo_set_planet_source): four rounds of step, gas force, kick and
    Cash-Karp step, against the same loop in the oracle (the planet's
    position fed to its potential each step)."""
    import torch
    w = lumpy_disk(12)
    eps = w.planet_eps
    o = oracle.Oracle(w)
    st = w.copy().state
    c = make_ctx(w)
    q = w.planet_q
    y = np.array([[1.0, 0.0, 0.0, 0.0, math.sqrt(1.0 + q), 0.0],
                  [1.45, 0.35, 0.0, -0.2, 0.75, 0.0]])
    m = np.array([q, 1e-5])
    yd, md = dev(y), dev(m)
    c.set_planet_source(yd.data_ptr())
    t = 0.0
    for n in range(4):
        dt_g = c.step()
        c.planets_advance_async(2, yd.data_ptr(), md.data_ptr(), eps, False, True)
        o.set_planet_position(y[0, :3])
        dt_o = o.step(st, t)
        t += dt_o
        assert abs(dt_g - dt_o) <= 1e-12 * dt_o, (n, dt_g, dt_o)
        acc = np.array([o.planet_force(st, tuple(y[i, :3]), eps)[:3] for i in range(2)])
        acc -= np.array(o.planet_force(st, (0.0, 0.0, 0.0), 0.0)[:3])[None, :]
        y = NB.nbody_step(y, m, 1.0, dt_o, kick=acc)
    torch.cuda.synchronize()
    compare_state(w, c.get_state(), st, 1e-11)
    e = np.max(np.abs(yd.cpu().numpy() - y))
    record("planet_coupled_vs_oracle", max_abs=e)
    assert e < 1e-12
    c.close()


def test_two_planets_in_the_potential_coupled_to_the_step_match_oracle():
    """Both integrated planets drive the step's potential (n = 2, masses on
    the device): four coupled rounds against the oracle's loop."""
    import torch
    w = lumpy_disk(14)
    eps = w.planet_eps
    o = oracle.Oracle(w)
    st = w.copy().state
    c = make_ctx(w)
    y = np.array([[1.0, 0.0, 0.0, 0.0, math.sqrt(1.0 + w.planet_q), 0.0],
                  [1.5, 0.4, 0.0, -0.25, 0.76, 0.0]])
    m = np.array([w.planet_q, 3e-4])
    yd, md = dev(y), dev(m)
    c.set_planet_source(yd.data_ptr(), 2, 6, md.data_ptr())
    t = 0.0
    for n in range(4):
        dt_g = c.step()
        c.planets_advance_async(2, yd.data_ptr(), md.data_ptr(), eps, False, True)
        o.set_planet_position(y[:, :3], m)
        dt_o = o.step(st, t)
        t += dt_o
        assert abs(dt_g - dt_o) <= 1e-12 * dt_o, (n, dt_g, dt_o)
        acc = np.array([o.planet_force(st, tuple(y[i, :3]), eps)[:3] for i in range(2)])
        acc -= np.array(o.planet_force(st, (0.0, 0.0, 0.0), 0.0)[:3])[None, :]
        y = NB.nbody_step(y, m, 1.0, dt_o, kick=acc)
    torch.cuda.synchronize()
    compare_state(w, c.get_state(), st, 1e-11)
    e = np.max(np.abs(yd.cpu().numpy() - y))
    record("two_planets_coupled_vs_oracle", max_abs=e)
    assert e < 1e-12
    c.close()


def test_clearing_the_planet_source_restores_the_circular_orbit():
    import paper_1602_02359_b300 as fb
    w = lumpy_disk(13)
    a, b = make_ctx(w), make_ctx(w)
    pos = dev([0.9, 0.3, 0.0])
    a.set_planet_source(pos.data_ptr())
    a.step()                       # rewrites the planet tables
    a.set_state(w.state)
    a.set_time(0.0)
    a.set_planet_source(None)      # back to the circular orbit
    a.step()
    b.step()
    ga, gb = a.get_state(), b.get_state()
    for k in ("rho", "vx", "vy"):
        assert np.array_equal(ga[k], gb[k]), k
    with pytest.raises(fb.FargoError):
        make_ctx(W.random_box(W.CART, 16, 8, 1, seed=1, planet=False)).set_planet_source(pos.data_ptr())
    with pytest.raises(fb.FargoError):   # several planets need their masses
        a.set_planet_source(pos.data_ptr(), 2, 3)
    big = dev(np.zeros((9, 3)))
    with pytest.raises(fb.FargoError):   # beyond FARGO_MAX_POT_PLANETS
        a.set_planet_source(big.data_ptr(), 9, 3, dev(np.ones(9)).data_ptr())
    a.close()
    b.close()
