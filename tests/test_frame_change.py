"""Pins of the oracle's frame change (Sec. 3.2, Eq. 13): it conserves the
angular momentum exactly (up to rounding), keeps the planet where it is,
and leaves the physics unchanged: stepping in a rotating frame and changing
back reproduces the steps taken in the original frame."""
import numpy as np
import pytest

import oracle
import workloads as W


@pytest.mark.parametrize("geom", [W.CYL, W.SPH])
def test_frame_change_conserves_angular_momentum(geom):
    """The X momentum total includes R^2 Omega_f rho: a wrong sign or lever
    arm in Eq. 13 changes it by about 2 (Omega' - Omega) sum rho R^2 V."""
    dims = (40, 24, 1) if geom == W.CYL else (32, 20, 10)
    w = W.random_box(geom, *dims, g=3, seed=5, omega_f=0.7)
    o = oracle.Oracle(w)
    st = w.copy().state
    m0, e0, l0 = o.sums(st)
    o.change_frame(st, 0.2, 0.37)
    m1, e1, l1 = o.sums(st)
    assert m1 == m0 and e1 == e0
    assert abs(l1 - l0) <= 1e-13 * abs(l0), (l0, l1)
    assert o.p.omega_f == 0.2


def test_frame_change_keeps_the_planet_in_place():
    w = W.disk2d(nx=64, ny=24, q=1e-3)
    o = oracle.Oracle(w)
    t1 = 3.1
    before = o.potential(t1)
    o.change_frame(w.copy().state, 0.6, t1)
    after = o.potential(t1)
    assert np.max(np.abs(after - before)) <= 1e-12 * np.max(np.abs(before))
    # and then it moves at the new relative rate
    om_p = np.sqrt(1.0 + w.planet_q)
    assert abs(o.p.planet_phase0 - 0.6 * t1) < 1e-15
    assert abs((o.p.planet_phase0 + (om_p - 0.6) * t1) - om_p * t1) < 1e-14


def test_steps_in_a_rotating_frame_match_the_inertial_frame():
    """An axisymmetric viscous disk (the orbital step is then the identity):
    five fixed steps in the inertial frame, against a change to Omega = 0.8,
    the same five steps and a change back.  Only the Coriolis and
    centrifugal bookkeeping and the frame terms of the discrete viscous
    stress (which cancel only to truncation order) differ: measured 8e-12
    (density) and 7e-10 (v_phi) relative to each field's size, and 2e-6 for
    v_r, the small residual of gravity and rotation, measured against its
    own much smaller size.  Changing the rate without Eq. 13 departs by
    more than a thousand times v_r's size."""
    w = W.disk2d(nx=32, ny=48, q=0.0, nu=1e-4)
    a = w.copy().state
    b = w.copy().state
    oa, ob = oracle.Oracle(w), oracle.Oracle(w)
    dt = 2e-3
    ob.change_frame(b, 0.8, 0.0)
    t = 0.0
    for _ in range(5):
        oa.step(a, t, dt_fixed=dt)
        ob.step(b, t, dt_fixed=dt)
        t += dt
    ob.change_frame(b, 0.0, t)
    for k, tol in (("rho", 1e-10), ("vx", 1e-8), ("vy", 1e-5)):
        d = np.max(np.abs(w.active(a[k]) - w.active(b[k])))
        assert d <= tol * np.max(np.abs(w.active(a[k]))), (k, d)
