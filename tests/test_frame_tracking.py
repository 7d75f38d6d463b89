"""Pins of oracle/frame.py, the frame tracking of a planet (Sec. 3.2, Eq. 13),
against closed forms, and of the oracle's tracked, coupled loop against
the conservation Eq. 13 guarantees."""
import math

import numpy as np

import oracle
import workloads as W
from oracle import frame as FR
from oracle import nbody as NB


def test_rate_of_a_circular_orbit_is_keplerian():
    """A body on a circular orbit of radius a about M + m moves at
    sqrt((M + m)/a^3); the rate is independent of its azimuth and of z."""
    for a, mu, ph in ((1.0, 1.0, 0.3), (2.5, 1.001, -2.0), (0.6, 1.0, 3.1)):
        w = math.sqrt(mu / a ** 3)
        y = [a * math.cos(ph), a * math.sin(ph), 0.07, -a * w * math.sin(ph), a * w * math.cos(ph), 0.01]
        assert abs(FR.tracking_rate(y) - w) <= 1e-15 * w


def test_rate_of_a_radial_motion_is_zero_and_sign_follows_the_sense():
    assert FR.tracking_rate([0.8, 0.6, 0.0, 0.8, 0.6, 0.0]) == 0.0
    assert FR.tracking_rate([1.0, 0.0, 0.0, 0.0, -0.5, 0.0]) == -0.5


def test_frame_angle_is_continuous_at_a_rate_change():
    c = FR.FrameClock(0.5)
    t = 3.7
    before = c.angle(t)
    c.change(1.25, t)
    assert abs(c.angle(t) - before) <= 1e-15
    assert abs(c.angle(t + 2.0) - (before + 1.25 * 2.0)) <= 1e-14


def test_rotations_round_trip_and_preserve_length():
    rng = np.random.default_rng(3)
    for _ in range(20):
        v = rng.standard_normal(3)
        th = rng.uniform(-10, 10)
        m = FR.to_mesh(v, th)
        assert np.allclose(FR.from_mesh(m, th), v, rtol=0, atol=1e-15)
        assert abs(np.linalg.norm(m) - np.linalg.norm(v)) <= 1e-15
        assert m[2] == v[2]


def test_tracked_planet_keeps_its_mesh_azimuth():
    """A planet integrated on its circular orbit, the frame set to its rate
    at t = 0: its azimuth on the mesh stays at its initial value (the
    orbit's rate equals the frame's), to the integrator's accuracy."""
    a, ph0 = 1.3, 0.4
    w = math.sqrt(1.0 / a ** 3)
    y = np.array([[a * math.cos(ph0), a * math.sin(ph0), 0.0, -a * w * math.sin(ph0), a * w * math.cos(ph0), 0.0]])
    clock = FR.FrameClock(0.0)
    clock.change(FR.tracking_rate(y[0]), 0.0)
    t, h = 0.0, 0.01
    for _ in range(200):
        y = NB.nbody_step(y, np.array([0.0]), 1.0, h)
        t += h
        p = FR.to_mesh(y[0, :3], clock.angle(t))
        assert abs(math.atan2(p[1], p[0]) - ph0) < 1e-9


def test_tracking_changes_conserve_angular_momentum():
    """Eq. 13 at every rate update: the total angular momentum of the gas
    (the inertial one, frame term included) is unchanged by each change, to
    round-off, while the rate follows an integrated, eccentric planet."""
    w = W.perturb(W.disk2d(nx=96, ny=32), seed=5, amp=1e-2)
    o = oracle.Oracle(w)
    st = w.copy().state
    y = np.array([[1.0, 0.0, 0.0, 0.0, 1.08, 0.0]])
    clock = FR.FrameClock(w.omega_f)
    t = 0.0
    for _ in range(5):
        before = o.sums(st)[2]
        om = FR.tracking_rate(y[0])
        o.change_frame(st, om, t)
        clock.change(om, t)
        after = o.sums(st)[2]
        assert abs(after - before) <= 1e-13 * abs(before)
        o.set_planet_position(FR.to_mesh(y[0, :3], clock.angle(t)))
        t += o.step(st, t)
        y = NB.nbody_step(y, np.array([w.planet_q]), 1.0, 0.05)
