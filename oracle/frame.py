"""Frame tracking of a planet (Sec. 3.2, "Splitting source and transport in
practice", and Eq. 13): test infrastructure, FP64, plain Python.

The mesh rotates about the polar axis at Omega_f(t).  When the frame is
made to track a planet (the x axis following it), the rate is updated
before the step (flow-chart cell 5b) to the planet's angular velocity, and
the azimuthal velocities are corrected by Eq. 13 (or_change_frame); the
paper handles the frame's time derivative that way, not as a source term.

The planets are integrated in the star's non-rotating frame
(oracle.nbody).  The mesh axes are those axes rotated by the frame angle
theta(t), the integral of Omega_f: with the rate piecewise constant,
theta(t) = theta_0 + Omega_f t, and a rate change at time t moves theta_0
so that theta is continuous there.  A planet's position enters the mesh's
potential rotated by -theta; a force computed on the mesh is rotated by
+theta back to the integrator's axes.

Pins: tests/test_frame_tracking.py (closed forms: the rate of a circular
orbit, the constant mesh azimuth of a planet on it, continuity of theta,
rotation round trips).
"""
import math

import numpy as np


def tracking_rate(y):
    """Angular velocity about the polar axis of a body with state y =
    (x, y, z, vx, vy, vz): (x vy - y vx) / (x^2 + y^2), the frame rate that
    keeps its azimuth fixed on the mesh."""
    x, yy, vx, vy = y[0], y[1], y[3], y[4]
    return (x * vy - yy * vx) / (x * x + yy * yy)


class FrameClock:
    """theta(t) = theta0 + omega t for a piecewise constant rate omega."""

    def __init__(self, omega=0.0, theta0=0.0):
        self.omega = float(omega)
        self.theta0 = float(theta0)

    def angle(self, t):
        return self.theta0 + self.omega * t

    def change(self, omega_new, t):
        """The rate becomes omega_new at time t; theta is continuous at t."""
        self.theta0 -= (omega_new - self.omega) * t
        self.omega = float(omega_new)


def to_mesh(v, theta):
    """Components (x, y, z) in the integrator's axes -> the mesh's axes
    (rotation by -theta about z)."""
    c, s = math.cos(theta), math.sin(theta)
    v = np.asarray(v, dtype=np.float64)
    return np.array([c * v[0] + s * v[1], -s * v[0] + c * v[1], v[2]])


def from_mesh(v, theta):
    """Components in the mesh's axes -> the integrator's (rotation by +theta)."""
    c, s = math.cos(theta), math.sin(theta)
    v = np.asarray(v, dtype=np.float64)
    return np.array([c * v[0] - s * v[1], s * v[0] + c * v[1], v[2]])
