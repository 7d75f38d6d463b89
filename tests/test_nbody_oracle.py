"""Pins of the planetary-integrator oracle (Sec. 3.7, Tab. rk): the
Cash-Karp step's order of accuracy and its quadrature exactness, a
circular two-body orbit, and a three-body run against SciPy's DOP853
integrating Newton's equations for star and planets in an inertial frame
(which checks the star-centred frame's indirect terms)."""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle import nbody as NB


def step_error(f, exact, t0, y0, h):
    return abs(NB.rk_step(f, t0, np.array([y0]), h)[0] - exact(t0 + h))


@pytest.mark.parametrize("case", ["exp", "ty"])
def test_local_error_is_sixth_order(case):
    """One step of a fifth-order method errs by O(h^6): halving h divides
    the error by about 64.  y' = y exercises the weights and the stage
    matrix; y' = t y (non-autonomous) also the nodes against the row sums."""
    if case == "exp":
        f, exact, t0, y0 = (lambda t, y: y), (lambda t: math.exp(t)), 0.0, 1.0
    else:
        f, exact, t0, y0 = (lambda t, y: t * y), (lambda t: math.exp(0.5 * t * t)), 0.3, math.exp(0.045)
    e1 = step_error(f, exact, t0, y0, 0.2)
    e2 = step_error(f, exact, t0, y0, 0.1)
    assert 50.0 < e1 / e2 < 80.0, (e1, e2)


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_polynomial_quadrature_is_exact_to_degree_four(p):
    """y' = t^p, y(0) = 0: a fifth-order method integrates it exactly up to
    p = 4 (sum_i b_i c_i^p = 1/(p+1)); p = 5 is not exact."""
    h = 0.7
    y = NB.rk_step(lambda t, y: np.array([t ** p]), 0.0, np.array([0.0]), h)[0]
    assert abs(y - h ** (p + 1) / (p + 1)) < 1e-15


def test_degree_five_quadrature_is_not_exact():
    h = 0.7
    y = NB.rk_step(lambda t, y: np.array([t ** 5]), 0.0, np.array([0.0]), h)[0]
    assert abs(y - h ** 6 / 6) > 1e-6


def test_circular_two_body_orbit_closes_with_the_reduced_mass():
    """A planet of mass m on a circular orbit of radius 1 around a unit
    star, in the star's frame, has the period 2 pi / sqrt(1 + m); after 400
    steps of one period it is back where it started."""
    m = 1e-3
    om = math.sqrt(1.0 + m)
    y = np.array([[1.0, 0.0, 0.0, 0.0, om, 0.0]])
    n = 400
    h = 2 * math.pi / om / n
    for _ in range(n):
        y = NB.nbody_step(y, [m], 1.0, h)
    assert np.max(np.abs(y[0] - [1.0, 0.0, 0.0, 0.0, om, 0.0])) < 1e-9


def inertial_rhs(masses):
    """Newton's equations for all bodies (the star first) in an inertial frame."""
    nb = len(masses)

    def f(t, s):
        s = s.reshape(nb, 6)
        out = np.zeros_like(s)
        out[:, :3] = s[:, 3:]
        for i in range(nb):
            for j in range(nb):
                if i != j:
                    d = s[j, :3] - s[i, :3]
                    out[i, 3:] += masses[j] * d / np.linalg.norm(d) ** 3
        return out.ravel()
    return f


def three_body_ics():
    m = np.array([1e-3, 5e-4])
    y = np.array([[1.0, 0.0, 0.0, 0.0, 1.0005, 0.0],
                  [-1.1, 1.2, 0.05, -0.5, -0.45, 0.02]])
    return m, y


def test_three_bodies_match_an_inertial_integration():
    """Star (mass 1) and two planets, integrated for about two inner orbits:
    the oracle's star-centred positions and velocities against SciPy's
    DOP853 on the inertial equations, converted to the star's frame.  A
    missing or mis-signed indirect term errs by ~1e-3."""
    m, y = three_body_ics()
    masses = np.concatenate([[1.0], m])
    s0 = np.zeros((3, 6))
    s0[1:] = y                        # star at rest at the origin at t = 0
    T, n = 12.0, 2400
    sol = solve_ivp(inertial_rhs(masses), (0.0, T), s0.ravel(), method="DOP853", rtol=1e-13, atol=1e-15)
    s = sol.y[:, -1].reshape(3, 6)
    ref = s[1:] - s[0]
    h = T / n
    for _ in range(n):
        y = NB.nbody_step(y, m, 1.0, h)
    assert np.max(np.abs(y - ref)) < 1e-8


def test_fixed_star_matches_an_inertial_integration_with_the_star_pinned():
    """indirect=False: the star stays at the origin of an inertial frame."""
    m, y = three_body_ics()
    masses = np.concatenate([[1.0], m])
    f_all = inertial_rhs(masses)

    def f(t, s):
        full = np.concatenate([np.zeros(6), s])
        return f_all(t, full)[6:]

    T, n = 12.0, 2400
    sol = solve_ivp(f, (0.0, T), y.ravel(), method="DOP853", rtol=1e-13, atol=1e-15)
    ref = sol.y[:, -1].reshape(2, 6)
    h = T / n
    for _ in range(n):
        y = NB.nbody_step(y, m, 1.0, h, indirect=False)
    assert np.max(np.abs(y - ref)) < 1e-8


def test_kick_updates_the_velocity_before_the_drift():
    """Free particles (no star, massless): one step with a kick a moves
    x0 by (v0 + h a) h and leaves the velocity at v0 + h a, exactly."""
    y = np.array([[0.3, -0.2, 0.1, 1.0, 2.0, -0.5], [1.0, 1.0, 1.0, 0.0, 0.0, 0.0]])
    a = np.array([[0.5, -1.0, 2.0], [3.0, 0.0, -1.0]])
    h = 0.25
    out = NB.nbody_step(y, [0.0, 0.0], 0.0, h, kick=a)
    v = y[:, 3:] + h * a
    assert np.allclose(out[:, 3:], v, rtol=0, atol=1e-15)
    assert np.allclose(out[:, :3], y[:, :3] + h * v, rtol=0, atol=1e-15)


def test_integrated_planet_on_the_circular_orbit_gives_the_same_potential():
    """The oracle's potential with the planet placed at a given position
    (an integrated planet) reproduces the circular orbit's at that
    position, in a cylindrical and a spherical mesh, and clearing it
    restores the circular orbit."""
    import oracle
    import workloads as W
    for w in (W.disk2d(nx=64, ny=24, q=1e-3), W.random_box(W.SPH, 48, 16, 10, seed=4)):
        o = oracle.Oracle(w)
        t = 1.7
        om = math.sqrt((w.star_mass + w.planet_q) / w.planet_a ** 3) - w.omega_f
        ref = o.potential(t)
        o.set_planet_position((w.planet_a * math.cos(om * t), w.planet_a * math.sin(om * t), 0.0))
        live = o.potential(t)
        assert np.max(np.abs(live - ref)) <= 1e-14 * np.max(np.abs(ref))
        o.set_planet_position(None)
        assert np.array_equal(o.potential(t), ref)


def test_potential_of_several_integrated_planets_superposes():
    """Two integrated planets (one off the midplane) in a spherical mesh:
    the potential is the sum of each planet's alone, less the star's,
    which a massless planet leaves (phi_AB - phi_A - phi_B + phi_0 = 0)."""
    import oracle
    import workloads as W
    w = W.random_box(W.SPH, 48, 16, 10, seed=4)
    o = oracle.Oracle(w)
    a, b = (0.9, 0.3, 0.02), (-0.6, 1.1, -0.05)
    o.set_planet_position([a, b], [1e-3, 4e-4])
    ab = o.potential(0.5)
    o.set_planet_position([a], [1e-3])
    pa = o.potential(0.5)
    o.set_planet_position([b], [4e-4])
    pb = o.potential(0.5)
    o.set_planet_position([a], [0.0])
    p0 = o.potential(0.5)
    assert np.max(np.abs(ab - pa - pb + p0)) <= 1e-14 * np.max(np.abs(ab))
    assert np.max(np.abs(pa - p0)) > 1e-6
