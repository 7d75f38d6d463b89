"""Pins of the oracle's shearing sheet (Sec. 2, Tab. momenta and the
shearing-sheet source terms of Sec. 3.3): the shear flow v_x = 2 A y is an
exact steady state, and a uniform velocity perturbation riding on it
performs the epicycle of the sheet's equations,
    du/dt = -2 (Omega + A) w,   dw/dt = 2 Omega u,
at the epicyclic frequency kappa = sqrt(4 Omega (Omega + A)) with
u = -(kappa / (2 Omega)) w0 sin(kappa t), w = w0 cos(kappa t)."""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def test_shear_flow_is_an_exact_steady_state():
    w = W.shearing_sheet()
    o = oracle.Oracle(w)
    st = w.copy().state
    t = 0.0
    for _ in range(20):
        t += o.step(st, t)
    for k in ("rho", "vx", "vy"):
        assert np.array_equal(st[k], w.state[k]), k


@pytest.mark.parametrize("oort_a", [-0.75, -0.5])
def test_uniform_perturbation_performs_the_epicycle(oort_a):
    w0, dt = 1e-3, 0.01
    w = W.shearing_sheet(w0=w0, oort_a=oort_a)
    o = oracle.Oracle(w)
    st = w.copy().state
    kappa = math.sqrt(4.0 * (1.0 + oort_a))
    jc = w.gy + w.ny // 2
    yc = W.centres(w.yf)[jc]
    n = int(round(2 * math.pi / kappa / dt))
    t = 0.0
    ws, us = [], []
    for _ in range(n):
        o.step(st, t, dt_fixed=dt)
        t += dt
        ws.append(st["vy"][0, jc, 0])
        us.append(st["vx"][0, jc, 0] - 2.0 * oort_a * yc)
    ts = dt * np.arange(1, n + 1)
    w_ex = w0 * np.cos(kappa * ts)
    u_ex = -(kappa / 2.0) * w0 * np.sin(kappa * ts)
    assert np.max(np.abs(np.array(ws) - w_ex)) < 1e-2 * w0
    assert np.max(np.abs(np.array(us) - u_ex)) < 1e-2 * w0
