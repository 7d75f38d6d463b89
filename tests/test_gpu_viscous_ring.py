"""Viscous spreading of a gaseous ring (Sec. 5.1) through the C ABI
(fargo_step, fargo_run_to): FP64 against the oracle step for step and run
against run, and FP64 and FP32 against the analytic solution at the
paper's last comparison time.

The ring is axisymmetric, one azimuthal cell; 512 evenly spaced radial
cells on 0.1 <= r <= 1.6, nu = 1e-5, started from the analytic profile at
t = 100, Courant number 0.3.  Bounds on the analytic error are those the
oracle meets with about a factor two to spare (its own errors: 0.16 % at
t = 300, 0.58 % at t = 1100, L1).
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.gpu_util import active_faces, make_ctx, record, rel_l1

pytestmark = pytest.mark.gpu

NU = 1e-5


def ring_l1(w, rho, t):
    r = W.centres(w.yf)[w.gy:w.gy + w.ny]
    sig = w.active(rho)[0, :, 0].astype(np.float64)
    ana, _ = W.viscous_ring_profile(r, t, NU)
    return np.sum(np.abs(sig - ana)) / np.sum(ana)


def test_viscous_ring_fp64_lockstep_with_oracle():
    """300 steps side by side: each Courant step within 1e-9 relative
    (measured 1.2e-11) and the density within 1e-11 relative L1 (measured
    1.8e-13) after 300 steps."""
    w = W.viscous_ring()
    o = oracle.Oracle(w)
    st = w.copy().state
    c = make_ctx(w, t=w.t0, t_end=w.t_end)
    t, worst = w.t0, 0.0
    for n in range(300):
        dto = o.step(st, t, w.t_end)
        dtg = c.step()
        worst = max(worst, abs(dtg - dto) / dto)
        t += dto
    e = rel_l1(w.active(c.get_field("rho")), w.active(st["rho"]))
    record("viscous_ring_fp64_lockstep", steps=300, dt_rel=worst, rho_rel_l1=e)
    assert worst < 1e-9 and e < 1e-11, (worst, e)
    c.close()


def test_viscous_ring_fp64_run_matches_oracle_run_and_analytic():
    """Independent runs to t = 300 (each with its own Courant steps: 4025 on
    the GPU and in the oracle) agree to 2.2e-11 relative L1, against their
    error of 1.6e-3 against the analytic solution; the GPU run then follows
    the analytic solution to t = 1100 (0.62 %)."""
    w = W.viscous_ring()
    o = oracle.Oracle(w)
    st = w.copy().state
    t_o, n_o = o.run(st, w.t0, 300.0)
    c = make_ctx(w, t=w.t0, t_end=300.0)
    c.run_to(300.0, poll=256)
    t_g, _, n_g, err = c.scalars()
    assert err == 0 and t_g == t_o == 300.0
    assert n_g == n_o, (n_g, n_o)
    rho = c.get_field("rho")
    e_go = rel_l1(w.active(rho), w.active(st["rho"]))
    e_ga = ring_l1(w, rho, 300.0)
    record("viscous_ring_fp64_t300", steps=n_g, oracle_steps=n_o, rel_l1_vs_oracle=e_go, rel_l1_vs_analytic=e_ga)
    assert e_go < 1e-9 and e_ga < 3e-3, (e_go, e_ga)
    c.set_time(300.0, w.t_end)
    c.run_to(w.t_end, poll=256)
    t_g, _, n_g, err = c.scalars()
    assert err == 0 and t_g == w.t_end
    e = ring_l1(w, c.get_field("rho"), w.t_end)
    record("viscous_ring_fp64_vs_analytic", t=w.t_end, rel_l1=e, steps=n_g)
    assert e < 1.2e-2
    c.close()


def test_viscous_ring_fp32_follows_analytic():
    """FP32 fields: 0.20 % L1 at t = 300 and 0.64 % at t = 1100, against
    0.16 % and 0.62 % in FP64.  Each step changes the Keplerian v_phi by
    about 3e-7 of itself through the viscous torque, a few FP32 units in
    the last place of v_phi; the FP32 step keeps v_phi relative to a
    per-ring reference, so the torque is not rounded away (stored as v_phi
    itself it was: 0.95 % and 2.3 %, the precision question of Sec. 6).  Bounds at about twice
    the measured errors."""
    import paper_1602_02359_b300 as fb
    w = W.viscous_ring()
    c = make_ctx(w, fb.F32, t=w.t0, t_end=300.0)
    c.run_to(300.0, poll=256)
    assert c.scalars()[3] == 0
    e300 = ring_l1(w, c.get_field("rho"), 300.0)
    c.set_time(300.0, w.t_end)
    c.run_to(w.t_end, poll=256)
    t_g, _, n_g, err = c.scalars()
    assert err == 0 and t_g == w.t_end
    e = ring_l1(w, c.get_field("rho"), w.t_end)
    record("viscous_ring_fp32_vs_analytic", l1_t300=e300, l1_t1100=e, steps=n_g)
    assert e300 < 4e-3 and e < 1.3e-2, (e300, e)
    c.close()
