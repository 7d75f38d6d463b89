"""Orbital advection of the magnetic field (Sec. 3.6, cell 11) through the C
ABI against the oracle, on Cartesian shearing sheets with a magnetic field:
full steps with their Courant steps (2D and 3D, frozen walls and periodic
Y, resistive and ideal, an azimuthal ring of 300 cells: a ragged tail over
the 256-wide blocks), the divergence constraint, and the closed form of a
uniform field wound up by the Keplerian shear (Eq. 52).

Tolerances as the other MHD parity tests: FP64 1e-11 of each field's
largest value after ten steps and 1e-12 on the Courant steps; FP32 2e-5
(density) and 1e-4 (velocities, field) in relative L1 after twenty steps."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.gpu_util import make_ctx, rel_l1
from tests.test_gpu_mhd import GAS, worst

pytestmark = pytest.mark.gpu


def sheets():
    return [
        ("2d-walls", W.mhd_shearing_sheet(300, 24, 1, amp=0.002, seed=1, vamp=0.02, eta=0.002)),
        ("3d-walls", W.mhd_shearing_sheet(64, 12, 8, amp=0.002, seed=2, vamp=0.02)),
        ("2d-periodic", W.mhd_shearing_sheet(128, 16, 1, amp=0.002, seed=3, vamp=0.02, bcy=W.BC_PERIODIC)),
        ("3d-passive", W.mhd_shearing_sheet(48, 10, 6, amp=0.002, seed=4, vamp=0.02, passive=True)),
    ]


@pytest.mark.parametrize("name,w", sheets())
def test_sheet_steps_match_oracle(name, w):
    import paper_1602_02359_b300 as fb
    o = oracle.Oracle(w)
    st = w.copy().state
    c = make_ctx(w, fb.F64)
    assert c.mhd
    t = 0.0
    for n in range(10):
        dt_o = o.step(st, t)
        dt_g = c.step()
        assert abs(dt_g - dt_o) <= 1e-12 * dt_o, (n, dt_g, dt_o)
        t += dt_o
    r = worst(w, c.get_state(), st, GAS + W.MHD_FIELDS)
    assert max(r.values()) <= 1e-11, r
    c.close()


def test_sheet_fp32_within_stated_tolerance():
    import paper_1602_02359_b300 as fb
    w = W.mhd_shearing_sheet(300, 24, 1, amp=0.002, seed=5, vamp=0.02)
    o = oracle.Oracle(w)
    st = w.copy().state
    c = make_ctx(w, fb.F32)
    t = 0.0
    for _ in range(20):
        dt = o.step(st, t)
        c.step_fixed(dt)
        t += dt
    g = c.get_state()
    assert rel_l1(w.active(g["rho"]), w.active(st["rho"])) <= 2e-5
    for k in ("vx", "vy") + W.MHD_FIELDS:
        if np.abs(w.active(st[k])).max() > 0:
            assert rel_l1(w.active(g[k]), w.active(st[k])) <= 1e-4, k
    c.close()


def test_sheet_divergence_and_winding_on_the_gpu():
    """Forty steps of a perturbed 3D sheet keep the net flux out of every
    cell at round-off; a uniform field in the Keplerian sheet winds up as
    B_x = 2 A t B_y0 in the rows the walls have not reached."""
    import paper_1602_02359_b300 as fb
    w = W.mhd_shearing_sheet(64, 12, 8, amp=0.002, seed=6, vamp=0.02)
    o = oracle.Oracle(w)
    c = make_ctx(w, fb.F64)
    st0 = w.copy().state
    dx, dy, dz = (w.xmax - w.xmin) / w.nx, w.yf[1] - w.yf[0], w.zf[1] - w.zf[0]
    scale = max(np.abs(st0[k]).max() for k in W.MHD_FIELDS) * max(dy * dz, dx * dz, dx * dy)
    for _ in range(40):
        c.step()
    g = c.get_state()
    assert np.abs(o.mhd_divb(g)).max() <= 1e-13 * scale
    c.close()

    by0, A = 0.05, -0.75
    w = W.mhd_shearing_sheet(300, 40, 1, b0=(0.0, by0, 0.0), oort_a=A)
    c = make_ctx(w, fb.F64)
    t = 0.0
    for _ in range(3):
        t += c.step()
    g = c.get_state()
    inner = w.active(g["bx"])[:, 12:-12, :]
    assert np.abs(inner - 2 * A * t * by0).max() <= 1e-12, t
    c.close()


def test_sheet_fp32_two_hundred_steps():
    """The FP32 MHD sheet with orbital advection of the field over 200 steps
    of its own Courant step against the FP64 oracle stepped with the same
    steps: 2e-5 relative L1 on density, 1e-4 on the velocities and the
    field."""
    import paper_1602_02359_b300 as fb
    w = W.mhd_shearing_sheet(128, 24, 1, amp=0.002, seed=8, vamp=0.02, eta=0.001)
    o = oracle.Oracle(w)
    st = w.copy().state
    c = make_ctx(w, fb.F32)
    t = 0.0
    for _ in range(200):
        dt = o.step(st, t)
        c.step_fixed(dt)
        t += dt
    g = c.get_state()
    errs = {"rho": rel_l1(w.active(g["rho"]), w.active(st["rho"]))}
    for k in ("vx", "vy") + W.MHD_FIELDS:
        if np.abs(w.active(st[k])).max() > 0:
            errs[k] = rel_l1(w.active(g[k]), w.active(st[k]))
    assert errs["rho"] <= 2e-5, errs
    assert max(v for k, v in errs.items() if k != "rho") <= 1e-4, errs
    c.close()
