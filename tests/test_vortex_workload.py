"""The Keplerian vortex of Sec. 6 (impact of orbital advection) and the
vortensity diagnostic its study reads, pinned on flows whose vorticity is
known in closed form."""
import math

import numpy as np

import workloads as W


def test_vortensity_of_keplerian_flow_is_half_omega():
    """(1/r) d(r v_K)/dr = Omega/2 = r^-1.5 / 2, to second order in the
    radial spacing (the corner estimate of the unperturbed disk)."""
    errs = []
    for ny in (64, 128):
        w = W.keplerian_vortex(nx=32, ny=ny, k_amp=0.0)
        z = W.vortensity(w, w.state)
        r = w.yf[w.gy + 1:w.gy + w.ny][:, None]
        errs.append(np.max(np.abs(z - 0.5 * r ** -1.5)))
    assert errs[0] < 1e-3 and 3.5 < errs[0] / errs[1] < 4.5, errs


def test_vortensity_of_solid_rotation_and_of_a_radial_shear_free_field():
    """v_phi = 2 r (solid rotation) has curl 4 exactly; adding
    v_r = sin(phi) (curl -(1/r) cos(phi) in the limit) checks the azimuthal
    derivative term and its sign; Sigma = 2 halves both."""
    w = W.keplerian_vortex(nx=256, ny=64, k_amp=0.0)
    st = w.copy().state
    rc = W.centres(w.yf)
    st["vx"][0, :w.ny_t, :] = 2.0 * rc[:, None]
    st["rho"][...] = 2.0
    z = W.vortensity(w, st)
    assert np.max(np.abs(z - 2.0)) < 1e-12
    pc = (np.arange(w.nx) + 0.5) * 2 * math.pi / w.nx
    st["vy"][0, :w.ny_t + 1, :] = np.sin(pc)[None, :]
    z = W.vortensity(w, st)
    r = w.yf[w.gy + 1:w.gy + w.ny][:, None]
    pf = np.arange(w.nx) * 2 * math.pi / w.nx
    expect = (4.0 - np.cos(pf)[None, :] / r) / 2.0
    assert np.max(np.abs(z - expect)) < 1e-3


def test_vortex_initial_condition():
    """Uniform Sigma = 1 and pressure 1/(gamma M^2) (c_s = 0.1); far from
    the vortex the flow is Keplerian; at its centre the vortensity is near
    2K + Omega/2 = -1.5 when the vortex (h = 0.05) is resolved."""
    w = W.keplerian_vortex(nx=1024, ny=256)
    g = w.gamma
    e = w.active(w.state["e"])
    assert np.allclose(w.active(w.state["rho"]), 1.0)
    assert np.allclose(g * (g - 1.0) * e, 0.01)
    z = W.vortensity(w, w.state)
    assert -1.55 < z.min() < -1.4, z.min()
    rc = W.centres(w.yf)[w.gy:w.gy + w.ny]
    far = np.abs(rc - 1.0) > 0.4
    assert np.allclose(w.active(w.state["vx"])[0][far], np.sqrt(1.0 / rc[far])[:, None], atol=1e-12)
