"""Orbital advection and vortensity (Sec. 6, impact of orbital advection):
the vortex in a Keplerian disk, FP64, with and without orbital advection,
through the C ABI.  The paper finds vortensity far better conserved with
orbital advection; here, at 512 x 128 over two orbits of the vortex, the
vortensity minimum must stay deeper with it, and orbital advection must
take several times fewer steps (its Courant step is set by the sound speed,
not by the Keplerian flow).  The full study is
`python bench.py --workload vortex-study`."""
import math

import pytest

import workloads as W
from tests.gpu_util import make_ctx, record

pytestmark = pytest.mark.gpu


def test_orbital_advection_keeps_the_vortex():
    out = {}
    for fargo in (True, False):
        w = W.keplerian_vortex(nx=512, ny=128, fargo=fargo, orbits=2.0)
        z0 = W.vortensity(w, w.state).min()
        c = make_ctx(w, t=0.0, t_end=w.t_end)
        c.run_to(w.t_end, poll=1024)
        t, _, n, err = c.scalars()
        assert err == 0 and t == w.t_end
        z = W.vortensity(w, c.get_state()).min()
        out[fargo] = (z, n)
        record("vortex_512x128_2orbits", fargo=int(fargo), vortensity_min_t0=z0, vortensity_min=z, steps=n)
        c.close()
    (z_f, n_f), (z_s, n_s) = out[True], out[False]
    assert z_f < z_s, (z_f, z_s)
    assert n_s > 3 * n_f, (n_f, n_s)
