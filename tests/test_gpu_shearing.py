"""The Cartesian shearing sheet (Sec. 2, Tab. momenta, Sec. 3.3) through
the C ABI: FP64 parity with the oracle on a perturbed sheet, the steady
shear flow, and the epicycle of a uniform perturbation in FP64 and FP32."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from tests.gpu_util import compare_state, make_ctx, record

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fargo", [True, False])
def test_shearing_sheet_fp64_matches_oracle(fargo):
    w = W.perturb(W.shearing_sheet(nx=40, ny=48, cs=0.05, u0=5e-4, w0=1e-3, fargo=fargo), seed=9, amp=1e-2,
                  fields=("rho", "vx", "vy"))
    o = oracle.Oracle(w)
    st = w.copy().state
    c = make_ctx(w, t=0.0)
    t = 0.0
    for n in range(5):
        dt_o = o.step(st, t)
        t += dt_o
        dt_g = c.step()
        if n == 0:
            assert dt_g == dt_o, (dt_g, dt_o)
        else:
            assert abs(dt_g - dt_o) <= 1e-12 * dt_o, (n, dt_g, dt_o)
    compare_state(w, c.get_state(), st, 1e-11)
    c.close()


def test_shear_flow_stays_steady():
    w = W.shearing_sheet()
    c = make_ctx(w, t=0.0)
    for _ in range(20):
        c.step()
    g = c.get_state()
    for k in ("rho", "vx", "vy"):
        assert np.max(np.abs(w.active(g[k]) - w.active(w.state[k]))) <= 1e-15, k
    c.close()


@pytest.mark.parametrize("prec_name", ["F64", "F32"])
def test_epicycle(prec_name):
    import paper_1602_02359_b300 as fb
    w0, dt, oort = 1e-3, 0.01, -0.75
    w = W.shearing_sheet(w0=w0, oort_a=oort)
    c = make_ctx(w, getattr(fb, prec_name), t=0.0)
    kappa = math.sqrt(4.0 * (1.0 + oort))
    n = int(round(2 * math.pi / kappa / dt))
    jc = w.gy + w.ny // 2
    yc = W.centres(w.yf)[jc]
    errs = []
    for s in range(1, n + 1):
        c.step_fixed(dt)
        if s % 20 == 0 or s == n:
            g = c.get_state()
            ww = float(g["vy"][0, jc, 0])
            uu = float(g["vx"][0, jc, 0]) - 2.0 * oort * yc
            errs.append(max(abs(ww - w0 * math.cos(kappa * s * dt)),
                            abs(uu + (kappa / 2.0) * w0 * math.sin(kappa * s * dt))))
    record("shearing_epicycle", fp32=int(prec_name == "F32"), max_err_over_w0=max(errs) / w0)
    assert max(errs) < 1e-2 * w0, max(errs) / w0
    c.close()


def test_shearing_needs_a_cartesian_mesh():
    import paper_1602_02359_b300 as fb
    w = W.disk2d(nx=32, ny=16)
    w.shearing = True
    with pytest.raises(fb.FargoError):
        fb.Fargo(w, fb.F64)
