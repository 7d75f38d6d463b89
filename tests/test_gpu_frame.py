"""Frame change (Sec. 3.2, Eq. 13) through the C ABI (fargo_change_frame)
against the oracle: the corrected state, the angular momentum, and the
steps that follow in the new frame (planet included), FP64; the FP32
correction is the FP64 one rounded once."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.gpu_util import compare_state, make_ctx

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("geom", [W.CYL, W.SPH])
def test_change_frame_then_steps_match_oracle(geom):
    dims = (70, 33, 1) if geom == W.CYL else (64, 24, 14)
    w = W.random_box(geom, *dims, g=3, seed=11, iso=geom == W.CYL, nu=1e-3, omega_f=0.3)
    o = oracle.Oracle(w)
    st = w.copy().state
    c = make_ctx(w, t=0.25)
    t = 0.25
    for _ in range(2):
        t += o.step(st, t)
        c.step()
    l0 = c.sums()[2]
    o.change_frame(st, 1.1, t)
    c.change_frame(1.1)
    assert abs(c.sums()[2] - l0) <= 1e-13 * abs(l0)
    compare_state(w, c.get_state(), st, 1e-12)
    for n in range(3):
        dt_o = o.step(st, t)
        t += dt_o
        dt_g = c.step()
        assert abs(dt_g - dt_o) <= 1e-12 * dt_o, (n, dt_g, dt_o)
    compare_state(w, c.get_state(), st, 1e-11)
    c.close()


def test_change_frame_fp32_is_the_rounded_fp64_correction():
    import paper_1602_02359_b300 as fb
    w = W.disk2d(nx=96, ny=40)
    c = make_ctx(w, fb.F32)
    v = c.get_field("vx").astype(np.float64)
    c.change_frame(0.9)
    R = W.centres(w.yf)[None, :, None]
    ref = (v[:w.nz_t, :w.ny_t] - 0.9 * R).astype(np.float32)
    assert np.array_equal(c.get_field("vx")[:w.nz_t, :w.ny_t], ref)
    c.close()


def test_change_frame_refusals():
    import paper_1602_02359_b300 as fb
    c = make_ctx(W.random_box(W.CART, 16, 8, 1, seed=1, planet=False))
    with pytest.raises(fb.FargoError):
        c.change_frame(0.5)
    c.close()
    a, b = make_ctx(W.disk2d(nx=64, ny=16)), make_ctx(W.disk2d(nx=64, ny=20))
    bt = fb.FargoBatch([a, b])
    with pytest.raises(fb.FargoError):
        a.change_frame(0.5)
    with pytest.raises(fb.FargoError):
        a.change_frame(float("nan"))
    bt.close()
    a.change_frame(0.5)   # no longer held by a batch
    a.close()
    b.close()
