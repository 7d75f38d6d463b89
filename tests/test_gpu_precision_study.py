"""Single versus double precision on the laminar planet disk of Sec. 6
(single or double precision): the paper's 4000 x 2000 inviscid disk with
an Earth-mass planet, corotating frame, run in FP64 and in this library's
FP32 path (FP32 fields with FP64 islands) side by side for one orbit, the
specific torque of the disk on the planet sampled every quarter orbit.

While the planet's wake is set up the two torques agree: within 10 % of the
largest FP64 torque of the orbit (measured: 0.9 %, 0.4 %, 2.6 %, 6 %).  The
paper's single-precision torque departs after 3-4 orbits; the eight-orbit
study is `python bench.py --workload precision-study`.  The azimuthal
velocities of the two runs differ at t = 0 by the FP32 rounding alone."""
import math

import numpy as np
import pytest

import workloads as W
from tests.gpu_util import make_ctx, record

pytestmark = pytest.mark.gpu


def test_sp_dp_torques_agree_over_the_first_orbit():
    import paper_1602_02359_b300 as fb
    w = W.laminar_disk(orbits=1.0)
    c64 = make_ctx(w, fb.F64, t=0.0, t_end=w.t_end)
    c32 = make_ctx(w, fb.F32, t=0.0, t_end=w.t_end)
    v64 = w.active(c64.get_field("vx"))
    v32 = w.active(c32.get_field("vx")).astype(np.float64)
    assert np.array_equal(v32, v64.astype(np.float32).astype(np.float64))
    w.state = None
    rp = (w.planet_a, 0.0, 0.0)
    hist = []
    for k in range(1, 5):
        t = 0.25 * k * 2 * math.pi
        c64.run_to(t, poll=512)
        c32.run_to(t, poll=512)
        s64, s32 = c64.scalars(), c32.scalars()
        assert s64[3] == 0 and s32[3] == 0, (s64, s32)
        g64 = c64.planet_force(rp, w.planet_eps)[3]
        g32 = c32.planet_force(rp, w.planet_eps)[3]
        hist.append((0.25 * k, g64, g32))
        record("sp_dp_torque_first_orbit", orbits=0.25 * k, torque_fp64=g64, torque_fp32=g32,
               steps_fp64=s64[2], steps_fp32=s32[2])
    h = np.array(hist)
    scale = np.max(np.abs(h[:, 1]))
    assert np.all(np.isfinite(h)) and scale > 0
    assert np.max(np.abs(h[:, 2] - h[:, 1])) < 0.1 * scale, h
    c64.close()
    c32.close()
