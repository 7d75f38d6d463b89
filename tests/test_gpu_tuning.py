"""Launch-shape autotuner and the bounded-wait failure check.

The tuned shapes (azimuths per block of the per-cell kernels, segment lengths
of the Y/Z sweeps) run the same compiled kernels on the same cells, so every
result is bit-identical whatever the shape; the autotuner leaves the state
and the time unchanged.  The wait check makes a bounded mbarrier wait run
out on purpose (an arrival that never comes) and reads the error code: no
hang, no fault, and the device stays usable."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import make_ctx

pytestmark = pytest.mark.gpu


def box3d():
    return W.random_box(W.SPH, 300, 70, 20, seed=21, iso=False, nu=1e-3, bc=W.BC_FROZEN)


@pytest.mark.parametrize("shape", [(128, 16, 16), (64, 32, 0), (256, 128, 5)])
def test_launch_shapes_give_identical_results(shape):
    import paper_1602_02359_b300 as fb
    w = box3d()
    a = make_ctx(w, fb.F32)
    b = make_ctx(w, fb.F32)
    b.set_launch_shape(*shape)
    for _ in range(3):
        a.step(want_dt=False)
        b.step(want_dt=False)
    assert a.scalars() == b.scalars()
    ga, gb = a.get_state(), b.get_state()
    for k in ga:
        assert np.array_equal(ga[k], gb[k]), k


def test_autotune_leaves_the_run_unchanged():
    import paper_1602_02359_b300 as fb
    w = box3d()
    a = make_ctx(w, fb.F64, t=0.25)
    b = make_ctx(w, fb.F64, t=0.25)
    cfg = a.autotune(reps=2)
    assert cfg[0] in (64, 128, 256) and cfg[1] >= 1 and cfg[2] >= 1
    assert a.scalars() == b.scalars()
    for k, v in a.get_state().items():
        assert np.array_equal(v, b.get_state()[k]), k
    for _ in range(2):
        a.step(want_dt=False)
        b.step(want_dt=False)
    assert a.scalars() == b.scalars()
    for k, v in a.get_state().items():
        assert np.array_equal(v, b.get_state()[k]), k


def test_launch_shape_outside_the_compiled_bounds_is_rejected():
    import paper_1602_02359_b300 as fb
    c = make_ctx(W.disk2d(nx=96, ny=32), fb.F64)
    with pytest.raises(fb.FargoError) as e:
        c.set_launch_shape(512, 0, 0)
    assert e.value.code == -1


def test_bounded_wait_reports_a_timeout_and_the_device_stays_usable():
    import paper_1602_02359_b300 as fb
    assert fb.debug_wait_timeout(1000) == -7
    assert fb.debug_wait_timeout(1) == -7
    c = make_ctx(W.disk2d(nx=96, ny=32), fb.F64)
    dt = c.step()
    assert dt > 0 and c.scalars()[3] == 0


def test_batch_autotune_leaves_the_run_unchanged():
    """The batch autotuner changes the per-cell grouping and the sweep
    segments of a batch of unequal disks, results-invariant shapes: after
    tuning, the members' states and times are those before it, and steps
    from there agree bit for bit with an untuned batch's."""
    import paper_1602_02359_b300 as fb
    ps = W.batch_params(n=6, seed=5)
    ps = [dict(p, ny=p["ny"] // 4, nx=3 * (p["ny"] // 4)) for p in ps]
    ws = [W.batch_instance(p) for p in ps]
    ca = [make_ctx(w, fb.F32, t=0.0, t_end=w.t_end) for w in ws]
    cb = [make_ctx(w, fb.F32, t=0.0, t_end=w.t_end) for w in ws]
    A, B = fb.FargoBatch(ca), fb.FargoBatch(cb)
    A.step()
    B.step()
    cfg, ms0, ms1 = A.autotune(reps=2)
    assert cfg["cells_per_thread"] in (4, 8, 16, 32) and cfg["segment"] in (-1, 0, 16, 32, 64, 128)
    assert 0 < ms1 <= ms0
    A.status()
    for x, y in zip(ca, cb):
        assert x.scalars() == y.scalars()
        for k, v in x.get_state().items():
            assert np.array_equal(v, y.get_state()[k]), k
    for _ in range(3):
        A.step(sync=False)
        B.step(sync=False)
    A.status()
    B.status()
    for x, y in zip(ca, cb):
        assert x.scalars() == y.scalars()
        for k, v in x.get_state().items():
            assert np.array_equal(v, y.get_state()[k]), k
    A.close()
    B.close()
