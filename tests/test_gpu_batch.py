"""The batched engine (fargo_batch_* through the C ABI).

Members run the single-instance kernels' per-cell and per-ring source code,
compiled into other kernels: the compiler may fuse a multiply and an add
into one rounding in one kernel and not in the other, so a member stepped
inside a batch agrees with the same context stepped alone to rounding, not
bit for bit (measured: 8e-15 relative L-inf in FP64 and 5e-6 in FP32 after
four steps of the mixed set below; the FP32 figure is larger because a
one-ulp change can flip a slope limiter).  The FP64 oracle closes the loop
for the batched path directly: first-step dt bit-exact, fields within the
stated tolerances.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.gpu_util import compare_state, make_ctx, momentum_density, rel_l1

pytestmark = pytest.mark.gpu


def mixed_members():
    """Uneven meshes, geometries, equations of state and boundary conditions:
    several ring-chunk groups (nx 37 .. 1100), every quantity count of the
    sweeps (3 .. 8), with and without viscosity, FARGO and a planet."""
    ws = [
        W.disk2d(nx=96, ny=32),
        W.disk2d(nx=600, ny=40, h=0.04, nu=1e-6, q=1e-4),
        W.disk2d(nx=1100, ny=24, h=0.06, nu=3e-6, q=3e-4),
        W.random_box(W.CART, 37, 21, 1, seed=3, iso=False, nu=1e-3, planet=False, bc=W.BC_REFLECT),
        W.random_box(W.CART, 19, 13, 11, seed=4, iso=False, nu=1e-3, planet=False, bc=W.BC_ZEROGRAD),
        W.random_box(W.CYL, 41, 17, 9, seed=5, iso=False, nu=1e-3, bc=W.BC_REFLECT),
        W.random_box(W.SPH, 64, 24, 14, seed=6, iso=False, nu=1e-3, bc=W.BC_FROZEN),
        W.random_box(W.SPH, 33, 19, 10, seed=7, iso=True, nu=0.0, bc=W.BC_REFLECT),
        W.random_box(W.CYL, 70, 33, 1, seed=8, iso=True, nu=1e-3, fargo=False, bc=W.BC_FROZEN),
    ]
    return ws


def fields(c):
    return {k: v.copy() for k, v in c.get_state().items()}


# batch vs alone: relative L-inf on every field, relative difference of dt
TOL_SOLO = {"f64": (1e-13, 1e-13), "f32": (5e-5, 1e-5)}


def assert_close(a, b, tol, where):
    for k in a:
        x, y = a[k].astype(np.float64), b[k].astype(np.float64)
        s = np.max(np.abs(y))
        d = np.max(np.abs(x - y))
        assert d <= tol * (s if s > 0 else 1.0), (where, k, d, s)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("graph", [True, False])
def test_batch_equals_members_stepped_alone(prec, graph):
    import paper_1602_02359_b300 as fb
    p = fb.F64 if prec == "f64" else fb.F32
    ws = mixed_members()
    solo = [make_ctx(w, p, t=0.0, t_end=w.t_end) for w in ws]
    mem = [make_ctx(w, p, t=0.0, t_end=w.t_end) for w in ws]
    tol_f, tol_dt = TOL_SOLO[prec]
    b = fb.FargoBatch(mem)
    b.use_graph(graph)
    assert b.launches_per_step() >= 14
    for n in range(4):
        b.step()
        for s in solo:
            s.step(want_dt=False)
        for i, (s, m) in enumerate(zip(solo, mem)):
            ts, dts, ns, es = s.scalars()
            tm, dtm, nm, em = m.scalars()
            assert (ns, es) == (nm, em) == (n + 1, 0), (i, n)
            if n == 0:
                assert dts == dtm, (i, dts, dtm)      # identical inputs
            assert abs(dtm - dts) <= tol_dt * dts and abs(tm - ts) <= tol_dt * ts, (i, n)
    dts = {m.scalars()[1] for m in mem}
    assert len(dts) == len(mem)            # every member took its own step
    for i, (s, m) in enumerate(zip(solo, mem)):
        assert_close(fields(m), fields(s), tol_f, i)
    b.close()


def test_batch_fp64_matches_oracle():
    import paper_1602_02359_b300 as fb
    ws = [W.disk2d(nx=96, ny=32), W.random_box(W.SPH, 64, 24, 14, seed=6, nu=1e-3, bc=W.BC_FROZEN),
          W.random_box(W.CART, 19, 13, 11, seed=4, planet=False, bc=W.BC_ZEROGRAD)]
    mem = [make_ctx(w, fb.F64, t=0.0, t_end=w.t_end) for w in ws]
    b = fb.FargoBatch(mem)
    ors = [oracle.Oracle(w) for w in ws]
    sts = [w.copy().state for w in ws]
    ts = [0.0] * len(ws)
    for n in range(3):
        b.step()
        for i, (o, st, m, w) in enumerate(zip(ors, sts, mem, ws)):
            dt_o = o.step(st, ts[i], w.t_end)
            ts[i] += dt_o
            dt_g = m.scalars()[1]
            if n == 0:
                assert dt_g == dt_o, (i, dt_g, dt_o)
            else:
                assert abs(dt_g - dt_o) <= 1e-12 * dt_o, (i, n, dt_g, dt_o)
    for w, m, st in zip(ws, mem, sts):
        compare_state(w, m.get_state(), st, 3e-12)
    b.close()


def test_batch_fp32_disks_within_stated_tolerance():
    """Three batch-sweep style disks (FP32) against the FP64 oracle after 60
    steps: 2e-5 relative L1 on density, 1e-4 on the momentum density."""
    import paper_1602_02359_b300 as fb
    ps = W.batch_params(n=3, seed=1602)
    ws = [W.disk2d(nx=3 * r, ny=r, h=pp["h"], nu=pp["nu"], q=pp["q"])
          for r, pp in zip((40, 56, 72), ps)]
    mem = [make_ctx(w, fb.F32, t=0.0, t_end=w.t_end) for w in ws]
    b = fb.FargoBatch(mem)
    ors = [oracle.Oracle(w) for w in ws]
    sts = [w.copy().state for w in ws]
    ts = [0.0] * len(ws)
    for n in range(60):
        b.step(sync=False)
        for i, (o, st, w) in enumerate(zip(ors, sts, ws)):
            ts[i] += o.step(st, ts[i], w.t_end)
    assert b.status() == (3, -1)
    for w, m, st in zip(ws, mem, sts):
        g = m.get_state()
        assert rel_l1(w.active(g["rho"]), w.active(st["rho"])) < 2e-5
        assert rel_l1(momentum_density(w, g), momentum_density(w, st)) < 1e-4
    b.close()


def test_batch_run_lands_every_member_on_its_own_end_time():
    import paper_1602_02359_b300 as fb
    ws = [W.sod(ny=64), W.sod(ny=96), W.disk2d(nx=96, ny=32)]
    ends = [0.03, 0.05, 0.02]
    mem = [make_ctx(w, fb.F64, t=0.0, t_end=te) for w, te in zip(ws, ends)]
    solo = [make_ctx(w, fb.F64, t=0.0, t_end=te) for w, te in zip(ws, ends)]
    b = fb.FargoBatch(mem)
    steps, running = b.run(poll=5)
    assert running == 0
    for i, (m, s, te) in enumerate(zip(mem, solo, ends)):
        s.run_to(te, poll=5)
        tm, _, nm, em = m.scalars()
        ts, _, ns, es = s.scalars()
        assert tm == te == ts and em == es == 0
        assert abs(nm - ns) <= 1
        assert_close(fields(m), fields(s), 1e-12, i)
    assert steps >= max(m.scalars()[2] for m in mem)
    n_before = [m.scalars()[2] for m in mem]
    b.step()                                       # all done: void steps
    assert [m.scalars()[2] for m in mem] == n_before
    b.close()


def test_batch_isolates_a_failing_member():
    """A member with a non-finite density latches NONFINITE and is reported
    by index; the other members keep stepping exactly as alone."""
    import paper_1602_02359_b300 as fb
    ws = [W.disk2d(nx=96, ny=32), W.random_box(W.CART, 37, 21, 1, seed=3, planet=False, bc=W.BC_REFLECT),
          W.disk2d(nx=120, ny=40)]
    ws[1].state["rho"][ws[1].gz, ws[1].gy + 2, 3] = float("nan")
    mem = [make_ctx(w, fb.F64, t=0.0, t_end=w.t_end) for w in ws]
    solo = make_ctx(ws[2], fb.F64, t=0.0, t_end=ws[2].t_end)
    b = fb.FargoBatch(mem)
    with pytest.raises(fb.FargoError) as e:
        b.step()
    assert e.value.code == -4 and "member 1" in str(e.value)
    for _ in range(2):
        b.step(sync=False)
    with pytest.raises(fb.FargoError):
        b.status()                               # synchronises; member 1 still failed
    for _ in range(3):
        solo.step()
    assert mem[1].scalars()[3] == -4
    assert mem[0].scalars()[2] == 3
    assert solo.scalars()[2] == mem[2].scalars()[2] == 3
    assert_close(fields(mem[2]), fields(solo), 1e-13, 2)
    b.close()


def test_batch_rejects_bad_members():
    import paper_1602_02359_b300 as fb
    a = make_ctx(W.disk2d(nx=96, ny=32), fb.F64)
    c = make_ctx(W.disk2d(nx=96, ny=32), fb.F32)
    with pytest.raises(fb.FargoError) as e:
        fb.FargoBatch([a, c])                    # mixed precision
    assert e.value.code == -1
    with pytest.raises(fb.FargoError) as e:
        fb.FargoBatch([a, a])                    # duplicate member
    assert e.value.code == -1


def test_full_size_sweep_sampled_members():
    """The 256-disk sweep at full size, as the benchmark runs it (FP32,
    batched, CUDA graph): after two batched steps, the smallest and the
    largest disk against the oracle stepping the same disk alone (2e-5
    relative L1 on density, 1e-4 on the momentum density); the first
    step's dt of both is bit-exact."""
    import paper_1602_02359_b300 as fb
    ps = W.batch_params(n=256, seed=1602)
    sizes = [p["ny"] for p in ps]
    pick = [int(np.argmin(sizes)), int(np.argmax(sizes))]
    mem, ws = [], {}
    for i, p in enumerate(ps):
        w = W.batch_instance(p)
        mem.append(make_ctx(w, fb.F32, t=0.0, t_end=w.t_end))
        if i in pick:
            ws[i] = w
        else:
            w.state = None
    b = fb.FargoBatch(mem)
    for n in range(2):
        b.step()
        for i in pick:
            w = ws[i]
            if n == 0:
                o = oracle.Oracle(w)
                st = {k: v.astype(np.float32).astype(np.float64) for k, v in w.state.items()}
                ws[i] = (w, o, st, [0.0])
            w, o, st, t = ws[i]
            dt_o = o.step(st, t[0], w.t_end)
            t[0] += dt_o
            if n == 0:
                assert mem[i].scalars()[1] == dt_o, i
    for i in pick:
        w, o, st, _ = ws[i]
        g = mem[i].get_state()
        assert rel_l1(w.active(g["rho"]), w.active(st["rho"])) < 2e-5, i
        assert rel_l1(momentum_density(w, g), momentum_density(w, st)) < 1e-4, i
    b.close()
    for m in mem:
        m.close()


def test_packed_field_transfers_equal_member_transfers():
    """fargo_batch_set_field_packed / get_field_packed move one field of every
    member as one buffer (active cells, member order): an upload then a step
    gives what the per-member uploads give, and the packed read equals the
    per-member reads concatenated."""
    import torch
    import paper_1602_02359_b300 as fb
    ws = [w for w in mixed_members() if w.iso][:4] or mixed_members()[:1]
    a = [make_ctx(w, fb.F32, t=0.0, t_end=w.t_end) for w in ws]
    b = [make_ctx(w, fb.F32, t=0.0, t_end=w.t_end) for w in ws]
    ba, bb = fb.FargoBatch(a), fb.FargoBatch(b)
    names = ["rho", "vx", "vy"] + (["vz"] if all(w.nz > 1 for w in ws) else [])
    rng = np.random.default_rng(11)
    packed = {}
    for n in names:
        parts = [(rng.uniform(0.5, 1.5, size=c.active_shape) if n == "rho" else
                  rng.normal(0, 0.01, size=c.active_shape)).astype(np.float32) for c in a]
        t = torch.empty(sum(p.size for p in parts), dtype=torch.float32, pin_memory=True)
        t.numpy()[...] = np.concatenate([p.ravel() for p in parts])
        packed[n] = (t, parts)
        ba.set_field_packed(n, t)
        for c, p in zip(b, parts):
            c.set_field(n, p, region=fb.ACTIVE)
    ba.step(sync=False)
    bb.step(sync=True)
    for n in names:
        out = torch.empty_like(packed[n][0])
        ba.get_field_packed(n, out)
        ref = np.concatenate([c.get_field(n, region=fb.ACTIVE).ravel() for c in b])
        np.testing.assert_array_equal(out.numpy(), ref, err_msg=n)
    with pytest.raises(fb.FargoError):
        ba.set_field_packed("rho", packed["rho"][0][:-1])
    ba.close()
    bb.close()
    for c in a + b:
        c.close()


@pytest.mark.parametrize("region", ["active", "full"])
def test_batch_field_transfers_equal_member_transfers(region):
    """fargo_batch_set_field / get_field (every member in one call, queued on
    the batch's stream, one synchronisation) move exactly the bytes the
    per-member accessors move, and the upload is ordered before the step
    that follows it without any host synchronisation in between."""
    import torch
    import paper_1602_02359_b300 as fb
    reg = fb.ACTIVE if region == "active" else fb.FULL
    ws = mixed_members()[:4]
    a = [make_ctx(w, fb.F32, t=0.0, t_end=w.t_end) for w in ws]
    b = [make_ctx(w, fb.F32, t=0.0, t_end=w.t_end) for w in ws]
    ba = fb.FargoBatch(a)
    bb = fb.FargoBatch(b)
    ba.step(sync=True)
    bb.step(sync=True)
    names = [n for n in ("rho", "e", "vx", "vy", "vz")]
    # new, distinct contents for every member and field, from pinned host memory
    rng = np.random.default_rng(7)
    host = {}
    for n in names:
        host[n] = []
        for c in a:
            shp = c.active_shape if reg == fb.ACTIVE else c.shape
            t = torch.empty(shp, dtype=torch.float32, pin_memory=True)
            t.numpy()[...] = rng.uniform(0.5, 1.5, size=shp) if n in ("rho", "e") else rng.normal(0, 0.01, size=shp)
            host[n].append(t)
    for n in names:
        ba.set_field(n, host[n], region=reg)           # queued, no synchronisation
        for c, t in zip(b, host[n]):
            c.set_field(n, t.numpy(), region=reg)
    ba.step(sync=False)                                # ordered after the uploads
    bb.step(sync=True)
    out = {n: [torch.empty_like(t) for t in host[n]] for n in names}
    for n in names:
        ba.get_field(n, out[n], region=reg)
    ba.status()
    for n in names:
        for k, c in enumerate(b):
            ref = c.get_field(n, region=reg)
            np.testing.assert_array_equal(out[n][k].numpy(), ref, err_msg=f"{n} member {k}")
    # a wrong byte count is refused
    bad = [t[..., :1].contiguous() for t in host["rho"]]
    with pytest.raises(fb.FargoError):
        ba.set_field("rho", bad, region=reg)
    ba.close()
    bb.close()
    for c in a + b:
        c.close()
