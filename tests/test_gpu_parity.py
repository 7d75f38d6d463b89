"""Parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances: dt, v0 and the ghost fill bit-exact; FP64 fields within 1e-12
relative L-infinity after one step or sub-step; FP64 Sod run within 1e-9
relative L1; FP32 fields within 2e-5 relative L1 (density) and 1e-4
(momenta/velocities) against the FP64 oracle.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from tests.gpu_util import active_faces, compare_state, fields_of, make_ctx, momentum_density, record, rel_l1, rel_linf

pytestmark = pytest.mark.gpu

TOL64 = 1e-12

# (geom, nx, ny, nz, iso, nu, bc): small meshes that still span several
# thread blocks and rings, with ragged sizes
CASES = [
    (W.CART, 37, 21, 1, False, 1e-3, W.BC_REFLECT),
    (W.CART, 19, 13, 11, False, 1e-3, W.BC_ZEROGRAD),
    (W.CYL, 70, 33, 1, True, 1e-3, W.BC_FROZEN),
    (W.CYL, 41, 17, 9, False, 1e-3, W.BC_REFLECT),
    (W.SPH, 64, 24, 14, False, 1e-3, W.BC_FROZEN),
    (W.SPH, 33, 19, 10, True, 0.0, W.BC_REFLECT),
    # rings long enough for several cells per thread in the ring kernels
    # (in FP64: three per thread, lanes exchanging the orbital step's stencil
    # halo, at 600 cells; two at 480)
    (W.CYL, 600, 9, 1, True, 1e-3, W.BC_FROZEN),
    (W.SPH, 480, 10, 6, False, 1e-3, W.BC_REFLECT),
    # one azimuthal cell: an axisymmetric disk (no X derivatives, no X sweep)
    (W.CYL, 1, 40, 1, True, 1e-3, W.BC_ZEROGRAD),
    # rings too long for two FP64 staging buffers: the ring kernels stage
    # one ring at a time
    (W.CYL, 4000, 6, 1, True, 1e-3, W.BC_FROZEN),
    # periodic boundaries: a Cartesian box periodic in Y and Z, a 2D one in
    # Y, a cylinder periodic in z (frozen radial walls)
    (W.CART, 37, 21, 9, False, 1e-3, W.BC_PERIODIC),
    (W.CART, 33, 20, 1, True, 1e-3, W.BC_PERIODIC),
    (W.CYL, 41, 17, 12, False, 1e-3, W.BC_PERIODIC),
]
IDS = [f"g{c[0]}-{c[1]}x{c[2]}x{c[3]}-{'iso' if c[4] else 'adi'}-nu{c[5]}-bc{c[6]}" for c in CASES]


def box(case, seed=1):
    geom, nx, ny, nz, iso, nu, bc = case
    w = W.random_box(geom, nx, ny, nz, g=3, seed=seed, iso=iso, nu=nu, planet=(geom != W.CART), bc=bc)
    if bc == W.BC_PERIODIC:
        if geom != W.CART:
            w.bc_y = (W.BC_FROZEN, W.BC_FROZEN)    # only z is periodic in a cylinder
        W.periodic_tables(w)
    return w


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_ghost_fill_bit_exact(case):
    w = box(case)
    c = make_ctx(w)
    c.debug_phase(0, 1.0)
    o = oracle.Oracle(w)
    st = w.copy().state
    o.bc_fill(st)
    g = c.get_state()
    for k in fields_of(w):
        assert np.array_equal(g[k][:w.nz_t + 1, :w.ny_t + 1], st[k]), k


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_courant_step_and_v0_bit_exact(case):
    w = box(case)
    o = oracle.Oracle(w)
    st = w.copy().state
    o.bc_fill(st)
    c = make_ctx(w)
    c.set_state(st)
    c.debug_phase(1)
    v0_gpu = c.get_aux(6)
    v0 = o.v0(st)
    assert np.array_equal(v0_gpu, v0)
    rc, dt = o.cfl(st, v0)
    assert rc == 0
    t, dt_gpu, _, err = c.scalars()
    assert err == 0
    assert dt_gpu == dt, (dt_gpu, dt)


def _phase_case(case, phase):
    w = box(case, seed=3)
    o = oracle.Oracle(w)
    st = w.copy().state
    o.bc_fill(st)
    dt = 2e-3
    c = make_ctx(w, t=0.3)
    c.set_state(st)
    ref = {k: v.copy() for k, v in st.items()}
    if phase == 2:
        phi = o.potential(0.3) if (w.star_mass > 0 or w.planet_q > 0) and w.geom != W.CART else None
        o.substep1(ref, phi, dt)
    elif phase == 3:
        o.artificial_viscosity(ref, dt)
        o.compression_heating(ref, dt)
    elif phase == 4:
        o.viscosity(ref, dt)
    c.debug_phase(phase, dt)
    return w, c.get_state(), ref


@pytest.mark.parametrize("case", CASES, ids=IDS)
@pytest.mark.parametrize("phase", [2, 3, 4])
def test_source_substeps_fp64(case, phase):
    w, g, ref = _phase_case(case, phase)
    compare_state(w, g, ref, TOL64)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_momenta_and_x_sweep_fp64(case):
    w = box(case, seed=4)
    o = oracle.Oracle(w)
    st = w.copy().state
    o.bc_fill(st)
    v0 = o.v0(st)
    dt = 0.05 if w.geom != W.CART else 0.01
    c = make_ctx(w)
    c.set_state(st)
    c.set_aux(6, v0)
    c.debug_phase(5, dt)
    pis = o.momenta(st)
    o.transport_x(st, pis, v0, dt)
    g = c.get_state()
    for k in ["rho"] + ([] if w.iso else ["e"]):
        assert rel_linf(w.active(g[k]), w.active(st[k])) < TOL64, k
    for q in range(6):
        if (q >= 2 and w.ny == 1) or (q >= 4 and w.nz == 1):
            continue
        a = c.get_aux(q)
        assert rel_linf(a[:w.nz_t, :w.ny_t], pis[q][:w.nz_t, :w.ny_t]) < TOL64, q


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_orbital_shift_fp64(case):
    """Integer shift + PPA fractional step (phase 9) against the oracle."""
    w = box(case, seed=10)
    if w.geom == W.CART:
        pytest.skip("no bulk rotation")
    o = oracle.Oracle(w)
    st = w.copy().state
    o.bc_fill(st)
    v0 = o.v0(st)
    pis = o.momenta(st)
    dt = 0.137
    c = make_ctx(w)
    c.set_state(st)
    c.set_aux(6, v0)
    for q in range(6):
        c.set_aux(q, pis[q])
    c.debug_phase(9, dt)
    o.orbital_shift(st, pis, v0, dt)
    g = c.get_state()
    for k in ["rho"] + ([] if w.iso else ["e"]):
        assert rel_linf(w.active(g[k]), w.active(st[k])) < TOL64, k
    for q in range(6):
        if (q >= 2 and w.ny == 1) or (q >= 4 and w.nz == 1):
            continue
        assert rel_linf(w.active(c.get_aux(q)), w.active(pis[q])) < TOL64, q


@pytest.mark.parametrize("case", CASES, ids=IDS)
@pytest.mark.parametrize("axis", ["y", "z"])
def test_y_and_z_sweeps_fp64(case, axis):
    w = box(case, seed=5)
    if (axis == "y" and w.ny == 1) or (axis == "z" and w.nz == 1):
        pytest.skip("axis absent")
    o = oracle.Oracle(w)
    st = w.copy().state
    o.bc_fill(st)
    pis = o.momenta(st)
    dt = 0.01
    c = make_ctx(w)
    c.set_state(st)
    for q in range(6):
        c.set_aux(q, pis[q])
    c.debug_phase(6 if axis == "y" else 7, dt)
    (o.transport_y if axis == "y" else o.transport_z)(st, pis, dt)
    g = c.get_state()
    for k in ["rho"] + ([] if w.iso else ["e"]):
        assert rel_linf(w.active(g[k]), w.active(st[k])) < TOL64, k
    for q in range(6):
        if (q >= 2 and w.ny == 1) or (q >= 4 and w.nz == 1):
            continue
        assert rel_linf(w.active(c.get_aux(q)), w.active(pis[q])) < TOL64, q


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_new_velocities_fp64(case):
    w = box(case, seed=6)
    o = oracle.Oracle(w)
    st = w.copy().state
    rng = np.random.default_rng(0)
    pis = o.momenta(st)
    for p in pis:
        p *= 1.0 + 0.05 * rng.uniform(-1, 1, size=p.shape)
    c = make_ctx(w)
    c.set_state(st)
    for q in range(6):
        c.set_aux(q, pis[q])
    c.debug_phase(8, 1e-3)
    o.new_velocities(st, pis)
    compare_state(w, c.get_state(), st, TOL64)


@pytest.mark.parametrize("case", CASES, ids=IDS)
@pytest.mark.parametrize("graph", [True, False])
def test_full_step_fp64(case, graph):
    w = box(case, seed=7)
    o = oracle.Oracle(w)
    st = w.copy().state
    c = make_ctx(w, t=0.1)
    c.use_graph(graph)
    t = 0.1
    for n in range(3):
        dt_o = o.step(st, t)
        t += dt_o
        dt_g = c.step()
        # bit-exact for identical inputs (first step); afterwards the fields
        # differ by round-off, so dt may differ in its last bits
        if n == 0:
            assert dt_g == dt_o, (dt_g, dt_o)
        else:
            assert abs(dt_g - dt_o) <= 1e-12 * dt_o, (n, dt_g, dt_o)
        compare_state(w, c.get_state(), st, TOL64 * (1 + n))


def test_sod_run_fp64_matches_oracle():
    w = W.sod()
    o = oracle.Oracle(w)
    st = w.copy().state
    t_o, n_o = o.run(st, 0.0, w.t_end)
    c = make_ctx(w, t=0.0, t_end=w.t_end)
    n_g = c.run_to(w.t_end, poll=64)
    t_g, _, nsteps, err = c.scalars()
    assert err == 0 and t_g == t_o and abs(nsteps - n_o) <= 1
    g = c.get_state()
    for k in ("rho", "e", "vy"):
        assert rel_l1(active_faces(w, k, g[k]), active_faces(w, k, st[k])) < 1e-9, k


def test_disk2d_fp64_ten_steps_full_size():
    """The 256 x 768 planet disk, FP64, in the step configuration the
    benchmark uses (CUDA graph): ten steps against the oracle, bit-exact dt."""
    w = W.disk2d()
    o = oracle.Oracle(w)
    st = w.copy().state
    c = make_ctx(w, t=0.0, t_end=w.t_end)
    t = 0.0
    for n in range(10):
        dt_o = o.step(st, t, w.t_end)
        t += dt_o
        dt_g = c.step()
        if n == 0:
            assert dt_g == dt_o, (dt_g, dt_o)
        else:
            assert abs(dt_g - dt_o) <= 1e-12 * dt_o, (n, dt_g, dt_o)
    compare_state(w, c.get_state(), st, 1e-11)


def test_corotating_laminar_disk_fp64_steps():
    """The precision study's disk (frame corotating with the planet, uniform
    surface density, linear radial spacing), reduced to 300 x 120: five
    steps against the oracle, bit-exact first dt.  The disk starts in
    equilibrium, so v_r is the small residual of gravity, the centrifugal
    force and the pressure, each of order one: its round-off is measured
    against the velocity scale max |v_phi| (1e-13), the other fields
    against their own size (1e-11)."""
    w = W.laminar_disk(nx=300, ny=120)
    o = oracle.Oracle(w)
    st = w.copy().state
    c = make_ctx(w, t=0.0, t_end=w.t_end)
    t = 0.0
    for n in range(5):
        dt_o = o.step(st, t, w.t_end)
        t += dt_o
        dt_g = c.step()
        if n == 0:
            assert dt_g == dt_o, (dt_g, dt_o)
        else:
            assert abs(dt_g - dt_o) <= 1e-12 * dt_o, (n, dt_g, dt_o)
    g = c.get_state()
    for k in ("rho", "vx"):
        assert rel_linf(active_faces(w, k, g[k]), active_faces(w, k, st[k])) < 1e-11, k
    dvy = np.max(np.abs(active_faces(w, "vy", g["vy"]) - active_faces(w, "vy", st["vy"])))
    assert dvy < 1e-13 * np.max(np.abs(w.active(st["vx"]))), dvy


@pytest.mark.parametrize("fargo", [True, False])
def test_keplerian_vortex_fp64_steps(fargo):
    """The vortex of the orbital-advection study (adiabatic, no planet,
    uniform surface density) at 160 x 48, with and without orbital
    advection: five steps against the oracle, bit-exact first dt."""
    w = W.keplerian_vortex(nx=160, ny=48, fargo=fargo)
    o = oracle.Oracle(w)
    st = w.copy().state
    c = make_ctx(w, t=0.0, t_end=w.t_end)
    t = 0.0
    for n in range(5):
        dt_o = o.step(st, t, w.t_end)
        t += dt_o
        dt_g = c.step()
        if n == 0:
            assert dt_g == dt_o, (dt_g, dt_o)
        else:
            assert abs(dt_g - dt_o) <= 1e-12 * dt_o, (n, dt_g, dt_o)
    compare_state(w, c.get_state(), st, 1e-11)


@pytest.mark.parametrize("case", [c for c in CASES if c[6] == W.BC_PERIODIC and c[0] == W.CART],
                         ids=[i for c, i in zip(CASES, IDS) if c[6] == W.BC_PERIODIC and c[0] == W.CART])
def test_periodic_box_conserves_mass_on_the_gpu(case):
    """Periodic boundaries take and give no mass: 20 FP64 steps keep the
    total within round-off, as in the oracle."""
    w = box(case, seed=12)
    c = make_ctx(w)
    m0 = c.sums()[0]
    for _ in range(20):
        c.step(want_dt=False)
    assert c.scalars()[3] == 0
    assert abs(c.sums()[0] - m0) <= 2e-14 * m0


def test_periodic_boundary_rules_are_enforced():
    """Periodic on one side only, on a spherical or cylindrical radius, or
    with ghost widths that differ from their images is refused."""
    import paper_1602_02359_b300 as fb
    w = box(CASES[-3])
    w.bc_y = (W.BC_PERIODIC, W.BC_FROZEN)
    with pytest.raises(fb.FargoError) as e:
        fb.Fargo(w)
    assert e.value.code == -1
    w = W.random_box(W.CYL, 16, 12, 1, g=3, seed=1, bc=W.BC_PERIODIC)
    with pytest.raises(fb.FargoError):
        fb.Fargo(w)
    w = box(CASES[-3])
    w.yf = w.yf.copy()
    w.yf[0] -= 0.01                      # a ghost wider than its image
    with pytest.raises(fb.FargoError):
        fb.Fargo(w)
    w = box(CASES[-3])
    w.nu = w.nu.copy()
    w.nu[:, 0] *= 2.0                    # a ghost ring's viscosity unlike its image's
    with pytest.raises(fb.FargoError):
        fb.Fargo(w)
    fb.Fargo(box(CASES[-3])).close()


def test_fp32_disk_within_stated_tolerance():
    """FP32 bulk with FP64 islands against the FP64 oracle after 100 steps of
    a planet disk: 2e-5 relative L1 on density, 1e-4 relative L1 on the
    momentum density vector (both components together; the radial part alone
    is small and its own relative norm is ill-conditioned)."""
    w = W.disk2d(nx=192, ny=64)
    o = oracle.Oracle(w)
    st = w.copy().state
    import paper_1602_02359_b300 as fb
    c = make_ctx(w, fb.F32, t=0.0, t_end=w.t_end)
    t = 0.0
    for n in range(100):
        t += o.step(st, t, w.t_end)
        c.step(want_dt=False)
    g = c.get_state()
    e_rho = rel_l1(w.active(g["rho"]), w.active(st["rho"]))
    e_mom = rel_l1(momentum_density(w, g), momentum_density(w, st))
    record("fp32_disk_192x64_100steps", rel_l1_rho=e_rho, rel_l1_momentum=e_mom)
    assert e_rho < 2e-5
    assert e_mom < 1e-4


def test_fp32_longest_ring_within_stated_tolerance():
    """The longest azimuthal ring a 2D isothermal disk can stage (4000 cells,
    eight per thread in the ring kernels, the orbital step in its per-thread
    form), ten steps against the FP64 oracle at the FP32 tolerances; the
    Courant step stays bit-exact on the promoted state."""
    w = W.perturb(W.disk2d(nx=4000, ny=6), seed=41, amp=1e-2)
    o = oracle.Oracle(w)
    st = w.copy().state
    import paper_1602_02359_b300 as fb
    c = make_ctx(w, fb.F32, t=0.0, t_end=w.t_end)
    t = 0.0
    for n in range(10):
        t += o.step(st, t, w.t_end)
        c.step(want_dt=False)
    g = c.get_state()
    e_rho = rel_l1(w.active(g["rho"]), w.active(st["rho"]))
    e_mom = rel_l1(momentum_density(w, g), momentum_density(w, st))
    record("fp32_longest_ring_4000x6_10steps", rel_l1_rho=e_rho, rel_l1_momentum=e_mom)
    assert e_rho < 2e-5
    assert e_mom < 1e-4


@pytest.mark.parametrize("nx", [700, 1101, 1700])
def test_fp32_orbital_chunk_classes_within_stated_tolerance(nx):
    """Rings whose orbital step takes each FP32 form: 700 cells (four per
    lane, packed cell pairs), 1101 (six per lane, packed pairs, a ragged last
    warp), 1700 (beyond the packed forms' thread caps: the per-thread form
    with eight cells per thread); ten steps of a perturbed disk against the
    FP64 oracle at the FP32 tolerances."""
    w = W.perturb(W.disk2d(nx=nx, ny=6), seed=43, amp=1e-2)
    o = oracle.Oracle(w)
    st = w.copy().state
    import paper_1602_02359_b300 as fb
    c = make_ctx(w, fb.F32, t=0.0, t_end=w.t_end)
    t = 0.0
    for n in range(10):
        t += o.step(st, t, w.t_end)
        c.step(want_dt=False)
    g = c.get_state()
    e_rho = rel_l1(w.active(g["rho"]), w.active(st["rho"]))
    e_mom = rel_l1(momentum_density(w, g), momentum_density(w, st))
    record(f"fp32_orbital_ring_{nx}x6_10steps", rel_l1_rho=e_rho, rel_l1_momentum=e_mom)
    assert e_rho < 2e-5
    assert e_mom < 1e-4
    c.close()


def test_fp32_courant_step_bit_exact_on_promoted_state():
    """dt and v0 are FP64 islands: from the FP32 fields promoted to FP64 they
    equal the oracle's bit for bit."""
    import paper_1602_02359_b300 as fb
    w = box(CASES[4], seed=9)
    o = oracle.Oracle(w)
    st = w.copy().state
    o.bc_fill(st)
    st32 = {k: v.astype(np.float32).astype(np.float64) for k, v in st.items()}
    c = make_ctx(w, fb.F32)
    c.set_state(st32)
    c.debug_phase(1)
    v0 = o.v0(st32)
    assert np.array_equal(c.get_aux(6), v0)
    rc, dt = o.cfl(st32, v0)
    assert c.scalars()[1] == dt


@pytest.mark.parametrize("case", CASES[:4], ids=IDS[:4])
def test_conserved_sums(case):
    w = box(case, seed=8)
    o = oracle.Oracle(w)
    c = make_ctx(w)
    got = c.sums()
    want = o.sums(w.state)
    for a, b in zip(got, want):
        assert abs(a - b) <= 1e-14 * max(abs(b), 1e-300) + 1e-300


def test_nonfinite_state_is_reported_without_fault():
    w = box(CASES[0])
    w.state["rho"][0, 5, 3] = float("nan")
    w.state["rho"][w.gz, w.gy + 2, 3] = float("nan")
    c = make_ctx(w)
    import paper_1602_02359_b300 as fb
    with pytest.raises(fb.FargoError) as e:
        c.step()
    assert e.value.code == -4
    # the state is left as it was
    assert np.isnan(c.get_field("rho")[w.gz, w.gy + 2, 3])


def test_bad_arguments_are_rejected():
    import paper_1602_02359_b300 as fb
    w = box(CASES[0])
    w.g = 1
    with pytest.raises(fb.FargoError) as e:
        fb.Fargo(w)
    assert e.value.code == -1
    w = box(CASES[0])
    c = make_ctx(w)
    with pytest.raises(fb.FargoError) as e:
        c.set_field("rho", np.zeros(5))
    assert e.value.code == -6


def test_rings_beyond_one_staging_buffer_are_refused():
    """An FP64 2D disk of 8000-cell rings: the orbital step's five staged
    rows need about 320 KB even in one buffer, over the 227 KB a CTA can
    have, so fargo_create refuses the mesh (FARGO_ERR_SIZE) before any
    launch; 4000-cell rings (one buffer, 161 KB) are accepted."""
    import paper_1602_02359_b300 as fb
    with pytest.raises(fb.FargoError) as e:
        fb.Fargo(W.disk2d(nx=8000, ny=8), fb.F64)
    assert e.value.code == -6
    fb.Fargo(W.disk2d(nx=4000, ny=8), fb.F64).close()


def test_run_to_lands_on_end_time_and_stops():
    w = W.sod(ny=64)
    c = make_ctx(w, t=0.0, t_end=0.05)
    c.run_to(0.05, poll=7)
    t, _, n, err = c.scalars()
    assert t == 0.05 and err == 0
    c.run_to(0.05, max_steps=5)        # nothing left to do
    assert c.scalars()[2] == n


def test_disk3d_full_size_sampled_slab():
    """The 1536 x 512 x 96 disk in FP32, in the benchmark's launch
    configuration (CUDA graph), one step at a fixed dt from a perturbed
    state, sampled against the oracle run on a 1536 x 40 x 40 slab cut from
    the same state.  The slab's ghosts are frozen while the full mesh updates
    those cells, and every sub-step carries that difference at most a few
    cells inward, so only cells 10 or more rows and planes inside the slab
    are compared.  v0 of the sampled rings is bit-exact."""
    import paper_1602_02359_b300 as fb
    w = W.perturb(W.disk3d(), seed=31, amp=1e-2)
    c = make_ctx(w, fb.F32)
    st32 = {k: v.astype(np.float32).astype(np.float64) for k, v in w.state.items()}
    w.state = None
    j0, nj, k0, nk, edge = 200, 40, 28, 40, 10
    ws = W.disk3d(slab=(j0, nj, k0, nk))
    g = ws.g
    sub = {k: v[k0:k0 + nk + 2 * g + 1, j0:j0 + nj + 2 * g + 1, :].copy() for k, v in st32.items()}
    dt = 2e-3
    c.step_fixed(dt)
    o = oracle.Oracle(ws)
    o.step(sub, 0.0, dt_fixed=dt)
    full = c.get_state()
    v0 = c.get_aux(6)
    vo = o.v0({k: v[k0:k0 + nk + 2 * g + 1, j0:j0 + nj + 2 * g + 1, :].copy() for k, v in st32.items()})
    zs, ys = slice(g + edge, g + nk - edge), slice(g + edge, g + nj - edge)
    assert np.array_equal(v0[k0 + g + edge:k0 + g + nk - edge, j0 + g + edge:j0 + g + nj - edge], vo[zs, ys])
    cut = lambda a: a[k0 + g + edge:k0 + g + nk - edge, j0 + g + edge:j0 + g + nj - edge, :]  # noqa: E731
    e_rho = rel_l1(cut(full["rho"]), sub["rho"][zs, ys])
    e_e = rel_l1(cut(full["e"]), sub["e"][zs, ys])
    mg = np.stack([cut(full[k]) * cut(full["rho"]) for k in ("vx", "vy", "vz")])
    mo = np.stack([sub[k][zs, ys] * sub["rho"][zs, ys] for k in ("vx", "vy", "vz")])
    e_mom = rel_l1(mg, mo)
    record("disk3d_full_size_slab_fp32_1step", rel_l1_rho=e_rho, rel_l1_e=e_e, rel_l1_momentum=e_mom)
    assert e_rho < 2e-5 and e_e < 2e-5 and e_mom < 1e-4, (e_rho, e_e, e_mom)
    c.close()
