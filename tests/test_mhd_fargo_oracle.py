"""Pins of the oracle's orbital advection of the magnetic field (Sec. 3.6,
cell 11): the upstream-averaged EMF of the orbital motion, applied by
constrained transport, against what the paper and the mathematics fix.

- An arc of a whole number of cells and no shear moves every component by
  that many cells, up to the round-off of the sums (Eqs. 60, 64).
- A residual arc (xi != 0) with no shear is, for the components across the
  orbital motion, the PPA transport of the hydrodynamic orbital step
  (Sec. 3.4.1) applied to the shifted ring (the telescoping of Eq. 59).
- A uniform field in a linear shear v0 = q y gains q dt B_y on B_x per step
  (Eqs. 51-52): the sign of the EMF, the face-averaged v0 and the CT signs.
- The divergence of B stays at round-off over full steps with orbital
  advection, and the full step of a uniform field in the Keplerian
  shearing sheet follows B_x(t) = B_x0 + 2 A t B_y0 in the rows the walls
  have not reached."""
import math

import numpy as np

import oracle
import workloads as W


def _box(dims, seed=5, fargo=True):
    w = W.random_mhd_box(*dims, seed=seed, b0=(0.4, 0.3, 0.25))
    w.fargo = fargo
    return w


def _apply_orbital(o, st, v0all, dt):
    E = o.mhd_fargo_emf(st, v0all, dt)
    o.mhd_ct(st, E, dt)
    return E


def test_whole_cell_arcs_shift_every_component():
    for dims in ((16, 8, 4), (16, 8, 1), (20, 1, 6)):
        for N in (3, -2, 0, 17):
            w = _box(dims)
            o = oracle.Oracle(w)
            st = w.copy().state
            dX = (w.xmax - w.xmin) / w.nx
            dt = 0.01
            v0 = np.full((w.nz_t, w.ny_t), N * dX / dt)
            b0 = {k: st[k].copy() for k in W.MHD_FIELDS}
            _apply_orbital(o, st, v0, dt)
            scale = max(np.abs(b0[k]).max() for k in W.MHD_FIELDS)
            for k in W.MHD_FIELDS:
                want = np.roll(b0[k], N, axis=2)
                err = np.abs(w.active(st[k]) - w.active(want)).max()
                assert err <= 1e-13 * scale * max(1, abs(N)), (dims, N, k, err)


def test_residual_arc_is_the_ppa_step_across_the_motion():
    """With no shear the components across the orbital motion (B_y, B_z)
    each take the hydrodynamic orbital step of a conserved density: the
    ring shifted by N, then the upwind PPA flux of Sec. 3.4.1 at xi."""
    for dims in ((16, 8, 4), (24, 6, 1)):
        for X in (2.3, -1.7, 0.45, -0.38):
            w = _box(dims, seed=7)
            o = oracle.Oracle(w)
            st = w.copy().state
            dX = (w.xmax - w.xmin) / w.nx
            dt = 0.02
            v0 = np.full((w.nz_t, w.ny_t), X * dX / dt)
            b0 = {k: st[k].copy() for k in W.MHD_FIELDS}
            _apply_orbital(o, st, v0, dt)
            N = int(math.floor(X + 0.5)) if X >= 0 else -int(math.floor(-X + 0.5))
            xi = X - N
            comps = ["by"] + (["bz"] if dims[2] > 1 else [])
            for k in comps:
                a = w.active(b0[k])
                got = w.active(st[k])
                want = np.empty_like(a)
                for kk in range(a.shape[0]):
                    for jj in range(a.shape[1]):
                        r = np.roll(a[kk, jj], N)
                        fs = oracle.ppa_faces(r, xi)
                        want[kk, jj] = r - xi * (np.roll(fs, -1) - fs)
                err = np.abs(got - want).max()
                assert err <= 1e-13 * np.abs(a).max() * (1 + abs(N)), (dims, X, k, err)


def test_uniform_field_in_linear_shear():
    """Eq. 52: B_x(t) = B_x0 + t q B_y0 for v0 = q y; B_y, B_z unchanged."""
    bx0, by0, bz0 = 0.35, -0.6, 0.2
    for nz in (1, 4):
        w = W.uniform_mhd_box(16, 12, nz, b=(bx0, by0, bz0))
        w.fargo = True
        o = oracle.Oracle(w)
        st = w.copy().state
        q, dt = -1.5, 0.03
        yc = W.centres(w.yf)[:w.ny_t]
        v0 = np.repeat((q * yc)[None, :], w.nz_t, axis=0)
        _apply_orbital(o, st, v0, dt)
        inner = w.active(st["bx"])[:, 1:-1, :]
        assert np.abs(inner - (bx0 + q * dt * by0)).max() <= 1e-13, nz
        for k, b in (("by", by0), ("bz", bz0)):
            assert np.abs(w.active(st[k]) - b).max() <= 1e-13, (nz, k)


def test_divergence_stays_at_round_off_with_orbital_advection():
    for dims, bcy, eta in (((16, 12, 4), W.BC_FROZEN, 0.0), ((24, 16, 1), W.BC_FROZEN, 0.01),
                           ((16, 12, 4), W.BC_PERIODIC, 0.0)):
        w = W.mhd_shearing_sheet(*dims, amp=0.004, seed=11, vamp=0.02, bcy=bcy, eta=eta)
        o = oracle.Oracle(w)
        st = w.copy().state
        dx, dy = (w.xmax - w.xmin) / w.nx, w.yf[1] - w.yf[0]
        dz = w.zf[1] - w.zf[0]
        area = max(dy * dz, dx * dz, dx * dy)
        scale = max(np.abs(st[k]).max() for k in W.MHD_FIELDS) * area
        b0 = {k: st[k].copy() for k in W.MHD_FIELDS}
        t = 0.0
        for _ in range(10):
            t += o.step(st, t)
        assert np.abs(o.mhd_divb(st)).max() <= 1e-13 * scale, dims
        moved = max(np.abs(w.active(st[k] - b0[k])).max() for k in W.MHD_FIELDS)
        assert moved > 1e-5, dims


def test_sheet_uniform_field_grows_linearly():
    """Full steps of the Keplerian sheet (v_x = 2 A y, equilibrium) with a
    uniform field B = (0, B_y0, 0): the residual velocity vanishes, the
    field stays uniform where the walls have not reached, and the orbital
    EMF alone winds B_x up at 2 A B_y0 per unit time (Eq. 52)."""
    by0, A = 0.05, -0.75
    for nz in (1, 4):
        w = W.mhd_shearing_sheet(16, 40, nz, b0=(0.0, by0, 0.0), oort_a=A)
        o = oracle.Oracle(w)
        st = w.copy().state
        t = 0.0
        for _ in range(3):
            t += o.step(st, t)
        inner = w.active(st["bx"])[:, 12:-12, :]
        assert np.abs(inner - 2 * A * t * by0).max() <= 1e-12, (nz, t)
        assert np.abs(w.active(st["by"])[:, 12:-12, :] - by0).max() <= 1e-14


def test_orbital_advection_and_standard_transport_agree_on_a_smooth_sheet():
    """The same sheet with a smooth perturbed field, stepped with orbital
    advection and with standard transport over the same times: the two
    discretisations of the same equations differ by much less than the
    field's change."""
    w1 = W.mhd_shearing_sheet(32, 32, 1, amp=0.002, seed=2, cs=0.2)
    w2 = W.mhd_shearing_sheet(32, 32, 1, amp=0.002, seed=2, cs=0.2, fargo=False)
    o1, o2 = oracle.Oracle(w1), oracle.Oracle(w2)
    s1, s2 = w1.copy().state, w2.copy().state
    t = 0.0
    for _ in range(20):
        dt = o2.step(s2, t)
        o1.step(s1, t, dt_fixed=dt)
        t += dt
    sl = (slice(None), slice(8, -8), slice(None))
    for k in ("bx", "by"):
        d = np.abs(w1.active(s1[k])[sl] - w2.active(s2[k])[sl]).max()
        ch = np.abs(w1.active(s2[k])[sl] - w1.active(w1.state[k])[sl]).max()
        assert d < 0.1 * ch, (k, d, ch)


def test_uniform_field_emf_is_v0_at_the_face_times_b():
    """For a uniform field the upstream average is the field itself, so
    each EMF is the orbital velocity at its face, the two-point mean of the
    rings on both sides (Sec. 3.6), times the field: e_z = v0 B_y and
    e_y = -v0 B_z, for any (here random) ring velocities and arcs of many
    cells."""
    bx0, by0, bz0 = 0.35, -0.6, 0.2
    w = W.uniform_mhd_box(16, 10, 6, b=(bx0, by0, bz0))
    w.fargo = True
    o = oracle.Oracle(w)
    st = w.copy().state
    rng = np.random.Generator(np.random.PCG64(9))
    dt = 0.05
    v0 = rng.uniform(-4.0, 4.0, (w.nz_t, w.ny_t))
    ex, ey, ez = o.mhd_fargo_emf(st, v0, dt)
    assert not ex.any()
    j0, j1, k0, k1 = w.gy, w.gy + w.ny, w.gz, w.gz + w.nz
    for k in range(k0, k1):
        for j in range(j0, j1 + 1):
            vf = 0.5 * (v0[k, j - 1] + v0[k, j])
            assert np.abs(ez[k, j] - vf * by0).max() <= 1e-13 * (1 + abs(vf)), (k, j)
    for k in range(k0, k1 + 1):
        for j in range(j0, j1):
            vf = 0.5 * (v0[k - 1, j] + v0[k, j])
            assert np.abs(ey[k, j] + vf * bz0).max() <= 1e-13 * (1 + abs(vf)), (k, j)
