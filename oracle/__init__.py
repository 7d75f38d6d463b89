"""ctypes wrapper of the plain FP64 CPU oracle (fargo_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check
and by the CPU-baseline leg of the benchmark.  The product path never imports
it.  It shares no code with the CUDA library.

The oracle takes a `workloads.Workload`-like object (mesh, switches, tables)
and a dict of FP64 field arrays of shape (nz_t+1, ny_t+1, nx).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fargo_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

P = C.POINTER(C.c_double)


class OrParams(C.Structure):
    _fields_ = [("geom", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("g", C.c_int),
                ("xmin", C.c_double), ("xmax", C.c_double), ("yf", P), ("zf", P),
                ("gamma", C.c_double), ("iso", C.c_int), ("cs", P), ("nu", P),
                ("cfl", C.c_double), ("cq", C.c_double), ("av_dt_literal", C.c_int),
                ("omega_f", C.c_double), ("fargo", C.c_int),
                ("bc_ylo", C.c_int), ("bc_yhi", C.c_int), ("bc_zlo", C.c_int), ("bc_zhi", C.c_int),
                ("star_mass", C.c_double), ("planet_q", C.c_double), ("planet_a", C.c_double),
                ("planet_eps", C.c_double), ("indirect", C.c_int), ("planet_phase0", C.c_double),
                ("shearing", C.c_int), ("oort_a", C.c_double), ("planet_live", C.c_int),
                ("planet_pos", C.c_double * 24), ("planet_mass", C.c_double * 8),
                ("mhd", C.c_int), ("mhd_passive", C.c_int), ("eta", C.c_double)]


class OrState(C.Structure):
    _fields_ = [("rho", P), ("e", P), ("vx", P), ("vy", P), ("vz", P), ("bx", P), ("by", P), ("bz", P)]


def build(force=False):
    """Compile liboracle.so with gcc (no FMA contraction, IEEE double)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "fargo_oracle.h"))):
        return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-o", LIB + ".tmp", SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        pp, ps = C.POINTER(OrParams), C.POINTER(OrState)
        L.or_set_threads.argtypes = [C.c_int]
        L.or_set_threads.restype = None
        L.or_get_threads.restype = C.c_int
        L.or_set_threads(int(os.environ.get("FARGO_ORACLE_THREADS", "1")))
        L.or_step.argtypes = [pp, ps, C.c_double, C.c_double, C.c_double, P]
        L.or_step.restype = C.c_int
        for name in ("or_bc_fill",):
            getattr(L, name).argtypes = [pp, ps]
        L.or_v0.argtypes = [pp, ps, P]
        L.or_cfl.argtypes = [pp, ps, P, C.c_double, C.c_double, P]
        L.or_cfl.restype = C.c_int
        L.or_potential.argtypes = [pp, C.c_double, P]
        L.or_change_frame.argtypes = [pp, ps, C.c_double, C.c_double]
        L.or_substep1.argtypes = [pp, ps, P, C.c_double]
        for name in ("or_artificial_viscosity", "or_compression_heating", "or_viscosity"):
            getattr(L, name).argtypes = [pp, ps, C.c_double]
        PP6 = P * 6
        L.or_momenta.argtypes = [pp, ps, PP6]
        L.or_transport_x.argtypes = [pp, ps, PP6, P, C.c_double]
        L.or_orbital_shift.argtypes = [pp, ps, PP6, P, C.c_double]
        L.or_transport_y.argtypes = [pp, ps, PP6, C.c_double]
        L.or_transport_z.argtypes = [pp, ps, PP6, C.c_double]
        L.or_new_velocities.argtypes = [pp, ps, PP6]
        L.or_geometry.argtypes = [pp, P, P, P, P, P, P]
        L.or_planet_force.argtypes = [pp, ps, P, C.c_double, C.c_int, P]
        L.or_planet_torque_profile.argtypes = [pp, ps, P, C.c_double, C.c_int, P]
        L.or_vanleer_slope.argtypes = [C.c_double] * 5
        L.or_vanleer_slope.restype = C.c_double
        L.or_ppa_faces.argtypes = [C.c_int, P, C.c_double, P]
        L.or_shift_ring.argtypes = [C.c_int, P, C.c_longlong]
        L.or_mhd_pressure.argtypes = [pp, ps, C.c_double]
        L.or_mhd_tension.argtypes = [pp, ps, C.c_double]
        L.or_mhd_emf.argtypes = [pp, ps, C.c_double, P, P, P]
        L.or_mhd_ct.argtypes = [pp, ps, P, P, P, C.c_double]
        L.or_mhd_fargo_emf.argtypes = [pp, ps, P, C.c_double, P, P, P]
        L.or_v0_all.argtypes = [pp, ps, P]
        L.or_mhd_divb.argtypes = [pp, ps, C.c_int, C.c_int, C.c_int]
        L.or_mhd_divb.restype = C.c_double
        L.or_nearest_int.argtypes = [C.c_double]
        L.or_nearest_int.restype = C.c_longlong
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(P) if a is not None else None


class Oracle:
    """Holds the parameter block of one workload (keeps arrays alive)."""

    def __init__(self, w):
        self.w = w
        self._keep = []

        def arr(a):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64)
            self._keep.append(a)
            return a

        yf, zf, cs, nu = arr(w.yf), arr(w.zf), arr(w.cs), arr(w.nu)
        self.p = OrParams(w.geom, w.nx, w.ny, w.nz, w.g, w.xmin, w.xmax, _ptr(yf), _ptr(zf),
                          w.gamma, int(w.iso), _ptr(cs), _ptr(nu), w.cfl, w.cq, int(w.av_dt_literal),
                          w.omega_f, int(w.fargo), w.bc_y[0], w.bc_y[1], w.bc_z[0], w.bc_z[1],
                          w.star_mass, w.planet_q, w.planet_a, w.planet_eps, int(w.indirect))
        self.p.shearing = int(bool(getattr(w, "shearing", False)))
        self.p.oort_a = float(getattr(w, "oort_a", 0.0))
        self.p.mhd = int(bool(getattr(w, "mhd", False)))
        self.p.mhd_passive = int(bool(getattr(w, "mhd_passive", False)))
        self.p.eta = float(getattr(w, "eta", 0.0))
        self.shape = w.shape
        self.nrings = w.nz_t * w.ny_t

    def _state(self, st):
        names = ("rho", "e", "vx", "vy", "vz") + (("bx", "by", "bz") if self.p.mhd else ())
        for k in names:
            a = st[k]
            assert a.dtype == np.float64 and a.flags.c_contiguous and a.shape == self.shape, k
        b = [_ptr(st[k]) if self.p.mhd else None for k in ("bx", "by", "bz")]
        return OrState(_ptr(st["rho"]), _ptr(st["e"]), _ptr(st["vx"]), _ptr(st["vy"]), _ptr(st["vz"]), *b)

    def step(self, st, t, t_end=1e30, dt_fixed=0.0):
        """One full update in place; returns dt.  Raises on a nonzero status."""
        dt = C.c_double(0.0)
        rc = lib().or_step(C.byref(self.p), C.byref(self._state(st)), t, t_end, dt_fixed, C.byref(dt))
        if rc:
            raise RuntimeError(f"oracle step failed with status {rc}")
        return dt.value

    def run(self, st, t, t_end, max_steps=10 ** 9):
        n = 0
        while t < t_end and n < max_steps:
            dt = self.step(st, t, t_end)
            t = t + dt
            n += 1
        return t, n

    def set_planet_position(self, pos, mass=None):
        """The planets at pos (one (x, y, z) or several rows) with masses
        `mass` (default: the planet of the workload's mass, one planet) for
        the following steps (integrated planets); None returns to the
        circular orbit."""
        if pos is None:
            self.p.planet_live = 0
            return
        pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
        mass = [self.w.planet_q] if mass is None else list(mass)
        assert len(pos) == len(mass) <= 8
        self.p.planet_live = len(pos)
        for n in range(len(pos)):
            for q in range(3):
                self.p.planet_pos[3 * n + q] = float(pos[n, q])
            self.p.planet_mass[n] = float(mass[n])

    def change_frame(self, st, omega_new, t):
        """Frame change at time t to the rate omega_new (Eq. 13), in place."""
        lib().or_change_frame(C.byref(self.p), C.byref(self._state(st)), float(omega_new), float(t))

    def bc_fill(self, st):
        lib().or_bc_fill(C.byref(self.p), C.byref(self._state(st)))

    def v0(self, st):
        v0 = np.zeros(self.nrings)
        lib().or_v0(C.byref(self.p), C.byref(self._state(st)), _ptr(v0))
        return v0.reshape(self.w.nz_t, self.w.ny_t)

    def cfl(self, st, v0, t=0.0, t_end=1e30):
        dt = C.c_double(0.0)
        v0 = np.ascontiguousarray(v0, dtype=np.float64)
        rc = lib().or_cfl(C.byref(self.p), C.byref(self._state(st)), _ptr(v0), t, t_end, C.byref(dt))
        return rc, dt.value

    def potential(self, t):
        phi = np.zeros(self.shape)
        lib().or_potential(C.byref(self.p), t, _ptr(phi))
        return phi

    def substep1(self, st, phi, dt):
        lib().or_substep1(C.byref(self.p), C.byref(self._state(st)), _ptr(phi), dt)

    def artificial_viscosity(self, st, dt):
        lib().or_artificial_viscosity(C.byref(self.p), C.byref(self._state(st)), dt)

    def compression_heating(self, st, dt):
        lib().or_compression_heating(C.byref(self.p), C.byref(self._state(st)), dt)

    def viscosity(self, st, dt):
        lib().or_viscosity(C.byref(self.p), C.byref(self._state(st)), dt)

    def mhd_pressure(self, st, dt):
        """Cell 7a's magnetic part: the gradient of the transverse magnetic
        pressure on every velocity (Sec. 3.5, after Eq. 46)."""
        lib().or_mhd_pressure(C.byref(self.p), C.byref(self._state(st)), dt)

    def mhd_emf(self, st, dt):
        """Cells 8a-8c: the EMF (Eq. 45, minus eta curl B) on the edges;
        returns (e_x, e_y, e_z) as full arrays, zero outside the stencil's
        reach."""
        E = [np.zeros(self.shape) for _ in range(3)]
        lib().or_mhd_emf(C.byref(self.p), C.byref(self._state(st)), dt, *[_ptr(a) for a in E])
        return E

    def mhd_tension(self, st, dt):
        """Cell 8d: the magnetic tension on the velocities (Eq. 47)."""
        lib().or_mhd_tension(C.byref(self.p), C.byref(self._state(st)), dt)

    def mhd_ct(self, st, E, dt):
        """Cell 10: constrained transport of B by the EMF (Eq. 39)."""
        E = [np.ascontiguousarray(a, dtype=np.float64) for a in E]
        lib().or_mhd_ct(C.byref(self.p), C.byref(self._state(st)), *[_ptr(a) for a in E], dt)

    def v0_all(self, st):
        """Eq. 37 on every ring, ghost rings included (the velocity whose
        residual the MHD sub-steps see under orbital advection)."""
        v0 = np.zeros(self.nrings)
        lib().or_v0_all(C.byref(self.p), C.byref(self._state(st)), _ptr(v0))
        return v0.reshape(self.w.nz_t, self.w.ny_t)

    def mhd_fargo_emf(self, st, v0all, dt):
        """Cell 11: the upstream averages of the orbital motion's EMF
        (Sec. 3.6, Eq. 54) on the edges; returns (e_x, e_y, e_z), e_x = 0."""
        E = [np.zeros(self.shape) for _ in range(3)]
        v0all = np.ascontiguousarray(v0all, dtype=np.float64)
        lib().or_mhd_fargo_emf(C.byref(self.p), C.byref(self._state(st)), _ptr(v0all), dt,
                               *[_ptr(a) for a in E])
        return E

    def mhd_divb(self, st):
        """The discrete divergence of B, sum over the faces of B times area
        (outward), of every active cell: shape (nz, ny, nx)."""
        w, s = self.w, self._state(st)
        out = np.zeros((w.nz, w.ny, w.nx))
        for k in range(w.nz):
            for j in range(w.ny):
                for i in range(w.nx):
                    out[k, j, i] = lib().or_mhd_divb(C.byref(self.p), C.byref(s), i, w.gy + j, w.gz + k)
        return out

    def momenta(self, st):
        pis = [np.zeros(self.shape) for _ in range(6)]
        arr = (P * 6)(*[_ptr(a) for a in pis])
        lib().or_momenta(C.byref(self.p), C.byref(self._state(st)), arr)
        return pis

    def _pis(self, pis):
        return (P * 6)(*[_ptr(a) for a in pis])

    def transport_x(self, st, pis, v0, dt):
        v0 = np.ascontiguousarray(v0, dtype=np.float64)
        lib().or_transport_x(C.byref(self.p), C.byref(self._state(st)), self._pis(pis), _ptr(v0), dt)

    def orbital_shift(self, st, pis, v0, dt):
        v0 = np.ascontiguousarray(v0, dtype=np.float64)
        lib().or_orbital_shift(C.byref(self.p), C.byref(self._state(st)), self._pis(pis), _ptr(v0), dt)

    def transport_y(self, st, pis, dt):
        lib().or_transport_y(C.byref(self.p), C.byref(self._state(st)), self._pis(pis), dt)

    def transport_z(self, st, pis, dt):
        lib().or_transport_z(C.byref(self.p), C.byref(self._state(st)), self._pis(pis), dt)

    def new_velocities(self, st, pis):
        lib().or_new_velocities(C.byref(self.p), C.byref(self._state(st)), self._pis(pis))

    def geometry(self):
        n = (self.w.nz_t + 1) * (self.w.ny_t + 1)
        out = [np.zeros(n) for _ in range(6)]
        lib().or_geometry(C.byref(self.p), *[_ptr(a) for a in out])
        return [a.reshape(self.w.nz_t + 1, self.w.ny_t + 1) for a in out]

    def planet_force(self, st, rp, eps, bm08=False):
        """Force of the gas on a planet at rp = (x, y, z), per unit planet
        mass (G = 1), Plummer softening eps; bm08 removes each ring's mean
        density first.  Returns (a_x, a_y, a_z, specific torque z)."""
        out = np.zeros(4)
        r = np.ascontiguousarray(rp, dtype=np.float64)
        rho = st["rho"]       # the only field the force reads
        assert rho.dtype == np.float64 and rho.flags.c_contiguous and rho.shape == self.shape
        s = OrState(_ptr(rho), None, None, None, None)
        lib().or_planet_force(C.byref(self.p), C.byref(s), _ptr(r), float(eps), int(bm08), _ptr(out))
        return out

    def planet_torque_profile(self, st, rp, eps, bm08=False):
        """Each active ring's share of the specific torque, shape (nz, ny)."""
        w = self.w
        out = np.zeros((w.nz, w.ny))
        r = np.ascontiguousarray(rp, dtype=np.float64)
        rho = st["rho"]
        assert rho.dtype == np.float64 and rho.flags.c_contiguous and rho.shape == self.shape
        s = OrState(_ptr(rho), None, None, None, None)
        lib().or_planet_torque_profile(C.byref(self.p), C.byref(s), _ptr(r), float(eps), int(bm08), _ptr(out))
        return out

    def sums(self, st):
        """Conserved totals (mass, internal energy, X momentum), exactly rounded sums.

        Mass = sum rho V, energy = sum e V, X momentum = sum (Pi-_x + Pi+_x)/2 V
        over active cells (flow-chart diagnostics, Sec. 4.2).
        """
        w = self.w
        _, _, _, _, vol, _ = self.geometry()
        V = vol[:w.nz_t, :w.ny_t][w.gz:w.gz + w.nz, w.gy:w.gy + w.ny][:, :, None]
        rho = w.active(st["rho"])
        pis = self.momenta(st)
        mom = 0.5 * (w.active(pis[0]) + w.active(pis[1]))
        m = math.fsum((rho * V).ravel())
        e = math.fsum((w.active(st["e"]) * V).ravel())
        lx = math.fsum((mom * V).ravel())
        return m, e, lx


def set_threads(n):
    """Threads of the oracle's loops (results are bit-identical for any n)."""
    lib().or_set_threads(int(n))


def threads():
    return lib().or_get_threads()


def vanleer_slope(qm, q0, qp, dxm, dxp):
    return lib().or_vanleer_slope(qm, q0, qp, dxm, dxp)


def ppa_faces(q, xi):
    q = np.ascontiguousarray(q, dtype=np.float64)
    out = np.zeros_like(q)
    lib().or_ppa_faces(len(q), _ptr(q), xi, _ptr(out))
    return out


def shift_ring(q, n):
    q = np.ascontiguousarray(q, dtype=np.float64).copy()
    lib().or_shift_ring(len(q), _ptr(q), n)
    return q


def nearest_int(x):
    return lib().or_nearest_int(x)
