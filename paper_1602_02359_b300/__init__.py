"""Python binding of the B300 FARGO3D hydro step (C ABI in include/fargo.h).

Argument marshalling only: every step of the method runs in the CUDA kernels
of libfargo_b300.so.  There is no CPU fallback; a missing library or device
raises.  PyTorch, when used, only provides device buffers and the stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libfargo_b300.so")

CART, CYL, SPH = 0, 1, 2
F64, F32 = 0, 1
RHO, ENERGY, VX, VY, VZ, BX, BY, BZ = range(8)
ACTIVE, FULL = 0, 1
FIELD_IDS = {"rho": RHO, "e": ENERGY, "vx": VX, "vy": VY, "vz": VZ, "bx": BX, "by": BY, "bz": BZ}
GAS_FIELDS = ("rho", "e", "vx", "vy", "vz")
MHD_FIELDS = ("bx", "by", "bz")

ERRORS = {0: "ok", -1: "BADARG", -2: "OOM", -3: "CUDA", -4: "NONFINITE", -5: "DT", -6: "SIZE",
          -7: "BARRIER_TIMEOUT", -8: "NOTBUILT"}

EXPORTED = ("fargo_create", "fargo_destroy", "fargo_set_field", "fargo_get_field", "fargo_set_time",
            "fargo_step", "fargo_step_fixed", "fargo_run_to", "fargo_get_scalars", "fargo_sums",
            "fargo_debug_phase", "fargo_get_aux", "fargo_set_aux", "fargo_use_graph",
            "fargo_launches_per_step", "fargo_strerror", "fargo_profile_step", "fargo_sums_noalloc",
            "fargo_alu_peaks", "fargo_batch_create", "fargo_batch_destroy", "fargo_batch_step", "fargo_batch_status",
            "fargo_batch_run", "fargo_batch_use_graph", "fargo_batch_launches_per_step",
            "fargo_batch_profile_step", "fargo_batch_autotune", "fargo_batch_set_field_packed",
            "fargo_batch_get_field_packed", "fargo_planet_force", "fargo_planet_force_async", "fargo_planets_force_async", "fargo_nbody_rk5_async", "fargo_planets_advance_async", "fargo_change_frame", "fargo_track_frame", "fargo_enable_mhd", "fargo_set_planet_source", "fargo_planet_torque_profile", "fargo_batch_set_field", "fargo_batch_get_field", "fargo_autotune", "fargo_set_launch_shape", "fargo_debug_wait_timeout",
            "fargo_mlp_create", "fargo_mlp_destroy", "fargo_mlp_num_params", "fargo_mlp_set_params",
            "fargo_mlp_get_params", "fargo_mlp_get_grads", "fargo_mlp_set_input_map", "fargo_mlp_set_output_map",
            "fargo_mlp_set_optimizer",
            "fargo_mlp_forward", "fargo_mlp_backward", "fargo_mlp_adam", "fargo_mlp_train_step", "fargo_mlp_status",
            "fargo_mlp_ensemble")

PD = C.POINTER(C.c_double)


def nbody_rk5_async(n, y_ptr, mass_ptr, mstar, h=0.0, h_ptr=None, kick_ptr=None, kick_stride=4,
                    kick_star_ptr=None, indirect=True, stream=None):
    """fargo_nbody_rk5_async: one Cash-Karp step of n planets (device arrays
    y [n][6], mass [n]), queued on `stream` (a CUDA stream handle or None)."""
    vp = C.c_void_p
    _check(lib().fargo_nbody_rk5_async(int(n), vp(y_ptr), vp(mass_ptr), float(mstar), float(h), vp(h_ptr),
                                       vp(kick_ptr), int(kick_stride), vp(kick_star_ptr), int(bool(indirect)),
                                       vp(stream)), "fargo_nbody_rk5_async")


class FargoError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({code})")


class Planet(C.Structure):
    _fields_ = [("q", C.c_double), ("a", C.c_double), ("eps", C.c_double), ("indirect", C.c_int)]


class Params(C.Structure):
    _fields_ = [("xmin", C.c_double), ("xmax", C.c_double), ("yfaces", PD), ("zfaces", PD),
                ("cs", PD), ("nu", PD), ("cfl", C.c_double), ("cq", C.c_double),
                ("av_dt_literal", C.c_int), ("omega_frame", C.c_double), ("fargo", C.c_int),
                ("bc_y", C.c_int * 2), ("bc_z", C.c_int * 2), ("star_mass", C.c_double),
                ("precision", C.c_int), ("stream", C.c_void_p), ("shearing", C.c_int), ("oort_a", C.c_double)]


_lib = None


def lib():
    """Load libfargo_b300.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIBPATH):
            raise RuntimeError(f"{LIBPATH} is missing: run `python -m paper_1602_02359_b300.build`")
        L = C.CDLL(LIBPATH)
        vp = C.c_void_p
        L.fargo_create.argtypes = [C.POINTER(vp), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                   C.POINTER(Planet), C.POINTER(Params)]
        L.fargo_destroy.argtypes = [vp]
        L.fargo_destroy.restype = None
        L.fargo_set_field.argtypes = [vp, C.c_int, C.c_int, vp, C.c_size_t, C.c_int]
        L.fargo_get_field.argtypes = [vp, C.c_int, C.c_int, vp, C.c_size_t, C.c_int]
        L.fargo_set_time.argtypes = [vp, C.c_double, C.c_double]
        L.fargo_step.argtypes = [vp, PD]
        L.fargo_step_fixed.argtypes = [vp, C.c_double]
        L.fargo_run_to.argtypes = [vp, C.c_double, C.c_longlong, C.c_int, C.POINTER(C.c_longlong)]
        L.fargo_get_scalars.argtypes = [vp, PD, PD, C.POINTER(C.c_longlong), C.POINTER(C.c_int)]
        L.fargo_sums.argtypes = [vp, PD]
        L.fargo_planet_force.argtypes = [vp, PD, C.c_double, C.c_int, PD]
        L.fargo_planet_force_async.argtypes = [vp, PD, C.c_double, C.c_int, vp]
        L.fargo_planets_force_async.argtypes = [vp, C.c_int, vp, C.c_int, C.c_double, C.c_int, vp]
        L.fargo_nbody_rk5_async.argtypes = [C.c_int, vp, vp, C.c_double, C.c_double, vp, vp, C.c_int, vp, C.c_int,
                                            vp]
        L.fargo_planets_advance_async.argtypes = [vp, C.c_int, vp, vp, C.c_double, C.c_int, C.c_int]
        L.fargo_change_frame.argtypes = [vp, C.c_double]
        L.fargo_enable_mhd.argtypes = [vp, C.c_int, C.c_double]
        L.fargo_track_frame.argtypes = [vp, vp, C.c_int, PD]
        L.fargo_set_planet_source.argtypes = [vp, vp, C.c_int, C.c_int, vp]
        L.fargo_planet_torque_profile.argtypes = [vp, PD, C.c_double, C.c_int, vp, PD]
        L.fargo_debug_phase.argtypes = [vp, C.c_int, C.c_double]
        L.fargo_get_aux.argtypes = [vp, C.c_int, vp, C.c_size_t]
        L.fargo_set_aux.argtypes = [vp, C.c_int, vp, C.c_size_t]
        L.fargo_use_graph.argtypes = [vp, C.c_int]
        L.fargo_launches_per_step.argtypes = [vp]
        L.fargo_profile_step.argtypes = [vp, C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_int),
                                         C.POINTER(C.c_char_p)]
        L.fargo_sums_noalloc.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp,
                                         C.c_double, C.c_int, vp, vp]
        L.fargo_alu_peaks.argtypes = [PD, vp]
        L.fargo_batch_create.argtypes = [C.POINTER(vp), C.POINTER(vp), C.c_int, vp]
        L.fargo_batch_destroy.argtypes = [vp]
        L.fargo_batch_destroy.restype = None
        L.fargo_batch_step.argtypes = [vp]
        L.fargo_batch_status.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.fargo_batch_run.argtypes = [vp, C.c_longlong, C.c_int, C.POINTER(C.c_longlong), C.POINTER(C.c_int)]
        L.fargo_batch_use_graph.argtypes = [vp, C.c_int]
        L.fargo_batch_set_field.argtypes = [vp, C.c_int, C.c_int, C.POINTER(vp), C.POINTER(C.c_size_t)]
        L.fargo_batch_get_field.argtypes = [vp, C.c_int, C.c_int, C.POINTER(vp), C.POINTER(C.c_size_t)]
        L.fargo_batch_launches_per_step.argtypes = [vp]
        L.fargo_batch_autotune.argtypes = [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_float),
                                           C.POINTER(C.c_float)]
        L.fargo_batch_set_field_packed.argtypes = [vp, C.c_int, vp, C.c_size_t]
        L.fargo_batch_get_field_packed.argtypes = [vp, C.c_int, vp, C.c_size_t]
        L.fargo_batch_profile_step.argtypes = [vp, C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_int),
                                               C.POINTER(C.c_char_p)]
        L.fargo_autotune.argtypes = [vp, C.c_int, C.POINTER(C.c_int)]
        L.fargo_set_launch_shape.argtypes = [vp, C.c_int, C.c_int, C.c_int]
        L.fargo_debug_wait_timeout.argtypes = [C.c_uint]
        L.fargo_strerror.argtypes = [C.c_int]
        L.fargo_strerror.restype = C.c_char_p
        _lib = L
    return _lib


def _check(rc, where):
    if rc != 0:
        raise FargoError(rc, where)


def _dptr(a):
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(PD)


class Fargo:
    """One simulation context on the current CUDA device.

    `w` carries the mesh and physics parameters (see workloads.Workload:
    geom, nx, ny, nz, g, xmin, xmax, yf, zf, gamma, iso, cs, nu, cfl, cq,
    fargo, omega_f, bc_y, bc_z, star_mass, planet_*).
    """

    def __init__(self, w, precision=F64, stream=None):
        L = lib()
        self.w = w
        self.prec = precision
        self.dtype = np.float64 if precision == F64 else np.float32
        self._keep = [np.ascontiguousarray(a, dtype=np.float64) if a is not None else None
                      for a in (w.yf, w.zf, w.cs, w.nu)]
        yf, zf, cs, nu = self._keep
        p = Params()
        p.xmin, p.xmax = w.xmin, w.xmax
        p.yfaces, p.zfaces = _dptr(yf), _dptr(zf)
        p.cs = _dptr(cs) if (w.iso and cs is not None) else None
        p.nu = _dptr(nu) if nu is not None else None
        p.cfl, p.cq = w.cfl, w.cq
        p.av_dt_literal = int(getattr(w, "av_dt_literal", False))
        p.omega_frame = w.omega_f
        p.fargo = int(w.fargo)
        p.bc_y[0], p.bc_y[1] = w.bc_y
        p.bc_z[0], p.bc_z[1] = w.bc_z
        p.star_mass = w.star_mass
        p.precision = precision
        p.stream = stream
        p.shearing = int(bool(getattr(w, "shearing", False)))
        p.oort_a = float(getattr(w, "oort_a", 0.0))
        pl = Planet(w.planet_q, w.planet_a, w.planet_eps, int(w.indirect))
        h = C.c_void_p()
        gamma = -1.0 if w.iso else w.gamma
        _check(L.fargo_create(C.byref(h), w.geom, w.nx, w.ny, w.nz, w.g, gamma,
                              C.byref(pl) if w.planet_q > 0 else None, C.byref(p)), "fargo_create")
        self.h = h
        self.shape = w.shape
        self.active_shape = (w.nz, w.ny, w.nx)
        self.mhd = False
        if getattr(w, "mhd", False):
            self.enable_mhd(bool(getattr(w, "mhd_passive", False)), float(getattr(w, "eta", 0.0)))

    def close(self):
        if getattr(self, "h", None):
            lib().fargo_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- fields
    def set_field(self, name, a, region=FULL):
        if hasattr(a, "data_ptr"):      # torch tensor on the device
            _check(lib().fargo_set_field(self.h, FIELD_IDS[name], region, C.c_void_p(a.data_ptr()),
                                         a.numel() * a.element_size(), 1), "fargo_set_field")
            return
        a = np.ascontiguousarray(a, dtype=self.dtype)
        _check(lib().fargo_set_field(self.h, FIELD_IDS[name], region, a.ctypes.data, a.nbytes, 0),
               "fargo_set_field")

    def get_field(self, name, region=FULL, out=None):
        if out is not None and hasattr(out, "data_ptr"):
            _check(lib().fargo_get_field(self.h, FIELD_IDS[name], region, C.c_void_p(out.data_ptr()),
                                         out.numel() * out.element_size(), 1), "fargo_get_field")
            return out
        shp = self.shape if region == FULL else self.active_shape
        a = np.empty(shp, dtype=self.dtype) if out is None else out
        _check(lib().fargo_get_field(self.h, FIELD_IDS[name], region, a.ctypes.data, a.nbytes, 0),
               "fargo_get_field")
        return a

    def set_state(self, st, region=FULL):
        for k in GAS_FIELDS + (MHD_FIELDS if self.mhd else ()):
            self.set_field(k, st[k], region)

    def get_state(self, region=FULL):
        return {k: self.get_field(k, region) for k in GAS_FIELDS + (MHD_FIELDS if self.mhd else ())}

    def enable_mhd(self, passive=False, eta=0.0):
        """fargo_enable_mhd: a magnetic field (B_x, B_y, B_z, zero until set,
        fields "bx", "by", "bz") on this Cartesian context; `passive` keeps
        the gas free of magnetic forces, `eta` is the Ohmic diffusivity."""
        _check(lib().fargo_enable_mhd(self.h, int(bool(passive)), float(eta)), "fargo_enable_mhd")
        self.mhd = True

    # ---- time stepping
    def set_time(self, t, t_end=1e300):
        _check(lib().fargo_set_time(self.h, t, t_end), "fargo_set_time")

    def step(self, want_dt=True):
        if want_dt:
            dt = C.c_double()
            _check(lib().fargo_step(self.h, C.byref(dt)), "fargo_step")
            return dt.value
        _check(lib().fargo_step(self.h, None), "fargo_step")
        return None

    def step_fixed(self, dt):
        _check(lib().fargo_step_fixed(self.h, dt), "fargo_step_fixed")

    def run_to(self, t_end, max_steps=10 ** 12, poll=64):
        """fargo_run_to: step until t_end, which becomes the context's end
        time (later steps are void until set_time moves it)."""
        n = C.c_longlong()
        _check(lib().fargo_run_to(self.h, t_end, max_steps, poll, C.byref(n)), "fargo_run_to")
        return n.value

    def scalars(self):
        t, dt, n, e = C.c_double(), C.c_double(), C.c_longlong(), C.c_int()
        _check(lib().fargo_get_scalars(self.h, C.byref(t), C.byref(dt), C.byref(n), C.byref(e)),
               "fargo_get_scalars")
        return t.value, dt.value, n.value, e.value

    def sums(self):
        out = (C.c_double * 3)()
        _check(lib().fargo_sums(self.h, out), "fargo_sums")
        return tuple(out)

    def planet_force(self, rp, eps, bm08=False):
        """Force of the gas on a planet at rp = (x, y, z) per unit planet mass
        (fargo_planet_force): (a_x, a_y, a_z, specific z torque)."""
        r = (C.c_double * 3)(*[float(v) for v in rp])
        out = (C.c_double * 4)()
        _check(lib().fargo_planet_force(self.h, r, float(eps), int(bool(bm08)), out), "fargo_planet_force")
        return tuple(out)

    def planet_torque_profile(self, rp, eps, bm08=False):
        """fargo_planet_torque_profile: each active ring's share of the
        specific torque, shape (nz, ny), and the call's (a_x, a_y, a_z,
        torque)."""
        r = (C.c_double * 3)(*[float(v) for v in rp])
        ring = np.empty((self.w.nz, self.w.ny), dtype=np.float64)
        out = (C.c_double * 4)()
        _check(lib().fargo_planet_torque_profile(self.h, r, float(eps), int(bool(bm08)), ring.ctypes.data, out),
               "fargo_planet_torque_profile")
        return ring, tuple(out)

    def planet_force_async(self, rp, eps, out_ptr, bm08=False):
        """fargo_planet_force_async: queue the force on the context's stream,
        its 4 FP64 results written to the device address out_ptr."""
        r = (C.c_double * 3)(*[float(v) for v in rp])
        _check(lib().fargo_planet_force_async(self.h, r, float(eps), int(bool(bm08)), C.c_void_p(out_ptr)),
               "fargo_planet_force_async")

    def set_planet_source(self, pos_ptr, n=1, stride=3, mass_ptr=None):
        """fargo_set_planet_source: read the step's n planets' positions from
        the device address pos_ptr (rows of `stride` doubles) each step, with
        masses at mass_ptr (None for n = 1: the planet of creation's mass);
        pos_ptr None: the fixed circular orbit."""
        _check(lib().fargo_set_planet_source(self.h, C.c_void_p(pos_ptr) if pos_ptr else None, int(n),
                                             int(stride), C.c_void_p(mass_ptr) if mass_ptr else None),
               "fargo_set_planet_source")

    def change_frame(self, omega_new):
        """fargo_change_frame: the frame's rotation rate becomes omega_new at
        the current time (Eq. 13)."""
        _check(lib().fargo_change_frame(self.h, float(omega_new)), "fargo_change_frame")

    def track_frame(self, y_ptr, index=0):
        """fargo_track_frame: the frame rate becomes the angular velocity of
        body `index` of the device planetary state at y_ptr (rows of 6
        doubles), with the Eq. 13 correction; returns the new rate."""
        om = C.c_double()
        _check(lib().fargo_track_frame(self.h, C.c_void_p(y_ptr), int(index), C.byref(om)), "fargo_track_frame")
        return om.value

    def planets_force_async(self, n, y_ptr, stride, eps, out_ptr, bm08=False):
        """fargo_planets_force_async: the gas force on n planets whose
        positions are on the device (planet i at y_ptr + 8*stride*i)."""
        _check(lib().fargo_planets_force_async(self.h, int(n), C.c_void_p(y_ptr), int(stride), float(eps),
                                               int(bool(bm08)), C.c_void_p(out_ptr)), "fargo_planets_force_async")

    def planets_advance_async(self, n, y_ptr, mass_ptr, eps, bm08=False, indirect=True):
        """fargo_planets_advance_async: gas force, kick and one Cash-Karp step
        of the planets (device arrays y [n][6], mass [n]) by the last dt."""
        _check(lib().fargo_planets_advance_async(self.h, int(n), C.c_void_p(y_ptr), C.c_void_p(mass_ptr),
                                                 float(eps), int(bool(bm08)), int(bool(indirect))),
               "fargo_planets_advance_async")

    def debug_phase(self, phase, dt=0.0):
        _check(lib().fargo_debug_phase(self.h, phase, dt), f"fargo_debug_phase({phase})")

    def get_aux(self, which):
        if which == 6:
            a = np.empty((self.w.nz_t, self.w.ny_t), dtype=np.float64)
        else:
            a = np.empty(self.shape, dtype=self.dtype)
        _check(lib().fargo_get_aux(self.h, which, a.ctypes.data, a.nbytes), "fargo_get_aux")
        return a

    def set_aux(self, which, a):
        a = np.ascontiguousarray(a, dtype=np.float64 if which == 6 else self.dtype)
        _check(lib().fargo_set_aux(self.h, which, a.ctypes.data, a.nbytes), "fargo_set_aux")

    def profile_step(self):
        """One step launched kernel by kernel; returns [(kernel, ms), ...]."""
        ms = (C.c_float * 64)()
        names = (C.c_char_p * 64)()
        n = C.c_int()
        _check(lib().fargo_profile_step(self.h, 64, ms, C.byref(n), names), "fargo_profile_step")
        return [(names[i].decode(), ms[i]) for i in range(n.value)]

    def use_graph(self, on=True):
        _check(lib().fargo_use_graph(self.h, int(on)), "fargo_use_graph")

    def autotune(self, reps=3):
        """Pick the per-cell block width and the sweep segment lengths by
        timing; the state is left unchanged.  Returns (block, seg_y, seg_z)."""
        cfg = (C.c_int * 3)()
        _check(lib().fargo_autotune(self.h, reps, cfg), "fargo_autotune")
        return tuple(cfg)

    def set_launch_shape(self, cell_bs=256, seg_y=0, seg_z=0):
        _check(lib().fargo_set_launch_shape(self.h, cell_bs, seg_y, seg_z), "fargo_set_launch_shape")

    def launches_per_step(self):
        return lib().fargo_launches_per_step(self.h)


def alu_peaks(stream=None):
    """Measured multiply-add throughput of the device in TFLOP/s:
    {"fp64": ..., "fp32": ..., "fp32x2": ...} (fargo_alu_peaks)."""
    out = (C.c_double * 3)()
    _check(lib().fargo_alu_peaks(out, stream), "fargo_alu_peaks")
    return {"fp64": out[0], "fp32": out[1], "fp32x2": out[2]}


def debug_wait_timeout(spin_limit=1000):
    """Run the bounded-wait failure check; returns the library's code
    (FARGO_ERR_BARRIER_TIMEOUT = -7 when the wait ran out, as expected)."""
    return lib().fargo_debug_wait_timeout(spin_limit)


def sums_noalloc(rho, e, vx, precision, nx, ny, nz, ghost, vol, R, omega_frame, out, nblocks=0, stream=None,
                 wframe=None):
    """Conserved totals of caller-owned device buffers without any device
    allocation by the library (see fargo_sums_noalloc in include/fargo.h).
    Buffers are torch CUDA tensors (or raw device addresses); `out` receives
    3 FP64 values on `stream` (a raw cudaStream_t, None = legacy default).
    wframe: the frame term of the X momentum per ring (None = R^2
    omega_frame; Cartesian callers pass it, zeros for a plain box)."""
    def addr(t):
        if t is None:
            return None
        return C.c_void_p(t.data_ptr() if hasattr(t, "data_ptr") else int(t))
    _check(lib().fargo_sums_noalloc(addr(rho), addr(e), addr(vx), precision, nx, ny, nz, ghost, addr(vol),
                                    addr(R), addr(wframe), omega_frame, nblocks, addr(out), stream),
           "fargo_sums_noalloc")


class FargoBatch:
    """Independent contexts (one precision) stepped together by the batched
    engine (fargo_batch_* in include/fargo.h), each with its own Courant step
    and time.  The batch keeps its members alive and must be closed before
    them; member accessors are valid after status()/run()."""

    def __init__(self, members, stream=None):
        self.members = list(members)
        arr = (C.c_void_p * len(self.members))(*[m.h for m in self.members])
        h = C.c_void_p()
        _check(lib().fargo_batch_create(C.byref(h), arr, len(self.members), stream), "fargo_batch_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().fargo_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, sync=True):
        """Queue one step of every member; with sync, wait and raise on a
        member's latched error."""
        _check(lib().fargo_batch_step(self.h), "fargo_batch_step")
        if sync:
            return self.status()
        return None

    def status(self):
        """(members still running, lowest failed member or -1); raises on error."""
        run, first = C.c_int(), C.c_int()
        rc = lib().fargo_batch_status(self.h, C.byref(run), C.byref(first))
        if rc != 0:
            raise FargoError(rc, f"fargo_batch_status (member {first.value})")
        return run.value, first.value

    def run(self, max_steps=10 ** 12, poll=64):
        """Step until every member reached its end time; returns (steps, running)."""
        n, run = C.c_longlong(), C.c_int()
        _check(lib().fargo_batch_run(self.h, max_steps, poll, C.byref(n), C.byref(run)), "fargo_batch_run")
        return n.value, run.value

    def use_graph(self, on=True):
        _check(lib().fargo_batch_use_graph(self.h, int(on)), "fargo_batch_use_graph")

    @staticmethod
    def _ptrs(arrays):
        """Pointers and byte counts of numpy arrays or torch tensors (contiguous)."""
        ptr, nb = [], []
        for a in arrays:
            if hasattr(a, "data_ptr"):
                ptr.append(a.data_ptr())
                nb.append(a.numel() * a.element_size())
            else:
                if not a.flags["C_CONTIGUOUS"]:
                    raise ValueError("field buffers must be contiguous")
                ptr.append(a.ctypes.data)
                nb.append(a.nbytes)
        n = len(ptr)
        return (C.c_void_p * n)(*ptr), (C.c_size_t * n)(*nb)

    def set_field(self, name, arrays, region=FULL):
        """Queue field `name` of every member from arrays[i] (one per member,
        the member's region shape; host arrays should be pinned).  No host
        synchronisation: keep the arrays unchanged until get_field/status."""
        if len(arrays) != len(self.members):
            raise ValueError("one array per member")
        ptr, nb = self._ptrs(arrays)
        _check(lib().fargo_batch_set_field(self.h, FIELD_IDS[name], region, ptr, nb), "fargo_batch_set_field")

    def get_field(self, name, arrays, region=FULL):
        """Copy field `name` of every member into arrays[i]; synchronises."""
        if len(arrays) != len(self.members):
            raise ValueError("one array per member")
        ptr, nb = self._ptrs(arrays)
        _check(lib().fargo_batch_get_field(self.h, FIELD_IDS[name], region, ptr, nb), "fargo_batch_get_field")
        return arrays

    def launches_per_step(self):
        return lib().fargo_batch_launches_per_step(self.h)

    @staticmethod
    def _ptr1(a):
        if hasattr(a, "data_ptr"):
            return C.c_void_p(a.data_ptr()), a.numel() * a.element_size()
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("the packed buffer must be contiguous")
        return C.c_void_p(a.ctypes.data), a.nbytes

    def set_field_packed(self, name, buf):
        """fargo_batch_set_field_packed: field `name` of every member from one
        buffer holding the members' active cells in member order (queued, no
        synchronisation: keep buf unchanged until get/status)."""
        p, nb = self._ptr1(buf)
        _check(lib().fargo_batch_set_field_packed(self.h, FIELD_IDS[name], p, nb), "fargo_batch_set_field_packed")

    def get_field_packed(self, name, buf):
        """fargo_batch_get_field_packed: field `name` of every member into one
        buffer (member order, active cells); synchronises."""
        p, nb = self._ptr1(buf)
        _check(lib().fargo_batch_get_field_packed(self.h, FIELD_IDS[name], p, nb), "fargo_batch_get_field_packed")
        return buf

    def autotune(self, reps=3):
        """fargo_batch_autotune: pick the per-cell grouping and the sweep
        segments by timing; the state is left unchanged.  Returns
        ({"cells_per_thread": .., "segment": ..}, ms_default, ms_tuned)."""
        cfg = (C.c_int * 2)()
        a, b = C.c_float(), C.c_float()
        _check(lib().fargo_batch_autotune(self.h, int(reps), cfg, C.byref(a), C.byref(b)), "fargo_batch_autotune")
        return {"cells_per_thread": cfg[0], "segment": cfg[1]}, a.value, b.value

    def profile_step(self):
        """One batched step launched kernel by kernel; returns [(kernel, ms), ...]."""
        ms = (C.c_float * 64)()
        names = (C.c_char_p * 64)()
        n = C.c_int()
        _check(lib().fargo_batch_profile_step(self.h, 64, ms, C.byref(n), names), "fargo_batch_profile_step")
        return [(names[i].decode(), ms[i]) for i in range(n.value)]
