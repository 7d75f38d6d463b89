"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no arithmetic of the time step itself: it only builds mesh
face coordinates and initial conditions (ICs) as plain FP64 NumPy arrays, plus
the parameter records that describe each workload.  Both the CPU oracle and the
CUDA library receive these arrays as *inputs*.

Array layout (identical for every field, ghost cells included):
    shape (nz_t + 1, ny_t + 1, nx), X fastest, where
    ny_t = ny + 2*g if ny > 1 else 1   (ghost layers in Y only when Y is active)
    nz_t = nz + 2*g if nz > 1 else 1
The extra row (j = ny_t) and plane (k = nz_t) exist so that the face-centred
v_y / v_z of the last ghost cell's upper face has storage (staggered mesh,
Sec. 2.3: a vector component is stored on the lower face of its cell).

Geometries follow the paper's axis naming (Tab. "corresp"): X = azimuth,
Y = radius, Z = z (cylindrical) or colatitude (spherical).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

CART, CYL, SPH = 0, 1, 2
BC_REFLECT, BC_FROZEN, BC_ZEROGRAD, BC_PERIODIC = 0, 1, 2, 3
FIELDS = ("rho", "e", "vx", "vy", "vz")


@dataclasses.dataclass
class Workload:
    """Everything a run needs: mesh, physics switches, tables and ICs."""
    name: str
    geom: int
    nx: int
    ny: int
    nz: int
    g: int
    xmin: float
    xmax: float
    yf: np.ndarray            # Y face coordinates, length ny_t + 1
    zf: np.ndarray            # Z face coordinates, length nz_t + 1
    gamma: float              # ratio of specific heats (adiabatic runs)
    iso: bool                 # locally isothermal EOS, Eq. eos1
    cs: Optional[np.ndarray]  # isothermal sound speed per ring, (nz_t, ny_t)
    nu: Optional[np.ndarray]  # kinematic viscosity per ring, (nz_t, ny_t)
    cfl: float
    cq: float                 # artificial-viscosity coefficient C_q
    fargo: bool
    omega_f: float
    bc_y: tuple
    bc_z: tuple
    star_mass: float
    planet_q: float           # 0 = no planet
    planet_a: float
    planet_eps: float
    indirect: bool
    t0: float
    t_end: float
    state: dict               # field name -> (nz_t+1, ny_t+1, nx) float64
    av_dt_literal: bool = False
    shearing: bool = False    # Cartesian shearing sheet (X along the shear flow)
    oort_a: float = 0.0       # its shear rate A: unperturbed v_x = 2 A y
    mhd: bool = False         # magnetic field (state keys bx, by, bz), Cartesian, STANDARD transport
    mhd_passive: bool = False # the field evolves passively (no magnetic force on the gas)
    eta: float = 0.0          # Ohmic diffusivity

    @property
    def ny_t(self):
        return self.ny + 2 * self.g if self.ny > 1 else 1

    @property
    def nz_t(self):
        return self.nz + 2 * self.g if self.nz > 1 else 1

    @property
    def shape(self):
        return (self.nz_t + 1, self.ny_t + 1, self.nx)

    @property
    def gy(self):
        return self.g if self.ny > 1 else 0

    @property
    def gz(self):
        return self.g if self.nz > 1 else 0

    def active(self, a):
        """Active-cell view (nz, ny, nx) of a full field array."""
        return a[self.gz:self.gz + self.nz, self.gy:self.gy + self.ny, :]

    @property
    def cells(self):
        return self.nx * self.ny * self.nz

    def copy(self):
        w = dataclasses.replace(self)
        w.state = {k: v.copy() for k, v in self.state.items()}
        return w


def faces(n, g, lo, hi, log=False):
    """Face coordinates of a 1D axis with n active cells and g ghosts per side."""
    if n == 1:
        return np.array([lo, hi], dtype=np.float64)
    j = np.arange(-g, n + g + 1, dtype=np.float64)
    if log:
        return lo * np.exp(j * (math.log(hi / lo) / n))
    return lo + j * ((hi - lo) / n)


def centres(f):
    return 0.5 * (f[:-1] + f[1:])


def _empty(shape):
    return {k: np.zeros(shape, dtype=np.float64) for k in FIELDS}


def sod(ny=512, g=2, axis="y"):
    """1D Sod shock tube (Sec. 5.1.1; parameters scaled to [0, 1], t = 0.2).

    Left state rho = P = 1, right rho = 0.125, P = 0.1, gamma = 1.4, v = 0.
    Run along Y with X and Z absent (one cell each); reflecting walls.
    With axis="x" the tube lies along the periodic X axis instead (nx = ny).
    """
    gamma = 1.4
    if axis == "y":
        nx, nyy = 1, ny
        yf = faces(ny, g, 0.0, 1.0)
    else:
        nx, nyy = ny, 1
        yf = faces(1, g, 0.0, 1.0)
    zf = faces(1, g, 0.0, 1.0)
    w = Workload("sod", CART, nx, nyy, 1, g, 0.0, 1.0, yf, zf, gamma, False,
                 None, None, 0.5, 1.41, False, 0.0,
                 (BC_REFLECT, BC_REFLECT), (BC_REFLECT, BC_REFLECT),
                 0.0, 0.0, 1.0, 0.0, False, 0.0, 0.2, {})
    st = _empty(w.shape)
    if axis == "y":
        ym = centres(yf)[None, :, None]
        left = np.broadcast_to(ym < 0.5, (w.nz_t, w.ny_t, 1))
    else:
        xc = (np.arange(nx) + 0.5) / nx
        left = np.broadcast_to((xc < 0.5)[None, None, :], (w.nz_t, w.ny_t, nx))
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    st["rho"][:w.nz_t, :w.ny_t, :] = rho
    st["e"][:w.nz_t, :w.ny_t, :] = p / (gamma - 1.0)
    w.state = st
    return w


def disk2d(nx=768, ny=256, h=0.05, nu=1e-5, q=1e-3, g=3, sigma0=1e-3,
           rmin=0.4, rmax=2.5, orbits=10.0, fargo=True, cq=1.41):
    """2D cylindrical locally isothermal Keplerian disk with one planet.

    Sigma = sigma0 r^-1/2, c_s = h r^-1/2, v_phi = sqrt((1 - 1.5 h^2)/r) (radial
    balance of gravity, pressure and centrifugal force), v_r = 0.  Non-rotating
    frame; planet on a circular orbit at a = 1, smoothing 0.6 H = 0.6 h a.
    Radial ghosts are frozen to the initial equilibrium.
    """
    yf = faces(ny, g, rmin, rmax, log=True)
    zf = faces(1, g, -0.5, 0.5)
    w = Workload("disk2d", CYL, nx, ny, 1, g, -math.pi, math.pi, yf, zf, 1.4, True,
                 None, None, 0.44, cq, fargo, 0.0,
                 (BC_FROZEN, BC_FROZEN), (BC_FROZEN, BC_FROZEN),
                 1.0, q, 1.0, 0.6 * h * 1.0, True, 0.0, orbits * 2.0 * math.pi, {})
    ym = centres(yf)
    cs = np.zeros((w.nz_t, w.ny_t))
    cs[:, :] = h * ym ** -0.5
    w.cs = cs
    w.nu = np.full((w.nz_t, w.ny_t), nu) if nu > 0 else None
    st = _empty(w.shape)
    st["rho"][:w.nz_t, :w.ny_t, :] = (sigma0 * ym ** -0.5)[None, :, None]
    st["vx"][:w.nz_t, :w.ny_t, :] = np.sqrt((1.0 - 1.5 * h * h) / ym)[None, :, None]
    w.state = st
    return w


def disk3d(nx=1536, ny=512, nz=96, h=0.05, alpha=1e-3, q=3e-4, g=3, rho0=1e-3,
           rmin=0.4, rmax=2.5, gamma=1.4, nsteps=200, fargo=True, cq=1.41, slab=None):
    """3D spherical adiabatic disk with one planet, vertically hydrostatic.

    Isothermal on spheres at t = 0: c_s^2 = h^2/r, rho = rho0 r^-1.5
    sin(theta)^(1/h^2 - 2.5), v_phi = sqrt((1 - 2.5 h^2)/r) (exact continuum
    equilibrium of the r and theta balances), e = c_s^2 rho/(gamma - 1).
    alpha viscosity nu = alpha c_s H = alpha h^2 r^(1/2), fixed in time.
    Colatitude spans pi/2 +- 3.5 h.  Ghosts frozen in r and theta.
    slab = (j0, nj, k0, nk) keeps only active rows j0..j0+nj-1 and planes
    k0..k0+nk-1 of the full mesh (same faces and ICs there): a bounded sample.
    """
    yf = faces(ny, g, rmin, rmax, log=True)
    zf = faces(nz, g, 0.5 * math.pi - 3.5 * h, 0.5 * math.pi + 3.5 * h)
    if slab is not None:
        j0, nj, k0, nk = slab
        yf = yf[j0:j0 + nj + 2 * g + 1]
        zf = zf[k0:k0 + nk + 2 * g + 1]
        ny, nz = nj, nk
    w = Workload("disk3d", SPH, nx, ny, nz, g, -math.pi, math.pi, yf, zf, gamma, False,
                 None, None, 0.44, cq, fargo, 0.0,
                 (BC_FROZEN, BC_FROZEN), (BC_FROZEN, BC_FROZEN),
                 1.0, q, 1.0, 0.6 * h * 1.0, True, 0.0, 1e30, {})
    w.nsteps = nsteps
    ym = centres(yf)[None, :]
    zm = centres(zf)[:, None]
    w.nu = np.broadcast_to(alpha * h * h * np.sqrt(ym), (w.nz_t, w.ny_t)).copy() if alpha > 0 else None
    st = _empty(w.shape)
    rho = rho0 * ym ** -1.5 * np.sin(zm) ** (1.0 / (h * h) - 2.5)
    st["rho"][:w.nz_t, :w.ny_t, :] = rho[:, :, None]
    st["e"][:w.nz_t, :w.ny_t, :] = ((h * h / ym) * rho / (gamma - 1.0))[:, :, None]
    st["vx"][:w.nz_t, :w.ny_t, :] = np.broadcast_to(np.sqrt((1.0 - 2.5 * h * h) / ym), (w.nz_t, w.ny_t))[:, :, None]
    w.state = st
    return w


def viscous_ring_profile(r, t, nu=1e-5, mass=1.0, r0=1.0):
    """Surface density and radial velocity of a ring of mass `mass`, started
    infinitely narrow at radius r0, spreading under a constant viscosity nu
    (Sec. 5.1, viscous spread of a gaseous ring): with u = r/r0 and
    tau = 12 nu t / r0^2,
        Sigma = mass / (pi r0^2) / (tau u^(1/4)) I_n(2u/tau) exp(-(1 + u^2)/tau),
        v_r   = 6 nu / (tau r0) (u - I_(n-1)(2u/tau) / I_n(2u/tau)),
    n = 1/4 (the order the paper leaves unnamed; with it the v_r expression
    follows from the flux r Sigma v_r = -3 sqrt(r) d/dr (nu sqrt(r) Sigma)).
    The Bessel functions are taken exponentially scaled, I_n(x) =
    ive(n, x) e^x, so that the exponents combine to -(1 - u)^2 / tau and
    nothing overflows for narrow rings."""
    from scipy.special import ive
    r = np.asarray(r, dtype=np.float64)
    tau = 12.0 * nu * t / (r0 * r0)
    u = r / r0
    x = 2.0 * u / tau
    i_n = ive(0.25, x)
    sigma = mass / (math.pi * r0 * r0) / (tau * u ** 0.25) * i_n * np.exp(-(1.0 - u) ** 2 / tau)
    vr = 6.0 * nu / (tau * r0) * (u - ive(-0.75, x) / i_n)
    return sigma, vr


def viscous_ring(ny=512, nx=1, nu=1e-5, t0=100.0, t_end=1100.0, cs=0.0, floor=1e-10, g=3, cq=1.41, cfl=0.3):
    """The viscous-ring test of Sec. 5.1: an axisymmetric Keplerian ring of
    unit mass at r0 = 1 around a unit-mass star, constant viscosity nu,
    0.1 <= r <= 1.6 on ny evenly spaced cylindrical cells, zero-gradient
    radial boundaries, started from the analytic profile at t0 and run to
    t_end.  Pressure is neglected, as in the analytic solution: isothermal
    with a uniform sound speed cs = 0 by default (already cs = 1e-3 spreads
    the ring by pressure about as fast as the viscosity does, since the
    viscous drift is only ~1e-4).  The density is floored at `floor` times its peak
    so that the exponentially small wings stay well inside FP32's range.
    v_phi is Keplerian at cell centres, v_r the analytic value at the radial
    faces.  nx azimuthal cells carry identical copies (no orbital advection:
    the ring is axisymmetric).  Courant number 0.3 rather than the usual
    0.44: at 0.44 the pressureless floor gas next to the inner edge, whose
    discrete centrifugal balance is not exact, runs a shock train that sets
    the time step, and that train runs away on some trajectories (1 in 12
    of the runs started from states perturbed at 1e-6, in either
    precision); at 0.3 it stays calm."""
    yf = faces(ny, g, 0.1, 1.6)
    zf = faces(1, g, -0.5, 0.5)
    w = Workload("viscous_ring", CYL, nx, ny, 1, g, -math.pi, math.pi, yf, zf, 1.4, True,
                 None, None, cfl, cq, False, 0.0,
                 (BC_ZEROGRAD, BC_ZEROGRAD), (BC_ZEROGRAD, BC_ZEROGRAD),
                 1.0, 0.0, 1.0, 0.0, False, t0, t_end, {})
    w.cs = np.full((w.nz_t, w.ny_t), cs)
    w.nu = np.full((w.nz_t, w.ny_t), nu)
    w.ring_nu = nu
    ym = centres(yf)
    sig, _ = viscous_ring_profile(ym, t0, nu)
    _, vr = viscous_ring_profile(yf[:w.ny_t + 1], t0, nu)
    sig = np.maximum(sig, floor * sig.max())
    st = _empty(w.shape)
    st["rho"][:w.nz_t, :w.ny_t, :] = sig[None, :, None]
    st["vx"][:w.nz_t, :w.ny_t, :] = np.sqrt(1.0 / ym)[None, :, None]
    st["vy"][:w.nz_t, :w.ny_t + 1, :] = vr[None, :, None]
    w.state = st
    return w


def laminar_disk(nx=4000, ny=2000, h=0.05, q=3e-6, sigma0=1e-3, g=3, rmin=0.6, rmax=1.4, eps_h=0.6,
                 orbits=8.0, cq=1.41):
    """The laminar disk of the precision study (Sec. 6, single or double
    precision): a 2D cylindrical, locally isothermal, inviscid disk of
    uniform surface density sigma0 and aspect ratio h (c_s = h r^-1/2), on
    rmin <= r <= rmax with ny evenly spaced radial cells (Delta r = 4e-4 at
    the paper's 2000) and nx azimuthal cells, an Earth-mass planet
    (q = 3e-6) at a = 1 with smoothing eps_h H.  The frame corotates with
    the planet (Omega_f = sqrt(1 + q), so the planet stays at azimuth 0);
    v_phi = sqrt((1 - h^2)/r) balances gravity and the pressure of this
    disk, less Omega_f r in the rotating frame; v_r = 0.  Radial ghosts are
    frozen to the initial state."""
    yf = faces(ny, g, rmin, rmax)
    zf = faces(1, g, -0.5, 0.5)
    om_f = math.sqrt(1.0 + q)
    w = Workload("laminar_disk", CYL, nx, ny, 1, g, -math.pi, math.pi, yf, zf, 1.4, True,
                 None, None, 0.44, cq, True, om_f,
                 (BC_FROZEN, BC_FROZEN), (BC_FROZEN, BC_FROZEN),
                 1.0, q, 1.0, eps_h * h, True, 0.0, orbits * 2.0 * math.pi, {})
    ym = centres(yf)
    w.cs = np.broadcast_to(h * ym ** -0.5, (w.nz_t, w.ny_t)).copy()
    st = _empty(w.shape)
    st["rho"][:w.nz_t, :w.ny_t, :] = sigma0
    st["vx"][:w.nz_t, :w.ny_t, :] = (np.sqrt((1.0 - h * h) / ym) - om_f * ym)[None, :, None]
    w.state = st
    return w


def keplerian_vortex(nx=1024, ny=256, fargo=True, mach=10.0, gamma=5.0 / 3.0, k_amp=-1.0, r0=1.0,
                     phi0=0.25 * math.pi, rmin=0.4, rmax=2.0, g=3, orbits=10.0, cq=1.41):
    """A vortex in a two-dimensional Keplerian disk (Sec. 6, impact of
    orbital advection): a disk around a unit mass, Phi = -1/r, of uniform
    surface density 1 and pressure 1/(gamma M^2) (M = 10, the Keplerian Mach
    number at r0 = 1: c_s = 1/M), adiabatic, inviscid, so the unperturbed
    flow is exactly Keplerian.  On it, a velocity perturbation
    K exp(-(x^2 + y^2)/h^2) (-y, x) in Cartesian components about the
    vortex centre (r0, phi0 = pi/4), turned into (v_phi, v_r) at each
    point, with h = c_s(r0) / (2 Omega(r0)) and K = -1 (anticyclonic).
    nx azimuthal by ny linearly spaced radial cells on [rmin, rmax]; radial
    ghosts frozen to the initial state; fargo toggles orbital advection."""
    yf = faces(ny, g, rmin, rmax)
    zf = faces(1, g, -0.5, 0.5)
    w = Workload("keplerian_vortex", CYL, nx, ny, 1, g, 0.0, 2.0 * math.pi, yf, zf, gamma, False,
                 None, None, 0.44, cq, fargo, 0.0,
                 (BC_FROZEN, BC_FROZEN), (BC_FROZEN, BC_FROZEN),
                 1.0, 0.0, 1.0, 0.0, False, 0.0, orbits * 2.0 * math.pi, {})
    cs0 = 1.0 / mach
    h = cs0 / (2.0 * r0 ** -1.5)
    p = 1.0 / (gamma * mach * mach)
    w.vortex = dict(r0=r0, phi0=phi0, h=h, k=k_amp)
    st = _empty(w.shape)
    rc = centres(yf)                                  # cell-centre radii (v_phi, rho, e)
    pc = (np.arange(nx) + 0.5) * (2.0 * math.pi / nx)  # cell-centre azimuths (v_r)
    pf = np.arange(nx) * (2.0 * math.pi / nx)          # azimuthal faces (v_phi)
    xc0, yc0 = r0 * math.cos(phi0), r0 * math.sin(phi0)

    def pert(r, ph):
        x = r * np.cos(ph) - xc0
        y = r * np.sin(ph) - yc0
        a = k_amp * np.exp(-(x * x + y * y) / (h * h))
        ux, uy = -y * a, x * a
        return -ux * np.sin(ph) + uy * np.cos(ph), ux * np.cos(ph) + uy * np.sin(ph)

    dvp, _ = pert(rc[:, None], pf[None, :])
    _, dvr = pert(yf[:w.ny_t + 1, None], pc[None, :])
    st["rho"][:w.nz_t, :w.ny_t, :] = 1.0
    st["e"][:w.nz_t, :w.ny_t, :] = p / (gamma - 1.0)
    st["vx"][:w.nz_t, :w.ny_t, :] = (np.sqrt(1.0 / rc)[:, None] + dvp)[None]
    st["vy"][:w.nz_t, :w.ny_t + 1, :] = dvr[None]
    w.state = st
    return w


def vortensity(w, st):
    """Vertical vortensity (curl v)_z / Sigma in the inertial frame at the
    cell corners (r_j faces, phi_i faces) of the active mesh, from the
    staggered fields: ((1/r) d(r v_phi)/dr - (1/r) dv_r/dphi) / Sigma, with
    Sigma the mean of the four cells around the corner.  A diagnostic of the
    flow, not a step of the method."""
    rc = centres(w.yf)
    rf = w.yf
    dphi = (w.xmax - w.xmin) / w.nx
    gy = w.gy
    vp = st["vx"][0, :w.ny_t, :] + w.omega_f * rc[:, None]     # at (rc_j, phi-face i)
    vr = st["vy"][0, :w.ny_t + 1, :]                           # at (r-face j, phi-centre i)
    rho = st["rho"][0, :w.ny_t, :]
    j = np.arange(gy + 1, gy + w.ny)                           # interior radial faces
    r = rf[j][:, None]
    d_rvp = (rc[j][:, None] * vp[j] - rc[j - 1][:, None] * vp[j - 1]) / (rc[j] - rc[j - 1])[:, None]
    d_vr = (vr[j] - np.roll(vr[j], 1, axis=1)) / dphi          # at phi-face i (between cells i-1, i)
    curl = (d_rvp - d_vr) / r
    sig = 0.25 * (rho[j] + rho[j - 1] + np.roll(rho[j], 1, axis=1) + np.roll(rho[j - 1], 1, axis=1))
    return curl / sig


def shearing_sheet(nx=16, ny=64, omega=1.0, oort_a=-0.75, cs=1e-3, ly=2.0, lx=0.5, u0=0.0, w0=0.0,
                   fargo=True, g=3, cq=1.41):
    """A 2D Cartesian shearing sheet (Sec. 2 and Sec. 3.3): the frame turns
    at Omega, X runs along the shear flow v_x = 2 A y (A = -3/4 Omega for
    Keplerian shear) and Y across it, y in [-ly/2, ly/2] on ny cells and x
    periodic over lx on nx cells.  Uniform density 1, isothermal with sound
    speed cs, no potential.  A uniform velocity perturbation (u0 along X,
    w0 along Y) rides on the shear flow.  Y ghosts frozen to the initial
    state."""
    yf = faces(ny, g, -0.5 * ly, 0.5 * ly)
    zf = faces(1, g, -0.5, 0.5)
    w = Workload("shearing_sheet", CART, nx, ny, 1, g, 0.0, lx, yf, zf, 1.4, True,
                 None, None, 0.44, cq, fargo, omega,
                 (BC_FROZEN, BC_FROZEN), (BC_FROZEN, BC_FROZEN),
                 0.0, 0.0, 1.0, 0.0, False, 0.0, 1e30, {}, shearing=True, oort_a=oort_a)
    w.cs = np.full((w.nz_t, w.ny_t), cs)
    ym = centres(yf)
    st = _empty(w.shape)
    st["rho"][:w.nz_t, :w.ny_t, :] = 1.0
    st["vx"][:w.nz_t, :w.ny_t, :] = (2.0 * oort_a * ym + u0)[None, :, None]
    st["vy"][:w.nz_t, :w.ny_t + 1, :] = w0
    w.state = st
    return w


def batch_params(n=256, seed=1602):
    """Parameter draws of the batched disk sweep (numpy PCG64, fixed seed).

    Nr ~ U{128..512}, Nphi = 3 Nr, q log-uniform [1e-5, 1e-3], h uniform
    [0.03, 0.07], nu log-uniform [1e-6, 1e-5].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    nr = rng.integers(128, 513, size=n)
    q = 10.0 ** rng.uniform(-5.0, -3.0, size=n)
    h = rng.uniform(0.03, 0.07, size=n)
    nu = 10.0 ** rng.uniform(-6.0, -5.0, size=n)
    return [dict(nx=int(3 * r), ny=int(r), q=float(a), h=float(b), nu=float(c))
            for r, a, b, c in zip(nr, q, h, nu)]


def batch_instance(p, orbits=500.0):
    return disk2d(nx=p["nx"], ny=p["ny"], h=p["h"], nu=p["nu"], q=p["q"], orbits=orbits)


def perturb(w, seed, amp=1e-2, fields=FIELDS):
    """Add seeded multiplicative/additive noise to every cell (ghosts included).

    Used to build generic, non-symmetric states for parity tests.  Density and
    energy stay positive; velocities get an additive perturbation scaled by the
    local sound-speed-like magnitude.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    st = w.state
    for f in fields:
        a = st[f]
        if f in ("rho", "e"):
            if np.any(a):
                a *= 1.0 + amp * rng.uniform(-1.0, 1.0, size=a.shape)
        else:
            if w.nx == 1 and f == "vx" and w.geom == CART:
                continue
            if w.ny == 1 and f == "vy":
                continue
            if w.nz == 1 and f == "vz":
                continue
            scale = max(np.abs(a).max(), 1.0) if f != "vx" else 1.0
            a += amp * scale * rng.uniform(-1.0, 1.0, size=a.shape) * (0.1 if f == "vx" else 1.0)
    return w


def random_box(geom, nx, ny, nz, g=3, seed=0, iso=False, nu=1e-3, planet=True,
               fargo=True, bc=BC_FROZEN, cq=1.41, omega_f=0.0):
    """A small generic mesh with a smooth random state, for sub-step parity.

    Densities/energies ~ 1 with O(10%) structure; velocities O(0.1-1) with a
    rotation-like v_x so that FARGO shifts are non-trivial.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if geom == CART:
        yf = faces(ny, g, 0.0, 1.0)
        zf = faces(nz, g, 0.0, 1.0)
        xmin, xmax = 0.0, 1.0
        star, pq = 0.0, 0.0
    elif geom == CYL:
        yf = faces(ny, g, 0.5, 1.5, log=True)
        zf = faces(nz, g, -0.1, 0.1)
        xmin, xmax = -math.pi, math.pi
        star, pq = 1.0, (1e-3 if planet else 0.0)
    else:
        yf = faces(ny, g, 0.5, 1.5, log=True)
        zf = faces(nz, g, 0.5 * math.pi - 0.2, 0.5 * math.pi + 0.2)
        xmin, xmax = -math.pi, math.pi
        star, pq = 1.0, (1e-3 if planet else 0.0)
    w = Workload("box", geom, nx, ny, nz, g, xmin, xmax, yf, zf, 1.4, iso,
                 None, None, 0.44, cq, fargo, omega_f, (bc, bc), (bc, bc),
                 star, pq, 1.0, 0.05, True, 0.3, 1e30, {})
    shp = w.shape
    nzt, nyt = w.nz_t, w.ny_t
    ym = centres(yf)
    if iso:
        w.cs = 0.05 + 0.05 * rng.uniform(size=(nzt, nyt))
    if nu > 0:
        w.nu = nu * (1.0 + 0.5 * rng.uniform(size=(nzt, nyt)))
    st = _empty(shp)
    x = 2 * math.pi * (np.arange(nx) + 0.5) / nx

    def smooth(amp):
        a = np.zeros(shp)
        for _ in range(3):
            kx = rng.integers(0, 3)
            ph = rng.uniform(0, 2 * math.pi)
            a += amp * rng.uniform(0.2, 1.0) * np.cos(kx * x + ph)[None, None, :] * \
                rng.uniform(0.5, 1.0, size=(shp[0], shp[1], 1))
        return a + amp * 0.3 * rng.uniform(-1, 1, size=shp)

    st["rho"] = 1.0 + smooth(0.1)
    st["rho"] = np.abs(st["rho"]) + 0.2
    st["e"] = 2.0 + smooth(0.2)
    st["e"] = np.abs(st["e"]) + 0.2
    if geom == CART:
        st["vx"] = 0.5 + smooth(0.2) if nx > 1 else np.zeros(shp)
    else:
        vk = np.zeros(shp)
        vk[:, :nyt, :] = (ym[:nyt] ** -0.5)[None, :, None]
        st["vx"] = vk + smooth(0.05)
    st["vy"] = smooth(0.1) if ny > 1 else np.zeros(shp)
    st["vz"] = smooth(0.1) if nz > 1 else np.zeros(shp)
    if iso:
        st["e"][:] = 0.0
    w.state = st
    return w


def periodic_tables(w):
    """On a periodic Y or Z axis the per-ring inputs (sound speed, viscosity)
    of the ghost rings must repeat the active rings one period away, as the
    state does: rewrite them so."""
    for name in ("cs", "nu"):
        a = getattr(w, name)
        if a is None:
            continue
        a = a.copy()
        if w.ny > 1 and w.bc_y[0] == BC_PERIODIC:
            g, n = w.g, w.ny
            a[:, :g] = a[:, n:n + g]
            a[:, g + n:] = a[:, g:2 * g]
        if w.nz > 1 and w.bc_z[0] == BC_PERIODIC:
            g, n = w.g, w.nz
            a[:g] = a[n:n + g]
            a[g + n:] = a[g:2 * g]
        setattr(w, name, a)
    return w


# ---------------------------------------------------------------------------
# Learned surrogate of the batched disk sweep (no counterpart in the paper):
# seeded inputs only.  The network maps (log10 q, h, log10 nu) and the
# initial surface density on SURR_BINS radial bins to the azimuthally
# averaged Sigma / Sigma_0 after a fixed number of orbits on the same bins.
# ---------------------------------------------------------------------------
SURR_BINS = 256


def mlp_dims(n_in=3 + SURR_BINS, width=256, hidden=4, n_out=SURR_BINS):
    """Layer widths: input, `hidden` hidden layers, output."""
    return [n_in] + [width] * hidden + [n_out]


def mlp_init(dims, seed):
    """Seeded initial parameters: He-uniform weights W_l of shape
    (dims[l+1], dims[l]) drawn from U(-sqrt(6/fan_in), +sqrt(6/fan_in)),
    zero biases.  Returns [(W_0, b_0), (W_1, b_1), ...] in FP64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for a, b in zip(dims[:-1], dims[1:]):
        lim = math.sqrt(6.0 / a)
        out.append((rng.uniform(-lim, lim, size=(b, a)), np.zeros(b)))
    return out


def surrogate_bins(n=SURR_BINS, rmin=0.4, rmax=2.5):
    """Bin centres, logarithmically spaced on [rmin, rmax]."""
    e = np.linspace(math.log(rmin), math.log(rmax), n + 1)
    return np.exp(0.5 * (e[:-1] + e[1:]))


def surrogate_params(n=4096, seed=1602, nr=(48, 96)):
    """Parameter draws of the surrogate's training sweep: the batched sweep's
    distributions of q, h and nu (seeded PCG64) on reduced meshes,
    Nr ~ U{nr[0]..nr[1]}, Nphi = 3 Nr."""
    rng = np.random.Generator(np.random.PCG64(seed))
    r = rng.integers(nr[0], nr[1] + 1, size=n)
    q = 10.0 ** rng.uniform(-5.0, -3.0, size=n)
    h = rng.uniform(0.03, 0.07, size=n)
    nu = 10.0 ** rng.uniform(-6.0, -5.0, size=n)
    return [dict(nx=int(3 * a), ny=int(a), q=float(b), h=float(c), nu=float(d))
            for a, b, c, d in zip(r, q, h, nu)]


def regression_set(n, n_in, n_out, seed):
    """A smooth synthetic regression task (inputs U(-1, 1), targets a fixed
    random two-layer tanh map) for training tests of the network kernels."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.uniform(-1.0, 1.0, size=(n, n_in))
    a = rng.normal(size=(n_in, 64)) / math.sqrt(n_in)
    b = rng.normal(size=(64, n_out)) / 8.0
    return x, np.tanh(x @ a) @ b


# ---------------------------------------------------------------------------
# MHD (Sec. 3.5; tests of Sec. 5.2): Cartesian boxes with a face-centred B,
# state keys bx, by, bz beside the hydrodynamic ones; STANDARD transport.
# ---------------------------------------------------------------------------
MHD_FIELDS = ("bx", "by", "bz")


def _mhd_base(name, nx, ny, nz, g, xr, yr, zr, gamma, iso, cs, bcy, bcz, cfl=0.44, cq=1.41, eta=0.0,
              passive=False, t_end=1e30):
    yf = faces(ny, g, *yr)
    zf = faces(nz, g, *zr)
    w = Workload(name, CART, nx, ny, nz, g, xr[0], xr[1], yf, zf, gamma, iso, None, None, cfl, cq, False, 0.0,
                 bcy, bcz, 0.0, 0.0, 1.0, 0.0, False, 0.0, t_end, {})
    w.mhd, w.mhd_passive, w.eta = True, passive, eta
    if iso:
        w.cs = np.full((w.nz_t, w.ny_t), cs)
    st = _empty(w.shape)
    st.update({k: np.zeros(w.shape) for k in MHD_FIELDS})
    w.state = st
    return w


def _mhd_coords(w):
    """Cell-centre and face coordinates along X, Y, Z (full ghosted ranges)."""
    dx = (w.xmax - w.xmin) / w.nx
    xf = w.xmin + dx * np.arange(w.nx)
    xc = xf + 0.5 * dx
    return xc, xf, centres(w.yf), w.yf[:w.ny_t + 1], centres(w.zf), w.zf[:w.nz_t + 1], dx


def curl_field(w, ax, ay, az):
    """A face-centred B = curl A from a vector potential given as functions
    A_x(x, y, z) at the X edges (x centre, y and z faces), A_y at the Y
    edges, A_z at the Z edges: each face's B is the circulation of A around
    it over its area, so the discrete divergence of every cell vanishes to
    round-off (the constrained-transport invariant)."""
    xc, xf, yc, yfa, zc, zfa, dx = _mhd_coords(w)
    nzt, nyt, nx = w.nz_t, w.ny_t, w.nx
    xfp = np.append(xf, xf[-1] + dx)                  # x faces 0..nx (periodic wrap)
    dy = np.diff(w.yf)[:nyt]
    dz = np.diff(w.zf)[:nzt]
    g = lambda f, z, y, x: f(x[None, None, :], y[None, :, None], z[:, None, None])  # noqa: E731
    Ax = g(ax, zfa, yfa, xc)                          # (nzt+1, nyt+1, nx)
    Ay = g(ay, zfa, yc, xfp)                          # (nzt+1, nyt, nx+1)
    Az = g(az, zc, yfa, xfp)                          # (nzt, nyt+1, nx+1)
    bx = np.zeros(w.shape)
    by = np.zeros(w.shape)
    bz = np.zeros(w.shape)
    if w.ny > 1:
        bx[:nzt, :nyt, :] += (Az[:, 1:, :nx] - Az[:, :nyt, :nx]) / dy[None, :, None]
        bz[:, :nyt, :] -= (Ax[:, 1:, :] - Ax[:, :nyt, :]) / dy[None, :, None]
    if w.nz > 1:
        bx[:nzt, :nyt, :] -= (Ay[1:, :, :nx] - Ay[:nzt, :, :nx]) / dz[:, None, None]
        by[:nzt, :, :] += (Ax[1:, :, :] - Ax[:nzt, :, :]) / dz[:, None, None]
    by[:nzt, :, :] -= (Az[:, :, 1:] - Az[:, :, :nx]) / dx
    bz[:, :nyt, :] += (Ay[:, :, 1:] - Ay[:, :, :nx]) / dx
    return bx, by, bz


def random_mhd_box(nx, ny, nz, g=3, seed=0, iso=False, b0=(0.6, 0.3, 0.2), amp=0.3, eta=0.0, passive=False,
                   nu=0.0, bc=BC_PERIODIC):
    """A Cartesian box (X periodic; Y and Z periodic, or walls of type bc)
    with a smooth random state and a divergence-free random field: uniform
    b0 plus the curl of a potential of a few integer Fourier modes of the
    box, evaluated at the ghosts' positions too."""
    rng = np.random.Generator(np.random.PCG64(seed))
    L = (1.0, ny / nx if ny > 1 else 1.0, nz / nx if nz > 1 else 1.0)
    w = _mhd_base("mhd_box", nx, ny, nz, g, (0.0, L[0]), (0.0, L[1]), (0.0, L[2]), 5.0 / 3.0, iso, 0.8,
                  (bc, bc), (bc, bc), eta=eta, passive=passive)
    if nu > 0:
        w.nu = np.full((w.nz_t, w.ny_t), nu)
    xc, xf, yc, yfa, zc, zfa, dx = _mhd_coords(w)

    def modes(a):
        terms = []
        for _ in range(3):
            k = [rng.integers(0, 3), rng.integers(0, 3) if ny > 1 else 0, rng.integers(0, 3) if nz > 1 else 0]
            ph = rng.uniform(0, 2 * math.pi)
            c = a * rng.uniform(-1, 1)
            terms.append((k, ph, c))

        def f(x, y, z):
            out = 0.0
            for k, ph, c in terms:
                out = out + c * np.cos(2 * math.pi * (k[0] * x / L[0] + k[1] * y / L[1] + k[2] * z / L[2]) + ph)
            return out
        return f

    def cell(f, z, y, x):
        return f(x[None, None, :], y[None, :, None], z[:, None, None]) + 0.0 * np.zeros((len(z), len(y), len(x)))

    st = w.state
    nzt, nyt = w.nz_t, w.ny_t
    st["rho"][:nzt, :nyt] = 1.0 + cell(modes(0.2), zc, yc, xc)
    if not iso:
        st["e"][:nzt, :nyt] = 1.5 * (1.0 + cell(modes(0.2), zc, yc, xc))
    st["vx"][:nzt, :nyt] = cell(modes(amp), zc, yc, xf)
    st["vy"][:nzt, :nyt + 1] = cell(modes(amp), zc, yfa, xc)
    if nz > 1:
        st["vz"][:nzt + 1, :nyt] = cell(modes(amp), zfa, yc, xc)
    bx, by, bz = curl_field(w, modes(0.05), modes(0.05), modes(0.05))
    st["bx"][:] = bx
    st["by"][:] = by
    st["bz"][:] = bz
    st["bx"][:nzt, :nyt] += b0[0]
    st["by"][:nzt, :nyt + 1] += b0[1]
    st["bz"][:nzt + 1, :nyt] += b0[2]
    return w


def current_sheet(nz=512, eta=0.25, b0=1.0, t0=None, g=3, cfl=0.44):
    """Resistive spreading of a current sheet (Sec. 5.2): a 1.5D column along
    Z on [-1, 1], gas at rest (rho = 1, P = 1, adiabatic), B_y = b0 erf(z /
    sqrt(4 eta t)) at t = t0, the field passive, zero-gradient Z boundaries.
    The field obeys dB_y/dt = eta d2B_y/dz2, whose solution stays the erf
    with t growing (current_sheet_profile).  t0 defaults to the test's
    (2.5 dz)^2 (with eta = 0.25: sqrt(4 eta t0) = 2.5 cells)."""
    w = _mhd_base("current_sheet", 1, 1, nz, g, (0.0, 1.0), (0.0, 1.0), (-1.0, 1.0), 5.0 / 3.0, False, 0.0,
                  (BC_ZEROGRAD, BC_ZEROGRAD), (BC_ZEROGRAD, BC_ZEROGRAD), cfl=cfl, eta=eta, passive=True)
    dz = 2.0 / nz
    if t0 is None:
        t0 = (2.5 * dz) ** 2
    w.t0 = t0
    st = w.state
    st["rho"][:] = 1.0
    st["e"][:] = 1.0 / (w.gamma - 1.0)
    zc = centres(w.zf)
    st["by"][:w.nz_t, :, :] = current_sheet_profile(zc, t0, eta, b0)[:, None, None]
    return w


def current_sheet_profile(z, t, eta=0.25, b0=1.0):
    return b0 * np.array([math.erf(v / math.sqrt(4.0 * eta * t)) for v in np.ravel(z)]).reshape(np.shape(z))


def _wave_box(name, nx, ny, g, cfl=0.44):
    return _mhd_base(name, nx, ny, 1, g, (0.0, 1.0), (0.0, ny / nx), (0.0, 1.0), 5.0 / 3.0, False, 0.0,
                     (BC_PERIODIC, BC_PERIODIC), (BC_ZEROGRAD, BC_ZEROGRAD), cfl=cfl)


def alfven_wave(nx=64, ny=4, amp=1e-3, bx=1.0, rho=1.0, pressure=0.6, g=3, modes=1, right=True):
    """A linear Alfven wave along X in a periodic X-Y box (1 x ny/nx): uniform
    rho and B_x, v_y = amp sin(k x), B_y = -+ amp sqrt(rho) sin(k x) (the
    minus sign for the wave moving in +x at v_A = B_x / sqrt(rho)),
    k = 2 pi modes.  Constant along Y; ny cells there keep v_y and B_y
    dynamical (a present direction)."""
    w = _wave_box("alfven_wave", nx, ny, g)
    st = w.state
    xc, xf, yc, yfa, zc, zfa, dx = _mhd_coords(w)
    k = 2.0 * math.pi * modes
    s = np.sin(k * xc)[None, None, :]
    nzt, nyt = w.nz_t, w.ny_t
    st["rho"][:nzt, :nyt] = rho
    st["e"][:nzt, :nyt] = pressure / (w.gamma - 1.0)
    st["bx"][:nzt, :nyt] = bx
    st["vy"][:nzt, :nyt + 1] = amp * s
    st["by"][:nzt, :nyt + 1] = (-1.0 if right else 1.0) * amp * math.sqrt(rho) * s
    return w


def fast_wave(nx=64, ny=4, amp=1e-3, bz=1.0, rho=1.0, pressure=0.6, g=3, modes=1):
    """A linear fast magnetosonic wave along X across a uniform B_z in a
    periodic X-Y box: the sound wave of rho = 1, P = 0.6 (c_s = 1 with
    gamma = 5/3) moving in +x, B_z compressed with the gas; it travels at
    sqrt(c_s^2 + B_z^2 / rho).  v_x = amp sin(k x) at the X faces, the
    density, pressure and B_z perturbed in phase: delta rho / rho =
    delta B_z / B_z = v_x / c_f, delta P = gamma P delta rho / rho."""
    w = _wave_box("fast_wave", nx, ny, g)
    st = w.state
    xc, xf, yc, yfa, zc, zfa, dx = _mhd_coords(w)
    k = 2.0 * math.pi * modes
    cs2 = w.gamma * pressure / rho
    cf = math.sqrt(cs2 + bz * bz / rho)
    sc = np.sin(k * xc)[None, None, :]
    nzt, nyt = w.nz_t, w.ny_t
    d = amp / cf * sc
    st["rho"][:nzt, :nyt] = rho * (1.0 + d)
    st["e"][:nzt, :nyt] = (pressure * (1.0 + w.gamma * d)) / (w.gamma - 1.0)
    st["bz"][:nzt, :nyt] = bz * (1.0 + d)
    st["vx"][:nzt, :nyt] = amp * np.sin(k * xf)[None, None, :]
    return w


def magnetostatic_column(nx=64, ny=4, b0=1.0, p0=2.0, g=3):
    """B_z(x) = b0 (1 + 0.5 sin 2 pi x) with the gas pressure P = p0 -
    B_z^2 / 2 (total pressure uniform), rho = 1, at rest: a magnetostatic
    equilibrium with no tension (B_z does not vary along z)."""
    w = _wave_box("magnetostatic_column", nx, ny, g)
    st = w.state
    xc, xf, yc, yfa, zc, zfa, dx = _mhd_coords(w)
    b = b0 * (1.0 + 0.5 * np.sin(2.0 * math.pi * xc))[None, None, :]
    nzt, nyt = w.nz_t, w.ny_t
    st["rho"][:nzt, :nyt] = 1.0
    st["bz"][:nzt, :nyt] = b
    st["e"][:nzt, :nyt] = (p0 - 0.5 * b * b) / (w.gamma - 1.0)
    return w


def mhd_shearing_sheet(nx=32, ny=32, nz=1, omega=1.0, oort_a=-0.75, cs=0.1, lx=1.0, ly=1.0, lz=0.5,
                       b0=(0.0, 0.05, 0.0), amp=0.0, seed=0, fargo=True, bcy=BC_FROZEN, g=3, eta=0.0,
                       passive=False, vamp=0.0):
    """A Cartesian shearing sheet with a magnetic field (Sec. 2 and Sec. 3.6):
    the frame turns at Omega, X runs along the shear flow v_x = 2 A y
    (A = -3/4 Omega, Keplerian) over lx, Y across it on [-ly/2, ly/2] with
    walls of type bcy (frozen: the initial state) or periodic, Z periodic
    over lz.  Uniform density 1, isothermal (sound speed cs), no potential.
    The field is the uniform b0 plus, with amp > 0, the curl of a seeded
    vector potential of a few Fourier modes (divergence-free to round-off);
    vamp > 0 adds a seeded smooth velocity perturbation."""
    rng = np.random.Generator(np.random.PCG64(seed))
    yf = faces(ny, g, -0.5 * ly, 0.5 * ly)
    zf = faces(nz, g, -0.5 * lz, 0.5 * lz)
    w = Workload("mhd_shearing_sheet", CART, nx, ny, nz, g, 0.0, lx, yf, zf, 5.0 / 3.0, True, None, None, 0.44,
                 1.41, fargo, omega, (bcy, bcy), (BC_PERIODIC, BC_PERIODIC), 0.0, 0.0, 1.0, 0.0, False, 0.0,
                 1e30, {}, shearing=True, oort_a=oort_a)
    w.mhd, w.mhd_passive, w.eta = True, passive, eta
    w.cs = np.full((w.nz_t, w.ny_t), cs)
    st = _empty(w.shape)
    st.update({k: np.zeros(w.shape) for k in MHD_FIELDS})
    w.state = st
    L = (lx, ly, lz)

    def modes(a):
        terms = []
        for _ in range(3):
            k = [rng.integers(1, 3), rng.integers(0, 3) if ny > 1 else 0, rng.integers(0, 3) if nz > 1 else 0]
            terms.append((k, rng.uniform(0, 2 * math.pi), a * rng.uniform(-1, 1)))

        def f(x, y, z):
            out = 0.0
            for k, ph, c in terms:
                out = out + c * np.cos(2 * math.pi * (k[0] * x / L[0] + k[1] * y / L[1] + k[2] * z / L[2]) + ph)
            return out
        return f

    xc, xf, yc, yfa, zc, zfa, dx = _mhd_coords(w)
    nzt, nyt = w.nz_t, w.ny_t
    st["rho"][:nzt, :nyt] = 1.0
    st["vx"][:nzt, :nyt] = (2.0 * oort_a * yc[:nyt])[None, :, None]
    if vamp > 0:
        fx, fy = modes(vamp), modes(vamp)
        st["vx"][:nzt, :nyt] += fx(xf[None, None, :], yc[None, :nyt, None], zc[:nzt, None, None])
        st["vy"][:nzt, :nyt + 1] += fy(xc[None, None, :], yfa[None, :, None], zc[:nzt, None, None])
    if amp > 0:
        bx, by, bz = curl_field(w, modes(amp), modes(amp), modes(amp))
        st["bx"][:] = bx
        st["by"][:] = by
        st["bz"][:] = bz
    st["bx"][:nzt, :nyt] += b0[0]
    st["by"][:nzt, :nyt + 1] += b0[1]
    st["bz"][:nzt + 1, :nyt] += b0[2]
    return w


def uniform_mhd_box(nx, ny, nz, rho=1.0, e=1.5, v=(0.0, 0.0, 0.0), b=(0.0, 0.0, 0.0), periodic=True, g=3,
                    eta=0.0, passive=False):
    """A Cartesian MHD box holding a uniform state (ghosts included);
    periodic or zero-gradient Y and Z boundaries.  The starting point of
    the closed-form pins (each test shapes the fields it needs)."""
    bc = (BC_PERIODIC, BC_PERIODIC) if periodic else (BC_ZEROGRAD, BC_ZEROGRAD)
    w = _mhd_base("mhd_uniform", nx, ny, nz, g, (0.0, 1.0), (0.0, ny / nx), (0.0, nz / nx), 5.0 / 3.0, False, 0.0,
                  bc, bc, eta=eta, passive=passive)
    st = w.state
    for k, val in (("rho", rho), ("e", e), ("vx", v[0]), ("vy", v[1]), ("vz", v[2]),
                   ("bx", b[0]), ("by", b[1]), ("bz", b[2])):
        st[k][:] = val
    return w


def resistive_mode(nz=32, mode=2, eta=0.1, g=3):
    """A passive field B_y = sin(2 pi mode z) in a periodic column along Z
    (unit length) with the gas at rest: Ohmic diffusion alone, each Fourier
    mode of the discrete Laplacian decaying by its own factor per step."""
    w = _mhd_base("resistive_mode", 1, 1, nz, g, (0.0, 1.0), (0.0, 1.0), (0.0, 1.0), 5.0 / 3.0, False, 0.0,
                  (BC_ZEROGRAD, BC_ZEROGRAD), (BC_PERIODIC, BC_PERIODIC), eta=eta, passive=True)
    st = w.state
    st["rho"][:] = 1.0
    st["e"][:] = 1.5
    zc = centres(w.zf)[:w.nz_t]
    st["by"][:w.nz_t, :, :] = np.sin(2.0 * math.pi * mode * zc)[:, None, None]
    return w


def field_loop(ny=128, nz=64, vy=math.sqrt(5.0) / 2.0, vz=0.0, a0=1e-3, radius=0.3, g=3):
    """The magnetic field loop advected across a periodic Y-Z box (Sec. 5.2,
    the loop test): y in [-1, 1], z in [-0.5, 0.5], rho = 1, P = 1,
    gamma = 5/3, uniform velocity (v_y, v_z), B = curl A with
    A_x = a0 (radius - r) inside r < radius (r the distance to the box
    centre, measured to the nearest periodic image), 0 outside."""
    w = _mhd_base("field_loop", 1, ny, nz, g, (0.0, 1.0), (-1.0, 1.0), (-0.5, 0.5), 5.0 / 3.0, False, 0.0,
                  (BC_PERIODIC, BC_PERIODIC), (BC_PERIODIC, BC_PERIODIC))
    st = w.state
    nzt, nyt = w.nz_t, w.ny_t
    st["rho"][:] = 1.0
    st["e"][:] = 1.0 / (w.gamma - 1.0)
    st["vy"][:] = vy
    st["vz"][:] = vz

    def ax(x, y, z):
        yy = (y + 1.0) % 2.0 - 1.0
        zz = (z + 0.5) % 1.0 - 0.5
        r = np.sqrt(yy * yy + zz * zz)
        return np.where(r < radius, a0 * (radius - r), 0.0)

    zero = lambda x, y, z: 0.0 * (x + y + z)  # noqa: E731
    bx, by, bz = curl_field(w, ax, zero, zero)
    st["bx"][:] = bx
    st["by"][:] = by
    st["bz"][:] = bz
    return w


def magnetic_energy(w, st):
    """Mean over the active cells of B^2, each component the zone-centred
    two-point mean of its faces (the single value along an absent axis)."""
    out = 0.0
    for d, k in enumerate(MHD_FIELDS):
        b = st[k]
        gz, gy = w.gz, w.gy
        lo = b[gz:gz + w.nz, gy:gy + w.ny, :]
        if d == 0:
            up = np.roll(lo, -1, axis=2)
        elif d == 1 and w.ny > 1:
            up = b[gz:gz + w.nz, gy + 1:gy + w.ny + 1, :]
        elif d == 2 and w.nz > 1:
            up = b[gz + 1:gz + w.nz + 1, gy:gy + w.ny, :]
        else:
            up = lo
        out = out + (0.5 * (lo + up)) ** 2
    return float(np.mean(out))


def _yz_box(name, ny, nz, yr, zr, gamma, bc, g=3, cfl=0.44):
    """A Y-Z plane (one cell in X) Cartesian MHD box with the boundary
    condition bc on both axes."""
    return _mhd_base(name, 1, ny, nz, g, (0.0, 1.0), yr, zr, gamma, False, 0.0, (bc, bc), (bc, bc), cfl=cfl)


def orszag_tang(n=128, plane="yz", g=3):
    """The Orszag-Tang vortex (Sec. 5.2): the unit square, periodic,
    gamma = 5/3, rho = 25/(36 pi), P = 5/(12 pi), v = (-sin 2 pi z,
    sin 2 pi y), B = B0 (-sin 2 pi z, sin 4 pi y), B0 = (4 pi)^-1/2, in the
    Y-Z plane as printed; plane="xy" lays the same problem in the X-Y plane
    (y -> x, z -> y), where the azimuthal lanes of the kernels are filled."""
    b0 = 1.0 / math.sqrt(4.0 * math.pi)
    if plane == "yz":
        w = _yz_box("orszag_tang", n, n, (0.0, 1.0), (0.0, 1.0), 5.0 / 3.0, BC_PERIODIC, g)
        xc, xf, yc, yfa, zc, zfa, dx = _mhd_coords(w)
        st = w.state
        nzt, nyt = w.nz_t, w.ny_t
        st["vy"][:nzt, :nyt + 1] = -np.sin(2 * math.pi * zc)[:, None, None]
        st["vz"][:nzt + 1, :nyt] = np.sin(2 * math.pi * yc)[None, :, None]
        st["by"][:nzt, :nyt + 1] = -b0 * np.sin(2 * math.pi * zc)[:, None, None]
        st["bz"][:nzt + 1, :nyt] = b0 * np.sin(4 * math.pi * yc)[None, :, None]
    else:
        w = _mhd_base("orszag_tang_xy", n, n, 1, g, (0.0, 1.0), (0.0, 1.0), (0.0, 1.0), 5.0 / 3.0, False, 0.0,
                      (BC_PERIODIC, BC_PERIODIC), (BC_ZEROGRAD, BC_ZEROGRAD))
        xc, xf, yc, yfa, zc, zfa, dx = _mhd_coords(w)
        st = w.state
        nzt, nyt = w.nz_t, w.ny_t
        st["vx"][:nzt, :nyt] = -np.sin(2 * math.pi * yc)[None, :, None]
        st["vy"][:nzt, :nyt + 1] = np.sin(2 * math.pi * xc)[None, None, :]
        st["bx"][:nzt, :nyt] = -b0 * np.sin(2 * math.pi * yc)[None, :, None]
        st["by"][:nzt, :nyt + 1] = b0 * np.sin(4 * math.pi * xc)[None, None, :]
    st["rho"][:] = 25.0 / (36.0 * math.pi)
    st["e"][:] = 5.0 / (12.0 * math.pi) / (w.gamma - 1.0)
    return w


def brio_wu(nz=800, g=3):
    """The MHD Riemann problem of Brio & Wu (Sec. 5.2) along Z: z in
    [0, 800], the discontinuity at 400, rho = 1 / 0.1, P = 1 / 0.1,
    B_z = 0.75, B_y = 1 / -1, gamma = 2, reflecting walls, shown at t = 80.
    The paper runs it as a 1.5D problem; here Y holds four periodic cells
    so that v_y and B_y, the transverse pair, are dynamical (an axis of a
    single cell is absent in this implementation)."""
    w = _mhd_base("brio_wu", 1, 4, nz, g, (0.0, 1.0), (0.0, 4.0), (0.0, 800.0), 2.0, False, 0.0,
                  (BC_PERIODIC, BC_PERIODIC), (BC_REFLECT, BC_REFLECT), t_end=80.0)
    zc = centres(w.zf)[:w.nz_t]
    left = (zc < 400.0)[:, None, None]
    st = w.state
    st["rho"][:w.nz_t] = np.where(left, 1.0, 0.1)
    st["e"][:w.nz_t] = np.where(left, 1.0, 0.1) / (w.gamma - 1.0)
    st["by"][:w.nz_t] = np.where(left, 1.0, -1.0)
    st["bz"][:] = 0.75
    return w


def mhd_rotor(n=128, g=3):
    """The MHD rotor (Sec. 5.2), Cartesian, in the Y-Z plane: the unit box
    centred on 0, reflecting walls, gamma = 1.4, P = 1, B_y = 5/sqrt(4 pi);
    rho = 10 and a solid rotation of angular speed v0/r1 (v0 = 2) for
    r0 <= r <= r1, with a linear taper to the background (rho = 1, at rest)
    over r1 < r < r2, and the inner hole r < r0 at rest with rho = 1
    (r0 = 0.05, r1 = 0.1, r2 = 0.115; r from the box centre)."""
    w = _yz_box("mhd_rotor", n, n, (-0.5, 0.5), (-0.5, 0.5), 1.4, BC_REFLECT, g)
    xc, xf, yc, yfa, zc, zfa, dx = _mhd_coords(w)
    r0, r1, r2, v0 = 0.05, 0.1, 0.115, 2.0

    def prof(y, z):
        r = np.sqrt(y * y + z * z)
        f = np.clip((r2 - r) / (r2 - r1), 0.0, 1.0)
        rho = np.where(r < r0, 1.0, np.where(r <= r1, 10.0, 1.0 + 9.0 * f))
        s = np.where(r < r0, 0.0, np.where(r <= r1, 1.0, f))
        return rho, s

    st = w.state
    rho, _ = prof(yc[None, :], zc[:, None])
    st["rho"][:w.nz_t, :w.ny_t, 0] = rho
    _, s = prof(yfa[None, :], zc[:, None])
    st["vy"][:w.nz_t, :w.ny_t + 1, 0] = -s * v0 * zc[:, None] / r1
    _, s = prof(yc[None, :], zfa[:, None])
    st["vz"][:w.nz_t + 1, :w.ny_t, 0] = s * v0 * yc[None, :] / r1
    st["e"][:] = 1.0 / (w.gamma - 1.0)
    st["by"][:] = 5.0 / math.sqrt(4.0 * math.pi)
    return w


def current_sheet_2d(n=256, v0=0.1, g=3):
    """The current sheet of Sec. 5.2 (after Gardiner & Stone): (y, z) in
    [0, 2]^2, periodic, rho = 1, P = 0.1, gamma = 5/3, B_z = 1 where
    |y - 1| < 0.5 and -1 elsewhere, v_y = v0 sin(pi z), no physical
    resistivity."""
    w = _yz_box("current_sheet_2d", n, n, (0.0, 2.0), (0.0, 2.0), 5.0 / 3.0, BC_PERIODIC, g)
    xc, xf, yc, yfa, zc, zfa, dx = _mhd_coords(w)
    st = w.state
    st["rho"][:] = 1.0
    st["e"][:] = 0.1 / (w.gamma - 1.0)
    st["bz"][:, :w.ny_t, 0] = np.where(np.abs(yc - 1.0) < 0.5, 1.0, -1.0)[None, :]
    st["vy"][:w.nz_t, :, 0] = (v0 * np.sin(math.pi * zc))[:, None]
    return w
