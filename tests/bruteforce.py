"""Independent brute-force restatement of one step of the method, for tiny meshes.

Test infrastructure, written from the paper's equations and the readings
listed with the oracle, in a deliberately different form from the C oracle:
every quantity lives at a position of the staggered mesh given in doubled
logical coordinates (cell centres odd, faces and edges even), values at
other positions are arithmetic averages of the neighbouring samples, and
every derivative is a difference of two samples divided by the difference
of their coordinates, the metric factors of the printed equations written
out term by term.  Geometry (face areas, volumes) comes from the closed-form
integrals of the metric, not from the product tables of App. A.  Plain
Python loops: meant for meshes of a few hundred cells.

State arrays follow the shared layout (nz_t + 1, ny_t + 1, nx), X fastest.
"""
from __future__ import annotations

import math

import numpy as np

CART, CYL, SPH = 0, 1, 2
# staggering of each quantity: 1 = centred along that axis (odd doubled
# coordinate), 0 = on the lower face (even), for axes (x, y, z)
CENTRE = (1, 1, 1)
STAG = {"rho": CENTRE, "e": CENTRE, "vx": (0, 1, 1), "vy": (1, 0, 1), "vz": (1, 1, 0),
        "txx": CENTRE, "tyy": CENTRE, "tzz": CENTRE, "txy": (0, 0, 1), "txz": (0, 1, 0), "tyz": (1, 0, 0)}


class Mesh:
    def __init__(self, w):
        self.w = w
        self.geom = w.geom
        self.nx, self.ny, self.nz = w.nx, w.ny, w.nz
        self.hasX, self.hasY, self.hasZ = w.nx > 1, w.ny > 1, w.nz > 1
        self.yf = np.asarray(w.yf, dtype=float)
        self.zf = np.asarray(w.zf, dtype=float)
        self.nyt, self.nzt = len(self.yf) - 1, len(self.zf) - 1
        self.j0, self.j1 = w.gy, w.gy + w.ny
        self.k0, self.k1 = w.gz, w.gz + w.nz
        self.dx = (w.xmax - w.xmin) / w.nx

    # ---- coordinates at doubled logical positions
    def phi(self, x2):
        return self.w.xmin + 0.5 * x2 * self.dx

    def y(self, y2):
        if y2 % 2 == 0:
            return self.yf[y2 // 2]
        return 0.5 * (self.yf[(y2 - 1) // 2] + self.yf[(y2 + 1) // 2])

    def z(self, z2):
        if z2 % 2 == 0:
            return self.zf[z2 // 2]
        return 0.5 * (self.zf[(z2 - 1) // 2] + self.zf[(z2 + 1) // 2])

    def R(self, y2, z2):
        """Distance to the rotation axis (lever arm of the azimuthal motion)."""
        if self.geom == CYL:
            return self.y(y2)
        if self.geom == SPH:
            return self.y(y2) * math.sin(self.z(z2))
        return 1.0

    def coord_step(self, axis, lo, hi):
        """Coordinate difference between two positions along `axis` (doubled coords)."""
        if axis == 0:
            return 0.5 * (hi - lo) * self.dx
        if axis == 1:
            return self.y(hi) - self.y(lo)
        return self.z(hi) - self.z(lo)

    # ---- exact geometry of a cell (j, k): integrals of the metric
    def volume(self, j, k):
        r0, r1 = self.yf[j], self.yf[j + 1]
        z0, z1 = self.zf[k], self.zf[k + 1]
        if self.geom == CART:
            return self.dx * (r1 - r0) * (z1 - z0)
        if self.geom == CYL:      # int r dr dphi dz
            return 0.5 * (r1 * r1 - r0 * r0) * self.dx * (z1 - z0)
        # int r^2 sin(theta) dr dtheta dphi
        return (r1 ** 3 - r0 ** 3) / 3.0 * self.dx * (math.cos(z0) - math.cos(z1))

    def area(self, axis, j, k):
        """Area of the lower face of cell (j, k) normal to `axis`."""
        r0, r1 = self.yf[j], self.yf[j + 1]
        z0, z1 = self.zf[k], self.zf[k + 1]
        if self.geom == CART:
            return [(r1 - r0) * (z1 - z0), self.dx * (z1 - z0), self.dx * (r1 - r0)][axis]
        if self.geom == CYL:
            if axis == 0:      # phi = const: dr dz
                return (r1 - r0) * (z1 - z0)
            if axis == 1:      # r = r0: r dphi dz
                return r0 * self.dx * (z1 - z0)
            return 0.5 * (r1 * r1 - r0 * r0) * self.dx     # z = z0: r dr dphi
        if axis == 0:          # phi = const: r dr dtheta
            return 0.5 * (r1 * r1 - r0 * r0) * (z1 - z0)
        if axis == 1:          # r = r0: r^2 sin(theta) dtheta dphi
            return r0 * r0 * self.dx * (math.cos(z0) - math.cos(z1))
        return 0.5 * (r1 * r1 - r0 * r0) * self.dx * math.sin(z0)   # theta = z0: r sin(theta) dr dphi


class Field:
    """A staggered quantity read at doubled logical positions; positions of
    the other parity along an axis read the average of the two neighbours.
    The quantity is an array, or a function `fn(x2, y2, z2)` evaluated at
    its own positions only (so a derived value such as v_phi + R Omega_f is
    formed at each sample before the average)."""

    def __init__(self, mesh, a, stag, fn=None):
        self.m, self.a, self.s, self.fn = mesh, a, stag, fn

    def __call__(self, x2, y2, z2):
        m = self.m
        p = [x2, y2, z2]
        for ax in range(3):
            if [m.hasX, m.hasY, m.hasZ][ax] and (p[ax] - self.s[ax]) % 2 != 0:
                lo, hi = list(p), list(p)
                lo[ax] -= 1
                hi[ax] += 1
                return 0.5 * (self(*lo) + self(*hi))
        if self.fn is not None:
            return self.fn(x2, y2, z2)
        i = ((x2 - self.s[0]) // 2) % m.nx
        j = (y2 - self.s[1]) // 2 if m.hasY else 0
        k = (z2 - self.s[2]) // 2 if m.hasZ else 0
        return self.a[k, j, i]


def deriv(m, f, axis, p):
    """d f / d(coordinate of `axis`) at p from the two samples at p -+ 1."""
    lo, hi = list(p), list(p)
    lo[axis] -= 1
    hi[axis] += 1
    return (f(*hi) - f(*lo)) / m.coord_step(axis, lo[axis], hi[axis])


def scaled(f, g):
    """Pointwise product of a sampler f and a position function g."""
    return lambda x2, y2, z2: f(x2, y2, z2) * g(x2, y2, z2)


def ring(w, a, j, k):
    return a[k, j] if a is not None else 0.0


# ---------------------------------------------------------------------------
# Pressure and potential (cells 4 and 5)
# ---------------------------------------------------------------------------
def pressure(w, st):
    P = np.zeros_like(st["rho"])
    for k in range(len(w.zf) - 1):
        for j in range(len(w.yf) - 1):
            if w.iso:
                P[k, j] = w.cs[k, j] ** 2 * st["rho"][k, j]
            else:
                P[k, j] = (w.gamma - 1.0) * st["e"][k, j]
    return P


def potential(w, t):
    """Star -M/r (spherical distance) plus a planet on its circular orbit at
    azimuth (Omega_p - Omega_f) t, Plummer-softened, with the indirect term
    q R a cos(phi - phi_p)/a^3, by the law of cosines in the midplane."""
    m = Mesh(w)
    phi = np.zeros_like(w.state["rho"])
    q, a, M = w.planet_q, w.planet_a, w.star_mass
    om_p = math.sqrt((M + q) / a ** 3) if q > 0 else 0.0
    ph_p = (om_p - w.omega_f) * t
    for k in range(m.nzt):
        for j in range(m.nyt):
            for i in range(m.nx):
                x2, y2, z2 = 2 * i + 1, 2 * j + 1, 2 * k + 1
                v = 0.0
                if w.geom == CART:
                    pass
                else:
                    if w.geom == CYL:
                        Rc, Zc = m.y(y2), m.z(z2)
                    else:
                        Rc, Zc = m.y(y2) * math.sin(m.z(z2)), m.y(y2) * math.cos(m.z(z2))
                    if M > 0:
                        v -= M / math.sqrt(Rc * Rc + Zc * Zc)
                    if q > 0:
                        cdp = math.cos(m.phi(x2) - ph_p)
                        d2 = Rc * Rc + a * a - 2.0 * Rc * a * cdp + Zc * Zc
                        v -= q / math.sqrt(d2 + w.planet_eps ** 2)
                        if w.indirect:
                            v += q * Rc * cdp / (a * a)
                phi[k, j, i] = v
    return phi


# ---------------------------------------------------------------------------
# Sub-step 1 (cell 7a, Sec. 3.3): pressure and potential gradients with the
# face density (rho_L + rho_R)/2 (Eq. 20), the centrifugal terms with the
# four-point average of the inertial azimuthal velocity (Eq. 12), the
# shearing sheet's Coriolis and tidal terms.  Jacobi; interior faces only.
# ---------------------------------------------------------------------------
def substep1(w, st, phi, dt):
    m = Mesh(w)
    out = {k: v.copy() for k, v in st.items()}
    P = Field(m, pressure(w, st), CENTRE)
    Ph = Field(m, phi if phi is not None else np.zeros_like(st["rho"]), CENTRE)
    rho = Field(m, st["rho"], CENTRE)
    vx, vz = Field(m, st["vx"], STAG["vx"]), Field(m, st["vz"], STAG["vz"])
    om = w.omega_f
    # inertial azimuthal velocity, formed at each v_phi face with its own R
    vt = Field(m, None, STAG["vx"], fn=lambda x2, y2, z2: vx(x2, y2, z2) + m.R(y2, z2) * om)
    for k in range(m.k0, m.k1):
        for j in range(m.j0, m.j1):
            for i in range(m.nx):
                if m.hasX:
                    p = (2 * i, 2 * j + 1, 2 * k + 1)
                    h = m.R(p[1], p[2])        # (1/r) or 1/(r sin theta) of the azimuthal derivative
                    acc = -deriv(m, P, 0, p) / h / rho(*p) - deriv(m, Ph, 0, p) / h
                    out["vx"][k, j, i] = st["vx"][k, j, i] + dt * acc
                if m.hasY and j > m.j0:
                    p = (2 * i + 1, 2 * j, 2 * k + 1)
                    acc = -deriv(m, P, 1, p) / rho(*p) - deriv(m, Ph, 1, p)
                    r = m.y(p[1])
                    if w.geom == CYL:
                        acc += vt(*p) ** 2 / r
                    elif w.geom == SPH:
                        cen = vt(*p) ** 2
                        if m.hasZ:
                            cen += vz(*p) ** 2
                        acc += cen / r
                    elif w.shearing:
                        acc += 2.0 * om * vx(*p) - 4.0 * w.oort_a * om * r
                    out["vy"][k, j, i] = st["vy"][k, j, i] + dt * acc
                if m.hasZ and k > m.k0:
                    p = (2 * i + 1, 2 * j + 1, 2 * k)
                    h = m.y(p[1]) if w.geom == SPH else 1.0   # 1/r of the colatitude derivative
                    acc = -deriv(m, P, 2, p) / h / rho(*p) - deriv(m, Ph, 2, p) / h
                    if w.geom == SPH:
                        th = m.z(p[2])
                        acc += vt(*p) ** 2 * (math.cos(th) / math.sin(th)) / m.y(p[1])
                    out["vz"][k, j, i] = st["vz"][k, j, i] + dt * acc
    return out


def _cell_width(m, axis, j, k):
    if axis == 0:
        return m.R(2 * j + 1, 2 * k + 1) * m.dx
    if axis == 1:
        return m.yf[j + 1] - m.yf[j]
    dz = m.zf[k + 1] - m.zf[k]
    return m.y(2 * j + 1) * dz if m.geom == SPH else dz


def _centre_distance(m, axis, p):
    """Physical distance between the two cell centres on either side of face p."""
    if axis == 0:
        return m.R(p[1], p[2]) * m.dx
    if axis == 1:
        return m.coord_step(1, p[1] - 1, p[1] + 1)
    d = m.coord_step(2, p[2] - 1, p[2] + 1)
    return m.y(p[1]) * d if m.geom == SPH else d


# ---------------------------------------------------------------------------
# Sub-step 2 (cell 7b): von Neumann-Richtmyer viscosity, component-wise, in
# the ZEUS form: q = C_q^2 rho (dv)^2 for a compression dv < 0 of the cell's
# two face velocities; faces accelerated by -(q_R - q_L)/(distance x face
# density); the gas heated by -q dv / width.
# ---------------------------------------------------------------------------
def artificial_viscosity(w, st, dt):
    if w.cq <= 0:
        return {k: v.copy() for k, v in st.items()}
    m = Mesh(w)
    out = {k: v.copy() for k, v in st.items()}
    names = ["vx", "vy", "vz"]
    active = [m.hasX, m.hasY, m.hasZ]
    q = [np.zeros_like(st["rho"]) for _ in range(3)]
    dv = [np.zeros_like(st["rho"]) for _ in range(3)]
    c2 = w.cq * w.cq
    for k in range(m.k0, m.k1):
        for j in range(m.j0, m.j1):
            for i in range(m.nx):
                up = [(k, j, (i + 1) % m.nx), (k, j + 1, i), (k + 1, j, i)]
                for ax in range(3):
                    if not active[ax]:
                        continue
                    d = st[names[ax]][up[ax]] - st[names[ax]][k, j, i]
                    dv[ax][k, j, i] = d
                    q[ax][k, j, i] = c2 * st["rho"][k, j, i] * d * d if d < 0 else 0.0
    rho = Field(m, st["rho"], CENTRE)
    if not w.iso:
        for k in range(m.k0, m.k1):
            for j in range(m.j0, m.j1):
                for i in range(m.nx):
                    heat = sum(q[ax][k, j, i] * dv[ax][k, j, i] / _cell_width(m, ax, j, k)
                               for ax in range(3) if active[ax])
                    out["e"][k, j, i] = st["e"][k, j, i] - dt * heat
    for ax in range(3):
        if not active[ax]:
            continue
        Q = Field(m, q[ax], CENTRE)
        for k in range(m.k0 + (1 if ax == 2 else 0), m.k1):
            for j in range(m.j0 + (1 if ax == 1 else 0), m.j1):
                for i in range(m.nx):
                    p = [2 * i + 1, 2 * j + 1, 2 * k + 1]
                    p[ax] -= 1
                    lo, hi = list(p), list(p)
                    lo[ax] -= 1
                    hi[ax] += 1
                    acc = -(Q(*hi) - Q(*lo)) / _centre_distance(m, ax, p) / rho(*p)
                    out[names[ax]][k, j, i] = st[names[ax]][k, j, i] + dt * acc
    return out


def divergence(m, st, i, j, k):
    """Gauss theorem on cell (i, j, k): (1/V) sum over faces of area x normal velocity."""
    f = 0.0
    if m.hasX:
        f += m.area(0, j, k) * (st["vx"][k, j, (i + 1) % m.nx] - st["vx"][k, j, i])
    if m.hasY:
        f += m.area(1, j + 1, k) * st["vy"][k, j + 1, i] - m.area(1, j, k) * st["vy"][k, j, i]
    if m.hasZ:
        f += m.area(2, j, k + 1) * st["vz"][k + 1, j, i] - m.area(2, j, k) * st["vz"][k, j, i]
    return f / m.volume(j, k)


# Sub-step 3 (cell 7c): -P div v for a gamma-law gas, time-centred:
# e' = e (1 - theta)/(1 + theta), theta = dt (gamma - 1) div v / 2.
def compression_heating(w, st, dt):
    out = {k: v.copy() for k, v in st.items()}
    if w.iso:
        return out
    m = Mesh(w)
    for k in range(m.k0, m.k1):
        for j in range(m.j0, m.j1):
            for i in range(m.nx):
                th = 0.5 * dt * (w.gamma - 1.0) * divergence(m, st, i, j, k)
                out["e"][k, j, i] = st["e"][k, j, i] * (1.0 - th) / (1.0 + th)
    return out


# ---------------------------------------------------------------------------
# Cell 7d: viscous stress tensor (App. B, Eqs. 72-74) and the velocity
# update (Eqs. 75-77), every term as printed with explicit metric factors;
# diagonal components at cell centres, tau_xy on (x-, y-) edges, tau_xz on
# (x-, z-) edges, tau_yz on (y-, z-) edges; rho and nu on an edge averaged
# over the cells sharing it; Eq. 75 divided by the face density.
# ---------------------------------------------------------------------------
def viscosity(w, st, dt):
    out = {k: v.copy() for k, v in st.items()}
    if w.nu is None:
        return out
    m = Mesh(w)
    g = w.geom
    rho = Field(m, st["rho"], CENTRE)
    nu = Field(m, _pad_ring(w, st), CENTRE)
    vx, vy, vz = (Field(m, st[n], STAG[n]) for n in ("vx", "vy", "vz"))
    r_ = lambda x2, y2, z2: m.y(y2)                               # noqa: E731
    s_ = lambda x2, y2, z2: math.sin(m.z(z2))                     # noqa: E731
    T = {n: np.zeros_like(st["rho"]) for n in ("txx", "tyy", "tzz", "txy", "txz", "tyz")}
    d = lambda f, ax, p: deriv(m, f, ax, p)                       # noqa: E731
    # diagonal components at active cell centres
    for k in range(m.k0, m.k1):
        for j in range(m.j0, m.j1):
            for i in range(m.nx):
                p = (2 * i + 1, 2 * j + 1, 2 * k + 1)
                rn = rho(*p) * nu(*p)
                div = divergence(m, st, i, j, k)
                r = m.y(p[1])
                dvx = d(vx, 0, p) if m.hasX else 0.0
                dvy = d(vy, 1, p) if m.hasY else 0.0
                dvz = d(vz, 2, p) if m.hasZ else 0.0
                vr = vy(*p) if m.hasY else 0.0
                if g == CART:
                    xx, yy, zz = dvx, dvy, dvz
                elif g == CYL:
                    xx, yy, zz = dvx / r + vr / r, dvy, dvz
                else:
                    th = m.z(p[2])
                    vth = vz(*p) if m.hasZ else 0.0
                    xx = dvx / (r * math.sin(th)) + vr / r + vth * (math.cos(th) / math.sin(th)) / r
                    yy = dvy
                    zz = dvz / r + vr / r
                T["txx"][k, j, i] = -rn * (2.0 * xx - 2.0 / 3.0 * div)
                T["tyy"][k, j, i] = -rn * (2.0 * yy - 2.0 / 3.0 * div)
                T["tzz"][k, j, i] = -rn * (2.0 * zz - 2.0 / 3.0 * div)
    # tau_xy (tau_phi r) on the edges (i-1/2, j-1/2, k)
    if m.hasY:
        for k in range(m.k0, m.k1):
            for j in range(m.j0, m.j1 + 1):
                for i in range(m.nx):
                    p = (2 * i, 2 * j, 2 * k + 1)
                    r = m.y(p[1])
                    if g == CART:
                        t = d(vy, 0, p) + d(vx, 1, p)
                    elif g == CYL:
                        t = d(vx, 1, p) - vx(*p) / r + d(vy, 0, p) / r
                    else:
                        t = d(vy, 0, p) / (r * math.sin(m.z(p[2]))) + d(vx, 1, p) - vx(*p) / r
                    T["txy"][k, j, i] = -rho(*p) * nu(*p) * t
    # tau_xz (tau_phi z / tau_phi theta) on the edges (i-1/2, j, k-1/2)
    if m.hasZ:
        for k in range(m.k0, m.k1 + 1):
            for j in range(m.j0, m.j1):
                for i in range(m.nx):
                    p = (2 * i, 2 * j + 1, 2 * k)
                    r = m.y(p[1])
                    if g == CART:
                        t = d(vz, 0, p) + d(vx, 2, p)
                    elif g == CYL:
                        t = d(vx, 2, p) + d(vz, 0, p) / r
                    else:
                        th = m.z(p[2])
                        vs = Field(m, None, STAG["vx"], fn=lambda x2, y2, z2: vx(x2, y2, z2) / math.sin(m.z(z2)))
                        t = math.sin(th) / r * d(vs, 2, p) + d(vz, 0, p) / (r * math.sin(th))
                    T["txz"][k, j, i] = -rho(*p) * nu(*p) * t
    # tau_yz (tau_rz / tau_r theta) on the edges (i, j-1/2, k-1/2)
    if m.hasY and m.hasZ:
        for k in range(m.k0, m.k1 + 1):
            for j in range(m.j0, m.j1 + 1):
                for i in range(m.nx):
                    p = (2 * i + 1, 2 * j, 2 * k)
                    r = m.y(p[1])
                    if g == SPH:
                        t = d(vz, 1, p) - vz(*p) / r + d(vy, 2, p) / r
                    else:
                        t = d(vz, 1, p) + d(vy, 2, p)
                    T["tyz"][k, j, i] = -rho(*p) * nu(*p) * t
    txx, tyy, tzz, txy, txz, tyz = (Field(m, T[n], STAG[n]) for n in ("txx", "tyy", "tzz", "txy", "txz", "tyz"))
    r2 = lambda x2, y2, z2: m.y(y2) ** 2                          # noqa: E731
    r3 = lambda x2, y2, z2: m.y(y2) ** 3                          # noqa: E731
    # v_x (v_phi) on the active faces
    for k in range(m.k0, m.k1):
        for j in range(m.j0, m.j1):
            for i in range(m.nx):
                p = (2 * i, 2 * j + 1, 2 * k + 1)
                r = m.y(p[1])
                f = 0.0
                if g == CART:
                    f += d(txx, 0, p)
                    if m.hasY:
                        f += d(txy, 1, p)
                    if m.hasZ:
                        f += d(txz, 2, p)
                elif g == CYL:
                    if m.hasY:
                        f += d(scaled(txy, r2), 1, p) / (r * r)
                    f += d(txx, 0, p) / r
                    if m.hasZ:
                        f += d(txz, 2, p)
                else:
                    th = m.z(p[2])
                    if m.hasY:
                        f += d(scaled(txy, r2), 1, p) / (r * r)
                    if m.hasZ:
                        f += d(txz, 2, p) / r
                    f += d(txx, 0, p) / (r * math.sin(th))
                    if m.hasY:
                        f += txy(*p) / r
                    if m.hasZ:
                        f += 2.0 * txz(*p) * (math.cos(th) / math.sin(th)) / r
                out["vx"][k, j, i] = st["vx"][k, j, i] - dt * f / rho(*p)
    # v_y (v_r) on the interior faces
    if m.hasY:
        for k in range(m.k0, m.k1):
            for j in range(m.j0 + 1, m.j1):
                for i in range(m.nx):
                    p = (2 * i + 1, 2 * j, 2 * k + 1)
                    r = m.y(p[1])
                    f = 0.0
                    if g == CART:
                        f += d(txy, 0, p) + d(tyy, 1, p)
                        if m.hasZ:
                            f += d(tyz, 2, p)
                    elif g == CYL:
                        f += d(scaled(tyy, r_), 1, p) / r + d(txy, 0, p) / r - txx(*p) / r
                        if m.hasZ:
                            f += d(tyz, 2, p)
                    else:
                        th = m.z(p[2])
                        f += d(scaled(tyy, r2), 1, p) / (r * r)
                        if m.hasZ:
                            f += d(scaled(tyz, s_), 2, p) / (r * math.sin(th))
                        f += d(txy, 0, p) / (r * math.sin(th))
                        f -= (tzz(*p) + txx(*p)) / r
                    out["vy"][k, j, i] = st["vy"][k, j, i] - dt * f / rho(*p)
    # v_z (v_theta) on the interior faces
    if m.hasZ:
        for k in range(m.k0 + 1, m.k1):
            for j in range(m.j0, m.j1):
                for i in range(m.nx):
                    p = (2 * i + 1, 2 * j + 1, 2 * k)
                    r = m.y(p[1])
                    f = 0.0
                    if g == CART:
                        f += d(txz, 0, p) + d(tzz, 2, p)
                        if m.hasY:
                            f += d(tyz, 1, p)
                    elif g == CYL:
                        if m.hasY:
                            f += d(scaled(tyz, r_), 1, p) / r
                        f += d(txz, 0, p) / r + d(tzz, 2, p)
                    else:
                        th = m.z(p[2])
                        if m.hasY:
                            f += d(scaled(tyz, r3), 1, p) / r ** 3
                        f += d(scaled(tzz, s_), 2, p) / (r * math.sin(th))
                        f += d(txz, 0, p) / (r * math.sin(th))
                        f -= txx(*p) * (math.cos(th) / math.sin(th)) / r
                    out["vz"][k, j, i] = st["vz"][k, j, i] - dt * f / rho(*p)
    return out


def _pad_ring(w, st):
    a = np.zeros_like(st["rho"])
    nu = np.asarray(w.nu)
    a[:nu.shape[0], :nu.shape[1], :] = nu[:, :, None]
    return a


# ---------------------------------------------------------------------------
# Transport (cells 12a-d): left/right momenta (Eqs. 16-17, Tab. momenta),
# upwind sweeps with van Leer interface values (Eqs. 14-15) and consistent
# transport, the orbital shift (Eqs. 28-37, PPA), the new velocities (Eq. 18).
# ---------------------------------------------------------------------------
def frame_term(m, w, y2, z2):
    """Frame share of the X momentum per unit mass (Tab. momenta)."""
    if w.geom == CART:
        return 2.0 * w.omega_f * m.y(y2) if w.shearing else 0.0
    return m.R(y2, z2) ** 2 * w.omega_f


def momenta(w, st):
    m = Mesh(w)
    shp = st["rho"].shape
    pm = {n: np.zeros(shp) for n in ("xm", "xp", "ym", "yp", "zm", "zp")}
    for k in range(m.nzt):
        for j in range(m.nyt):
            y2, z2 = 2 * j + 1, 2 * k + 1
            R, wf = m.R(y2, z2), frame_term(m, w, y2, z2)
            zfac = m.y(y2) if w.geom == SPH else 1.0
            for i in range(m.nx):
                r = st["rho"][k, j, i]
                pm["xm"][k, j, i] = r * (R * st["vx"][k, j, i] + wf)
                pm["xp"][k, j, i] = r * (R * st["vx"][k, j, (i + 1) % m.nx] + wf)
                if m.hasY:
                    pm["ym"][k, j, i] = r * st["vy"][k, j, i]
                    pm["yp"][k, j, i] = r * st["vy"][k, j + 1, i]
                if m.hasZ:
                    pm["zm"][k, j, i] = r * zfac * st["vz"][k, j, i]
                    pm["zp"][k, j, i] = r * zfac * st["vz"][k + 1, j, i]
    return pm


def quantities(w):
    m_y, m_z = w.ny > 1, w.nz > 1
    out = ["rho"] + ([] if w.iso else ["e"]) + ["xm", "xp"]
    if m_y:
        out += ["ym", "yp"]
    if m_z:
        out += ["zm", "zp"]
    return out


def _vanleer(qm, q0, qp, hm, hp):
    a, b = (q0 - qm) / hm, (qp - q0) / hp
    if a * b <= 0.0:
        return 0.0
    return 2.0 * a * b / (a + b)


def sweep_1d(Q, cen, wid, vel, area, vol, first, last, dt):
    """One conservative upwind sweep over cells first..last-1 of a line.
    Q: list of arrays (density first); face f sits between cells f-1, f."""
    def star(a, f, v):
        if v >= 0.0:
            c = f - 1
            s = _vanleer(a[c - 1], a[c], a[c + 1], cen[c] - cen[c - 1], cen[c + 1] - cen[c])
            return a[c] + 0.5 * s * (wid[c] - v * dt)
        c = f
        s = _vanleer(a[c - 1], a[c], a[c + 1], cen[c] - cen[c - 1], cen[c + 1] - cen[c])
        return a[c] - 0.5 * s * (wid[c] + v * dt)
    ratios = [Q[0]] + [Q[n] / Q[0] for n in range(1, len(Q))]
    flux = np.zeros((len(Q), len(vel)))
    for f in range(first, last + 1):
        mass = vel[f] * star(ratios[0], f, vel[f]) * area[f]
        flux[0, f] = mass
        for n in range(1, len(Q)):
            flux[n, f] = mass * star(ratios[n], f, vel[f])
    new = [a.copy() for a in Q]
    for n in range(len(Q)):
        for c in range(first, last):
            new[n][c] = Q[n][c] - dt * (flux[n, c + 1] - flux[n, c]) / vol[c]
    return new


def transport_x(w, st, pm, v0, dt):
    m = Mesh(w)
    names = quantities(w)
    arr = {**{"rho": st["rho"], "e": st["e"]}, **pm}
    out = {n: arr[n].copy() for n in names}
    if not m.hasX:
        return out
    nx = m.nx
    for k in range(m.k0, m.k1):
        for j in range(m.j0, m.j1):
            dX = m.R(2 * j + 1, 2 * k + 1) * m.dx
            base = v0[k, j] if w.fargo else 0.0
            # the periodic ring with two images on each side
            idx = [(c - 2) % nx for c in range(nx + 4)]
            Q = [np.array([arr[n][k, j, i] for i in idx]) for n in names]
            vel = np.array([st["vx"][k, j, i] - base for i in idx])
            res = sweep_1d(Q, np.arange(nx + 4) * dX, np.full(nx + 4, dX), vel, np.full(nx + 4, m.area(0, j, k)),
                           np.full(nx + 4, m.volume(j, k)), 2, nx + 2, dt)
            for n, a in zip(names, res):
                out[n][k, j, :] = a[2:nx + 2]
    return out


def transport_y(w, st, q, dt):
    m = Mesh(w)
    names = quantities(w)
    out = {n: q[n].copy() for n in names}
    if not m.hasY:
        return out
    cen = np.array([m.y(2 * j + 1) for j in range(m.nyt)])
    wid = np.array([m.yf[j + 1] - m.yf[j] for j in range(m.nyt)])
    for k in range(m.k0, m.k1):
        area = np.array([m.area(1, j, k) for j in range(m.nyt)] + [0.0])
        vol = np.array([m.volume(j, k) for j in range(m.nyt)])
        for i in range(m.nx):
            Q = [q[n][k, :m.nyt, i].copy() for n in names]
            res = sweep_1d(Q, cen, wid, st["vy"][k, :m.nyt + 1, i], area, vol, m.j0, m.j1, dt)
            for n, a in zip(names, res):
                out[n][k, m.j0:m.j1, i] = a[m.j0:m.j1]
    return out


def transport_z(w, st, q, dt):
    m = Mesh(w)
    names = quantities(w)
    out = {n: q[n].copy() for n in names}
    if not m.hasZ:
        return out
    for j in range(m.j0, m.j1):
        f = m.y(2 * j + 1) if w.geom == SPH else 1.0
        cen = np.array([f * m.z(2 * k + 1) for k in range(m.nzt)])
        wid = np.array([f * (m.zf[k + 1] - m.zf[k]) for k in range(m.nzt)])
        area = np.array([m.area(2, j, k) for k in range(m.nzt)] + [0.0])
        vol = np.array([m.volume(j, k) for k in range(m.nzt)])
        for i in range(m.nx):
            Q = [q[n][:m.nzt, j, i].copy() for n in names]
            res = sweep_1d(Q, cen, wid, st["vz"][:m.nzt + 1, j, i], area, vol, m.k0, m.k1, dt)
            for n, a in zip(names, res):
                out[n][m.k0:m.k1, j, i] = a[m.k0:m.k1]
    return out


def ppa_interface(q, xi):
    """Interface values Q*_{i+1/2} of a periodic ring for the uniform
    fractional Courant number xi (Eqs. 34-36 and the PPA interface value):
    returns a list whose entry i is the value on the face between cells
    i and i+1."""
    n = len(q)
    Q = lambda i: q[i % n]                                       # noqa: E731
    dm = []
    for i in range(n):
        a, b = Q(i) - Q(i - 1), Q(i + 1) - Q(i)
        if a * b <= 0.0:
            dm.append(0.0)
        else:
            dq = 0.5 * (Q(i + 1) - Q(i - 1))
            dm.append(math.copysign(min(2.0 * abs(a), 2.0 * abs(b), abs(dq)), dq))
    DM = lambda i: dm[i % n]                                     # noqa: E731
    QR = [Q(i) + 0.5 * (Q(i + 1) - Q(i)) - (DM(i + 1) - DM(i)) / 6.0 for i in range(n)]
    L, R = [], []
    for i in range(n):
        ql, qr = QR[(i - 1) % n], QR[i]
        if (Q(i + 1) - Q(i)) * (Q(i) - Q(i - 1)) <= 0.0:
            ql = qr = Q(i)
        else:
            D, Cc = qr - ql, Q(i) - 0.5 * (ql + qr)
            if D * Cc > D * D / 6.0:
                ql = 3.0 * Q(i) - 2.0 * qr
            elif -D * D / 6.0 > D * Cc:
                qr = 3.0 * Q(i) - 2.0 * ql
        L.append(ql)
        R.append(qr)
    out = []
    for i in range(n):
        if xi >= 0.0:
            x = xi
            out.append(R[i] + x * (Q(i) - R[i]) + x * (1.0 - x) * (2.0 * Q(i) - R[i] - L[i]))
        else:
            x, c = -xi, (i + 1) % n
            out.append(L[c] + x * (Q(c) - L[c]) + x * (1.0 - x) * (2.0 * Q(c) - R[c] - L[c]))
    return out


def nearest_integer(x):
    """E(X): the nearest integer, halves away from zero."""
    f = math.floor(abs(x) + 0.5)
    return int(math.copysign(f, x))


def orbital_shift(w, q, v0, dt):
    m = Mesh(w)
    names = quantities(w)
    out = {n: q[n].copy() for n in names}
    if not (m.hasX and w.fargo):
        return out
    nx = m.nx
    for k in range(m.k0, m.k1):
        for j in range(m.j0, m.j1):
            dX = m.R(2 * j + 1, 2 * k + 1) * m.dx
            X = v0[k, j] * dt / dX
            N = nearest_integer(X)
            xi = X - N
            rings = {n: np.array([q[n][k, j, (i - N) % nx] for i in range(nx)]) for n in names}
            if xi != 0.0:
                S, V = m.area(0, j, k), m.volume(j, k)
                vR = xi * dX / dt
                rs = ppa_interface(list(rings["rho"]), xi)
                mass = [vR * s * S for s in rs]           # flux through the face after cell i
                new = {}
                for n in names:
                    if n == "rho":
                        fl = mass
                    else:
                        rr = ppa_interface(list(rings[n] / rings["rho"]), xi)
                        fl = [a * b for a, b in zip(mass, rr)]
                    new[n] = np.array([rings[n][i] - dt * (fl[i] - fl[(i - 1) % nx]) / V for i in range(nx)])
                rings = new
            for n in names:
                out[n][k, j, :] = rings[n]
    return out


def new_velocities(w, st, q):
    """Eq. 18 with the factors of Tab. momenta undone; interior faces."""
    m = Mesh(w)
    out = {k: v.copy() for k, v in st.items()}
    rho = q["rho"]
    for k in range(m.k0, m.k1):
        for j in range(m.j0, m.j1):
            y2, z2 = 2 * j + 1, 2 * k + 1
            R, wf = m.R(y2, z2), frame_term(m, w, y2, z2)
            for i in range(m.nx):
                im = (i - 1) % m.nx
                mom = (q["xp"][k, j, im] + q["xm"][k, j, i]) / (rho[k, j, im] + rho[k, j, i])
                out["vx"][k, j, i] = (mom - wf) / R
                if m.hasY and j > m.j0:
                    out["vy"][k, j, i] = (q["yp"][k, j - 1, i] + q["ym"][k, j, i]) / (rho[k, j - 1, i] + rho[k, j, i])
                if m.hasZ and k > m.k0:
                    f = m.y(y2) if w.geom == SPH else 1.0
                    out["vz"][k, j, i] = (q["zp"][k - 1, j, i] + q["zm"][k, j, i]) / (rho[k - 1, j, i] + rho[k, j, i]) / f
    out["rho"] = q["rho"].copy()
    if not w.iso:
        out["e"] = q["e"].copy()
    return out


# ---------------------------------------------------------------------------
# Cells 3 and 6: bulk azimuthal velocity (Eq. 37) and the Courant step
# (Eq. cfl2 with the FARGO amendments and the shear limit, Eq. 38).
# ---------------------------------------------------------------------------
def v0_of(w, st):
    m = Mesh(w)
    v0 = np.zeros((m.nzt, m.nyt))
    if w.fargo:
        for k in range(m.k0, m.k1):
            for j in range(m.j0, m.j1):
                row = st["vx"][k, j, :]
                v0[k, j] = 0.5 * (max(row) + min(row))
    return v0


def courant(w, st, v0):
    m = Mesh(w)
    best = math.inf
    names = ["vx", "vy", "vz"]
    active = [m.hasX, m.hasY, m.hasZ]
    for k in range(m.k0, m.k1):
        for j in range(m.j0, m.j1):
            widths = [_cell_width(m, ax, j, k) for ax in range(3)]
            dmin = min(widths[ax] for ax in range(3) if active[ax])
            nu = w.nu[k, j] if w.nu is not None else 0.0
            for i in range(m.nx):
                rho = st["rho"][k, j, i]
                cs = w.cs[k, j] if w.iso else math.sqrt(w.gamma * (w.gamma - 1.0) * st["e"][k, j, i] / rho)
                terms = [dmin / cs if cs > 0 else math.inf]
                up = [(k, j, (i + 1) % m.nx), (k, j + 1, i), (k + 1, j, i)]
                t2, t3 = math.inf, math.inf
                for ax in range(3):
                    if not active[ax]:
                        continue
                    base = v0[k, j] if (ax == 0 and w.fargo) else 0.0
                    lo, hi = st[names[ax]][k, j, i] - base, st[names[ax]][up[ax]] - base
                    vmax = max(abs(lo), abs(hi))
                    if vmax > 0:
                        t2 = min(t2, widths[ax] / vmax)
                    dv = hi - lo
                    if w.cq > 0 and dv < 0:
                        t3 = min(t3, widths[ax] / (4.0 * w.cq * w.cq * -dv))
                terms += [t2, t3]
                if nu > 0:
                    terms.append(dmin * dmin / (4.0 * nu))
                s = sum(1.0 / (t * t) for t in terms if math.isfinite(t))
                best = min(best, 1.0 / math.sqrt(s))
    dt = w.cfl * best
    if w.fargo and m.hasY:
        for k in range(m.k0, m.k1):
            for j in range(m.j0, m.j1 - 1):
                a = v0[k, j] / (m.R(2 * j + 1, 2 * k + 1) * m.dx)
                b = v0[k, j + 1] / (m.R(2 * j + 3, 2 * k + 1) * m.dx)
                if a != b:
                    dt = min(dt, w.cfl / abs(a - b))
    return dt
