"""Plain FP64 oracle of the planetary integrator (Sec. 3.7, orbital
integrator for planets): one fixed step of the fifth-order Cash-Karp
Runge-Kutta method, with the Butcher tableau of Tab. rk, applied to the
positions and velocities of N point masses orbiting a central star.

TEST INFRASTRUCTURE ONLY (tests and the package smoke check); the product
path never imports it, and it shares no code with the CUDA library.

Readings (the paper writes the system only formally, dy/dt = f(t, y)):
- The frame is centred on the star (the mesh's origin), so each planet
  feels, besides the star's and the other planets' pull, the indirect
  acceleration of that frame: minus the star's acceleration by the planets,
      d2r_i/dt2 = -G (M + m_i) r_i/|r_i|^3
                  + sum_{j != i} G m_j [(r_j - r_i)/|r_j - r_i|^3 - r_j/|r_j|^3],
  G = 1, no softening between planets.  indirect=False drops the frame
  terms (the star then held fixed in an inertial frame):
      d2r_i/dt2 = -G M r_i/|r_i|^3 + sum_{j != i} G m_j (r_j - r_i)/|r_j - r_i|^3.
- The gas force, evaluated once per hydrodynamical step, updates the
  velocities: v_i += h * kick_i before the Runge-Kutta stages (kick = the
  gas acceleration of planet i, less the star's when the frame is the
  star's; the caller composes it).
"""
from __future__ import annotations

from fractions import Fraction as Fr

import numpy as np

# Tab. rk: nodes c_i, stage matrix a_ij (lower triangle), fifth-order weights b_i.
C_NODES = [Fr(0), Fr(1, 5), Fr(3, 10), Fr(3, 5), Fr(1), Fr(7, 8)]
A_STAGE = [
    [],
    [Fr(1, 5)],
    [Fr(3, 40), Fr(9, 40)],
    [Fr(3, 10), Fr(-9, 10), Fr(6, 5)],
    [Fr(-11, 54), Fr(5, 2), Fr(-70, 27), Fr(35, 27)],
    [Fr(1631, 55296), Fr(175, 512), Fr(575, 13824), Fr(44275, 110592), Fr(253, 4096)],
]
B_WEIGHT = [Fr(37, 378), Fr(0), Fr(250, 621), Fr(125, 594), Fr(0), Fr(512, 1771)]


def rk_step(f, t, y, h):
    """y(t + h) by one Cash-Karp step: k_i = f(t + c_i h, y + h sum_j a_ij k_j),
    y_new = y + h sum_i b_i k_i."""
    y = np.asarray(y, dtype=np.float64)
    k = []
    for i in range(6):
        yi = y.copy()
        for j, a in enumerate(A_STAGE[i]):
            yi = yi + h * float(a) * k[j]
        k.append(np.asarray(f(t + float(C_NODES[i]) * h, yi), dtype=np.float64))
    out = y.copy()
    for i in range(6):
        out = out + h * float(B_WEIGHT[i]) * k[i]
    return out


def nbody_rhs(y, mass, mstar, indirect=True):
    """dy/dt for y of shape (N, 6) = (x, y, z, vx, vy, vz) per planet."""
    y = np.asarray(y, dtype=np.float64).reshape(-1, 6)
    n = y.shape[0]
    r = y[:, :3]
    acc = np.zeros((n, 3))
    for i in range(n):
        d = np.linalg.norm(r[i])
        gm = mstar + (mass[i] if indirect else 0.0)
        acc[i] -= gm * r[i] / d ** 3
        for j in range(n):
            if j == i:
                continue
            dij = r[j] - r[i]
            acc[i] += mass[j] * dij / np.linalg.norm(dij) ** 3
            if indirect:
                acc[i] -= mass[j] * r[j] / np.linalg.norm(r[j]) ** 3
    return np.concatenate([y[:, 3:], acc], axis=1)


def nbody_step(y, mass, mstar, h, kick=None, indirect=True):
    """One planetary step: the gas kick on the velocities, then one
    Cash-Karp step of length h.  y is (N, 6); returns the new (N, 6)."""
    y = np.array(y, dtype=np.float64).reshape(-1, 6)
    if kick is not None:
        y[:, 3:] += h * np.asarray(kick, dtype=np.float64).reshape(-1, 3)
    mass = np.asarray(mass, dtype=np.float64)
    return rk_step(lambda t, z: nbody_rhs(z, mass, mstar, indirect), 0.0, y, h)
