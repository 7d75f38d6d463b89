"""Exact solution of the 1D Riemann problem for a gamma-law gas.

Independent of the oracle: the classical construction (pressure function of
a shock or a rarefaction on each side, Newton iteration for the star
pressure, self-similar sampling in x/t) as given in standard textbooks on
Riemann solvers.  Used to pin the whole oracle step on the Sod tube.
"""
import math

import numpy as np


def _f(p, rho, pk, gamma):
    a = math.sqrt(gamma * pk / rho)
    if p > pk:  # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        return (p - pk) * math.sqrt(A / (p + B)), math.sqrt(A / (B + p)) * (1.0 - 0.5 * (p - pk) / (B + p))
    # rarefaction
    e = (gamma - 1.0) / (2.0 * gamma)
    return 2.0 * a / (gamma - 1.0) * ((p / pk) ** e - 1.0), (1.0 / (rho * a)) * (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma))


def star_state(rl, ul, pl, rr, ur, pr, gamma=1.4):
    p = 0.5 * (pl + pr)
    for _ in range(100):
        fl, dl = _f(p, rl, pl, gamma)
        fr, dr = _f(p, rr, pr, gamma)
        dp = (fl + fr + ur - ul) / (dl + dr)
        p = max(p - dp, 1e-12)
        if abs(dp) < 1e-15 * p:
            break
    fl, _ = _f(p, rl, pl, gamma)
    fr, _ = _f(p, rr, pr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(x, t, x0, left, right, gamma=1.4):
    """Density, velocity, pressure at positions x (array) and time t."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(rl, ul, pl, rr, ur, pr, gamma)
    al, ar = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    out = np.zeros((3, len(x)))
    for n, xi in enumerate((np.asarray(x) - x0) / t):
        if xi <= us:  # left of contact
            if ps > pl:
                rs = rl * (ps / pl + g1) / (g1 * ps / pl + 1.0)
                sl = ul - al * math.sqrt((gamma + 1) / (2 * gamma) * ps / pl + (gamma - 1) / (2 * gamma))
                val = (rl, ul, pl) if xi < sl else (rs, us, ps)
            else:
                rs = rl * (ps / pl) ** (1.0 / gamma)
                als = al * (ps / pl) ** ((gamma - 1) / (2 * gamma))
                shl, stl = ul - al, us - als
                if xi < shl:
                    val = (rl, ul, pl)
                elif xi > stl:
                    val = (rs, us, ps)
                else:
                    u = 2.0 / (gamma + 1) * (al + (gamma - 1) / 2 * ul + xi)
                    c = 2.0 / (gamma + 1) * (al + (gamma - 1) / 2 * (ul - xi))
                    r = rl * (c / al) ** (2.0 / (gamma - 1))
                    val = (r, u, pl * (c / al) ** (2 * gamma / (gamma - 1)))
        else:
            if ps > pr:
                rs = rr * (ps / pr + g1) / (g1 * ps / pr + 1.0)
                sr = ur + ar * math.sqrt((gamma + 1) / (2 * gamma) * ps / pr + (gamma - 1) / (2 * gamma))
                val = (rr, ur, pr) if xi > sr else (rs, us, ps)
            else:
                rs = rr * (ps / pr) ** (1.0 / gamma)
                ars = ar * (ps / pr) ** ((gamma - 1) / (2 * gamma))
                shr, str_ = ur + ar, us + ars
                if xi > shr:
                    val = (rr, ur, pr)
                elif xi < str_:
                    val = (rs, us, ps)
                else:
                    u = 2.0 / (gamma + 1) * (-ar + (gamma - 1) / 2 * ur + xi)
                    c = 2.0 / (gamma + 1) * (ar - (gamma - 1) / 2 * (ur - xi))
                    r = rr * (c / ar) ** (2.0 / (gamma - 1))
                    val = (r, u, pr * (c / ar) ** (2 * gamma / (gamma - 1)))
        out[:, n] = val
    return out


def shock_speed(rr, ur, pr, ps, gamma=1.4):
    ar = math.sqrt(gamma * pr / rr)
    return ur + ar * math.sqrt((gamma + 1) / (2 * gamma) * ps / pr + (gamma - 1) / (2 * gamma))
