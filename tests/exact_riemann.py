"""Exact solution of the 1D Riemann problem for an ideal gas (textbook
pressure-function method: shock branch from the Rankine-Hugoniot relations,
rarefaction branch from the isentropic relations, Newton iteration for the
star pressure).  Used to pin the oracle on the shock tube (Sec. 5.2)."""
import math

import numpy as np


def _f_side(p, rho, pk, gamma):
    c = math.sqrt(gamma * pk / rho)
    if p > pk:  # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        s = math.sqrt(A / (p + B))
        f = (p - pk) * s
        df = s * (1.0 - 0.5 * (p - pk) / (p + B))
    else:  # rarefaction
        f = 2.0 * c / (gamma - 1.0) * ((p / pk) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)
        df = 1.0 / (rho * c) * (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma))
    return f, df


def star_state(left, right, gamma):
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)
    # two-rarefaction initial guess
    z = (gamma - 1.0) / (2.0 * gamma)
    p = ((cl + cr - 0.5 * (gamma - 1.0) * (ur - ul)) / (cl / pl ** z + cr / pr ** z)) ** (1.0 / z)
    for _ in range(100):
        fl, dfl = _f_side(p, rl, pl, gamma)
        fr, dfr = _f_side(p, rr, pr, gamma)
        step = (fl + fr + ur - ul) / (dfl + dfr)
        p_new = max(p - step, 1e-14)
        if abs(p_new - p) < 1e-15 * p:
            p = p_new
            break
        p = p_new
    fl, _ = _f_side(p, rl, pl, gamma)
    fr, _ = _f_side(p, rr, pr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(xi, left, right, gamma):
    """(rho, u, p) at similarity coordinate xi = (x - x0) / t."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, gamma)
    g = gamma
    if xi <= us:  # left of contact
        cl = math.sqrt(g * pl / rl)
        if ps > pl:  # left shock
            sl = ul - cl * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
            if xi <= sl:
                return rl, ul, pl
            r = rl * (ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1)
            return r, us, ps
        # left rarefaction
        csl = cl * (ps / pl) ** ((g - 1) / (2 * g))
        if xi <= ul - cl:
            return rl, ul, pl
        if xi >= us - csl:
            return rl * (ps / pl) ** (1 / g), us, ps
        u = 2 / (g + 1) * (cl + (g - 1) / 2 * ul + xi)
        c = 2 / (g + 1) * (cl + (g - 1) / 2 * (ul - xi))
        r = rl * (c / cl) ** (2 / (g - 1))
        return r, u, pl * (c / cl) ** (2 * g / (g - 1))
    cr = math.sqrt(g * pr / rr)
    if ps > pr:  # right shock
        sr = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
        if xi >= sr:
            return rr, ur, pr
        r = rr * (ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1)
        return r, us, ps
    csr = cr * (ps / pr) ** ((g - 1) / (2 * g))
    if xi >= ur + cr:
        return rr, ur, pr
    if xi <= us + csr:
        return rr * (ps / pr) ** (1 / g), us, ps
    u = 2 / (g + 1) * (-cr + (g - 1) / 2 * ur + xi)
    c = 2 / (g + 1) * (cr - (g - 1) / 2 * (ur - xi))
    r = rr * (c / cr) ** (2 / (g - 1))
    return r, u, pr * (c / cr) ** (2 * g / (g - 1))


def density_profile(x, t, x0=0.5, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1), gamma=1.4):
    return np.array([sample((xx - x0) / t, left, right, gamma)[0] for xx in np.ravel(x)]).reshape(
        np.shape(x))
