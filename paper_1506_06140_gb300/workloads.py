"""Seeded synthetic inputs: initial conditions and mesh recipes.

This module holds the problem definitions only -- closed-form primitive
fields turned into conserved variables at given points, random coefficient
states, and mesh descriptions.  It contains none of the DG method's
arithmetic, so both the CUDA library's tests and the CPU oracle draw their
inputs from it.

Workloads (shapes after the paper's tests, Sec. 5):
  * ``wave2d``    advected density wave, periodic [0,1]^2
  * ``vortex``    isentropic vortex (Sec. 5.1), periodic [-5,5]^2, boost (1,1)
  * ``sedov3d``   blast wave on a static two-level mesh (Sec. 5.3)
  * ``acoustic3d`` small-amplitude standing sound wave, periodic [0,1]^3
  * ``sod``       shock tube (Sec. 5.2) as a quasi-1D strip
  * ``square2d``  supersonic square advection (Sec. 5.4), periodic [0,1]^2
"""
import math

import numpy as np

BC_PERIODIC, BC_TRANSMISSIVE = 0, 1


def conserved(rho, vel, p, gamma):
    """Conserved state (rho, rho v, rho e) from primitive fields (eq. state_vector)."""
    vel = [np.asarray(v, dtype=np.float64) * np.ones_like(rho) for v in vel]
    kin = 0.5 * rho * sum(v * v for v in vel)
    return np.stack([rho] + [rho * v for v in vel] + [p / (gamma - 1.0) + kin])


# ---- initial conditions at points xyz[axis][...] ---------------------------

def wave2d(xyz, gamma=1.4, amp=0.2, vel=(1.0, 1.0), p=1.0, t=0.0):
    x, y = xyz[0], xyz[1]
    rho = 1.0 + amp * np.sin(2.0 * math.pi * ((x - vel[0] * t) + (y - vel[1] * t)))
    return conserved(rho, vel, p * np.ones_like(rho), gamma)


def vortex_primitive(xyz, gamma=1.4, beta=5.0, center=(0.0, 0.0), boost=(1.0, 1.0), t=0.0,
                     period=10.0):
    """Isentropic vortex (Sec. 5.1): rho, v, p at time t (translated IC)."""
    x = xyz[0] - boost[0] * t - center[0]
    y = xyz[1] - boost[1] * t - center[1]
    if period:
        x = (x + 0.5 * period) % period - 0.5 * period
        y = (y + 0.5 * period) % period - 0.5 * period
    r2 = x * x + y * y
    rho = (1.0 - (gamma - 1.0) * beta ** 2 / (8.0 * gamma * math.pi ** 2) * np.exp(1.0 - r2)) \
        ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    amp = beta / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
    vx = boost[0] - y * amp
    vy = boost[1] + x * amp
    return rho, (vx, vy), p


def vortex(xyz, gamma=1.4, beta=5.0, center=(0.0, 0.0), boost=(1.0, 1.0), t=0.0, period=10.0):
    rho, vel, p = vortex_primitive(xyz, gamma, beta, center, boost, t, period)
    return conserved(rho, vel, p, gamma)


def acoustic3d(xyz, gamma=1.4, amp=1e-3, vel=(0.0, 0.0, 0.0)):
    """rho = 1 + amp sin(2 pi x) sin(2 pi y) sin(2 pi z), uniform velocity vel
    (zero for the standing wave), p = 1/gamma (sound speed 1)."""
    x, y, z = xyz[0], xyz[1], xyz[2]
    rho = 1.0 + amp * np.sin(2 * math.pi * x) * np.sin(2 * math.pi * y) * np.sin(2 * math.pi * z)
    v = [np.full_like(rho, vv) for vv in vel]
    return conserved(rho, v, np.full_like(rho, 1.0 / gamma), gamma)


def square2d(xyz, gamma=1.4, rho_in=4.0, rho_out=1.0, p=2.5, vel=(100.0, 50.0), lo=0.25, hi=0.75,
             t=0.0):
    """Square advection (Sec. 5.4): a square overdensity in pressure equilibrium
    moving supersonically through the periodic unit box; the exact solution is
    the initial state translated by vel * t."""
    x = np.mod(xyz[0] - vel[0] * t, 1.0)
    y = np.mod(xyz[1] - vel[1] * t, 1.0)
    inside = (x > lo) & (x < hi) & (y > lo) & (y < hi)
    rho = np.where(inside, rho_in, rho_out)
    return conserved(rho, vel, np.full_like(rho, p), gamma)


def kelvin_helmholtz(xyz, gamma=1.4, w0=0.1, sigma=0.05 / np.sqrt(2.0)):
    """Kelvin-Helmholtz initial data (Sec. 5.6) on the periodic
    unit box: a dense band 0.25 < y < 0.75 (rho 2, v_x 0.5) in a lighter
    medium (rho 1, v_x -0.5), p = 2.5 everywhere, and a single-mode v_y
    perturbation w0 sin(4 pi x) localised at both interfaces with width sigma."""
    x, y = xyz[0], xyz[1]
    band = (y > 0.25) & (y < 0.75)
    rho = np.where(band, 2.0, 1.0)
    vx = np.where(band, 0.5, -0.5)
    env = np.exp(-(y - 0.25) ** 2 / (2 * sigma ** 2)) + np.exp(-(y - 0.75) ** 2 / (2 * sigma ** 2))
    vy = w0 * np.sin(4 * np.pi * x) * env
    return conserved(rho, [vx, vy], np.full_like(rho, 2.5), gamma)


def keplerian_disc(xyz, gamma=5.0 / 3.0, rho0=1e-5, p0=1e-5, rho_d=1.0, r_in=0.5, r_out=2.0, dr=0.1,
                   center=(3.0, 3.0)):
    """Cold Keplerian disc (Sec. 5.5) in the periodic box [0,6]^2: density
    rho_d between r_in and r_out with linear ramps of width dr to the
    background rho0, uniform pressure p0, Keplerian rotation
    v = (-y', x') / r'^(3/2) for r_in - 2 dr < r' < r_out + 2 dr, at rest
    elsewhere (primed coordinates from the box centre)."""
    x, y = xyz[0] - center[0], xyz[1] - center[1]
    r = np.sqrt(x * x + y * y)
    a0, a1 = r_in - dr / 2, r_in + dr / 2
    b0, b1 = r_out - dr / 2, r_out + dr / 2
    rho = np.full_like(r, rho0)
    ramp_in = (r >= a0) & (r < a1)
    rho = np.where(ramp_in, (rho_d - rho0) / dr * (r - a0) + rho0, rho)
    rho = np.where((r >= a1) & (r < b0), rho_d, rho)
    ramp_out = (r >= b0) & (r < b1)
    rho = np.where(ramp_out, (rho0 - rho_d) / dr * (r - b0) + rho_d, rho)
    rotating = (r > r_in - 2 * dr) & (r < r_out + 2 * dr)
    rs = np.where(rotating, r, 1.0)
    vx = np.where(rotating, -y / rs ** 1.5, 0.0)
    vy = np.where(rotating, x / rs ** 1.5, 0.0)
    return conserved(rho, [vx, vy], np.full_like(r, p0), gamma)


def keplerian_accel(xyz, r_in=0.5, dr=0.1, eps=0.25, center=(3.0, 3.0)):
    """External acceleration a = -grad Phi of the Keplerian disc (Sec. 5.5):
    -x'/r'^3 outside r_in - dr/2, softened to -x'/[r' (r'^2 + eps^2)] inside.
    Returns [2][...] like xyz."""
    x, y = xyz[0] - center[0], xyz[1] - center[1]
    r = np.sqrt(x * x + y * y)
    rs = np.where(r > 0, r, 1.0)
    g = np.where(r > r_in - dr / 2, 1.0 / rs ** 3, 1.0 / (rs * (rs * rs + eps * eps)))
    g = np.where(r > 0, g, 0.0)
    return np.stack([-x * g, -y * g])


def sod(xyz, gamma=1.4, x0=0.5):
    x = xyz[0]
    left = x < x0
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    zero = np.zeros_like(rho)
    return conserved(rho, [zero] * len(xyz), p, gamma)


def sedov3d(xyz, gamma=1.4, p0=1e-5, energy=1.0, half_width=1.0 / 64.0, center=0.5):
    """Blast: uniform rho=1, p=p0, plus `energy` spread uniformly as internal
    energy over the cube |x - center| < half_width (2x2x2 base cells of a 64^3 grid)."""
    x, y, z = xyz[0], xyz[1], xyz[2]
    inside = (np.abs(x - center) < half_width) & (np.abs(y - center) < half_width) & \
             (np.abs(z - center) < half_width)
    vol = (2.0 * half_width) ** 3
    rho = np.ones_like(x)
    p = np.where(inside, (gamma - 1.0) * energy / vol, p0)
    zero = np.zeros_like(rho)
    return conserved(rho, (zero, zero, zero), p, gamma)


# ---- random coefficient states --------------------------------------------

def random_weights(dim, n_basis, n_cells, seed, gamma=1.4, slope=0.05, rho_range=(0.7, 1.3),
                   vel_amp=0.5, p_range=(0.6, 1.4), dtype=np.float64):
    """Random weights W[var][coef][cell]: admissible cell means and small
    higher-order weights (decaying with the coefficient index)."""
    rng = np.random.default_rng(seed)
    nv = dim + 2
    rho = rng.uniform(*rho_range, n_cells)
    vel = [rng.uniform(-vel_amp, vel_amp, n_cells) for _ in range(dim)]
    p = rng.uniform(*p_range, n_cells)
    W = np.zeros((nv, n_basis, n_cells))
    W[:, 0, :] = conserved(rho, vel, p, gamma)
    if n_basis > 1:
        scale = np.abs(W[:, :1, :]) + 0.1
        decay = 1.0 / (1.0 + np.arange(1, n_basis))[None, :, None]
        W[:, 1:, :] = slope * decay * scale * rng.uniform(-1, 1, (nv, n_basis - 1, n_cells))
    return W.astype(dtype)


# ---- mesh recipes ---------------------------------------------------------

def mesh_uniform(dim, n, lo, hi, bc=None):
    return dict(dim=dim, n=list(n), lo=list(lo), hi=list(hi),
                bc=list(bc) if bc is not None else [BC_PERIODIC] * dim, refine_boxes=[])


def mesh_two_level_3d(n_base=64, refine_lo=16, refine_hi=47, lo=0.0, hi=1.0):
    """Static two-level 3D mesh: an n_base^3 base grid with the base-cell box
    [refine_lo, refine_hi]^3 refined once."""
    m = mesh_uniform(3, [n_base] * 3, [lo] * 3, [hi] * 3)
    m["refine_boxes"] = [[refine_lo] * 3 + [refine_hi] * 3]
    return m


def ensemble_problems(n_problems=512, sizes=(32, 48, 64, 96, 128), seed=1506061):
    """Uneven ensemble of vortex problems: (grid size, vortex strength) pairs."""
    rng = np.random.default_rng(seed)
    n = rng.choice(np.array(sizes), size=n_problems)
    beta = rng.uniform(3.0, 6.0, n_problems)
    return [(int(a), float(b)) for a, b in zip(n, beta)]
