"""Pins of the oracle's gravity source (eq. gravity_term, Sec. 2.4) and
gravity timestep (Sec. 2.5), each against something the oracle does not
compute itself:

* a uniform state in a linear acceleration field: the flux terms vanish and
  dW/dt is the projection of s = (0, rho a, m . a), known in closed form
  (mean and the two/three linear moments, nothing else);
* a smooth rotating equilibrium in a central Plummer field (centrifugal
  force balanced by gravity, uniform pressure): the cell-mean residual
  vanishes at second order or better with the mesh, while dropping the
  source leaves an O(1) residual -- a wrong sign or factor does not converge;
* angular momentum (Sec. 2.6): with a central field the discrete total
  L = sum_K int_K (x' m_y - y' m_x) dV of a state at rest near the periodic
  boundary has dL/dt = 0 to rounding, on uniform and two-level meshes;
* the timestep is the smaller of the hydro bound and
  c / (sqrt(2 gamma (gamma - 1)) |a|) (closed form on a uniform state).
"""
import numpy as np
import pytest

from oracle import pyoracle as O
from paper_1506_06140_gb300 import workloads as wl

GAMMA = 5.0 / 3.0
EPS = 0.3
S3 = np.sqrt(3.0)


def plummer(xyz, center=3.0):
    x, y = xyz[0] - center, xyz[1] - center
    g = 1.0 / (x * x + y * y + EPS * EPS) ** 1.5
    return np.stack([-x * g, -y * g])


def cell_centres(o):
    return np.array([o.quad_points()[a].mean(axis=0) for a in range(o.dim)])


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_uniform_state_in_linear_field(dim, k):
    n = [5, 4, 3][:dim]
    hi = [n[a] * 0.25 for a in range(dim)]
    o = O.Oracle(dim, n, [0.0] * dim, hi, k, GAMMA)
    xyz = o.quad_points()
    rho0, p0 = 1.3, 0.9
    v0 = np.array([0.4, -0.7, 0.2][:dim])
    g0 = np.array([0.5, -1.5, 0.8][:dim])
    alpha = np.array([2.0, -0.6, 1.1][:dim])
    x0 = 0.3
    accel = np.stack([g0[a] + alpha[a] * (xyz[a] - x0) for a in range(dim)])
    o.set_accel(accel)
    U = wl.conserved(np.full(xyz[0].shape, rho0), [np.full(xyz[0].shape, v) for v in v0],
                     np.full(xyz[0].shape, p0), GAMMA)
    W = o.project(U)
    d = o.rhs(W)
    xc, dx = cell_centres(o), 0.25
    expect = np.zeros_like(d)
    for a in range(dim):
        mean = rho0 * (g0[a] + alpha[a] * (xc[a] - x0))       # rho a_a at the centre
        slope = rho0 * alpha[a] * (dx / 2) / S3                # its linear moment along a
        expect[1 + a, 0] = mean
        expect[1 + a, 1 + a] = slope
        expect[-1, 0] += v0[a] * mean                          # m . a
        expect[-1, 1 + a] = v0[a] * slope
    np.testing.assert_allclose(d, expect, rtol=0, atol=1e-12 * np.abs(expect).max())


def equilibrium(xyz):
    """rotation v_phi = r / (r^2 + eps^2)^(3/4) balancing the Plummer field,
    rho(r) smooth, p uniform: a steady state of the Euler equations"""
    x, y = xyz[0] - 3.0, xyz[1] - 3.0
    r2 = x * x + y * y
    w = 1.0 / (r2 + EPS * EPS) ** 0.75
    rho = 1.0 + 0.4 * np.cos(np.sqrt(r2))
    return wl.conserved(rho, [-y * w, x * w], np.ones_like(rho), GAMMA)


@pytest.mark.parametrize("k,min_ratio", [(1, 3.0), (2, 4.5)])
def test_rotating_equilibrium_residual_converges(k, min_ratio):
    res, res_nograv = [], []
    for n in (24, 48):
        o = O.Oracle(2, [n, n], [0.0, 0.0], [6.0, 6.0], k, GAMMA)
        xyz = o.quad_points()
        W = o.project(equilibrium(xyz))
        xc = cell_centres(o) - 3.0
        ring = (np.hypot(xc[0], xc[1]) > 0.9) & (np.hypot(xc[0], xc[1]) < 1.5)
        o.set_accel(plummer(xyz))
        res.append(np.abs(o.rhs(W)[:, 0, ring]).max())
        o.set_accel(None)
        res_nograv.append(np.abs(o.rhs(W)[:, 0, ring]).max())
    assert res[0] / res[1] > min_ratio, res
    assert min(res_nograv) > 0.5 and res_nograv[0] / res_nograv[1] < 1.5  # the source is what balances


def bump(r, r1):
    """C-infinity bump: 1 at r = 0, 0 for r >= r1"""
    t = np.clip(r / r1, 0.0, 1.0 - 1e-12)
    return np.where(r < r1, np.exp(1.0 - 1.0 / (1.0 - t * t)), 0.0)


def angular_momentum_rate(o, d):
    """d/dt sum_K int_K (x' m_y - y' m_x) dV from dW/dt: on a cell with
    centre c and edge dx, int_K x' m_y = |K| (x'_c w_0 + (dx/2) w_x / sqrt(3))"""
    xc = cell_centres(o) - 3.0
    dx = o.cell_dx()
    vol = dx ** 2
    h = dx / 2 / S3
    terms = [vol * xc[0] * d[2, 0], vol * h * d[2, 1], -vol * xc[1] * d[1, 0], -vol * h * d[1, 2]]
    return sum(t.sum() for t in terms), sum(np.abs(t).sum() for t in terms)


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("amr", [False, True], ids=["uniform", "two-level"])
def test_central_field_conserves_angular_momentum(k, amr):
    n = 16
    boxes = [[5, 5, 10, 10]] if amr else []
    o = O.Oracle(2, [n, n], [0.0, 0.0], [6.0, 6.0], k, GAMMA, refine_boxes=boxes)
    xyz = o.quad_points()
    x, y = xyz[0] - 3.0, xyz[1] - 3.0
    r = np.hypot(x, y)
    rho = 1.0 + 0.8 * bump(r, 2.0)
    w = 0.9 * bump(r, 2.2) / (r * r + EPS * EPS) ** 0.75
    U = wl.conserved(rho, [-y * w + 0.3 * bump(r, 1.5), x * w], np.ones_like(r), GAMMA)
    W = o.project(U)
    # generic higher moments inside, the state at rest and uniform near the boundary
    rng = np.random.default_rng(4)
    xc = cell_centres(o) - 3.0
    inner = np.hypot(xc[0], xc[1]) < 1.8
    W[:, 1:, inner] += 0.02 * rng.uniform(-1, 1, W[:, 1:, inner].shape)
    o.set_accel(plummer(xyz))
    rate, scale = angular_momentum_rate(o, o.rhs(W))
    assert scale > 1.0
    assert abs(rate) < 1e-13 * scale, (rate, scale)
    # a field with a tangential part exerts a torque the check sees
    swirl = 0.2 * np.stack([-y, x]) / (r * r + EPS * EPS) ** 1.5
    o.set_accel(plummer(xyz) + swirl)
    rate2, _ = angular_momentum_rate(o, o.rhs(W))
    assert abs(rate2) > 1e-2 * scale


def test_timestep_takes_the_gravity_bound():
    n, k, dx = 8, 2, 0.125
    o = O.Oracle(2, [n, n], [0.0, 0.0], [1.0, 1.0], k, GAMMA)
    xyz = o.quad_points()
    U = wl.conserved(np.ones(xyz[0].shape), [np.zeros(xyz[0].shape)] * 2, np.ones(xyz[0].shape), GAMMA)
    W = o.project(U)
    cs = np.sqrt(GAMMA)
    hydro = 0.2 / (2 * k + 1) / (2 * cs / dx)
    assert o.compute_dt(W) == pytest.approx(hydro, rel=1e-14)
    for g, expect_grav in ((5.0, False), (500.0, True)):
        a = np.stack([np.full(xyz[0].shape, g), np.zeros(xyz[0].shape)])
        a[0, 3, 5] *= 1.5  # one point of one cell: the largest |a| over the points decides
        o.set_accel(a)
        grav = cs / (np.sqrt(2 * GAMMA * (GAMMA - 1)) * 1.5 * g)
        assert o.compute_dt(W) == pytest.approx(min(hydro, grav), rel=1e-14)
        assert (grav < hydro) == expect_grav


@pytest.mark.parametrize("rk", [2, 3, 4])
def test_rk_step_with_constant_field_is_exact(rk):
    """A uniform state in a constant field: no flux divergence, so
    m(dt) = m0 + rho g dt and E(dt) = E0 + rho (v0 . g) dt + rho |g|^2 dt^2 / 2
    (SSP-RK of order >= 2 integrates these polynomials in t exactly)."""
    n, k = 6, 2
    o = O.Oracle(2, [n, n], [0.0, 0.0], [1.0, 1.0], k, GAMMA, rk_order=rk)
    xyz = o.quad_points()
    rho0, p0, v0, g = 1.3, 0.8, np.array([0.3, -0.2]), np.array([0.7, -1.1])
    o.set_accel(np.stack([np.full(xyz[0].shape, g[0]), np.full(xyz[0].shape, g[1])]))
    W = o.project(wl.conserved(np.full(xyz[0].shape, rho0), [np.full(xyz[0].shape, v) for v in v0],
                               np.full(xyz[0].shape, p0), GAMMA))
    dt = 0.01
    W1, _ = o.rk_step(W, dt)
    dm = rho0 * g * dt
    dE = rho0 * (v0 @ g) * dt + 0.5 * rho0 * (g @ g) * dt ** 2
    # the increments; RK4 uses the tableau's printed digits, whose weights sum
    # to 1 only to ~1e-10
    rtol = 1e-11 if rk < 4 else 2e-10
    np.testing.assert_allclose(W1[1, 0] - W[1, 0], dm[0], rtol=rtol)
    np.testing.assert_allclose(W1[2, 0] - W[2, 0], dm[1], rtol=rtol)
    np.testing.assert_allclose(W1[-1, 0] - W[-1, 0], dE, rtol=rtol)
    np.testing.assert_allclose(W1[0], W[0], atol=1e-14)
    np.testing.assert_allclose(W1[:, 1:], 0.0, atol=1e-13)  # still uniform
