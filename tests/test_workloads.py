"""Spot checks of the synthetic inputs against the setups the paper states
(the generators hold no method arithmetic, but a wrong initial state would
change what a workload measures)."""
import numpy as np

from paper_1506_06140_gb300 import workloads as wl


def prim(U, gamma):
    rho = U[0]
    v = U[1:-1] / rho
    p = (gamma - 1.0) * (U[-1] - 0.5 * rho * (v ** 2).sum(axis=0))
    return rho, v, p


def test_kelvin_helmholtz_setup():
    # Sec. 5.6: band 0.25 < y < 0.75 with rho 2, v_x 0.5; rho 1, v_x -0.5
    # outside; p 2.5; v_y = w0 sin(4 pi x) [two Gaussians of width sigma]
    x = np.array([0.1, 0.1, 0.3, 0.6, 0.125])
    y = np.array([0.5, 0.1, 0.25 + 1e-9, 0.9, 0.75])
    rho, v, p = prim(wl.kelvin_helmholtz(np.stack([x, y]), gamma=1.4), 1.4)
    np.testing.assert_allclose(rho, [2.0, 1.0, 2.0, 1.0, 1.0])
    np.testing.assert_allclose(v[0], [0.5, -0.5, 0.5, -0.5, -0.5])
    np.testing.assert_allclose(p, 2.5)
    sigma = 0.05 / np.sqrt(2.0)
    env = np.exp(-(y - 0.25) ** 2 / (2 * sigma ** 2)) + np.exp(-(y - 0.75) ** 2 / (2 * sigma ** 2))
    np.testing.assert_allclose(v[1], 0.1 * np.sin(4 * np.pi * x) * env, atol=1e-15)
    assert abs(v[1][4] - 0.1 * (1.0 + np.exp(-0.25 / (2 * sigma ** 2)))) < 1e-12  # sin(pi/2) at y = 0.75


def test_keplerian_disc_setup():
    # Sec. 5.5: centre (3, 3); rho_D = 1 on [0.5, 2] with 0.1 ramps to 1e-5;
    # p = 1e-5; v = (-y', x') / r'^1.5 on (0.3, 2.2), at rest elsewhere
    g = 5.0 / 3.0
    r = np.array([1.0, 0.5, 2.0, 0.25, 2.5, 0.42])
    x = 3.0 + r
    y = np.full_like(r, 3.0)
    rho, v, p = prim(wl.keplerian_disc(np.stack([x, y]), gamma=g), g)
    np.testing.assert_allclose(rho, [1.0, 0.5 * (1 + 1e-5), 0.5 * (1 + 1e-5), 1e-5, 1e-5, 1e-5], rtol=1e-12)
    np.testing.assert_allclose(p, 1e-5, rtol=1e-9)
    np.testing.assert_allclose(v[0], 0.0, atol=1e-15)
    np.testing.assert_allclose(v[1], [1.0, 0.5 ** -0.5, 2.0 ** -0.5, 0.0, 0.0, 0.42 ** -0.5], rtol=1e-12)
    # acceleration: -x'/r'^3 outside r' = 0.45, -x'/(r'(r'^2 + 0.25^2)) inside
    a = wl.keplerian_accel(np.stack([x, y]))
    inside = r <= 0.45
    expect = np.where(inside, -r / (r * (r * r + 0.0625)), -r / r ** 3)
    np.testing.assert_allclose(a[0], expect, rtol=1e-12)
    np.testing.assert_allclose(a[1], 0.0, atol=1e-15)


def test_sedov_energy_in_the_central_cells():
    # Sec. 5.3: E = 1 as internal energy in the 2^3 central cells of an n^3 grid
    n, g = 16, 5.0 / 3.0
    h = 1.0 / n
    c = (np.arange(n) + 0.5) * h
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    U = wl.sedov3d(np.stack([X.ravel(), Y.ravel(), Z.ravel()]), gamma=g, p0=1e-6, energy=1.0, half_width=h)
    _, _, p = prim(U, g)
    e_int = p / (g - 1.0) * h ** 3
    hot = p > 1.0
    assert hot.sum() == 8
    np.testing.assert_allclose(e_int[hot].sum(), 1.0, rtol=1e-12)
    np.testing.assert_allclose(p[~hot], 1e-6)
