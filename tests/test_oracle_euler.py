"""Pins of the oracle's Euler flux, HLLC flux and eigenvector matrices.

The flux is pinned by properties the mathematics fixes (homogeneity of degree
one, eigenvalues of its Jacobian); HLLC by consistency, upwinding, symmetry
and the exact isolated-contact flux; the Appendix E matrices by L R = I and
by being eigenvectors of the independently formed (dual-number) Jacobian.
"""
import numpy as np
import pytest

from oracle import pyoracle as O
from paper_1506_06140_gb300 import workloads as wl

GAMMA = 1.4


def _states(dim, seed, n=20):
    W = wl.random_weights(dim, 1, n, seed)
    return W[:, 0, :].T


def _prim(dim, u, gamma=GAMMA):
    rho = u[0]
    v = u[1:1 + dim] / rho
    p = (gamma - 1) * (u[dim + 1] - 0.5 * rho * np.dot(v, v))
    return rho, v, p


@pytest.mark.parametrize("dim", [2, 3])
def test_flux_homogeneous_and_eigenvalues(dim):
    for u in _states(dim, 1):
        rho, v, p = _prim(dim, u)
        c = np.sqrt(GAMMA * p / rho)
        for a in range(dim):
            J = O.flux_jacobian(dim, GAMMA, u, a)
            f = O.flux(dim, GAMMA, u, a)
            # Euler flux is homogeneous of degree one in u: A(u) u = f(u)
            np.testing.assert_allclose(J @ u, f, rtol=1e-13, atol=1e-13)
            ev = np.sort(np.linalg.eigvals(J).real)
            ref = np.sort([v[a] - c, v[a] + c] + [v[a]] * dim)
            np.testing.assert_allclose(ev, ref, rtol=1e-9, atol=1e-9)
            # mass flux is the momentum component
            assert f[0] == pytest.approx(u[1 + a], rel=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_eigen_matrices(dim):
    for u in _states(dim, 2):
        rho, v, p = _prim(dim, u)
        c = np.sqrt(GAMMA * p / rho)
        for a in range(dim):
            L, R = O.eigen_matrices(dim, GAMMA, u, a)
            np.testing.assert_allclose(L @ R, np.eye(dim + 2), atol=1e-12)
            J = O.flux_jacobian(dim, GAMMA, u, a)
            lam = np.array([v[a] - c, v[a], v[a] + c] + [v[a]] * (dim - 1))
            np.testing.assert_allclose(J @ R, R * lam[None, :], atol=1e-11)


@pytest.mark.parametrize("dim", [2, 3])
def test_hllc_consistency(dim):
    for u in _states(dim, 3):
        for a in range(dim):
            np.testing.assert_allclose(O.hllc(dim, GAMMA, u, u, a), O.flux(dim, GAMMA, u, a),
                                       rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_hllc_supersonic_upwind(dim):
    for sgn in (1.0, -1.0):
        uL = wl.conserved(np.array(1.0), [sgn * 5.0] + [0.3] * (dim - 1), np.array(1.0), GAMMA)
        uR = wl.conserved(np.array(0.5), [sgn * 4.0] + [-0.2] * (dim - 1), np.array(0.7), GAMMA)
        F = O.hllc(dim, GAMMA, uL, uR, 0)
        ref = O.flux(dim, GAMMA, uL if sgn > 0 else uR, 0)
        np.testing.assert_allclose(F, ref, rtol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_hllc_isolated_contact_is_upwind(dim):
    # equal normal velocity and pressure: HLLC resolves the contact exactly
    for vn in (0.7, -0.4):
        vel = [vn] + [0.25] * (dim - 1)
        velR = [vn] + [-0.6] * (dim - 1)
        uL = wl.conserved(np.array(1.3), vel, np.array(0.9), GAMMA)
        uR = wl.conserved(np.array(0.4), velR, np.array(0.9), GAMMA)
        F = O.hllc(dim, GAMMA, uL, uR, 0)
        ref = O.flux(dim, GAMMA, uL if vn > 0 else uR, 0)
        np.testing.assert_allclose(F, ref, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_hllc_mirror_and_rotation(dim):
    rng = np.random.default_rng(5)
    S = _states(dim, 4)
    for i in range(len(S) - 1):
        uL, uR = S[i], S[i + 1]
        F = O.hllc(dim, GAMMA, uL, uR, 0)
        # mirror x -> -x: swap sides and flip x momentum; flux flips sign except the x momentum
        mL, mR = uR.copy(), uL.copy()
        mL[1] *= -1
        mR[1] *= -1
        Fm = O.hllc(dim, GAMMA, mL, mR, 0)
        flip = -np.ones(dim + 2)
        flip[1] = 1.0
        np.testing.assert_allclose(Fm, flip * F, rtol=1e-12, atol=1e-13)
        # rotation: swapping the x and y axes turns a y-face into an x-face
        perm = list(range(dim + 2))
        perm[1], perm[2] = 2, 1
        Fy = O.hllc(dim, GAMMA, uL[perm], uR[perm], 1)
        np.testing.assert_allclose(Fy[perm], F, rtol=1e-13, atol=1e-14)
    _ = rng


def test_sod_star_state_pin():
    # the exact solver used as a pin reproduces the textbook Sod star state
    from exact_riemann import star_state
    p, u = star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4)
    assert p == pytest.approx(0.30313, abs=1e-5)
    assert u == pytest.approx(0.92745, abs=1e-5)
