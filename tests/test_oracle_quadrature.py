"""Pins of the oracle's Legendre polynomials, quadrature rules and basis.

Each check compares against something other than the oracle itself: the
polynomials printed in Appendix A, numpy's Gauss-Legendre routine, exactness
of the rules on monomials, closed-form Lobatto weights, and orthonormality
integrated with numpy's rule.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as npoly

import golden_values
from oracle import pyoracle as O

# Appendix A, eq. legendre_polys (tests/golden/legendre_polynomials.txt)
PRINTED = golden_values.legendre_polynomials()


@pytest.mark.parametrize("x", [-1.0, -0.73, -0.2, 0.0, 0.41, 0.999, 1.0])
def test_legendre_matches_printed_polynomials(x):
    P, dP = O.legendre(5, x)
    assert sorted(PRINTED) == list(range(6))
    for n in range(6):
        c = PRINTED[n]
        assert P[n] == pytest.approx(npoly.polyval(x, c), abs=1e-14)
        assert dP[n] == pytest.approx(npoly.polyval(x, npoly.polyder(c)), abs=1e-13)


def test_legendre_ode():
    # Legendre's equation (Appendix A): ((1-x^2) P')' + n(n+1) P = 0, checked by differences
    for n in range(0, 7):
        for x in (-0.6, 0.1, 0.8):
            h = 1e-4
            g = lambda t: (1 - t * t) * O.legendre(n, t)[1][n]
            lhs = (g(x + h) - g(x - h)) / (2 * h) + n * (n + 1) * O.legendre(n, x)[0][n]
            assert abs(lhs) < 1e-4  # O(h^2) difference error


@pytest.mark.parametrize("n", range(1, 10))
def test_gauss_legendre_matches_numpy(n):
    x, w = O.gauss_legendre(n)
    xr, wr = npleg.leggauss(n)
    np.testing.assert_allclose(x, xr, atol=2e-15, rtol=0)
    np.testing.assert_allclose(w, wr, atol=2e-15, rtol=0)
    assert abs(w.sum() - 2.0) < 1e-14


@pytest.mark.parametrize("n", range(1, 9))
def test_gauss_legendre_exact_to_degree_2n_minus_1(n):
    x, w = O.gauss_legendre(n)
    for p in range(0, 2 * n):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(np.dot(w, x ** p) - exact) < 1e-14
    p = 2 * n
    assert abs(np.dot(w, x ** p) - 2.0 / (p + 1)) > 1e-6  # not exact beyond


def test_gauss_legendre_k1_nodes():
    x, w = O.gauss_legendre(2)
    np.testing.assert_allclose(x, [-1 / math.sqrt(3), 1 / math.sqrt(3)], atol=1e-16)
    np.testing.assert_allclose(w, [1.0, 1.0], atol=1e-16)


@pytest.mark.parametrize("n", range(2, 9))
def test_gauss_lobatto(n):
    x, w = O.gauss_lobatto(n)
    assert x[0] == -1.0 and x[-1] == 1.0
    assert np.all(np.diff(x) > 0)
    assert abs(w.sum() - 2.0) < 1e-14
    # closed form 2 / (n (n-1) P_{n-1}(x)^2) at every node, endpoints included
    Pn1 = np.array([npleg.legval(t, [0] * (n - 1) + [1]) for t in x])
    np.testing.assert_allclose(w, 2.0 / (n * (n - 1) * Pn1 ** 2), atol=1e-14, rtol=0)
    # interior nodes are roots of P'_{n-1}
    dcoef = npleg.legder([0] * (n - 1) + [1])
    assert np.all(np.abs(npleg.legval(x[1:-1], dcoef)) < 1e-12)
    for p in range(0, 2 * n - 2):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(np.dot(w, x ** p) - exact) < 1e-14


def test_lobatto_small_rules():
    x, w = O.gauss_lobatto(2)
    np.testing.assert_allclose(w, [1, 1])
    x, w = O.gauss_lobatto(3)
    np.testing.assert_allclose(x, [-1, 0, 1], atol=1e-16)
    np.testing.assert_allclose(w, [1 / 3, 4 / 3, 1 / 3], atol=1e-15)


@pytest.mark.parametrize("k,w1", sorted(golden_values.lobatto_first_weight().items()))
def test_first_lobatto_weight_per_order(k, w1):
    # Sec. 3.4: m = smallest integer >= (k+3)/2; the printed first GLL weight
    # (tests/golden/lobatto_first_weight.txt: 1 for k=1, 1/3 for k=2,3)
    m = math.ceil((k + 3) / 2)
    x, w = O.gauss_lobatto(m)
    assert w[0] == pytest.approx(w1, abs=1e-15)


@pytest.mark.parametrize("dim,k", [(2, 0), (2, 1), (2, 2), (2, 3), (3, 0), (3, 1), (3, 2), (3, 3)])
def test_basis_count_and_order(dim, k):
    e = O.basis_exponents(dim, k)
    N = (k + 1) * (k + 2) * (k + 3) // 6 if dim == 3 else (k + 1) * (k + 2) // 2
    assert len(e) == N  # eq. nof_basis_functions
    assert len({tuple(r) for r in e}) == N
    assert all(r.sum() <= k for r in e)
    assert tuple(e[0]) == (0, 0, 0)
    if k >= 1:
        assert tuple(e[1]) == (1, 0, 0) and tuple(e[2]) == (0, 1, 0)
        if dim == 3:
            assert tuple(e[3]) == (0, 0, 1)
    deg = e.sum(axis=1)
    assert np.all(np.diff(deg) >= 0)


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 3), (3, 2)])
def test_basis_orthonormal(dim, k):
    # 2^-d int phi_i phi_j = delta_ij, integrated with numpy's rule
    xg, wg = npleg.leggauss(k + 2)
    e = O.basis_exponents(dim, k)
    N = len(e)
    pts = np.array(np.meshgrid(*([xg] * dim), indexing="ij")).reshape(dim, -1).T
    wts = np.prod(np.array(np.meshgrid(*([wg] * dim), indexing="ij")).reshape(dim, -1), axis=0)
    Phi = np.array([[O.basis_phi(dim, k, l, p) for p in pts] for l in range(N)])
    G = (Phi * wts) @ Phi.T / 2 ** dim
    np.testing.assert_allclose(G, np.eye(N), atol=1e-13)
    # phi_1 = 1 and the linear functions are sqrt(3) xi_a
    for p in pts[:5]:
        assert O.basis_phi(dim, k, 0, p) == pytest.approx(1.0)
        for a in range(dim):
            assert O.basis_phi(dim, k, 1 + a, p) == pytest.approx(math.sqrt(3) * p[a])


def test_basis_derivative_against_differences():
    rng = np.random.default_rng(3)
    for dim, k in ((2, 3), (3, 2)):
        for l in range(len(O.basis_exponents(dim, k))):
            xi = rng.uniform(-0.9, 0.9, dim)
            for a in range(dim):
                h = 1e-6
                xp, xm = xi.copy(), xi.copy()
                xp[a] += h
                xm[a] -= h
                fd = (O.basis_phi(dim, k, l, xp) - O.basis_phi(dim, k, l, xm)) / (2 * h)
                assert O.basis_dphi(dim, k, l, a, xi) == pytest.approx(fd, abs=1e-6)
