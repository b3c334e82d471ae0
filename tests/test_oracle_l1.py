"""Pins of the oracle's L1 density error against closed forms.

Sec. 5.1 defines the error as (1/V) * integral over the domain of
|rho_h - rho_exact| dV; the oracle evaluates it cell by cell with a
(k+3)^d Gauss-Legendre rule (the reading of "accuracy of order p+2").

The integrand is fixed here so that the value is known without the oracle:

* |rho_h - rho_exact| = p(x) with p a positive polynomial of degree 2k+4 in
  one coordinate: the (k+3)-point rule integrates it exactly, a (k+2)-point
  rule would not, so the expected value is (1/V) * integral of p, computed in
  closed form.  It is independent of the mesh, so a uniform and a two-level
  mesh must give the same number (pins the (dx/2)^d cell weight per level);
* |rho_h - rho_exact| = |a sqrt(3) xi| (a pure x slope against the cell mean):
  the value is |a| sqrt(3) G / 2 with G = sum_i w_i |x_i| of the (k+3)-point
  rule (numpy's Gauss-Legendre nodes), which pins that the absolute value is
  taken point by point, and the size of the rule.

rho_h is evaluated here from the weights with numpy's Legendre polynomials
(phi = prod sqrt(2n+1) P_n), independently of the oracle's basis code.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import pyoracle as O


def exponents(dim, k):
    """basis order: total degree, then the x exponent descending, then y descending"""
    out = []
    for g in range(k + 1):
        for a in range(g, -1, -1):
            if dim == 2:
                out.append((a, g - a, 0))
            else:
                for b in range(g - a, -1, -1):
                    out.append((a, b, g - a - b))
    return out


def leg(n, x):
    c = np.zeros(n + 1)
    c[n] = 1.0
    return math.sqrt(2 * n + 1) * npleg.legval(x, c)


def density_at(o, W, xyz):
    """rho_h at physical points xyz[axis][q][cell] from the density weights"""
    dim = o.dim
    dx = o.cell_dx()
    ctr = xyz.mean(axis=1)  # the L1 rule is symmetric: its mean point is the centre
    xi = [(xyz[a] - ctr[a][None, :]) / (0.5 * dx[None, :]) for a in range(dim)]
    rho = np.zeros(xyz.shape[1:])
    for l, e in enumerate(exponents(dim, o.k)):
        term = W[0, l][None, :] * np.ones_like(rho)
        for a in range(dim):
            term = term * leg(e[a], xi[a])
        rho += term
    return rho


def random_weights(o, seed):
    rng = np.random.default_rng(seed)
    W = rng.normal(size=o.shape) * 0.1
    W[0, 0] += 1.0
    return W


def closed_form_2d(k, L):
    """(1/V) * integral over [0,Lx]x[0,Ly] of 1 + x^2/2 + y^(2k+4)/4"""
    Lx, Ly = L
    n = 2 * k + 4
    integral = Lx * Ly + 0.5 * Lx ** 3 / 3.0 * Ly + 0.25 * Lx * Ly ** (n + 1) / (n + 1)
    return integral / (Lx * Ly)


def poly_2d(k, xyz):
    return 1.0 + 0.5 * xyz[0] ** 2 + 0.25 * xyz[1] ** (2 * k + 4)


@pytest.mark.parametrize("k", [0, 1, 2, 3])
@pytest.mark.parametrize("boxes", [(), ([1, 0, 2, 1],)])
@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_l1_positive_polynomial_2d(k, boxes, sign):
    # 4 x 2 cells of edge 0.5 on [0,2] x [0,1]; optionally the middle block refined
    o = O.Oracle(2, [4, 2], [0.0, 0.0], [2.0, 1.0], k, refine_boxes=list(boxes))
    W = random_weights(o, 11 + k)
    xyz = o.l1_points()
    rho_ex = density_at(o, W, xyz) - sign * poly_2d(k, xyz)
    got = o.l1_density(W, rho_ex)
    want = closed_form_2d(k, (2.0, 1.0))
    assert abs(got - want) < 1e-12 * want, (got, want)


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("boxes", [(), ([0, 0, 1, 0, 0, 1],)])
def test_l1_positive_polynomial_3d(k, boxes):
    # 2 x 2 x 2 cells of edge 0.5 on [0,1]^3: p = 1 + x^2 + z^(2k+4)
    o = O.Oracle(3, [2, 2, 2], [0.0] * 3, [1.0] * 3, k, refine_boxes=list(boxes))
    W = random_weights(o, 21 + k)
    xyz = o.l1_points()
    n = 2 * k + 4
    p = 1.0 + xyz[0] ** 2 + xyz[2] ** n
    got = o.l1_density(W, density_at(o, W, xyz) + p)
    want = 1.0 + 1.0 / 3.0 + 1.0 / (n + 1)
    assert abs(got - want) < 1e-12 * want, (got, want)


@pytest.mark.parametrize("dim,k", [(2, 0), (2, 1), (2, 3), (3, 2)])
def test_l1_sign_changing_slope(dim, k):
    # rho_h = w0 + a sqrt(3) xi in every cell against rho_exact = w0: the
    # integrand |a sqrt(3) xi| is not a polynomial, so the rule's own sum is
    # the value: |a| sqrt(3) G / 2 with G = sum_i w_i |x_i| over k+3 nodes
    n = [3, 2, 2][:dim]
    o = O.Oracle(dim, n, [0.0] * dim, [0.5 * m for m in n], k)
    a = -0.37
    W = np.zeros(o.shape)
    W[0, 0] = 1.3
    if k >= 1:
        W[0, 1] = a  # x slope (basis index 1)
    else:
        pytest.skip("k = 0 has no slope weight")
    got = o.l1_density(W, np.full((o.nq_l1, o.n_cells), 1.3))
    x, w = npleg.leggauss(k + 3)
    G = float((w * np.abs(x)).sum())
    want = abs(a) * math.sqrt(3.0) * G / 2.0
    assert abs(got - want) < 1e-13, (got, want)
    # a rule with one point less gives a different number: the pin sees the rule's size
    x2, w2 = npleg.leggauss(k + 2)
    assert abs(abs(a) * math.sqrt(3.0) * float((w2 * np.abs(x2)).sum()) / 2.0 - want) > 1e-3


def test_l1_piecewise_constant_k0():
    # k = 0 on a two-level mesh: |rho_h - rho_exact| constant per cell, so the
    # value is the volume-weighted mean of the cell constants
    o = O.Oracle(2, [3, 2], [0.0, 0.0], [1.5, 1.0], 0, refine_boxes=[[1, 0, 1, 0]])
    rng = np.random.default_rng(5)
    W = np.zeros(o.shape)
    W[0, 0] = rng.uniform(0.5, 1.5, o.n_cells)
    d = rng.uniform(-0.3, 0.3, o.n_cells)
    rho_ex = np.broadcast_to(W[0, 0] - d, (o.nq_l1, o.n_cells))
    dx = o.cell_dx()
    want = float((np.abs(d) * dx ** 2).sum() / 1.5)
    assert abs(o.l1_density(W, rho_ex) - want) < 1e-14
