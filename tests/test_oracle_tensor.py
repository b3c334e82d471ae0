"""Pins of the oracle's tensor-product basis option (Q_k: every exponent
<= k, (k+1)^d functions), the reading of the vortex workload's "k=3, 16
coefficients per cell and field" beside the paper's total-degree basis.

* the exponent set and its order (phi_1 = 1, then x, y; by total degree);
* orthonormality 2^-d int phi_i phi_j = delta_ij with numpy's Gauss rule and
  numpy's Legendre polynomials (independent of the oracle's own);
* the projection reproduces any polynomial of Q_k exactly (x^k y^k included,
  which the total-degree basis cannot);
* free stream and conservation to round-off; k+1 convergence on the vortex.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import pyoracle as O
from paper_1506_06140_gb300 import workloads as wl


def leg(n, x):
    c = np.zeros(n + 1)
    c[n] = 1.0
    return math.sqrt(2 * n + 1) * npleg.legval(x, c)


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2)])
def test_tensor_exponents(dim, k):
    e = O.basis_exponents_tensor(dim, k)
    assert len(e) == (k + 1) ** dim
    assert len({tuple(x) for x in e}) == len(e)
    assert (e[:, :dim] <= k).all() and (e[:, dim:] == 0).all()
    g = e.sum(axis=1)
    assert (np.diff(g) >= 0).all()  # by total degree
    assert tuple(e[0]) == (0, 0, 0)
    assert [tuple(x) for x in e[1:1 + dim]] == [tuple(np.eye(3, dtype=int)[a]) for a in range(dim)]


@pytest.mark.parametrize("dim,k", [(2, 2), (2, 3), (3, 1)])
def test_tensor_orthonormal(dim, k):
    e = O.basis_exponents_tensor(dim, k)
    x, w = npleg.leggauss(k + 2)
    grids = np.meshgrid(*([x] * dim), indexing="ij")
    wts = np.ones_like(grids[0])
    for a in range(dim):
        wts = wts * np.meshgrid(*([w] * dim), indexing="ij")[a]
    pts = np.stack([gg.ravel() for gg in grids], axis=1)
    # the oracle's phi at the points against numpy's Legendre product
    for l in range(len(e)):
        mine = np.prod([leg(int(e[l][a]), pts[:, a]) for a in range(dim)], axis=0)
        orc = np.array([O.basis_phi_tensor(dim, k, l, p) for p in pts[:7]])
        np.testing.assert_allclose(orc, mine[:7], rtol=1e-13, atol=1e-13)
    Phi = np.stack([np.prod([leg(int(e[l][a]), pts[:, a]) for a in range(dim)], axis=0)
                    for l in range(len(e))])
    G = (Phi * wts.ravel()) @ Phi.T / 2 ** dim
    np.testing.assert_allclose(G, np.eye(len(e)), atol=1e-13)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_tensor_projection_exact_for_qk(k):
    m = wl.mesh_uniform(2, [3, 2], [0.0, 0.0], [1.5, 1.0])
    # x^k y^k plus lower terms: in Q_k, not in P_k
    poly = lambda X, Y: 0.7 + X ** k * Y ** k - 0.3 * X * Y ** (k - 1) + 0.2 * Y ** k

    def check(basis):
        o = O.Oracle(2, m["n"], m["lo"], m["hi"], k, basis=basis)
        xyz = o.quad_points()
        U = np.zeros((4, o.nq, o.n_cells))
        U[0] = poly(xyz[0], xyz[1])
        W = o.project(U)
        x1 = o.l1_points()
        # rho_h at the (k+3)^2 points from the weights, with numpy's polynomials
        e = O.basis_exponents_tensor(2, k) if basis == "tensor" else O.basis_exponents(2, k)
        dx = o.cell_dx()
        ctr = x1.mean(axis=1)
        xi = [(x1[a] - ctr[a][None, :]) / (0.5 * dx[None, :]) for a in range(2)]
        rho = sum(W[0, l][None, :] * leg(int(e[l][0]), xi[0]) * leg(int(e[l][1]), xi[1]) for l in range(len(e)))
        return np.abs(rho - poly(x1[0], x1[1])).max()

    assert check("tensor") < 1e-12
    assert check("total") > 1e-3  # the paper's basis cannot hold x^k y^k


@pytest.mark.parametrize("k", [1, 2, 3])
def test_tensor_free_stream_and_conservation(k):
    m = dict(wl.mesh_uniform(2, [6, 5], [0.0, 0.0], [1.2, 1.0]), refine_boxes=[[1, 1, 3, 2]])
    o = O.Oracle(2, m["n"], m["lo"], m["hi"], k, basis="tensor", refine_boxes=m["refine_boxes"])
    assert o.N == (k + 1) ** 2
    W = np.zeros(o.shape)
    W[:, 0] = np.array([1.1, 0.3, -0.2, 2.7])[:, None]
    assert np.abs(o.rhs(W)).max() < 1e-12
    W = wl.random_weights(2, o.N, o.n_cells, seed=40 + k)
    d = o.rhs(W)
    vol = o.cell_dx() ** 2
    tot = (d[:, 0, :] * vol[None, :]).sum(axis=1)
    assert np.abs(tot).max() < 1e-12 * np.abs(d[:, 0, :] * vol[None, :]).sum()


@pytest.mark.parametrize("k", [1, 2])
def test_tensor_vortex_convergence(k):
    def l1(n):
        rk = {1: 2, 2: 3}[k]
        o = O.Oracle(2, [n, n], [-5, -5], [5, 5], k, rk_order=rk, basis="tensor")
        W = o.project(wl.vortex(o.quad_points()))
        t = 0.0
        while t < 0.5 - 1e-14:
            dt = min(o.compute_dt(W), 0.5 - t)
            W, _ = o.rk_step(W, dt)
            t += dt
        return o.l1_density(W, wl.vortex(o.l1_points(), t=0.5)[0])
    e1, e2 = l1(16), l1(32)
    assert math.log2(e1 / e2) > k + 1 - 0.4
