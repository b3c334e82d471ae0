"""Pins of the oracle's DG scheme against what the paper and the mathematics fix.

* the advected density wave reduces exactly to upwind DG for linear
  advection, whose operator is built here in exact arithmetic (sympy);
* free-stream preservation and conservation to round-off (uniform and AMR);
* RK tableau identities and observed order on scalar ODEs;
* L2 projection exact for polynomials of degree <= k;
* (k+1)-order convergence on the wave and the isentropic vortex, and on a
  two-level mesh (hanging faces);
* neighbour tables against an independent brute-force search;
* refinement matrices reproduce the coarse polynomial; refine->derefine = I;
* limiter invariants; positivity bounds; the Sod tube against the exact
  Riemann solution; JVPs of a step against central differences.
"""
import itertools
import math

import numpy as np
import pytest
import sympy as sp

from exact_riemann import density_profile
from oracle import pyoracle as O
from paper_1506_06140_gb300 import workloads as wl

GAMMA = 1.4


def wave_problem(n, k, rk=2, cfl=0.3, **kw):
    return O.Oracle(2, [n, n], [0, 0], [1, 1], k, GAMMA, rk_order=rk, cfl=cfl, **kw)


def eval_density(o, W, pts_ref, dim):
    """rho_h at reference points of every cell, [q][cell]."""
    Phi = np.array([[O.basis_phi(dim, o.k, l, p) for l in range(o.N)] for p in pts_ref])
    return Phi @ W[0]


# ---------------------------------------------------------------------------
# exact upwind DG operator for rho_t + v . grad rho = 0 (v = (1,1)) on a
# periodic n x n mesh, k = 1, in exact arithmetic

def upwind_dg_operator(n, k=1, v=(1, 1)):
    xi, eta = sp.symbols("xi eta")
    e = O.basis_exponents(2, k)
    leg = lambda m, x: sp.sqrt(2 * m + 1) * sp.legendre(m, x)
    phi = [leg(int(a), xi) * leg(int(b), eta) for a, b, _ in e]
    N = len(phi)
    dx = sp.Rational(1, n)
    pre = sp.Rational(1, 2) / dx  # 2^(1-d)/dx
    integ2 = lambda f: sp.integrate(sp.integrate(sp.expand(f), (xi, -1, 1)), (eta, -1, 1))
    integ1 = lambda f, var: sp.integrate(sp.expand(f), (var, -1, 1))
    # local matrices
    Vol = sp.zeros(N, N)
    for j in range(N):
        for l in range(N):
            Vol[j, l] = integ2(phi[l] * (v[0] * sp.diff(phi[j], xi) + v[1] * sp.diff(phi[j], eta)))
    # outflow faces (own trace) and inflow faces (neighbour trace at its far face)
    outx = sp.zeros(N, N); inx = sp.zeros(N, N)
    outy = sp.zeros(N, N); iny = sp.zeros(N, N)
    for j in range(N):
        for l in range(N):
            outx[j, l] = v[0] * integ1(phi[l].subs(xi, 1) * phi[j].subs(xi, 1), eta)
            inx[j, l] = -v[0] * integ1(phi[l].subs(xi, 1) * phi[j].subs(xi, -1), eta)
            outy[j, l] = v[1] * integ1(phi[l].subs(eta, 1) * phi[j].subs(eta, 1), xi)
            iny[j, l] = -v[1] * integ1(phi[l].subs(eta, 1) * phi[j].subs(eta, -1), xi)
    nc = n * n
    M = np.zeros((N * nc, N * nc))
    f = lambda A: np.array(A.evalf(30).tolist(), dtype=np.float64)
    Vol, outx, inx, outy, iny = map(f, (Vol, outx, inx, outy, iny))
    pref = float(pre)
    for iy in range(n):
        for ix in range(n):
            c = ix + n * iy
            west = (ix - 1) % n + n * iy
            south = ix + n * ((iy - 1) % n)
            blk = lambda cc: slice(cc * N, (cc + 1) * N)
            M[blk(c), blk(c)] += pref * (Vol - outx - outy)
            M[blk(c), blk(west)] += -pref * inx
            M[blk(c), blk(south)] += -pref * iny
    return M


def test_wave_rhs_equals_exact_upwind_dg():
    n, k = 4, 1
    o = wave_problem(n, k)
    rng = np.random.default_rng(11)
    Wr = np.zeros((o.N, o.n_cells))
    Wr[0] = 1.0 + 0.2 * rng.uniform(-1, 1, o.n_cells)
    Wr[1:] = 0.05 * rng.uniform(-1, 1, (o.N - 1, o.n_cells))
    v, p = np.array([1.0, 1.0]), 1.0
    W = np.zeros(o.shape)
    W[0] = Wr
    W[1] = v[0] * Wr
    W[2] = v[1] * Wr
    W[3] = 0.5 * v.dot(v) * Wr
    W[3, 0] += p / (GAMMA - 1)
    dW = o.rhs(W)
    M = upwind_dg_operator(n, k)
    # cell-major unknown vector (cell, coef)
    ref = (M @ Wr.T.reshape(-1)).reshape(o.n_cells, o.N).T
    np.testing.assert_allclose(dW[0], ref, atol=1e-12, rtol=0)
    # momentum and energy follow the density affinely
    np.testing.assert_allclose(dW[1], v[0] * ref, atol=1e-12)
    np.testing.assert_allclose(dW[2], v[1] * ref, atol=1e-12)
    np.testing.assert_allclose(dW[3], 0.5 * v.dot(v) * ref, atol=1e-12)


# ---------------------------------------------------------------------------

AMR_2D = dict(dim=2, n=[8, 8], lo=[0, 0], hi=[1, 1], boxes=[[2, 3, 4, 5]])
AMR_3D = dict(dim=3, n=[4, 4, 4], lo=[0, 0, 0], hi=[1, 1, 1], boxes=[[1, 1, 1, 2, 2, 2]])


def make(mesh, k, **kw):
    return O.Oracle(mesh["dim"], mesh["n"], mesh["lo"], mesh["hi"], k, GAMMA,
                    refine_boxes=mesh.get("boxes", []), **kw)


MESHES = [
    dict(dim=2, n=[6, 5], lo=[0, 0], hi=[1.2, 1.0]),
    AMR_2D,
    dict(dim=3, n=[3, 4, 3], lo=[0, 0, 0], hi=[0.75, 1.0, 0.75]),
    AMR_3D,
]


@pytest.mark.parametrize("mesh", MESHES, ids=["u2", "amr2", "u3", "amr3"])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_free_stream_and_conservation(mesh, k):
    o = make(mesh, k)
    const = wl.conserved(np.array(1.1), [0.3, -0.7, 0.2][: mesh["dim"]], np.array(0.8), GAMMA)
    W = np.zeros(o.shape)
    W[:, 0, :] = const[:, None]
    assert np.max(np.abs(o.rhs(W))) < 1e-12
    Wr = wl.random_weights(mesh["dim"], o.N, o.n_cells, seed=7 + k)
    dW = o.rhs(Wr)
    vol = o.cell_dx() ** mesh["dim"]
    tot = (dW[:, 0, :] * vol).sum(axis=1)
    scale = np.abs(dW[:, 0, :] * vol).sum(axis=1)
    assert np.all(np.abs(tot) <= 1e-13 * scale + 1e-15)


def test_rk_tableaux():
    for order in (1, 2, 3, 4):
        A, b, c = O.rk_tableau(order)
        assert abs(b.sum() - 1.0) < 1e-10  # printed RK4 weights sum to 1 - 8.8e-11
        np.testing.assert_allclose(A.sum(axis=1), c, atol=2e-14)
        assert np.all(np.triu(A) == 0)


@pytest.mark.parametrize("order", [1, 2, 3, 4])
@pytest.mark.parametrize("problem", [0, 1])
def test_rk_order_on_scalar_odes(order, problem):
    y0, T = (1.0, 1.0) if problem == 0 else (0.5, 1.0)
    exact = math.exp(-T) if problem == 0 else y0 / (1 - y0 * T)
    errs = [abs(O.rk_ode(order, problem, y0, T, n) - exact) for n in (20, 40)]
    rate = math.log2(errs[0] / errs[1])
    assert rate > order - 0.2


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 3), (3, 2)])
def test_projection_exact_for_polynomials(dim, k):
    mesh = MESHES[1] if dim == 2 else MESHES[3]
    o = make(mesh, k)
    rng = np.random.default_rng(1)
    # random polynomial of total degree k in physical coordinates, per variable
    exps = [e for e in itertools.product(range(k + 1), repeat=dim) if sum(e) <= k]
    coefs = rng.normal(size=(o.nv, len(exps)))
    poly = lambda xyz: np.stack([sum(cf * np.prod([xyz[a] ** e[a] for a in range(dim)], axis=0)
                                     for cf, e in zip(coefs[v], exps)) for v in range(o.nv)])
    W = o.project(poly(o.quad_points()))
    # compare at the L1 rule's points (distinct from the projection points)
    xyz = o.l1_points()
    from numpy.polynomial import legendre as npleg
    xg, _ = npleg.leggauss(k + 3)
    ref_pts = np.array(list(itertools.product(xg, repeat=dim)))[:, ::-1]
    Phi = np.array([[O.basis_phi(dim, k, l, p) for l in range(o.N)] for p in ref_pts])
    vals = np.einsum("ql,vlc->vqc", Phi, W)
    np.testing.assert_allclose(vals, poly(xyz), atol=1e-11, rtol=1e-11)


def _run(o, W, t_end):
    t = 0.0
    while t < t_end - 1e-14:
        dt = min(o.compute_dt(W), t_end - t)
        W, _ = o.rk_step(W, dt)
        t += dt
    return W


def _l1_wave(n, k, t_end):
    o = wave_problem(n, k, rk=k + 1, cfl=0.3)
    W = o.project(wl.wave2d(o.quad_points()))
    W = _run(o, W, t_end)
    rho_ex = wl.wave2d(o.l1_points(), t=t_end)[0]
    return o.l1_density(W, rho_ex)


@pytest.mark.parametrize("k", [1, 2])
def test_wave_convergence_order(k):
    e1, e2 = _l1_wave(8, k, 0.2), _l1_wave(16, k, 0.2)
    assert math.log2(e1 / e2) > k + 1 - 0.3


def _l1_vortex(n, k, t_end, boxes=()):
    rk = {1: 2, 2: 3, 3: 4}[k]
    o = O.Oracle(2, [n, n], [-5, -5], [5, 5], k, GAMMA, rk_order=rk, refine_boxes=boxes)
    W = o.project(wl.vortex(o.quad_points()))
    W = _run(o, W, t_end)
    return o.l1_density(W, wl.vortex(o.l1_points(), t=t_end)[0])


@pytest.mark.parametrize("k", [1, 2])
def test_vortex_convergence_order(k):
    e1, e2 = _l1_vortex(16, k, 0.5), _l1_vortex(32, k, 0.5)
    assert math.log2(e1 / e2) > k + 1 - 0.4


def test_vortex_convergence_on_two_level_mesh():
    # a refined central box: hanging faces must keep the order
    e1 = _l1_vortex(12, 2, 0.5, boxes=[[4, 4, 7, 7]])
    e2 = _l1_vortex(24, 2, 0.5, boxes=[[8, 8, 15, 15]])
    assert math.log2(e1 / e2) > 2.6


# ---------------------------------------------------------------------------

def brute_force_neighbours(o, mesh):
    """Neighbour table from cell boxes: the region beyond each face is matched
    against every cell's box and every refined base cell (node)."""
    dim = mesh["dim"]
    lo, hi = np.array(mesh["lo"], float), np.array(mesh["hi"], float)
    dx = o.cell_dx()
    xyz = o.quad_points().mean(axis=1)  # cell centres (rule is symmetric)
    L = hi - lo
    kids = o.node_children()
    node_ctr = np.array([xyz[:, ch].mean(axis=1) for ch in kids]) if len(kids) else np.zeros((0, dim))
    node_dx = np.array([2 * dx[ch[0]] for ch in kids])
    out = np.full((2 * dim, o.n_cells), -1, np.int32)
    for c in range(o.n_cells):
        for a in range(dim):
            for s in (0, 1):
                p = xyz[:, c].copy()
                p[a] += (1 if s else -1) * dx[c]
                p = lo + np.mod(p - lo, L)
                # a refined region of this size centred at p is a node
                nd = np.nonzero(np.all(np.abs(node_ctr - p[None, :]) < 1e-9, axis=1)
                                & (np.abs(node_dx - dx[c]) < 1e-12))[0] if len(kids) else []
                if len(nd):
                    assert len(nd) == 1
                    out[2 * a + s, c] = -(nd[0] + 2)
                    continue
                # otherwise exactly one leaf box contains the region centre p
                inside = np.all(np.abs(xyz - p[:, None]) < 0.5 * dx[None, :] * (1 - 1e-9), axis=0)
                hits = np.nonzero(inside)[0]
                assert len(hits) == 1
                assert dx[hits[0]] >= dx[c] * (1 - 1e-9)
                out[2 * a + s, c] = hits[0]
    return out


@pytest.mark.parametrize("mesh", MESHES, ids=["u2", "amr2", "u3", "amr3"])
def test_neighbour_table_brute_force(mesh):
    o = make(mesh, 1)
    np.testing.assert_array_equal(o.neighbor_table(), brute_force_neighbours(o, mesh))


def test_neighbour_table_transmissive():
    o = O.Oracle(2, [5, 1], [0, 0], [1, 0.2], 1, GAMMA, bc=[O.BC_TRANSMISSIVE, O.BC_PERIODIC])
    nb = o.neighbor_table()
    assert nb[0, 0] == -1 and nb[1, 4] == -1
    assert list(nb[1, :4]) == [1, 2, 3, 4]
    assert list(nb[2]) == list(range(5)) and list(nb[3]) == list(range(5))


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 3), (3, 2)])
def test_refinement_matrices(dim, k):
    rng = np.random.default_rng(2)
    N = len(O.basis_exponents(dim, k))
    Ps = [O.refinement_matrix(dim, k, ch) for ch in range(2 ** dim)]
    wK = rng.normal(size=N)
    for ch, P in enumerate(Ps):
        wA = P @ wK
        o = np.array([1.0 if (ch >> a) & 1 else -1.0 for a in range(dim)])
        for _ in range(5):
            eta = rng.uniform(-1, 1, dim)
            xi = 0.5 * (eta + o)
            coarse = sum(wK[l] * O.basis_phi(dim, k, l, xi) for l in range(N))
            fine = sum(wA[l] * O.basis_phi(dim, k, l, eta) for l in range(N))
            assert fine == pytest.approx(coarse, abs=1e-12)
    # refinement followed by derefinement (eq. deref_weights) is the identity
    G = sum(P.T @ P for P in Ps) / 2 ** dim
    np.testing.assert_allclose(G, np.eye(N), atol=1e-13)
    # the printed claim P_A P_A^T = I does not hold for k >= 1
    assert np.max(np.abs(Ps[0] @ Ps[0].T - np.eye(N))) > 1e-3


def test_node_weights_are_derefinement():
    o = make(AMR_3D, 2)
    rng = np.random.default_rng(4)
    wK = rng.normal(size=(o.nv, o.N))
    W = wl.random_weights(3, o.N, o.n_cells, 3)
    kids = o.node_children()
    for m, ch in enumerate(kids):  # fill node m's children with a refined coarse polynomial
        for s, c in enumerate(ch):
            W[:, :, c] = wK @ O.refinement_matrix(3, 2, s).T
    Wn = o.node_weights(W)
    for m in range(len(kids)):
        np.testing.assert_allclose(Wn[:, :, m], wK, atol=1e-12)


# ---------------------------------------------------------------------------

def test_minmod_tables():
    mm = lambda a, b, c, M=0.0, dx=1.0: O.minmod_b(a, b, c, M, dx)
    assert mm(1, 2, 3) == 1 and mm(-1, -2, -3) == -1
    assert mm(3, 2, 1) == 1 and mm(-3, -0.5, -2) == -0.5
    assert mm(1, -2, 3) == 0 and mm(0, 1, 1) == 0 and mm(1, 0, 1) == 0
    # TVB bound: |a| <= Mtilde dx returns a
    assert mm(0.05, -1, 1, M=0.5, dx=0.2) == 0.05
    assert mm(0.2, -1, 1, M=0.5, dx=0.2) == 0.0


@pytest.mark.parametrize("lim", [O.LIM_COMPONENT, O.LIM_CHARACTERISTIC])
@pytest.mark.parametrize("mesh", [MESHES[0], AMR_2D, AMR_3D], ids=["u2", "amr2", "amr3"])
def test_slope_limiter_invariants(lim, mesh):
    o = make(mesh, 2, limiter=lim, Mtilde=0.0)
    dim = mesh["dim"]
    W = wl.random_weights(dim, o.N, o.n_cells, 21, slope=0.3)
    Wl = o.slope_limit(W)
    np.testing.assert_array_equal(Wl[:, 0, :], W[:, 0, :])  # means unchanged
    changed = np.any(Wl != W, axis=(0, 1))
    assert changed.any()
    # limited cells keep only linear terms
    e = O.basis_exponents(dim, 2)
    high = e.sum(axis=1) >= 2
    assert np.all(Wl[:, high][:, :, changed] == 0)
    # limiting twice changes nothing more in the linear terms' limited cells' means
    np.testing.assert_array_equal(o.slope_limit(Wl)[:, 0, :], W[:, 0, :])


@pytest.mark.parametrize("lim", [O.LIM_COMPONENT, O.LIM_CHARACTERISTIC])
def test_slope_limiter_noop_on_linear_state(lim):
    # a globally linear field: slopes equal the mean differences, beta = 1 keeps them
    n = 8
    # a tiny TVB bound keeps characteristic components that are zero up to round-off
    o = O.Oracle(2, [n, n], [0, 0], [1, 1], 1, GAMMA, limiter=lim, Mtilde=1e-9,
                 bc=[O.BC_TRANSMISSIVE] * 2)
    xyz = o.quad_points()
    rho = 1.0 + 0.3 * xyz[0] - 0.2 * xyz[1]
    U = wl.conserved(rho, [0.1, 0.2], np.ones_like(rho), GAMMA)
    W = o.project(U)
    # interior cells only (boundary cells see a zero-gradient ghost)
    lvl = o.neighbor_table()
    interior = np.all(lvl >= 0, axis=0)
    Wl = o.slope_limit(W)
    np.testing.assert_array_equal(Wl[:, :, interior], W[:, :, interior])


@pytest.mark.parametrize("mesh", [MESHES[0], AMR_2D, AMR_3D], ids=["u2", "amr2", "amr3"])
def test_positivity_limiter(mesh):
    dim = mesh["dim"]
    k = 2
    o = make(mesh, k, positivity=True, eps=1e-10)
    rng = np.random.default_rng(8)
    W = wl.random_weights(dim, o.N, o.n_cells, 9, slope=0.0, rho_range=(0.05, 0.2),
                          p_range=(1e-3, 1e-2))
    W[:, 1:, :] = rng.uniform(-1, 1, (o.nv, o.N - 1, o.n_cells)) * np.abs(W[:, :1, :]) * 0.8
    Wl = o.positivity_limit(W)
    np.testing.assert_array_equal(Wl[:, 0, :], W[:, 0, :])
    # check rho and p at the union points S of every cell
    from numpy.polynomial import legendre as npleg
    m = math.ceil((k + 3) / 2)
    xl = np.concatenate([[-1.0], np.sort(npleg.legroots(npleg.legder([0] * (m - 1) + [1]))), [1.0]])
    xg, _ = npleg.leggauss(k + 1)
    pts = []
    for a in range(dim):
        for p in itertools.product(*[xl if b == a else xg for b in range(dim)]):
            pts.append(p)
    Phi = np.array([[O.basis_phi(dim, k, l, p) for l in range(o.N)] for p in pts])
    U = np.einsum("ql,vlc->vqc", Phi, Wl)
    rho = U[0]
    pres = (GAMMA - 1) * (U[dim + 1] - 0.5 * (U[1:dim + 1] ** 2).sum(axis=0) / rho)
    assert rho.min() >= 1e-10 - 1e-14
    assert pres.min() >= 1e-10 - 1e-9
    Ub = np.einsum("ql,vlc->vqc", Phi, W)
    assert Ub[0].min() < 0 or ((GAMMA - 1) * (Ub[dim + 1] - 0.5 * (Ub[1:dim + 1] ** 2).sum(0) / Ub[0])).min() < 0
    # an admissible state is left unchanged
    Wp = wl.random_weights(dim, o.N, o.n_cells, 10, slope=0.01)
    np.testing.assert_array_equal(o.positivity_limit(Wp), Wp)


def test_solve_tau_root():
    for seed in range(20):
        rng = np.random.default_rng(seed)
        ub = wl.conserved(np.array(1.0), rng.uniform(-1, 1, 2), np.array(0.5), GAMMA)
        u = wl.conserved(np.array(0.8), rng.uniform(-3, 3, 2), np.array(-0.3), GAMMA)
        tau = O.solve_tau(2, GAMMA, 1e-10, ub, u)
        s = ub + tau * (u - ub)
        p = (GAMMA - 1) * (s[3] - 0.5 * (s[1] ** 2 + s[2] ** 2) / s[0])
        assert 0 < tau < 1
        assert abs(p - 1e-10) < 1e-12


def test_timestep_closed_form():
    o = wave_problem(8, 2, cfl=0.3)
    W = np.zeros(o.shape)
    W[:, 0, :] = wl.conserved(np.array(1.0), [0.5, -0.25], np.array(1.0), GAMMA)[:, None]
    c = math.sqrt(GAMMA)
    ref = 0.3 / 5 / ((0.5 + c) * 8 + (0.25 + c) * 8)
    assert o.compute_dt(W) == pytest.approx(ref, rel=1e-14)
    op = O.Oracle(2, [8, 8], [0, 0], [1, 1], 2, GAMMA, cfl=0.3, positivity=True)
    assert op.compute_dt(W) == pytest.approx(0.3 * min(1 / 5, 1 / 6) / ((0.5 + c) * 8 + (0.25 + c) * 8),
                                             rel=1e-14)


def _sod(n, k, lim, t_end=0.228):
    o = O.Oracle(2, [n, 1], [0, 0], [1, 1.0 / n], k, GAMMA, rk_order=max(k + 1, 1) if k < 3 else 4,
                 bc=[O.BC_TRANSMISSIVE, O.BC_PERIODIC], limiter=lim, positivity=(k > 0))
    W = o.project(wl.sod(o.quad_points()))
    W = o.limit(W)
    W = _run(o, W, t_end)
    x = o.quad_points()[0].mean(axis=0)
    return np.abs(W[0, 0] - density_profile(x, t_end)).mean(), W, x, o


def test_sod_godunov_converges_to_exact():
    e1 = _sod(64, 0, O.LIM_NONE)[0]
    e2 = _sod(128, 0, O.LIM_NONE)[0]
    assert e2 < e1 and e2 < 0.02


def test_sod_dg3_characteristic_limiter():
    err, W, x, o = _sod(64, 2, O.LIM_CHARACTERISTIC)
    assert err < 0.01
    # shock position: the exact shock is at x0 + 1.7522 t; find the mean-density jump
    rho = W[0, 0]
    xs = 0.5 + 1.75216 * 0.228
    jump = x[np.argmin(np.diff(rho)) + 1]
    assert abs(jump - xs) < 2.0 / 64
    assert np.all(rho > 0)


def test_step_jvp_matches_central_differences():
    o = O.Oracle(2, [4, 4], [0, 0], [1, 1], 1, GAMMA, rk_order=3)
    W = wl.random_weights(2, o.N, o.n_cells, 31, slope=0.05)
    V = np.random.default_rng(2).normal(size=o.shape)
    dt = 0.5 * o.compute_dt(W)
    _, JV = o.rk_step_jvp(W, V, dt)
    h = 1e-6
    fd = (o.rk_step(W + h * V, dt)[0] - o.rk_step(W - h * V, dt)[0]) / (2 * h)
    assert np.max(np.abs(JV - fd)) < 1e-7 * np.max(np.abs(JV))


@pytest.mark.parametrize("mesh", MESHES + [dict(dim=2, n=[5, 1], lo=[0, 0], hi=[1, 0.2])],
                         ids=["u2", "amr2", "u3", "amr3", "strip"])
def test_per_cell_evaluations_match_full_mesh(mesh):
    """rhs_one / limit_one (used for sampled comparisons at full size) agree
    with the whole-mesh rhs and limiter."""
    o = make(mesh, 2, limiter=O.LIM_CHARACTERISTIC, positivity=True)
    W = wl.random_weights(mesh["dim"], o.N, o.n_cells, seed=41, slope=0.5, rho_range=(0.2, 2.0),
                          p_range=(0.05, 2.0))
    cells = np.arange(o.n_cells)
    np.testing.assert_allclose(o.rhs_cells(W, cells), o.rhs(W), rtol=0,
                               atol=1e-13 * np.abs(o.rhs(W)).max())
    np.testing.assert_array_equal(o.limit_cells(W, cells), o.limit(W))


# ---------------------------------------------------------------------------
# the oracle's all-core step (gather form on OpenMP threads) against its
# serial scatter form

@pytest.mark.parametrize("dim,n,k,boxes", [(2, [9, 7], 3, [[2, 2, 5, 4]]), (3, [4, 3, 3], 2, [[1, 0, 1, 2, 1, 1]])])
def test_parallel_step_matches_serial_step(dim, n, k, boxes):
    lo, hi = [-1.0] * dim, [-1.0 + 0.5 * m for m in n]
    rk = {2: 3, 3: 4}[k]
    o = O.Oracle(dim, n, lo, hi, k, GAMMA, rk_order=rk, refine_boxes=boxes)
    W = wl.random_weights(dim, o.N, o.n_cells, seed=31 + dim)
    dt = 0.5 * o.compute_dt(W)
    ref, _ = o.rk_step(W, dt)
    o.set_threads(4)
    par4, _ = o.rk_step(W, dt)
    o.set_threads(3)
    par3, _ = o.rk_step(W, dt)
    # the gather form's result does not depend on the thread count
    np.testing.assert_array_equal(par3, par4)
    # and agrees with the scatter form to rounding (same terms, another order)
    d = np.abs(par4 - W).max()
    np.testing.assert_allclose(par4 - W, ref - W, rtol=0, atol=1e-13 * d)
