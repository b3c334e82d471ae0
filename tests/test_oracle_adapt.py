"""Pins of the oracle's mesh adaptation (Secs. 4.1, 4.3, 4.4) on the
two-level mesh: the refinement criterion of eq. cell_ref and the keep
criterion of eq. node_ref with their hysteresis, one buffer layer around
flagged base cells, refinement by the matrices of eq. ref_weights (exact for
the coarse polynomial), derefinement by eq. deref_weights (conserving the
means, and undoing a refinement exactly)."""

import numpy as np
import pytest

from oracle import pyoracle as O
from paper_1506_06140_gb300 import workloads as wl

WT, ALPHA = 0.01, 1.1


def oracle(dim, n, boxes=(), k=2, bc=None):
    hi = [n[a] / n[0] for a in range(dim)]
    return O.Oracle(dim, n, [0.0] * dim, hi, k, 1.4, bc=bc or [0] * dim, refine_boxes=list(boxes))


def boxes_of(flags, n):
    dim = len(n)
    out = []
    for b in np.nonzero(flags)[0]:
        p = [b % n[0], (b // n[0]) % n[1]] + ([b // (n[0] * n[1])] if dim == 3 else [])
        out.append(p + p)
    return out


def flat_state(o):
    """uniform means, no slopes"""
    return wl.random_weights(o.dim, o.N, o.n_cells, seed=3, slope=0.0, rho_range=(1.0, 1.0),
                             vel_amp=0.0, p_range=(1.0, 1.0))


def test_single_steep_cell_flags_its_3x3_block():
    o = oracle(2, [6, 5])
    W = flat_state(o)
    W[0, 1, 1 + 6 * 1] = 2 * ALPHA * WT  # density slope in x of base cell (1, 1)
    f = o.adapt_flags(W, WT, ALPHA).reshape(5, 6)
    expect = np.zeros((5, 6), int)
    expect[0:3, 0:3] = 1
    np.testing.assert_array_equal(f, expect)


@pytest.mark.parametrize("bc,expect_wrap", [(0, True), (1, False)], ids=["periodic", "transmissive"])
def test_buffer_layer_wraps_on_periodic_axes_3d(bc, expect_wrap):
    n = [4, 4, 3]
    o = oracle(3, n, bc=[bc] * 3)
    W = flat_state(o)
    W[0, 3, 0] = -2 * ALPHA * WT  # negative z-slope in the corner base cell (0, 0, 0)
    f = o.adapt_flags(W, WT, ALPHA).reshape(3, 4, 4)  # [z][y][x]
    assert f[0, 0, 0] == 1 and f[1, 1, 1] == 1 and f[2, 2, 2] == 0
    assert f[2, 3, 3] == (1 if expect_wrap else 0)  # the periodic image of (-1, -1, -1)
    assert f.sum() == (27 if expect_wrap else 8)


def test_hysteresis_between_refine_and_keep_thresholds():
    # leaf: refined above alpha w_t only
    o = oracle(2, [5, 5])
    for slope, refined in ((1.05 * WT, 0), (1.15 * WT, 1)):
        W = flat_state(o)
        W[0, 2, 12] = slope  # y-slope of the centre base cell
        assert o.adapt_flags(W, WT, ALPHA).reshape(5, 5)[2, 2] == refined
    # node: kept above w_t / alpha (its node weights), derefined below
    on = oracle(2, [5, 5], boxes=[[2, 2, 2, 2]])
    first = 12  # base cell 12 is refined: its 4 children start at cell 12
    for slope, kept in ((0.95 * WT, 1), (0.85 * WT, 0)):
        W = flat_state(on)
        Wc = np.zeros((on.nv, on.N, 1))
        Wc[0, 0, 0], Wc[0, 1, 0] = 1.0, slope  # a linear coarse density, refined exactly
        for ch in range(4):
            W[0, :, first + ch] = O.refinement_matrix(2, 2, ch) @ Wc[0, :, 0]
        assert np.allclose(on.node_weights(W)[0, 1, 0], slope, rtol=1e-13)
        assert on.adapt_flags(W, WT, ALPHA).reshape(5, 5)[2, 2] == kept


def _sample(o, W, c, xi):
    return sum(W[:, l, c] * O.basis_phi(o.dim, o.k, l, xi) for l in range(o.N))


@pytest.mark.parametrize("dim", [2, 3])
def test_refinement_is_exact_and_derefinement_undoes_it(dim):
    n = [3, 3] if dim == 2 else [3, 2, 2]
    k = 2
    coarse = oracle(dim, n, k=k)
    W = wl.random_weights(dim, coarse.N, coarse.n_cells, seed=11, slope=0.3)
    flags = np.zeros(int(np.prod(n)), int)
    flags[[1, 4]] = 1
    fine = oracle(dim, n, boxes=boxes_of(flags, n), k=k)
    Wf = fine.adapt_project(coarse, W)
    # base cell 1 (the second) is now 2^d children starting at cell 1; each
    # child's polynomial equals the parent's at the same physical points
    rng = np.random.default_rng(0)
    for ch in range(2 ** dim):
        off = np.array([((ch >> a) & 1) for a in range(dim)])
        for _ in range(3):
            eta = rng.uniform(-1, 1, dim)
            parent_xi = (eta + 2 * off - 1) / 2.0
            np.testing.assert_allclose(_sample(fine, Wf, 1 + ch, eta), _sample(coarse, W, 1, parent_xi),
                                       rtol=1e-12, atol=1e-13)
    # unchanged base cells are copied
    np.testing.assert_array_equal(Wf[:, :, 0], W[:, :, 0])
    # derefinement back to the coarse mesh restores the state
    back = coarse.adapt_project(fine, Wf)
    np.testing.assert_allclose(back, W, rtol=0, atol=1e-14 * np.abs(W).max())


def test_derefinement_conserves_means():
    n = [4, 3]
    fine = oracle(2, n, boxes=[[1, 1, 2, 1]])
    W = wl.random_weights(2, fine.N, fine.n_cells, seed=12, slope=0.4)
    coarse = oracle(2, n)
    Wc = coarse.adapt_project(fine, W)
    np.testing.assert_allclose(coarse.totals(Wc), fine.totals(W), rtol=1e-14)
    # a non-polynomial fine state is not restored by refining again (information is lost)
    again = fine.adapt_project(coarse, Wc)
    assert np.abs(again - W).max() > 1e-3


def test_adaptive_run_conserves_totals():
    """Steps and adaptations together keep the totals to rounding: the DG step
    is conservative on a periodic two-level mesh and both projections keep the
    cell means of every base cell (eqs. ref_weights, deref_weights)."""
    n = [12, 12]
    o = oracle(2, n)
    xyz = o.quad_points()
    r2 = (xyz[0] - 0.4) ** 2 + (xyz[1] - 0.5) ** 2
    rho = 1.0 + 0.6 * np.exp(-r2 / 0.15 ** 2)
    W = o.project(wl.conserved(rho, [np.full_like(rho, 1.0), np.full_like(rho, 0.4)], np.ones_like(rho), 1.4))
    t0 = o.totals(W)
    refined_any = False
    for _ in range(8):
        W, _ = o.rk_step(W, 0.0)
        flags = o.adapt_flags(W, WT, ALPHA)
        o_new = oracle(2, n, boxes=boxes_of(flags, n))
        W = o_new.adapt_project(o, W)
        o = o_new
        refined_any |= bool(flags.any())
        np.testing.assert_allclose(o.totals(W), t0, rtol=1e-13, atol=1e-13)
    assert refined_any
