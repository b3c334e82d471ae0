"""The 3D Sedov workload at its full size: 64^3 base cells, the central 32^3
refined once (491,520 cells), k=2, SSP-RK3, characteristic TVB limiter and
positivity limiter; FP32 state with FP64 totals and positivity check.

The oracle cannot advance 491,520 cells in seconds, so the CUDA results are
compared on sampled cells (every cell next to a level jump plus a seeded
random sample), with the oracle evaluating those cells one by one.
"""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O
from paper_1506_06140_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

GAMMA = 1.4
MESH = wl.mesh_two_level_3d(64, 16, 47)


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1506_06140_gb300 import build
    build.build()
    o = O.Oracle(3, MESH["n"], MESH["lo"], MESH["hi"], 2, GAMMA, bc=MESH["bc"],
                 refine_boxes=MESH["refine_boxes"], rk_order=3,
                 limiter=O.LIM_CHARACTERISTIC, positivity=True)
    nbr = o.neighbor_table()
    lev = o.levels()
    # cells at level jumps (a coarser neighbour or a node on some side) and a random sample
    jump = np.nonzero(np.any(nbr <= -2, axis=0) |
                      np.any((nbr >= 0) & (lev[np.maximum(nbr, 0)] != lev[None, :]), axis=0))[0]
    rng = np.random.default_rng(7)
    sample = np.unique(np.concatenate([jump[rng.choice(len(jump), 1500, replace=False)],
                                       rng.choice(o.n_cells, 1500, replace=False)]))
    return o, nbr, lev, sample


def solver(precision):
    from paper_1506_06140_gb300 import dg
    return dg.Solver(MESH, 2, GAMMA, rk_order=3, limiter="characteristic", positivity=True,
                     precision=precision)


def sedov_state(o, s):
    U = wl.sedov3d(o.quad_points())
    return U, o.project(U)


def rough_state(o):
    """large jumps and moments: the limiters act (pressure may be negative at points)"""
    return wl.random_weights(3, o.N, o.n_cells, seed=12, slope=0.4, rho_range=(0.1, 2.0),
                             p_range=(1e-4, 2.0))


def smooth_state(o):
    """admissible at every quadrature point, for the right-hand side"""
    return wl.random_weights(3, o.N, o.n_cells, seed=13, slope=0.1, rho_range=(0.5, 2.0),
                             p_range=(0.3, 2.0))


def test_sedov_mesh_tables_bit_exact(setup):
    o, nbr, lev, _ = setup
    s = solver("fp32")
    assert s.n_cells == 491520 == o.n_cells
    np.testing.assert_array_equal(s.neighbor_table(), nbr)
    np.testing.assert_array_equal(s.levels(), lev)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 2e-5)])
def test_sedov_rhs_sampled(setup, precision, tol):
    o, _, _, sample = setup
    s = solver(precision)
    W = smooth_state(o)
    Wd = torch.as_tensor(W, dtype=s.dtype, device="cuda")
    got = s.rhs(Wd).cpu().numpy()[:, :, sample]
    ref = o.rhs_cells(W.astype(np.float32).astype(np.float64) if precision == "fp32" else W, sample)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err < tol, err


def test_sedov_limiter_sampled_fp64(setup):
    o, _, _, sample = setup
    s = solver("fp64")
    W = rough_state(o)
    got = s.limit(torch.as_tensor(W, device="cuda")).cpu().numpy()[:, :, sample]
    ref = o.limit_cells(W, sample)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err < 1e-12, err
    assert np.any(ref != W[:, :, sample])


def test_sedov_projection_and_totals(setup):
    o, _, _, _ = setup
    s = solver("fp64")
    U, W = sedov_state(o, s)
    Wd = s.project(torch.as_tensor(U))
    np.testing.assert_allclose(Wd.cpu().numpy(), W, rtol=0, atol=1e-12 * np.abs(W).max())
    # sums of 491,520 terms in different orders: n * eps ~ 5e-11 relative at most
    np.testing.assert_allclose(s.totals(Wd).cpu().numpy(), o.totals(W), rtol=1e-10, atol=1e-14)
    # total energy is the deposited 1 plus the background p0/(gamma-1) over the unit box
    # (to the n * eps bound of a 491,520-term sum)
    expect = 1.0 + (1.0 - (2 / 64) ** 3) * 1e-5 / 0.4
    assert o.totals(W)[4] == pytest.approx(expect, rel=1e-10)
    assert s.totals(Wd)[4].item() == pytest.approx(expect, rel=1e-10)


def test_sedov_fp32_run_conserves_and_stays_positive(setup):
    o, _, _, _ = setup
    s = solver("fp32")
    U, W = sedov_state(o, s)
    Wd = s.project(torch.as_tensor(U))
    s.limit(Wd)
    t0 = s.totals(Wd).cpu().numpy()
    hist = s.scalar(20)
    s.advance(Wd, 20, hist)
    t1 = s.totals(Wd).cpu().numpy()
    torch.cuda.synchronize()
    assert s.status() == 0
    assert torch.isfinite(Wd).all().item()
    assert np.all(hist.cpu().numpy() > 0)
    # mass and energy to FP32 round-off of the per-cell updates; momentum stays ~0
    assert abs(t1[0] - t0[0]) < 1e-5 * abs(t0[0])
    assert abs(t1[4] - t0[4]) < 1e-5 * abs(t0[4])
    assert np.all(np.abs(t1[1:4]) < 1e-5)
    # cell-mean density and pressure positive everywhere
    Wm = Wd[:, 0, :].double().cpu().numpy()
    p = (GAMMA - 1) * (Wm[4] - 0.5 * (Wm[1] ** 2 + Wm[2] ** 2 + Wm[3] ** 2) / Wm[0])
    assert Wm[0].min() > 0 and p.min() > 0
