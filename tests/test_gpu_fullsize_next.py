"""Parity at the full sizes of the Keplerian-disc and adaptive Kelvin-Helmholtz
workloads (1024^2 base cells), in the launch configuration the benchmark
times, on sampled cells that the oracle evaluates one by one.

* Keplerian disc (Sec. 5.5), 1024^2, k=2, FP64, gravity source: dW/dt of
  the projected and positivity-limited initial state on cells of the disc's
  rims and a seeded random sample, against the oracle with the same
  acceleration field.
* Kelvin-Helmholtz (Sec. 5.6), 1024^2 base, k=3, FP64: the base cells around
  both interfaces refined through dg_adapt_set + dg_regrid (the mesh tables
  built on the device), dW/dt and the limiter on every cell next to a level
  jump plus a random sample, against an oracle built with the same
  refinement.
"""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O
from paper_1506_06140_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1506_06140_gb300 import build
    build.build()


def test_keplerian_disc_1024_rhs_sampled():
    from paper_1506_06140_gb300 import dg
    n, k, gamma = 1024, 2, 5.0 / 3.0
    m = wl.mesh_uniform(2, [n, n], [0.0, 0.0], [6.0, 6.0])
    s = dg.Solver(m, k, gamma, rk_order=3, positivity=True)
    xyz = s.quad_points().cpu().numpy()
    acc = wl.keplerian_accel(xyz)
    s.set_gravity(torch.as_tensor(acc))
    # the limited projection (the raw one undershoots to non-physical traces at
    # the disc's edges, where HLLC is undefined)
    W = s.limit(s.project(torch.as_tensor(wl.keplerian_disc(xyz))))
    got = s.rhs(W).cpu().numpy()
    Wh = W.cpu().numpy()
    c = xyz.mean(axis=1) - 3.0
    r = np.hypot(c[0], c[1])
    rims = np.nonzero((np.abs(r - 0.5) < 0.1) | (np.abs(r - 2.0) < 0.1) | (r < 0.3))[0]
    rng = np.random.default_rng(11)
    sample = np.unique(np.concatenate([rng.choice(rims, 1500, replace=False), rng.choice(n * n, 1500, replace=False)]))
    o = O.Oracle(2, [n, n], [0.0, 0.0], [6.0, 6.0], k, gamma, rk_order=3, positivity=True)
    o.set_accel(wl.keplerian_accel(o.quad_points()))  # sampled at the oracle's own points
    ref = o.rhs_cells(Wh, sample)
    err = np.max(np.abs(got[:, :, sample] - ref)) / np.max(np.abs(ref))
    assert err < 1e-11, err


def test_kelvin_helmholtz_1024_regridded_sampled():
    from paper_1506_06140_gb300 import dg
    n, k = 1024, 3
    m = wl.mesh_uniform(2, [n, n], [0.0, 0.0], [1.0, 1.0])
    s = dg.Solver(m, k, 1.4, rk_order=4, limiter="characteristic", positivity=True)
    W = s.project(torch.as_tensor(wl.kelvin_helmholtz(s.quad_points().cpu().numpy())))
    # refine the base cells within 3 cells of either interface, plus a few scattered ones
    yb = (np.arange(n) + 0.5) / n
    band = (np.abs(yb - 0.25) < 3.0 / n) | (np.abs(yb - 0.75) < 3.0 / n)
    flags = np.repeat(band[:, None], n, axis=1).astype(np.int32)
    flags.reshape(-1)[np.random.default_rng(12).choice(n * n, 2000, replace=False)] = 1
    s.set_refinement(flags.reshape(-1))
    W = s.regrid(W)
    # a generic state on the new mesh (smooth means, slopes of both signs)
    Wr = wl.random_weights(2, s.N, s.n_cells, seed=13, slope=0.1)
    Wd = torch.as_tensor(Wr, device="cuda")
    got_rhs = s.rhs(Wd).cpu().numpy()
    got_lim = s.limit(Wd.clone()).cpu().numpy()
    fb = np.nonzero(flags.reshape(-1))[0]
    boxes = [[b % n, b // n, b % n, b // n] for b in fb]
    o = O.Oracle(2, [n, n], [0.0, 0.0], [1.0, 1.0], k, 1.4, refine_boxes=boxes, rk_order=4,
                 limiter=O.LIM_CHARACTERISTIC, positivity=True)
    assert o.n_cells == s.n_cells
    nbr, lev = o.neighbor_table(), o.levels()
    np.testing.assert_array_equal(s.neighbor_table(), nbr)
    jump = np.nonzero(np.any(nbr <= -2, axis=0) |
                      np.any((nbr >= 0) & (lev[np.maximum(nbr, 0)] != lev[None, :]), axis=0))[0]
    rng = np.random.default_rng(14)
    sample = np.unique(np.concatenate([rng.choice(jump, 1500, replace=False),
                                       rng.choice(o.n_cells, 1500, replace=False)]))
    ref = o.rhs_cells(Wr, sample)
    assert np.max(np.abs(got_rhs[:, :, sample] - ref)) / np.max(np.abs(ref)) < 1e-11
    ref_lim = o.limit_cells(Wr, sample)
    assert np.max(np.abs(got_lim[:, :, sample] - ref_lim)) < 1e-12 * np.max(np.abs(ref_lim))
