"""Gravity source (eq. gravity_term) and gravity timestep bound (Sec. 2.5)
through the CUDA path, against the oracle.

* dW/dt with an external acceleration field: random states, uniform and
  two-level meshes, 2D k=1..3 and 3D k=1,2, FP64 (1e-12 of the largest
  weight rate) and FP32 (FP32 rounding of the same).
* the timestep: hydro bound or gravity bound, whichever is smaller (FP64
  to 1e-14, FP32 to 1e-6).
* the cold Keplerian disc of Sec. 5.5 (DG-2 with the positivity limiter
  only) for a few steps: the FP64 run follows the oracle's to 1e-10, and so
  does its angular momentum drift (the positivity limiter does not keep it).
* without a limiter, a rotating state in a central field keeps its total
  angular momentum to rounding (Sec. 2.6), on uniform and two-level meshes.
* the field is tied to the mesh: dg_regrid drops it (stepping refuses until
  it is set again); mixed and tensor-core precisions refuse it.
"""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O
from paper_1506_06140_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
GAMMA = 5.0 / 3.0
EPS = 0.3


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1506_06140_gb300 import build
    build.build()


def plummer(xyz, center):
    r2 = sum((xyz[a] - center) ** 2 for a in range(len(xyz))) + EPS * EPS
    return np.stack([-(xyz[a] - center) / r2 ** 1.5 for a in range(len(xyz))])


def make(dim, n, k, boxes, precision="fp64", **kw):
    from paper_1506_06140_gb300 import dg
    hi = [n[a] * 0.25 for a in range(dim)]
    m = wl.mesh_uniform(dim, n, [0.0] * dim, hi)
    m["refine_boxes"] = boxes
    s = dg.Solver(m, k, GAMMA, rk_order=3, precision=precision, **kw)
    o = O.Oracle(dim, n, [0.0] * dim, hi, k, GAMMA, refine_boxes=boxes, rk_order=3, **kw)
    return s, o


CASES = [(2, [12, 10], 1, []), (2, [12, 10], 2, [[3, 2, 7, 6]]), (2, [8, 8], 3, [[2, 2, 4, 5]]),
         (3, [5, 4, 4], 1, [[1, 1, 1, 3, 2, 2]]), (3, [4, 4, 4], 2, [])]


@pytest.mark.parametrize("dim,n,k,boxes", CASES, ids=["2d-k1", "2d-k2-amr", "2d-k3-amr", "3d-k1-amr", "3d-k2"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rhs_with_gravity_matches_oracle(dim, n, k, boxes, precision):
    s, o = make(dim, n, k, boxes, precision)
    center = 0.5 * n[0] * 0.25
    acc_s = plummer(s.quad_points().cpu().numpy(), center)
    s.set_gravity(torch.as_tensor(acc_s))
    o.set_accel(plummer(o.quad_points(), center))
    W = wl.random_weights(dim, s.N, s.n_cells, seed=7 + k, slope=0.1, vel_amp=0.8)
    Wd = torch.as_tensor(W, dtype=s.dtype, device="cuda")
    got = s.rhs(Wd).double().cpu().numpy()
    expect = o.rhs(Wd.double().cpu().numpy())
    scale = np.abs(expect).max()
    tol = 1e-12 if precision == "fp64" else 2e-5
    np.testing.assert_allclose(got, expect, rtol=0, atol=tol * scale)
    # without the field the source is gone again
    s.set_gravity(None)
    o.set_accel(None)
    np.testing.assert_allclose(s.rhs(Wd).double().cpu().numpy(), o.rhs(Wd.double().cpu().numpy()),
                               rtol=0, atol=tol * scale)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("g", [0.5, 400.0], ids=["hydro-bound", "gravity-bound"])
def test_timestep_with_gravity_matches_oracle(precision, g):
    s, o = make(2, [10, 10], 2, [[2, 2, 5, 5]], precision, positivity=True)
    W = wl.random_weights(2, s.N, s.n_cells, seed=3, slope=0.05)
    Wd = torch.as_tensor(W, dtype=s.dtype, device="cuda")
    for sv, xyz in ((s, s.quad_points().cpu().numpy()), (o, o.quad_points())):
        a = g * plummer(xyz, 1.25)
        (sv.set_gravity(torch.as_tensor(a)) if sv is s else sv.set_accel(a))
    got = s.compute_dt(Wd).item()
    expect = o.compute_dt(Wd.double().cpu().numpy())
    assert got == pytest.approx(expect, rel=1e-14 if precision == "fp64" else 1e-6)
    o.set_accel(None)
    hydro = o.compute_dt(Wd.double().cpu().numpy())
    assert (expect < hydro * (1 - 1e-9)) == (g > 1.0)


def angular_momentum(W, xyz_centres, dx, center=3.0):
    x, y = xyz_centres[0] - center, xyz_centres[1] - center
    h = dx / 2 / np.sqrt(3.0)
    return (dx * dx * (x * W[2, 0] + h * W[2, 1] - y * W[1, 0] - h * W[1, 2])).sum()


def test_keplerian_disc_follows_oracle():
    """Sec. 5.5 setup, DG-2 with the positivity limiter only (which does not
    keep the angular momentum: both runs lose the same ~1e-4 of it)"""
    from paper_1506_06140_gb300 import dg
    n, k, steps = 48, 1, 12
    m = wl.mesh_uniform(2, [n, n], [0.0, 0.0], [6.0, 6.0])
    s = dg.Solver(m, k, GAMMA, rk_order=2, positivity=True)
    o = O.Oracle(2, [n, n], [0.0, 0.0], [6.0, 6.0], k, GAMMA, rk_order=2, positivity=True)
    xs, xo = s.quad_points().cpu().numpy(), o.quad_points()
    s.set_gravity(torch.as_tensor(wl.keplerian_accel(xs)))
    o.set_accel(wl.keplerian_accel(xo))
    W = s.limit(s.project(torch.as_tensor(wl.keplerian_disc(xs))))
    Wo = o.limit(o.project(wl.keplerian_disc(xo)))
    centres = xo.mean(axis=1)
    L0 = angular_momentum(Wo, centres, 6.0 / n)
    for _ in range(steps):
        dt = o.compute_dt(Wo)
        assert s.compute_dt(W).item() == pytest.approx(dt, rel=1e-13)
        Wo, _ = o.rk_step(Wo, dt)
        s.rk_step(W, dt)
    assert s.status() == 0
    Wg = W.cpu().numpy()
    np.testing.assert_allclose(Wg, Wo, rtol=0, atol=1e-10 * np.abs(Wo).max())
    drift_gpu = angular_momentum(Wg, centres, 6.0 / n) - L0
    drift_orc = angular_momentum(Wo, centres, 6.0 / n) - L0
    assert abs(drift_gpu - drift_orc) < 1e-10 * abs(L0)


def bump(r, r1):
    t = np.clip(r / r1, 0.0, 1.0 - 1e-12)
    return np.where(r < r1, np.exp(1.0 - 1.0 / (1.0 - t * t)), 0.0)


@pytest.mark.parametrize("boxes", [[], [[5, 5, 10, 10]]], ids=["uniform", "two-level"])
def test_angular_momentum_conserved_without_limiter(boxes):
    """Sec. 2.6: unlimited DG (k >= 1) with a central field conserves the
    total angular momentum of a state at rest near the boundary to rounding"""
    from paper_1506_06140_gb300 import dg
    n, k = 16, 2
    m = wl.mesh_uniform(2, [n, n], [0.0, 0.0], [6.0, 6.0])
    m["refine_boxes"] = boxes
    s = dg.Solver(m, k, GAMMA, rk_order=3)
    xyz = s.quad_points().cpu().numpy()
    x, y = xyz[0] - 3.0, xyz[1] - 3.0
    r = np.hypot(x, y)
    w = 0.9 * bump(r, 2.2) / (r * r + EPS * EPS) ** 0.75
    U = wl.conserved(1.0 + 0.8 * bump(r, 2.0), [-y * w, x * w], np.ones_like(r), GAMMA)
    W = s.project(torch.as_tensor(U))
    # central, and zero beyond r = 2.6 so that the background stays at rest
    # near the periodic boundary (where x' and y' jump)
    s.set_gravity(torch.as_tensor(plummer(xyz, 3.0) * bump(r, 2.6)[None]))
    centres = xyz.mean(axis=1)
    dx = 6.0 / n / (1 + s.levels())
    L0 = angular_momentum(W.cpu().numpy(), centres, dx)
    for _ in range(10):
        s.rk_step(W)
    assert s.status() == 0
    L1 = angular_momentum(W.cpu().numpy(), centres, dx)
    assert abs(L1 - L0) < 1e-13 * abs(L0), (L0, L1)


def test_regrid_drops_the_field_and_unsupported_precisions_refuse():
    from paper_1506_06140_gb300 import dg
    s, _ = make(2, [8, 8], 2, [])
    s.set_gravity(torch.as_tensor(plummer(s.quad_points().cpu().numpy(), 1.0)))
    W = torch.as_tensor(wl.random_weights(2, s.N, s.n_cells, seed=1), device="cuda")
    s.set_refinement(np.eye(8, dtype=np.int32).reshape(-1))
    W = s.regrid(W)
    with pytest.raises(dg.DGError):
        s.rk_step(W, 1e-4)
    s.set_gravity(torch.as_tensor(plummer(s.quad_points().cpu().numpy(), 1.0)))
    s.rk_step(W, 1e-4)
    for precision in ("mixed", "fp32_tc"):
        t, _ = make(2, [8, 8], 2, [], precision)
        with pytest.raises(dg.DGError):
            t.set_gravity(torch.as_tensor(plummer(t.quad_points().cpu().numpy(), 1.0)))
