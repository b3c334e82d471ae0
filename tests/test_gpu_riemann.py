"""Shock-tube runs through the CUDA path with the characteristic TVB limiter
and the positivity limiter (Secs. 3.3, 3.4, 5.2), against the exact Riemann
solution and against the oracle's run of the same scheme.

* Sod along x and y of a 2D strip and along z of a 3D strip: the three
  characteristic decompositions of Appendix E (R_x, R_y, R_z) each decide the
  limiting once; mean density within 1% (L1) of the exact solution, the shock
  within two cells, and the FP64 run within 1e-10 (L1 of the cell-mean
  density; every limiter decision the same) of the oracle's run.
* The double rarefaction (u = -2 | +2): near-vacuum in the middle, where the
  positivity limiter acts and every cell mean keeps a positive density and
  pressure (the device status flag stays clear).
"""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O
from paper_1506_06140_gb300 import workloads as wl
from exact_riemann import density_profile

pytestmark = pytest.mark.gpu
GAMMA = 1.4
T_SOD = 0.228


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1506_06140_gb300 import build
    build.build()


def strip(dim, axis, n):
    """n cells along `axis`, one cell across; transmissive along the strip."""
    cells = [1] * dim
    cells[axis] = n
    hi = [1.0 / n] * dim
    hi[axis] = 1.0
    bc = [wl.BC_PERIODIC] * dim
    bc[axis] = wl.BC_TRANSMISSIVE
    return wl.mesh_uniform(dim, cells, [0.0] * dim, hi, bc=bc)


def riemann_state(xyz, axis, left, right, x0=0.5):
    """conserved state of a Riemann problem across x_axis = x0 (left/right = rho, u, p)"""
    x = xyz[axis]
    lo = x < x0
    rho = np.where(lo, left[0], right[0])
    p = np.where(lo, left[2], right[2])
    vel = [np.zeros_like(rho) for _ in range(len(xyz))]
    vel[axis] = np.where(lo, left[1], right[1])
    return wl.conserved(rho, vel, p, GAMMA)


def run_gpu(s, W, t_end):
    t = 0.0
    dt_buf = s.scalar()
    while t < t_end - 1e-14:
        s.compute_dt(W, dt_buf)
        dt = min(dt_buf.item(), t_end - t)
        s.rk_step(W, dt)
        t += dt
    return W


def run_oracle(o, W, t_end):
    t = 0.0
    while t < t_end - 1e-14:
        dt = min(o.compute_dt(W), t_end - t)
        W, _ = o.rk_step(W, dt)
        t += dt
    return W


@pytest.mark.parametrize("dim,axis", [(2, 0), (2, 1), (3, 2)], ids=["2d-x", "2d-y", "3d-z"])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_sod_shock_tube(dim, axis, precision):
    from paper_1506_06140_gb300 import dg
    n, k = 96, 2
    m = strip(dim, axis, n)
    left, right = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    s = dg.Solver(m, k, GAMMA, rk_order=3, limiter="characteristic", positivity=True,
                  precision=precision)
    U = riemann_state(s.quad_points().cpu().numpy(), axis, left, right)
    W = s.project(torch.as_tensor(U))
    s.limit(W)
    W = run_gpu(s, W, T_SOD)
    assert s.status() == 0
    rho = W[0, 0].double().cpu().numpy()
    x = s.quad_points()[axis].mean(dim=0).cpu().numpy()
    err = np.abs(rho - density_profile(x, T_SOD)).mean()
    print("sod %dD axis %d %s: L1 %.3e" % (dim, axis, precision, err))
    assert err < 0.01, err
    xs = 0.5 + 1.75216 * T_SOD
    jump = x[np.argmin(np.diff(rho)) + 1]
    assert abs(jump - xs) < 2.0 / n
    assert np.all(rho > 0)
    if precision == "fp64":
        o = O.Oracle(m["dim"], m["n"], m["lo"], m["hi"], k, GAMMA, bc=m["bc"], rk_order=3,
                     limiter=O.LIM_CHARACTERISTIC, positivity=True)
        Wo = o.limit(o.project(riemann_state(o.quad_points(), axis, left, right)))
        Wo = run_oracle(o, Wo, T_SOD)
        d = np.abs(Wo[0, 0] - rho).mean()
        print("fp64 vs oracle L1 of cell means: %.3e" % d)
        assert d < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_double_rarefaction_stays_positive(precision):
    from paper_1506_06140_gb300 import dg
    n, k, t_end = 128, 2, 0.15
    m = strip(2, 0, n)
    left, right = (1.0, -2.0, 0.4), (1.0, 2.0, 0.4)
    s = dg.Solver(m, k, GAMMA, rk_order=3, limiter="characteristic", positivity=True,
                  precision=precision)
    U = riemann_state(s.quad_points().cpu().numpy(), 0, left, right)
    W = s.project(torch.as_tensor(U))
    s.limit(W)
    W = run_gpu(s, W, t_end)
    assert s.status() == 0
    Wh = W.double().cpu().numpy()
    rho_mean = Wh[0, 0]
    assert np.all(rho_mean > 0)
    x = s.quad_points()[0].mean(dim=0).cpu().numpy()
    err = np.abs(rho_mean - density_profile(x, t_end, left=left, right=right)).mean()
    print("double rarefaction %s: L1 %.3e" % (precision, err))
    assert err < 0.02, err
    counts = s.limiter_counts().cpu().numpy()
    assert counts[1] > 0  # the positivity limiter acted near the vacuum


@pytest.mark.parametrize("dim,axis", [(2, 0), (3, 1)], ids=["2d-x", "3d-y"])
def test_sod_component_limiter_matches_oracle(dim, axis):
    """The component-wise variant of the slope limiter (Sec. 3.2): same run,
    same bars, FP64 against the oracle."""
    from paper_1506_06140_gb300 import dg
    n, k = 96, 2
    m = strip(dim, axis, n)
    left, right = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    s = dg.Solver(m, k, GAMMA, rk_order=3, limiter="component", positivity=True)
    W = s.project(torch.as_tensor(riemann_state(s.quad_points().cpu().numpy(), axis, left, right)))
    s.limit(W)
    W = run_gpu(s, W, T_SOD)
    rho = W[0, 0].cpu().numpy()
    x = s.quad_points()[axis].mean(dim=0).cpu().numpy()
    err = np.abs(rho - density_profile(x, T_SOD)).mean()
    print("sod component limiter %dD: L1 %.3e" % (dim, err))
    assert err < 0.015, err
    o = O.Oracle(m["dim"], m["n"], m["lo"], m["hi"], k, GAMMA, bc=m["bc"], rk_order=3,
                 limiter=O.LIM_COMPONENT, positivity=True)
    Wo = run_oracle(o, o.limit(o.project(riemann_state(o.quad_points(), axis, left, right))), T_SOD)
    assert np.abs(Wo[0, 0] - rho).mean() < 1e-10
