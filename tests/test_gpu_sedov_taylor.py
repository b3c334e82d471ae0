"""The Sedov-Taylor blast of Sec. 5.3 through the CUDA path: uniform gas
(rho = 1, p = 1e-6, gamma = 5/3) at rest in [0,1]^3, thermal energy E = 1 in
the eight central cells, characteristic TVB and positivity limiters.  The
self-similar shock radius is R(t) = R_0 (E t^2 / rho)^(1/5) with R_0 ~ 1.152
for gamma = 5/3 in 3D, the value the paper prints; at t = 0.05 that is
0.3477.  On 32^3 cells the front (the outermost radius where the spherically
averaged density crosses half of its peak rise) lies within 1.5 cells of it
for DG-2 and DG-3, the peak compression stays below the analytic 4, and
mass and energy are conserved.  The state is FP64 (DG-2) or FP64 with the
FP32 perturbation-form right-hand side (DG-3): near the blast's vacuum-like
centre, weights rounded to FP32 move point values by ~1e-7 of the weights,
more than the positivity limiter's eps = 1e-10, and an FP32 state breaks
down after a few hundred steps."""
import numpy as np
import pytest
import torch

import golden_values
from paper_1506_06140_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
GAMMA = 5.0 / 3.0
R0 = golden_values.validation_figures()["sedov_taylor_R0"]  # Sec. 5.3
T_END = 0.05


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1506_06140_gb300 import build
    build.build()


def run_to(s, W, t_end, chunk=200):
    """CFL steps to t_end: graph-recorded chunks while they fit, then single steps"""
    t, hist = 0.0, s.dt_buffer(chunk)
    last = 0.0
    while t + 1.5 * chunk * last < t_end:
        s.advance(W, chunk, hist)
        h = hist.cpu().numpy()
        t += h.sum()
        last = h[-1]
    dt_buf = s.scalar()
    while t < t_end - 1e-15:
        s.compute_dt(W, dt_buf)
        dt = min(dt_buf.item(), t_end - t)
        s.rk_step(W, dt)
        t += dt
    return t


def front_radius(s, W, n):
    c = s.quad_points().mean(dim=1).cpu().numpy()
    r = np.sqrt(((c - 0.5) ** 2).sum(axis=0))
    rho = W[0, 0].double().cpu().numpy()
    dr = 0.5 / n
    b = (r / dr).astype(int)
    prof = np.bincount(b, weights=rho) / np.maximum(np.bincount(b), 1)
    rc = (np.arange(len(prof)) + 0.5) * dr
    ip = int(np.argmax(prof))
    half = 1.0 + 0.5 * (prof[ip] - 1.0)
    out = ip + int(np.argmax(prof[ip:] < half))  # first bin outside the peak below half the rise
    return rc[out - 1] + dr * (prof[out - 1] - half) / (prof[out - 1] - prof[out]), prof[ip]


@pytest.mark.parametrize("k,rk,precision", [(1, 2, "fp64"), (2, 3, "mixed"), (1, 2, "fp32")],
                         ids=["DG-2", "DG-3", "DG-2-fp32"])
def test_sedov_taylor_shock_radius(k, rk, precision):
    from paper_1506_06140_gb300 import dg
    n = 32
    m = wl.mesh_uniform(3, [n] * 3, [0.0] * 3, [1.0] * 3, bc=[wl.BC_TRANSMISSIVE] * 3)
    s = dg.Solver(m, k, GAMMA, rk_order=rk, limiter="characteristic", positivity=True, precision=precision)
    U = wl.sedov3d(s.quad_points().cpu().numpy(), gamma=GAMMA, p0=1e-6, energy=1.0, half_width=1.0 / n)
    W = s.project(torch.as_tensor(U))
    s.limit(W)
    tot0 = s.totals(W).cpu().numpy()
    t = run_to(s, W, T_END)
    assert s.status() == 0 and abs(t - T_END) < 1e-12
    R, peak = front_radius(s, W, n)
    R_exact = R0 * (1.0 * T_END ** 2 / 1.0) ** 0.2
    print("DG-%d %d^3: front %.4f, analytic %.4f, peak compression %.2f" % (k + 1, n, R, R_exact, peak))
    assert abs(R - R_exact) < 1.5 / n
    assert 1.5 < peak < 4.0
    tot1 = s.totals(W).cpu().numpy()
    # FP64 conserves to rounding; the perturbation-form right-hand side to the
    # FP32 rounding of its face-flux differences
    tol = {"fp64": 1e-10, "mixed": 1e-7, "fp32": 1e-5}[precision]
    assert abs(tot1[0] - tot0[0]) < tol * tot0[0] and abs(tot1[-1] - tot0[-1]) < tol * tot0[-1]
