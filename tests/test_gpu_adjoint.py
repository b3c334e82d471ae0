"""The adjoint of one RK step (dg_rk_step_adjoint) and the differentiable
stepping built on it.

* element by element against the oracle's exact transpose J^T lam, with J
  assembled column by column from the oracle's dual-number JVPs (FP64,
  relative 1e-10), on uniform and two-level meshes, RK2/3/4, k=1..3;
* gradients of an L2 density misfit after several steps against central
  finite differences of the forward map (relative 1e-6), on the 3D acoustic
  wave at reduced size.
"""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O
from paper_1506_06140_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
GAMMA = 1.4


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1506_06140_gb300 import build
    build.build()


CASES = [
    ("u2_k1_rk2", wl.mesh_uniform(2, [4, 3], [0.0, 0.0], [4 / 3.0, 1.0]), 1, 2),
    ("u2_k3_rk4", wl.mesh_uniform(2, [3, 3], [0.0, 0.0], [1.0, 1.0]), 3, 4),
    ("u2t_k2_rk3", wl.mesh_uniform(2, [5, 2], [0.0, 0.0], [1.0, 0.4], bc=[1, 0]), 2, 3),
    ("amr2_k2_rk3", dict(wl.mesh_uniform(2, [4, 4], [0.0, 0.0], [1.0, 1.0]),
                         refine_boxes=[[1, 1, 1, 2]]), 2, 3),
    ("u3_k2_rk3", wl.mesh_uniform(3, [2, 2, 3], [0.0] * 3, [2 / 3.0, 2 / 3.0, 1.0]), 2, 3),
    ("amr3_k1_rk3", dict(wl.mesh_uniform(3, [3, 2, 2], [0.0] * 3, [1.5, 1.0, 1.0]),
                         refine_boxes=[[1, 0, 0, 1, 0, 0]]), 1, 3),
]


@pytest.mark.parametrize("name,mesh,k,rk", CASES, ids=[c[0] for c in CASES])
def test_adjoint_equals_oracle_transpose(name, mesh, k, rk):
    from paper_1506_06140_gb300 import dg
    o = O.Oracle(mesh["dim"], mesh["n"], mesh["lo"], mesh["hi"], k, GAMMA, bc=mesh["bc"],
                 refine_boxes=mesh["refine_boxes"], rk_order=rk)
    s = dg.Solver(mesh, k, GAMMA, rk_order=rk)
    W = wl.random_weights(mesh["dim"], o.N, o.n_cells, seed=17, slope=0.08)
    lam = np.random.default_rng(5).normal(size=o.shape)
    dt = 0.6 * o.compute_dt(W)
    # J^T lam from the oracle's JVP columns
    ref = np.zeros(W.size)
    for i in range(W.size):
        e = np.zeros(W.size)
        e[i] = 1.0
        _, JV = o.rk_step_jvp(W, e.reshape(o.shape), dt)
        ref[i] = np.dot(JV.ravel(), lam.ravel())
    ref = ref.reshape(o.shape)
    got = s.rk_step_adjoint(torch.as_tensor(W, device="cuda"), dt,
                            torch.as_tensor(lam, device="cuda")).cpu().numpy()
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err < 1e-10, err


def test_adjoint_in_place_and_repeatable():
    from paper_1506_06140_gb300 import dg
    m = wl.mesh_uniform(2, [9, 7], [0.0, 0.0], [9 / 7.0, 1.0])
    s = dg.Solver(m, 2, GAMMA, rk_order=3)
    W = torch.as_tensor(wl.random_weights(2, s.N, s.n_cells, seed=3), device="cuda")
    lam = torch.randn_like(W)
    a = s.rk_step_adjoint(W, 1e-3, lam)
    b = s.rk_step_adjoint(W, 1e-3, lam)
    c = lam.clone()
    s.rk_step_adjoint(W, 1e-3, c, out=c)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(a, c)


def test_adjoint_rejects_limited_handles_and_bad_dt():
    from paper_1506_06140_gb300 import dg
    m = wl.mesh_uniform(2, [4, 4], [0.0, 0.0], [1.0, 1.0])
    s = dg.Solver(m, 1, GAMMA, limiter="characteristic")
    W = torch.as_tensor(wl.random_weights(2, s.N, s.n_cells, seed=3), device="cuda")
    with pytest.raises(dg.DGError):
        s.rk_step_adjoint(W, 1e-3, W.clone())
    s2 = dg.Solver(m, 1, GAMMA)
    with pytest.raises(dg.DGError):
        s2.rk_step_adjoint(W, 0.0, W.clone())


def misfit_setup(n=8, k=2, steps=6, seed=1506062, vel=(0.3, 0.2, 0.1)):
    """Acoustic wave (rho = 1 + 1e-3 sin sin sin, p = 1/gamma) carried by a
    uniform flow, and an L2 density misfit
    J = 1/2 sum_K |K| sum_j (w_rho,j - w_target,j)^2.  The flow keeps the HLLC
    contact speed away from 0, where the flux is only piecewise smooth and a
    finite difference would straddle the kink."""
    from paper_1506_06140_gb300 import dg
    m = wl.mesh_uniform(3, [n] * 3, [0.0] * 3, [1.0] * 3)
    s = dg.Solver(m, k, GAMMA, rk_order=3)
    U = wl.acoustic3d(s.quad_points().cpu().numpy(), vel=vel)
    W0 = s.project(torch.as_tensor(U))
    dt = s.compute_dt(W0).item()
    rng = np.random.default_rng(seed)
    target = W0[0].clone() + torch.as_tensor(1e-4 * rng.normal(size=tuple(W0[0].shape)),
                                             device="cuda")
    vol = (1.0 / n) ** 3
    return s, W0, dt, steps, target, vol


def test_gradient_matches_central_differences():
    from paper_1506_06140_gb300.autograd import rk_steps
    s, W0, dt, steps, target, vol = misfit_setup()

    def J(W):
        WN = rk_steps(W, s, steps, dt)
        return 0.5 * vol * ((WN[0] - target) ** 2).sum()

    W = W0.clone().requires_grad_(True)
    val = J(W)
    val.backward()
    g = W.grad.detach()
    rng = np.random.default_rng(1506063)
    v = torch.as_tensor(rng.normal(size=tuple(W0.shape)), device="cuda")
    v = v / v.norm()
    dJ = (g * v).sum().item()
    best = None
    with torch.no_grad():
        for rel in (1e-3, 1e-4, 1e-5):
            eps = rel * W0.abs().max().item()
            fd = (J(W0 + eps * v).item() - J(W0 - eps * v).item()) / (2 * eps)
            e = abs(fd - dJ) / abs(dJ)
            best = e if best is None else min(best, e)
    assert best < 1e-6, best
