"""Mixed precision (FP64 state, FP32 right-hand side in perturbation form)
against the FP64 oracle.

The perturbation form leaves the discrete right-hand side unchanged (the
volume and surface integrals of a cell's constant reference flux cancel
exactly under the Gauss rules), so the oracle's FP64 RHS is the reference.
What changes is the size of the FP32 rounding: it scales with the variation
of the solution across a cell and its neighbours instead of with the fluxes.
On random states (cell means drawn independently, jumps of O(1) between
neighbours) that is no gain, and the FP32 bar of the plain FP32 kernels
applies.  On the smooth 256^2 vortex, where the plain FP32 RHS loses ~1e-4
of max |dW/dt| to cancellation, the mixed RHS must be an order of magnitude
closer to the oracle.
"""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O
from paper_1506_06140_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

GAMMA = 1.4
TOL32_MAX, TOL32_RMS = 2e-5, 2e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1506_06140_gb300 import build
    build.build()


MESHES = {
    "u2": wl.mesh_uniform(2, [37, 29], [0.0, 0.0], [37 / 29.0, 1.0]),
    "u2t": wl.mesh_uniform(2, [23, 3], [0.0, 0.0], [1.0, 3 / 23.0], bc=[1, 0]),
    "amr2": dict(wl.mesh_uniform(2, [16, 12], [0.0, 0.0], [4 / 3.0, 1.0]),
                 refine_boxes=[[4, 3, 9, 7], [13, 0, 15, 1]]),
    "u3": wl.mesh_uniform(3, [7, 6, 5], [0.0, 0.0, 0.0], [7 / 6.0, 1.0, 5 / 6.0]),
    "amr3": dict(wl.mesh_uniform(3, [6, 6, 6], [0.0] * 3, [1.0] * 3), refine_boxes=[[2, 2, 1, 3, 4, 3]]),
    "amr3t": dict(wl.mesh_uniform(3, [5, 4, 4], [0.0] * 3, [1.25, 1.0, 1.0], bc=[1, 0, 1]),
                  refine_boxes=[[0, 1, 1, 1, 2, 2]]),
}


def oracle_for(mesh, k, **kw):
    return O.Oracle(mesh["dim"], mesh["n"], mesh["lo"], mesh["hi"], k, GAMMA, bc=mesh["bc"],
                    refine_boxes=mesh["refine_boxes"], **kw)


def solver_for(mesh, k, **kw):
    from paper_1506_06140_gb300 import dg
    return dg.Solver(mesh, k, GAMMA, **kw)


def dev(W):
    return torch.as_tensor(W, dtype=torch.float64, device="cuda").contiguous()


def rel_err(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    scale = max(np.max(np.abs(b)), 1e-300)
    return np.max(np.abs(a - b)) / scale, np.sqrt(np.mean((a - b) ** 2)) / scale


@pytest.mark.parametrize("name", list(MESHES))
def test_rhs_mixed_random_states(name):
    m = MESHES[name]
    for k in ((0, 1, 2, 3) if m["dim"] == 2 else (0, 1, 2)):
        o = oracle_for(m, k)
        s = solver_for(m, k, precision="mixed")
        assert s.dtype == torch.float64
        W = wl.random_weights(m["dim"], o.N, o.n_cells, seed=1200 + k)
        ref = o.rhs(W)
        got = s.rhs(dev(W)).cpu().numpy()
        e, erms = rel_err(got, ref)
        assert e < TOL32_MAX and erms < TOL32_RMS, (name, k, e, erms)
        assert s.status() == 0


def test_rhs_mixed_smooth_vortex_full_size():
    """256^2 vortex, k=3: plain FP32 and mixed against the oracle."""
    m = wl.mesh_uniform(2, [256, 256], [-5.0, -5.0], [5.0, 5.0])
    o = oracle_for(m, 3)
    U = wl.vortex(o.quad_points())
    W = o.project(U)
    ref = o.rhs(W)
    s32 = solver_for(m, 3, precision="fp32")
    e32, r32 = rel_err(s32.rhs(torch.as_tensor(W, dtype=torch.float32, device="cuda")).cpu().numpy(), ref)
    smx = solver_for(m, 3, precision="mixed")
    emx, rmx = rel_err(smx.rhs(dev(W)).cpu().numpy(), ref)
    print("fp32 max %.3e rms %.3e | mixed max %.3e rms %.3e" % (e32, r32, emx, rmx))
    # perturbations ~ dx |grad u| ~ 0.04 against fluxes ~ 2: the cancellation
    # factor pre |df| |dphi| / |dW/dt| drops from ~1.4e3 to ~20, so FP32
    # rounding (6e-8) times it and the ~50 terms of a sum stays below 1e-5
    assert emx < 1e-5 and rmx < 3e-7, (emx, rmx)
    assert emx < 0.02 * e32 and rmx < 0.02 * r32, (emx, e32, rmx, r32)


def test_rhs_mixed_smooth_acoustic_3d():
    """32^3 acoustic wave with a uniform flow, k=2: perturbations are small,
    the fluxes are not."""
    m = wl.mesh_uniform(3, [32, 32, 32], [0.0] * 3, [1.0] * 3)
    o = oracle_for(m, 2)
    U = wl.acoustic3d(o.quad_points(), amp=1e-2, vel=(0.5, -0.3, 0.2))
    W = o.project(U)
    ref = o.rhs(W)
    s32 = solver_for(m, 2, precision="fp32")
    e32, r32 = rel_err(s32.rhs(torch.as_tensor(W, dtype=torch.float32, device="cuda")).cpu().numpy(), ref)
    smx = solver_for(m, 2, precision="mixed")
    emx, rmx = rel_err(smx.rhs(dev(W)).cpu().numpy(), ref)
    print("fp32 max %.3e rms %.3e | mixed max %.3e rms %.3e" % (e32, r32, emx, rmx))
    assert emx < 1e-5 and rmx < 3e-7, (emx, rmx)
    assert emx < 0.02 * e32, (emx, e32)


@pytest.mark.parametrize("order", [2, 3, 4])
@pytest.mark.parametrize("name", ["u2", "amr3"])
def test_rk_step_mixed(order, name):
    m = MESHES[name]
    k = min(order - 1, 2) if m["dim"] == 3 else order - 1
    o = oracle_for(m, k, rk_order=order)
    s = solver_for(m, k, rk_order=order, precision="mixed")
    W = wl.random_weights(m["dim"], o.N, o.n_cells, seed=1300 + order)
    dt = 0.5 * o.compute_dt(W)
    ref, _ = o.rk_step(W, dt)
    Wd = dev(W)
    s.rk_step(Wd, dt)
    got = Wd.cpu().numpy()
    # the increment carries the FP32 RHS error; the state itself stays FP64
    e, _ = rel_err(got - W, ref - W)
    assert e < 1e-4, (order, name, e)
    assert np.max(np.abs(got - ref)) < 1e-6 * np.max(np.abs(ref))


def test_limited_rk3_step_mixed():
    m = MESHES["amr3"]
    o = oracle_for(m, 2, rk_order=3, limiter=O.LIM_CHARACTERISTIC, positivity=True)
    s = solver_for(m, 2, rk_order=3, limiter="characteristic", positivity=True, precision="mixed")
    rng = np.random.default_rng(1400)
    W = wl.random_weights(3, o.N, o.n_cells, seed=1401, slope=0.3)
    W[:, 1:, rng.random(o.n_cells) < 0.3] *= 4.0
    W = o.limit(W)
    dt = o.compute_dt(W)
    ref, _ = o.rk_step(W, dt)
    Wd = dev(W)
    s.rk_step(Wd, dt)
    got = Wd.cpu().numpy()
    assert np.max(np.abs(got - ref)) < 1e-5 * np.max(np.abs(ref))
    assert s.status() == 0


def test_mixed_advance_graph_equals_steps():
    m = MESHES["amr2"]
    s = solver_for(m, 2, rk_order=3, precision="mixed")
    W = dev(wl.random_weights(2, s.N, s.n_cells, seed=1500))
    W2 = W.clone()
    hist = s.scalar(4)
    s.advance(W, 4, hist)
    for _ in range(4):
        s.rk_step(W2, 0.0)
    torch.cuda.synchronize()
    assert torch.equal(W, W2)


def test_mixed_batch_matches_problems_alone():
    problems = [(8, 5.0), (12, 3.5), (6, 6.0)]
    meshes = [wl.mesh_uniform(2, [n, n], [-5.0, -5.0], [5.0, 5.0]) for n, _ in problems]
    sb = solver_for(meshes, 2, rk_order=3, precision="mixed")
    xyz = sb.quad_points().cpu().numpy()
    U = np.empty((sb.nv, sb.nq, sb.n_cells))
    for p, (n, beta) in enumerate(problems):
        a, b = sb.cell_offsets[p], sb.cell_offsets[p + 1]
        U[:, :, a:b] = wl.vortex(xyz[:, :, a:b], beta=beta)
    W = sb.project(torch.as_tensor(U))
    dW = sb.rhs(W).cpu().numpy()
    for p, (n, beta) in enumerate(problems):
        a, b = sb.cell_offsets[p], sb.cell_offsets[p + 1]
        s1 = solver_for(meshes[p], 2, rk_order=3, precision="mixed")
        Wp = W[:, :, a:b].contiguous()
        assert np.array_equal(s1.rhs(Wp).cpu().numpy(), dW[:, :, a:b])


def test_mixed_adjoint_close_to_fp64():
    """The adjoint of a mixed handle recomputes its stage states with the
    mixed forward kernels and applies the FP64 stage adjoint: it differs from
    the FP64 handle's adjoint only through the FP32 right-hand side."""
    m = MESHES["u2"]
    s = solver_for(m, 1, rk_order=2, precision="mixed")
    s64 = solver_for(m, 1, rk_order=2)
    W = dev(wl.random_weights(2, s.N, s.n_cells, seed=1600))
    lam = dev(wl.random_weights(2, s.N, s.n_cells, seed=1601))
    dt = 0.5 * s64.compute_dt(W).item()
    a = s.rk_step_adjoint(W, dt, lam).cpu().numpy()
    b = s64.rk_step_adjoint(W, dt, lam).cpu().numpy()
    e, _ = rel_err(a - lam.cpu().numpy(), b - lam.cpu().numpy())
    assert e < 1e-4, e


# ---------------------------------------------------------------------------
# DG_MIXED_TC: the same scheme with the cell kernel's contractions on the
# tensor cores (split TF32 products, FP32 accumulation)

@pytest.mark.parametrize("k", [1, 2, 3])
def test_rhs_mixed_tc_random_states(k):
    for name in ("u2", "u2t"):
        m = MESHES[name]
        o = oracle_for(m, k)
        s = solver_for(m, k, precision="mixed_tc")
        W = wl.random_weights(2, o.N, o.n_cells, seed=1700 + k)
        ref = o.rhs(W)
        e, erms = rel_err(s.rhs(dev(W)).cpu().numpy(), ref)
        assert e < TOL32_MAX and erms < TOL32_RMS, (name, k, e, erms)
        assert s.status() == 0


def test_rhs_mixed_tc_smooth_vortex_full_size():
    m = wl.mesh_uniform(2, [256, 256], [-5.0, -5.0], [5.0, 5.0])
    o = oracle_for(m, 3)
    W = o.project(wl.vortex(o.quad_points()))
    ref = o.rhs(W)
    s = solver_for(m, 3, precision="mixed_tc")
    e, erms = rel_err(s.rhs(dev(W)).cpu().numpy(), ref)
    print("mixed_tc max %.3e rms %.3e" % (e, erms))
    assert e < 1e-5 and erms < 3e-7, (e, erms)


@pytest.mark.parametrize("order", [3, 4])
def test_rk_step_mixed_tc_matches_mixed(order):
    """Delta-register steps: the tensor-core and SIMT mixed kernels agree to
    the FP32 rounding of the right-hand side."""
    m = MESHES["u2"]
    k = order - 1
    o = oracle_for(m, k, rk_order=order)
    W = o.project(wl.wave2d(o.quad_points(), amp=0.1))
    dt = 0.5 * o.compute_dt(W)
    ref, _ = o.rk_step(W, dt)
    for prec in ("mixed", "mixed_tc"):
        s = solver_for(m, k, rk_order=order, precision=prec)
        Wd = dev(W)
        s.rk_step(Wd, dt)
        got = Wd.cpu().numpy()
        e, _ = rel_err(got - W, ref - W)
        assert e < 1e-4, (prec, e)
        assert s.status() == 0


def test_mixed_tc_advance_graph_and_rejections():
    from paper_1506_06140_gb300 import dg
    m = wl.mesh_uniform(2, [150, 131], [0.0, 0.0], [1.5, 1.31])  # ragged last tile, many tiles
    s = solver_for(m, 3, rk_order=4, precision="mixed_tc")
    W = dev(wl.random_weights(2, s.N, s.n_cells, seed=1800))
    W2 = W.clone()
    s.advance(W, 3)
    for _ in range(3):
        s.rk_step(W2)
    torch.cuda.synchronize()
    assert torch.equal(W, W2)
    with pytest.raises(dg.DGError):
        solver_for(MESHES["amr2"], 2, precision="mixed_tc")
    with pytest.raises(dg.DGError):
        solver_for(MESHES["u3"], 2, precision="mixed_tc")
