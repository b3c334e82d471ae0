"""Checkpoint and resume (Solver.save_checkpoint / Solver.from_checkpoint):
a run resumed from a checkpoint continues bit for bit as the run that wrote
it, on an adapted two-level mesh (the refinement is part of the checkpoint),
for an ensemble and for the FP64-state mixed mode."""
import numpy as np
import pytest
import torch

from paper_1506_06140_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1506_06140_gb300 import build
    build.build()


def dg_mod():
    from paper_1506_06140_gb300 import dg
    return dg


def steps_with_adaptation(s, W, n):
    """RK steps, each followed by an adaptation whose small threshold keeps
    refining wherever the density has a slope (both runs take the same path)."""
    for _ in range(n):
        s.rk_step(W)
        W, _ = s.adapt(W, w_t=1e-7)
    return W


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adaptive_run_resumes_bit_for_bit(tmp_path, precision):
    dg = dg_mod()
    m = wl.mesh_uniform(2, [16, 16], [0.0, 0.0], [1.0, 1.0])
    s = dg.Solver(m, 2, 1.4, rk_order=3, limiter="characteristic", positivity=True, precision=precision)
    W = s.project(torch.as_tensor(wl.kelvin_helmholtz(s.quad_points().cpu().numpy())))
    s.limit(W)
    # a refined band across the shear layers (69 of 256 base cells) and steps
    # on it; the checkpoint holds this mesh, the continuation adapts it
    flags = np.zeros((16, 16), np.int32)
    flags[3:6, :] = 1
    flags[10:13, 2:9] = 1
    s.set_refinement(flags.reshape(-1))
    W = s.regrid(W)
    for _ in range(3):
        s.rk_step(W)
    assert s.n_cells == 256 + 3 * 69
    path = tmp_path / "run.npz"
    s.save_checkpoint(path, W, t=0.125, step=3)
    ref_mesh, ref_nbr = s.refinement().copy(), s.neighbor_table()
    W_ref = steps_with_adaptation(s, W.clone(), 4)
    r, W2, meta = dg.Solver.from_checkpoint(path)
    assert meta == {"t": 0.125, "step": 3}
    np.testing.assert_array_equal(r.refinement(), ref_mesh)
    np.testing.assert_array_equal(r.neighbor_table(), ref_nbr)
    np.testing.assert_array_equal(W2.cpu().numpy(), W.cpu().numpy())
    W2 = steps_with_adaptation(r, W2, 4)
    np.testing.assert_array_equal(r.refinement(), s.refinement())
    np.testing.assert_array_equal(W2.cpu().numpy(), W_ref.cpu().numpy())
    assert r.status() == 0


def test_ensemble_resumes_bit_for_bit(tmp_path):
    dg = dg_mod()
    meshes = [wl.mesh_uniform(2, [n, n], [-5.0, -5.0], [5.0, 5.0]) for n in (12, 20, 9)]
    s = dg.Solver(meshes, 2, 1.4, rk_order=3, precision="fp32")
    W = torch.as_tensor(wl.random_weights(2, s.N, s.n_cells, seed=2300), dtype=s.dtype, device="cuda")
    s.advance(W, 2)
    s.save_checkpoint(tmp_path / "ens.npz", W, step=2)
    W_ref = W.clone()
    s.advance(W_ref, 3)
    r, W2, meta = dg.Solver.from_checkpoint(tmp_path / "ens.npz")
    assert meta == {"step": 2} and r.batch and r.n_problems == 3 and W2.dtype == torch.float32
    r.advance(W2, 3)
    np.testing.assert_array_equal(W2.cpu().numpy(), W_ref.cpu().numpy())
