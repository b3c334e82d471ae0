"""Ensembles of independent problems in one handle (dg_create_batch).

Each problem of the batch must evolve exactly as it would alone: its RHS,
its own CFL timestep and its RK steps are compared with the oracle run on
that problem separately.  The full workload -- 512 vortices with sizes drawn
from {32,48,64,96,128}^2, strengths U(3,6), k=2, SSP-RK3, FP32 -- is checked
on a 4-problem subset.
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


def vortex_mesh(n):
    return wl.mesh_uniform(2, [n, n], [-5.0, -5.0], [5.0, 5.0])


def batch_state(s, problems):
    xyz = s.quad_points().cpu().numpy()
    U = np.empty((s.nv, s.nq, s.n_cells))
    for p, (n, beta) in enumerate(problems):
        a, b = s.cell_offsets[p], s.cell_offsets[p + 1]
        U[:, :, a:b] = wl.vortex(xyz[:, :, a:b], beta=beta)
    return U


def test_batch_matches_problems_run_alone_fp64():
    from paper_1506_06140_gb300 import dg
    problems = [(8, 5.0), (12, 3.5), (6, 6.0), (10, 4.2)]
    s = dg.Solver([vortex_mesh(n) for n, _ in problems], 2, GAMMA, rk_order=3)
    assert s.n_problems == 4
    assert list(np.diff(s.cell_offsets)) == [n * n for n, _ in problems]
    U = batch_state(s, problems)
    W = s.project(torch.as_tensor(U))
    dW = s.rhs(W).cpu().numpy()
    dts = s.compute_dt(W).cpu().numpy()
    W1 = W.clone()
    dt_used = s.dt_buffer()
    s.rk_step(W1, 0.0, dt_used)
    W0h, W1h = W.cpu().numpy(), W1.cpu().numpy()
    for p, (n, beta) in enumerate(problems):
        a, b = s.cell_offsets[p], s.cell_offsets[p + 1]
        m = vortex_mesh(n)
        o = O.Oracle(2, m["n"], m["lo"], m["hi"], 2, GAMMA, rk_order=3)
        Wp = o.project(wl.vortex(o.quad_points(), beta=beta))
        np.testing.assert_allclose(W0h[:, :, a:b], Wp, rtol=0, atol=1e-14 * np.abs(Wp).max())
        ref = o.rhs(Wp)
        assert np.max(np.abs(dW[:, :, a:b] - ref)) < 1e-11 * np.max(np.abs(ref))
        dtp = o.compute_dt(Wp)
        assert dts[p] == pytest.approx(dtp, rel=1e-14)
        assert dt_used.cpu().numpy()[p] == pytest.approx(dtp, rel=1e-14)
        ref1, _ = o.rk_step(Wp, dt_used.cpu().numpy()[p])
        d = W1h[:, :, a:b] - Wp
        assert np.max(np.abs(d - (ref1 - Wp))) < 1e-10 * np.max(np.abs(ref1 - Wp))


def test_batch_advance_graph_equals_steps():
    from paper_1506_06140_gb300 import dg
    problems = [(8, 5.0), (16, 4.0), (4, 3.0)]
    s = dg.Solver([vortex_mesh(n) for n, _ in problems], 1, GAMMA, rk_order=2, precision="fp32")
    W = s.project(torch.as_tensor(batch_state(s, problems)))
    W2 = W.clone()
    hist = s.dt_buffer(6)
    s.advance(W, 6, hist)
    for i in range(6):
        d = s.dt_buffer()
        s.rk_step(W2, 0.0, d)
        assert torch.equal(d, hist[i * 3:(i + 1) * 3])
    torch.cuda.synchronize()
    assert torch.equal(W, W2)


def test_full_ensemble_fp32_subset_vs_oracle():
    """512 problems, 3.4M cells; one RK3 step; 4 problems against the oracle."""
    from paper_1506_06140_gb300 import dg
    problems = wl.ensemble_problems()
    s = dg.Solver([vortex_mesh(n) for n, _ in problems], 2, GAMMA, rk_order=3, precision="fp32")
    assert s.n_problems == 512
    W = s.project(torch.as_tensor(batch_state(s, problems)))
    W0 = W.double().cpu().numpy()
    dt = s.dt_buffer()
    s.advance(W, 1, dt)
    W1 = W.double().cpu().numpy()
    dt = dt.cpu().numpy()
    assert s.status() == 0
    rng = np.random.default_rng(3)
    sizes = np.array([n for n, _ in problems])
    picks = [int(np.nonzero(sizes == n)[0][0]) for n in (32, 128)] + \
        [int(i) for i in rng.choice(len(problems), 2, replace=False)]
    for p in picks:
        n, beta = problems[p]
        a, b = s.cell_offsets[p], s.cell_offsets[p + 1]
        m = vortex_mesh(n)
        o = O.Oracle(2, m["n"], m["lo"], m["hi"], 2, GAMMA, rk_order=3)
        Wp = W0[:, :, a:b]
        assert dt[p] == pytest.approx(o.compute_dt(Wp), rel=1e-6)
        ref, _ = o.rk_step(Wp, dt[p])
        # FP32 state: the new state is rounded to FP32 (ulp/2 ~ 6e-8 |W|); the FP32
        # right-hand side adds ~1e-5 of the increment
        err = np.max(np.abs(W1[:, :, a:b] - ref)) / np.max(np.abs(ref))
        assert err < 1e-6, (p, n, err)
        inc, ref_inc = W1[:, :, a:b] - Wp, ref - Wp
        rms = np.sqrt(np.mean((inc - ref_inc) ** 2)) / np.sqrt(np.mean(ref_inc ** 2))
        assert rms < 1e-2, (p, n, rms)  # gross errors in the increment (dt, prefactor)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_autotuned_tiles_change_no_result(precision):
    """The tiled kernels only regroup cells and faces into thread blocks: with
    any tile a handle steps bit-identically to one with the fixed tiles."""
    from paper_1506_06140_gb300 import dg
    problems = [(24, 5.0), (40, 3.5), (8, 4.5)]
    meshes = [vortex_mesh(n) for n, _ in problems]
    s0 = dg.Solver(meshes, 2, GAMMA, rk_order=3, precision=precision)
    s1 = dg.Solver(meshes, 2, GAMMA, rk_order=3, precision=precision, autotune=True)
    ct, ft = s1.tiles()
    assert ct in ((1, 16, 32, 64) if precision == "fp32" else (16, 32, 64)) and ft in (16, 32, 64)
    assert s0.tiles() == (32, 32)
    W0 = s0.project(torch.as_tensor(batch_state(s0, problems)))
    W1 = W0.clone()
    s0.advance(W0, 3)
    if ct == 1:  # the one-thread-per-cell kernel: same scheme, another summation order
        s1.set_tiles(32, ft)
    s1.advance(W1, 3)
    torch.cuda.synchronize()
    assert torch.equal(W0, W1)
