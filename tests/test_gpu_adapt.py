"""Mesh adaptation through the CUDA path (Secs. 4.1, 4.3-4.5) against the
oracle and against freshly created handles.

* dg_adapt_mark's refinement decision (criterion of eqs. cell_ref / node_ref,
  one buffer layer) equals the oracle's flag for flag, on meshes that already
  hold nodes, periodic and transmissive, 2D and 3D, FP64 and FP32 states.
* dg_regrid builds the mesh tables on the device: after a sequence of
  refinements and derefinements (growing and shrinking the buffers) the
  handle is indistinguishable from one created with the same refinement —
  neighbour table and levels equal, right-hand side, limiter, timestep and a
  graph-recorded advance bit-identical.
* the projected state equals the oracle's adapt_project (copy, refinement
  matrices, transposed merge) to rounding.
* an adaptive run (adaptation after every RK step, as in Sec. 4) follows the
  oracle's run: the same mesh after every step and the same state to 1e-10.
"""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O
from paper_1506_06140_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
WT, ALPHA = 0.01, 1.1


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1506_06140_gb300 import build
    build.build()


def boxes_of(flags, n):
    dim = len(n)
    out = []
    for b in np.nonzero(flags)[0]:
        p = [b % n[0], (b // n[0]) % n[1]] + ([b // (n[0] * n[1])] if dim == 3 else [])
        out.append(p + p)
    return out


def mesh(dim, n, flags=None, bc=wl.BC_PERIODIC):
    m = wl.mesh_uniform(dim, n, [0.0] * dim, [n[a] / n[0] for a in range(dim)], bc=[bc] * dim)
    if flags is not None:
        m["refine_boxes"] = boxes_of(flags, n)
    return m


def solver(m, k=2, precision="fp64", **kw):
    from paper_1506_06140_gb300 import dg
    return dg.Solver(m, k, 1.4, rk_order=3, precision=precision, **kw)


def oracle(m, k=2, **kw):
    return O.Oracle(m["dim"], m["n"], m["lo"], m["hi"], k, 1.4, bc=m["bc"],
                    refine_boxes=m.get("refine_boxes") or [], rk_order=3, **kw)


def steep_state(dim, N, nc, seed, frac=0.08, amp=0.03):
    """smooth random means; density slopes of a fraction of cells spread
    across both thresholds, the rest small"""
    rng = np.random.default_rng(seed)
    W = wl.random_weights(dim, N, nc, seed=seed, slope=0.004, rho_range=(0.995, 1.005))
    steep = rng.random(nc) < frac
    for a in range(dim):
        W[0, 1 + a, steep] = rng.uniform(-amp, amp, steep.sum())
    return W


def random_flags(nb, seed, frac=0.3):
    return (np.random.default_rng(seed).random(nb) < frac).astype(np.int32)


@pytest.mark.parametrize("dim,n", [(2, [12, 10]), (3, [6, 5, 4])], ids=["2d", "3d"])
@pytest.mark.parametrize("bc", [wl.BC_PERIODIC, wl.BC_TRANSMISSIVE], ids=["periodic", "transmissive"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_flags_match_oracle(dim, n, bc, precision):
    nb = int(np.prod(n))
    m = mesh(dim, n, random_flags(nb, 5), bc=bc)
    s, o = solver(m, precision=precision), oracle(m)
    for seed in range(3):
        W = steep_state(dim, s.N, s.n_cells, seed=20 + seed)
        Wd = torch.as_tensor(W, dtype=s.dtype, device="cuda")
        nc, changed, flags = s.adapt_mark(Wd, WT, ALPHA, flags=True)
        expect = o.adapt_flags(Wd.double().cpu().numpy(), WT, ALPHA)
        np.testing.assert_array_equal(flags, expect)
        assert 0 < expect.sum() < nb  # both outcomes occur
        assert nc == nb + ((1 << dim) - 1) * expect.sum()
        assert changed == int(np.sum(expect != s.refinement()))


def _same_handle(a, b, seed, limiter):
    """a (regridded) and b (created) give the same tables and the same bits"""
    np.testing.assert_array_equal(a.neighbor_table(), b.neighbor_table())
    np.testing.assert_array_equal(a.levels(), b.levels())
    assert a.n_cells == b.n_cells and a.n_nodes == b.n_nodes
    W = torch.as_tensor(wl.random_weights(a.dim, a.N, a.n_cells, seed=seed, slope=0.05),
                        dtype=a.dtype, device="cuda")
    assert torch.equal(a.rhs(W), b.rhs(W))
    assert torch.equal(a.compute_dt(W), b.compute_dt(W))
    if limiter:
        assert torch.equal(a.limit(W.clone()), b.limit(W.clone()))
    Wa, Wb = W.clone(), W.clone()
    a.advance(Wa, 2)
    b.advance(Wb, 2)
    assert torch.equal(Wa, Wb)
    np.testing.assert_allclose(a.totals(W).cpu().numpy(), b.totals(W).cpu().numpy(), rtol=1e-13)


@pytest.mark.parametrize("dim,n,k", [(2, [16, 12], 2), (3, [6, 6, 5], 1), (3, [5, 4, 4], 2)],
                         ids=["2d-k2", "3d-k1", "3d-k2"])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_regrid_sequence_matches_created_handles(dim, n, k, precision):
    nb = int(np.prod(n))
    bc = wl.BC_TRANSMISSIVE if dim == 3 and k == 1 else wl.BC_PERIODIC
    limiter = dict(limiter="characteristic", positivity=True) if precision != "mixed" else {}
    s = solver(mesh(dim, n, bc=bc), k=k, precision=precision, **limiter)
    W = torch.as_tensor(wl.random_weights(dim, s.N, s.n_cells, seed=1, slope=0.05), dtype=s.dtype,
                        device="cuda")
    seq = [random_flags(nb, 7, 0.25), np.ones(nb, np.int32), random_flags(nb, 8, 0.5),
           np.zeros(nb, np.int32), random_flags(nb, 9, 0.1)]
    for i, flags in enumerate(seq):
        nc, changed = s.set_refinement(flags)
        assert changed == int(np.sum(flags != s.refinement()))
        W = s.regrid(W)
        assert tuple(W.shape) == (s.nv, s.N, nc) and s.n_cells == nc
        np.testing.assert_array_equal(s.refinement(), flags)
        fresh = solver(mesh(dim, n, flags, bc=bc), k=k, precision=precision, **limiter)
        _same_handle(s, fresh, seed=30 + i, limiter=bool(limiter))


@pytest.mark.parametrize("dim,n,bc", [(2, [1, 1], wl.BC_PERIODIC), (2, [1, 3], wl.BC_TRANSMISSIVE),
                                      (3, [1, 1, 1], wl.BC_PERIODIC), (3, [2, 1, 1], wl.BC_TRANSMISSIVE)],
                         ids=["2d-1x1", "2d-1x3-open", "3d-1x1x1", "3d-2x1x1-open"])
def test_regrid_degenerate_meshes(dim, n, bc):
    """a single periodic base cell (refined: its children are each other's
    neighbours across the wrap) and one-cell-wide strips"""
    nb = int(np.prod(n))
    s = solver(mesh(dim, n, bc=bc), k=1)
    W = torch.as_tensor(wl.random_weights(dim, s.N, s.n_cells, seed=3, slope=0.05), device="cuda")
    seq = [np.ones(nb, np.int32), (np.arange(nb) % 2).astype(np.int32), np.zeros(nb, np.int32)]
    for i, flags in enumerate(seq):
        s.set_refinement(flags)
        W = s.regrid(W)
        fresh = solver(mesh(dim, n, flags, bc=bc), k=1)
        _same_handle(s, fresh, seed=50 + i, limiter=False)


@pytest.mark.parametrize("dim,n", [(2, [9, 7]), (3, [5, 4, 3])], ids=["2d", "3d"])
def test_projection_matches_oracle(dim, n):
    nb = int(np.prod(n))
    f0, f1 = random_flags(nb, 3, 0.4), random_flags(nb, 4, 0.4)
    m0, m1 = mesh(dim, n, f0), mesh(dim, n, f1)
    s = solver(m0)
    W0 = wl.random_weights(dim, s.N, s.n_cells, seed=2, slope=0.2)
    s.set_refinement(f1)
    W1 = s.regrid(torch.as_tensor(W0, device="cuda")).cpu().numpy()
    o0, o1 = oracle(m0), oracle(m1)
    expect = o1.adapt_project(o0, W0)
    np.testing.assert_allclose(W1, expect, rtol=0, atol=1e-14 * np.abs(W0).max())
    # derefinement conserves the totals
    assert o1.n_cells == s.n_cells
    np.testing.assert_allclose(s.totals(torch.as_tensor(W1, device="cuda")).cpu().numpy(),
                               o0.totals(W0), rtol=1e-13)


def pulse(xyz, dim, center, vel, width=0.09):
    r2 = sum((xyz[a] - center[a]) ** 2 for a in range(dim))
    rho = 1.0 + 0.6 * np.exp(-r2 / width ** 2)
    v = [np.full_like(rho, vel[a]) for a in range(dim)]
    return wl.conserved(rho, v, np.ones_like(rho), 1.4)


@pytest.mark.parametrize("dim,n,k,steps", [(2, [20, 20], 2, 24), (3, [8, 8, 8], 1, 8)], ids=["2d", "3d"])
def test_adaptive_run_follows_oracle(dim, n, k, steps):
    """Adapt after every step (Sec. 4): a density pulse advected across a
    periodic box; the refined region follows it."""
    center, vel = [0.35] * dim, [1.0, 0.6, 0.3][:dim]
    m = mesh(dim, n)
    s, o = solver(m, k=k), oracle(m, k=k)
    W = s.project(torch.as_tensor(pulse(s.quad_points().cpu().numpy(), dim, center, vel)))
    Wo = o.project(pulse(o.quad_points(), dim, center, vel))
    # adapt to the initial data first (twice: refine, then refine where the
    # finer projection now sees the slopes)
    history = []
    for step in range(steps + 2):
        if step >= 2:
            dt = o.compute_dt(Wo)
            Wo, _ = o.rk_step(Wo, dt)
            s.rk_step(W, dt)
        flags_o = o.adapt_flags(Wo, WT, ALPHA)
        nc, changed, flags = s.adapt_mark(W, WT, ALPHA, flags=True)
        np.testing.assert_array_equal(flags, flags_o)
        m1 = mesh(dim, n, flags_o)
        o1 = oracle(m1, k=k)
        Wo, o = o1.adapt_project(o, Wo), o1
        W = s.regrid(W)
        history.append(int(flags.sum()))
        np.testing.assert_allclose(W.cpu().numpy(), Wo, rtol=0, atol=1e-10)
    assert min(history) > 0 and max(history) < int(np.prod(n))
    # the refined region moved with the pulse: mass is conserved to rounding
    np.testing.assert_allclose(s.totals(W).cpu().numpy(), o.totals(Wo), rtol=1e-12)


def test_tensor_core_handle_refuses_a_refined_mesh():
    from paper_1506_06140_gb300 import dg
    s = solver(mesh(2, [8, 8]), k=2, precision="fp32_tc")
    W = torch.as_tensor(wl.random_weights(2, s.N, s.n_cells, seed=1), dtype=s.dtype, device="cuda")
    s.set_refinement(np.eye(8, dtype=np.int32).reshape(-1))
    with pytest.raises(dg.DGError):
        s.regrid(W)
    s.set_refinement(np.zeros(64, np.int32))  # a uniform mesh stays allowed
    W2 = s.regrid(W)
    assert torch.equal(W2, W)
