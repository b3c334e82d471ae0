"""The tensor-product basis Q_k (DG_BASIS_TENSOR) against the FP64 oracle
run with the same basis.

The stage kernels take the basis as a compile-time choice of the
sum-factorised loops' bounds and coefficient positions; these tests compare
projection, right-hand side, RK steps, timestep, totals and the L1 error with
the oracle on uniform, transmissive and two-level meshes at k = 1..3 (bars as
in the total-degree parity tests), check that every cell tile gives the same
result, that advance() repeats rk_step(), and that the calls and options the
basis does not have are refused.
"""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O
from paper_1506_06140_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

GAMMA = 1.4
TOL64 = 1e-11
TOL32_MAX, TOL32_RMS = 2e-5, 2e-6


@pytest.fixture(scope="session", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1506_06140_gb300 import build
    build.build()


def dg_mod():
    from paper_1506_06140_gb300 import dg
    return dg


MESHES = {
    "u2": wl.mesh_uniform(2, [37, 29], [0.0, 0.0], [37 / 29.0, 1.0]),
    "u2t": wl.mesh_uniform(2, [23, 3], [0.0, 0.0], [1.0, 3 / 23.0], bc=[1, 0]),
    "amr2": dict(wl.mesh_uniform(2, [16, 12], [0.0, 0.0], [4 / 3.0, 1.0]),
                 refine_boxes=[[4, 3, 9, 7], [13, 0, 15, 1]]),
}


def oracle_for(mesh, k, **kw):
    return O.Oracle(mesh["dim"], mesh["n"], mesh["lo"], mesh["hi"], k, GAMMA, bc=mesh["bc"],
                    refine_boxes=mesh["refine_boxes"], basis="tensor", **kw)


def solver_for(mesh, k, **kw):
    return dg_mod().Solver(mesh, k, GAMMA, basis="tensor", **kw)


def to_dev(s, W):
    return torch.as_tensor(W, dtype=s.dtype, device="cuda").contiguous()


def rel_err(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    scale = max(np.max(np.abs(b)), 1e-300)
    return np.max(np.abs(a - b)) / scale, np.sqrt(np.mean((a - b) ** 2)) / scale


def test_sizes():
    m = MESHES["u2"]
    for k in (0, 1, 2, 3):
        s = solver_for(m, k)
        assert s.N == (k + 1) ** 2 and s.N == oracle_for(m, k).N


@pytest.mark.parametrize("name", ["u2", "amr2"])
def test_projection(name):
    m = MESHES[name]
    for k in (1, 2, 3):
        o = oracle_for(m, k)
        s = solver_for(m, k)
        np.testing.assert_allclose(s.quad_points().cpu().numpy(), o.quad_points(), rtol=0, atol=1e-15)
        U = wl.vortex(o.quad_points(), center=(0.6, 0.5), period=0)
        Wg = s.project(torch.as_tensor(U, device="cuda")).cpu().numpy()
        e, _ = rel_err(Wg, o.project(U))
        assert e < 1e-14, (name, k, e)


@pytest.mark.parametrize("name", list(MESHES))
def test_rhs_fp64(name):
    m = MESHES[name]
    for k in (1, 2, 3):
        o = oracle_for(m, k)
        s = solver_for(m, k)
        W = wl.random_weights(2, o.N, o.n_cells, seed=1100 + k)
        e, _ = rel_err(s.rhs(to_dev(s, W)).cpu().numpy(), o.rhs(W))
        assert e < TOL64, (name, k, e)


@pytest.mark.parametrize("name", ["u2", "amr2"])
def test_rhs_fp32(name):
    m = MESHES[name]
    for k in (1, 2, 3):
        o = oracle_for(m, k)
        s = solver_for(m, k, precision="fp32")
        W = wl.random_weights(2, o.N, o.n_cells, seed=1200 + k).astype(np.float32)
        ref = o.rhs(W.astype(np.float64))
        e, erms = rel_err(s.rhs(to_dev(s, W)).cpu().numpy(), ref)
        assert e < TOL32_MAX and erms < TOL32_RMS, (name, k, e, erms)


def test_tensor_modes_reach_the_rhs():
    """A state whose only non-zero slopes are the modes outside the
    total-degree space (x^a y^b with a + b > k) has a non-zero right-hand
    side, equal to the oracle's: those coefficients enter the kernels."""
    m = MESHES["u2"]
    k = 2
    o = oracle_for(m, k)
    s = solver_for(m, k)
    W = wl.random_weights(2, o.N, o.n_cells, seed=1300)
    n_total = (k + 1) * (k + 2) // 2
    W[:, 1:n_total, :] = 0.0
    ref = o.rhs(W)
    assert np.abs(ref).max() > 0.0
    e, _ = rel_err(s.rhs(to_dev(s, W)).cpu().numpy(), ref)
    assert e < TOL64


@pytest.mark.parametrize("order,k", [(2, 1), (3, 2), (4, 3)])
@pytest.mark.parametrize("name", ["u2", "amr2"])
def test_rk_step_fp64(order, k, name):
    m = MESHES[name]
    o = oracle_for(m, k, rk_order=order)
    s = solver_for(m, k, rk_order=order)
    W = wl.random_weights(2, o.N, o.n_cells, seed=1400 + order)
    dt = 0.5 * o.compute_dt(W)
    ref, _ = o.rk_step(W, dt)
    Wd = to_dev(s, W)
    s.rk_step(Wd, dt)
    e, _ = rel_err(Wd.cpu().numpy() - W, ref - W)  # compare the increments
    assert e < 1e-10, (order, name, e)


@pytest.mark.parametrize("name", ["u2t", "amr2"])
def test_dt_totals_l1(name):
    m = MESHES[name]
    k = 3
    o = oracle_for(m, k, cfl=0.3)
    s = solver_for(m, k, cfl=0.3)
    W = wl.random_weights(2, o.N, o.n_cells, seed=1500)
    Wd = to_dev(s, W)
    assert s.compute_dt(Wd).item() == pytest.approx(o.compute_dt(W), rel=1e-14)
    ref_t = o.totals(W)
    np.testing.assert_allclose(s.totals(Wd).cpu().numpy(), ref_t, rtol=1e-14, atol=1e-14 * np.abs(ref_t).max())
    rho_ref = 1.0 + 0.1 * np.sin(o.l1_points()).sum(axis=0)
    assert s.l1_density(Wd, torch.as_tensor(rho_ref)).item() == pytest.approx(o.l1_density(W, rho_ref), rel=1e-13)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_every_tile_gives_the_same_rhs(precision):
    m = MESHES["amr2"]
    k = 3
    s = solver_for(m, k, precision=precision)
    W = to_dev(s, wl.random_weights(2, s.N, s.n_cells, seed=1600))
    base = s.rhs(W).cpu().numpy()
    for ct in (16, 32, 64):
        for ft in (16, 32, 64):
            try:
                s.set_tiles(ct, ft)
            except dg_mod().DGError as err:
                assert err.code == dg_mod().DG_ERR_UNSUPPORTED
                continue
            np.testing.assert_array_equal(s.rhs(W).cpu().numpy(), base)


def test_advance_repeats_rk_step():
    m = wl.mesh_uniform(2, [40, 40], [-5.0, -5.0], [5.0, 5.0])
    k = 3
    s = solver_for(m, k, rk_order=4)
    U = torch.as_tensor(wl.vortex(s.quad_points().cpu().numpy()))
    W0 = s.project(U)
    Wa = W0.clone()
    s.advance(Wa, 4)
    Wb = W0.clone()
    for _ in range(4):
        s.rk_step(Wb)
    np.testing.assert_array_equal(Wa.cpu().numpy(), Wb.cpu().numpy())
    # conservation of the totals on the periodic box
    t0, t1 = s.totals(W0).cpu().numpy(), s.totals(Wa).cpu().numpy()
    np.testing.assert_allclose(t1, t0, rtol=0, atol=1e-12 * np.abs(t0).max())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_vortex_256_k3_rk4_full_size(precision):
    """The benchmarked workload itself: the 256^2 vortex with Q_3 (16
    coefficients per variable), SSP-RK4.  Right-hand side, timestep and one
    CFL step through advance() -- the one-step graph the benchmark replays --
    against the oracle with the same basis.  FP64 at the total-degree bars;
    FP32 at the full-size FP32 bars (dW/dt is a ~1.4e3-fold cancellation of
    volume and surface terms on this smooth state, so FP32 rounding bounds the
    error near 6e-4 of max |dW/dt|)."""
    m = wl.mesh_uniform(2, [256, 256], [-5.0, -5.0], [5.0, 5.0])
    o = oracle_for(m, 3, rk_order=4)
    s = solver_for(m, 3, rk_order=4, precision=precision)
    assert s.N == 16
    U = wl.vortex(o.quad_points())
    Wd = s.project(torch.as_tensor(U, device="cuda"))
    W = Wd.double().cpu().numpy()
    ref_rhs = o.rhs(W)
    e, erms = rel_err(s.rhs(Wd).cpu().numpy(), ref_rhs)
    dt = o.compute_dt(W)
    dt_hist = torch.zeros(1, dtype=torch.float64, device="cuda")
    s.advance(Wd, 1, dt_hist)
    got = Wd.double().cpu().numpy()
    ref, _ = o.rk_step(W, dt)
    if precision == "fp64":
        assert e < TOL64, e
        assert dt_hist.item() == pytest.approx(dt, rel=1e-14)
        e_step, _ = rel_err(got - W, ref - W)
        assert e_step < 1e-10, e_step
    else:
        assert e < 1e-3 and erms < 5e-5, (e, erms)
        assert dt_hist.item() == pytest.approx(dt, rel=1e-6)
        assert np.max(np.abs(got - ref)) < 1e-6 * np.max(np.abs(ref))
    assert s.status() == 0


def test_vortex_error_below_the_total_degree_basis():
    """Q_3 contains P_3: on the isentropic vortex after one time unit the
    tensor basis' L1 density error is below the total-degree basis' (both
    solvers on the same mesh, same steps)."""
    dg = dg_mod()
    m = wl.mesh_uniform(2, [32, 32], [-5.0, -5.0], [5.0, 5.0])
    errs, n_steps = {}, None
    for basis in ("total", "tensor"):
        s = dg.Solver(m, 3, GAMMA, rk_order=4, cfl=0.2, basis=basis)
        W = s.project(torch.as_tensor(wl.vortex(s.quad_points().cpu().numpy())))
        if n_steps is None:  # the same steps for both: the CFL step of the initial state
            n_steps = int(np.ceil(1.0 / s.compute_dt(W).item()))
        for _ in range(n_steps):
            s.rk_step(W, 1.0 / n_steps)
        rho = torch.as_tensor(wl.vortex(s.l1_points().cpu().numpy(), t=1.0)[0])
        errs[basis] = s.l1_density(W, rho).item()
    assert errs["tensor"] < errs["total"], errs


def test_refused_options_and_calls():
    dg = dg_mod()
    m = MESHES["amr2"]
    for kw in (dict(precision="mixed"), dict(precision="fp32_tc"), dict(precision="mixed_tc"),
               dict(limiter="component"), dict(positivity=True)):
        with pytest.raises(dg.DGError) as ei:
            solver_for(m, 2, **kw)
        assert ei.value.code == dg.DG_ERR_UNSUPPORTED, kw
    m3 = wl.mesh_uniform(3, [4, 4, 4], [0.0] * 3, [1.0] * 3)
    with pytest.raises(dg.DGError) as ei:
        solver_for(m3, 1)
    assert ei.value.code == dg.DG_ERR_UNSUPPORTED
    s = solver_for(m, 2)
    W = to_dev(s, wl.random_weights(2, s.N, s.n_cells, seed=1700))
    calls = [lambda: s.limit(W.clone()),
             lambda: s.rk_step_adjoint(W, 1e-3, W.clone()),
             lambda: s.node_weights(W),
             lambda: s.set_gravity(torch.zeros((2, s.nq, s.n_cells), dtype=torch.float64)),
             lambda: s.adapt_mark(W),
             lambda: s.set_refinement(np.zeros(s.n_base, np.int32)),
             lambda: s.set_advance_mode("persistent"),
             lambda: s.set_tiles(32, 0)]
    for i, call in enumerate(calls):
        with pytest.raises(dg.DGError) as ei:
            call()
        assert ei.value.code == dg.DG_ERR_UNSUPPORTED, i
    assert s.advance_mode() == "graph"
    s.rhs(W)  # the handle still works
    assert s.status() == dg.DG_OK
    sf = solver_for(MESHES["u2"], 2, precision="fp32")
    with pytest.raises(dg.DGError) as ei:
        sf.set_tiles(1, 32)
    assert ei.value.code == dg.DG_ERR_UNSUPPORTED


def test_k0_is_the_total_degree_handle():
    m = MESHES["amr2"]
    dg = dg_mod()
    a = dg.Solver(m, 0, GAMMA, basis="tensor", limiter="component")  # the constants: every kernel exists
    b = dg.Solver(m, 0, GAMMA, limiter="component")
    W = wl.random_weights(2, 1, a.n_cells, seed=1800)
    np.testing.assert_array_equal(a.rhs(to_dev(a, W)).cpu().numpy(), b.rhs(to_dev(b, W)).cpu().numpy())


def test_autotune():
    s = solver_for(MESHES["u2"], 3, precision="fp32", autotune=True)
    ct, ft = s.tiles()
    assert ct in (16, 32, 64) and ft in (16, 32, 64)
    o = oracle_for(MESHES["u2"], 3)
    W = wl.random_weights(2, o.N, o.n_cells, seed=1900).astype(np.float32)
    e, erms = rel_err(s.rhs(to_dev(s, W)).cpu().numpy(), o.rhs(W.astype(np.float64)))
    assert e < TOL32_MAX and erms < TOL32_RMS
