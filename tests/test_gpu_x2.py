"""The packed-pair FP32 cell kernel (two variables per thread, paired FP32
multiply-adds; dg_set_tiles cell tile 2) against the one-variable-per-thread
cell kernel: per lane it performs the same operations in the same order, so
right-hand sides and RK steps must agree bit for bit, on uniform,
transmissive and two-level meshes, k = 0..3, and on an ensemble; the oracle
bar follows from that.  Handles without the kernel refuse the tile."""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O
from paper_1506_06140_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

GAMMA = 1.4


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


def to_dev(W):
    return torch.as_tensor(W, dtype=torch.float32, device="cuda").contiguous()


@pytest.mark.parametrize("name", list(MESHES))
def test_rhs_bit_identical_to_one_variable_per_thread(name):
    dg = dg_mod()
    m = MESHES[name]
    for k in (0, 1, 2, 3):
        s = dg.Solver(m, k, GAMMA, precision="fp32")
        W = to_dev(wl.random_weights(2, s.N, s.n_cells, seed=2100 + k).astype(np.float32))
        ref = s.rhs(W).cpu().numpy()
        s.set_tiles(2, 32)
        assert s.tiles() == (2, 32)
        got = s.rhs(W).cpu().numpy()
        np.testing.assert_array_equal(got, ref)
        if k == 3 and name == "amr2":
            o = O.Oracle(2, m["n"], m["lo"], m["hi"], k, GAMMA, bc=m["bc"], refine_boxes=m["refine_boxes"])
            exact = o.rhs(W.cpu().numpy().astype(np.float64))
            assert np.max(np.abs(got - exact)) < 2e-5 * np.max(np.abs(exact))


@pytest.mark.parametrize("order", [2, 3, 4])
def test_steps_bit_identical(order):
    dg = dg_mod()
    m = wl.mesh_uniform(2, [48, 48], [-5.0, -5.0], [5.0, 5.0])
    k = {2: 1, 3: 2, 4: 3}[order]
    a = dg.Solver(m, k, GAMMA, rk_order=order, precision="fp32")
    b = dg.Solver(m, k, GAMMA, rk_order=order, precision="fp32")
    b.set_tiles(2, 32)
    U = torch.as_tensor(wl.vortex(a.quad_points().cpu().numpy()))
    Wa, Wb = a.project(U), b.project(U)
    a.advance(Wa, 3)
    for _ in range(3):
        b.rk_step(Wb)
    np.testing.assert_array_equal(Wa.cpu().numpy(), Wb.cpu().numpy())
    b.advance(Wb, 2)
    a.advance(Wa, 2)
    np.testing.assert_array_equal(Wa.cpu().numpy(), Wb.cpu().numpy())


def test_ensemble_bit_identical():
    dg = dg_mod()
    meshes = [wl.mesh_uniform(2, [n, n], [-5.0, -5.0], [5.0, 5.0]) for n in (12, 20, 9)]
    a = dg.Solver(meshes, 2, GAMMA, rk_order=3, precision="fp32")
    b = dg.Solver(meshes, 2, GAMMA, rk_order=3, precision="fp32")
    b.set_tiles(2, 32)
    W = to_dev(wl.random_weights(2, a.N, a.n_cells, seed=2200).astype(np.float32))
    Wa, Wb = W.clone(), W.clone()
    a.advance(Wa, 2)
    b.advance(Wb, 2)
    np.testing.assert_array_equal(Wa.cpu().numpy(), Wb.cpu().numpy())


def test_refused_where_not_built():
    dg = dg_mod()
    m = MESHES["u2"]
    for kw in (dict(precision="fp64"), dict(precision="mixed"), dict(precision="fp32_tc"),
               dict(precision="fp32", basis="tensor")):
        s = dg.Solver(m, 2, GAMMA, **kw)
        with pytest.raises(dg.DGError) as ei:
            s.set_tiles(2, 32)
        assert ei.value.code == dg.DG_ERR_UNSUPPORTED, kw
    s = dg.Solver(m, 2, GAMMA, precision="fp32")
    with pytest.raises(dg.DGError) as ei:
        s.set_tiles(2, 0)  # the fused kernel has its own cell update
    assert ei.value.code == dg.DG_ERR_UNSUPPORTED
    m3 = wl.mesh_uniform(3, [4, 4, 4], [0.0] * 3, [1.0] * 3)
    s3 = dg.Solver(m3, 1, GAMMA, precision="fp32")
    with pytest.raises(dg.DGError) as ei:
        s3.set_tiles(2, 32)
    assert ei.value.code == dg.DG_ERR_UNSUPPORTED
