"""The fused face + cell kernel (a tile of 8 x 4 cells with its face halo,
dg_set_tiles(..., face_tile=0)) against the face kernel + cell kernel pair.

Both compute every trace, HLLC flux and integral with the same functions in
the same order; the compiler may still fuse a multiply and an add
differently in the two kernels, so the right-hand side and whole RK steps
must agree to rounding (1e-12 of the largest value in FP64, 1e-5 in FP32):
on meshes whose size is a multiple of the tile, on ragged ones, with
transmissive sides (mirrored states), and on meshes narrower than a tile,
where a periodic neighbour lies in the same tile; for FP64 and FP32 states
and k = 0..3.  The fused path is also checked against the FP64 oracle.
"""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O
from paper_1506_06140_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1506_06140_gb300 import build
    build.build()


MESHES = {
    "tiles": wl.mesh_uniform(2, [32, 16], [0.0, 0.0], [2.0, 1.0]),
    "ragged": wl.mesh_uniform(2, [37, 29], [0.0, 0.0], [37 / 29.0, 1.0]),
    "transmissive": wl.mesh_uniform(2, [23, 3], [0.0, 0.0], [1.0, 3 / 23.0], bc=[1, 0]),
    "narrow": wl.mesh_uniform(2, [5, 3], [0.0, 0.0], [5 / 3.0, 1.0]),
    "one_row_open": wl.mesh_uniform(2, [6, 1], [0.0, 0.0], [6.0, 1.0], bc=[1, 1]),
}


def close(x, y, precision):
    x, y = x.double(), y.double()
    tol = 1e-12 if precision == "fp64" else 1e-5
    d = (x - y).abs().max().item() / max(y.abs().max().item(), 1e-300)
    assert d <= tol, d


def pair(mesh, k, precision, rk=3):
    from paper_1506_06140_gb300 import dg
    a = dg.Solver(mesh, k, 1.4, rk_order=rk, precision=precision)
    b = dg.Solver(mesh, k, 1.4, rk_order=rk, precision=precision)
    b.set_tiles(32, 0)
    assert b.tiles() == (32, 0)
    return a, b


@pytest.mark.parametrize("name", sorted(MESHES))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_fused_rhs_and_step_bit_identical(name, precision, k):
    a, b = pair(MESHES[name], k, precision)
    dtype = np.float64 if precision == "fp64" else np.float32
    W = torch.as_tensor(wl.random_weights(2, a.N, a.n_cells, seed=3000 + k).astype(dtype), device="cuda")
    close(b.rhs(W), a.rhs(W), precision)
    Wa, Wb = W.clone(), W.clone()
    for _ in range(3):
        a.rk_step(Wa)
        b.rk_step(Wb)
    torch.cuda.synchronize()
    close(Wb - W, Wa - W, precision)
    assert a.status() == 0 and b.status() == 0


def test_fused_vortex_matches_the_oracle():
    m = wl.mesh_uniform(2, [64, 64], [-5.0, -5.0], [5.0, 5.0])
    o = O.Oracle(2, m["n"], m["lo"], m["hi"], 3, 1.4, rk_order=4)
    a, b = pair(m, 3, "fp64", rk=4)
    W = o.project(wl.vortex(o.quad_points()))
    Wd = torch.as_tensor(W, device="cuda")
    ref = o.rhs(W)
    got = b.rhs(Wd).cpu().numpy()
    assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()
    dt = o.compute_dt(W)
    W1, _ = o.rk_step(W, dt)
    b.rk_step(Wd, dt)
    d = Wd.cpu().numpy() - W
    assert np.abs(d - (W1 - W)).max() < 1e-10 * np.abs(W1 - W).max()


def test_fused_graph_advance_agrees():
    a, b = pair(wl.mesh_uniform(2, [48, 40], [-5.0, -5.0], [5.0, -5.0 + 40 * 10.0 / 48]), 2, "fp64")
    W = a.project(torch.as_tensor(wl.vortex(a.quad_points().cpu().numpy())))
    Wa, Wb = W.clone(), W.clone()
    ha, hb = a.dt_buffer(6), b.dt_buffer(6)
    a.advance(Wa, 6, ha)
    b.advance(Wb, 6, hb)
    torch.cuda.synchronize()
    close(Wb - W, Wa - W, "fp64")
    close(hb, ha, "fp64")


def test_fused_rejected_where_unsupported():
    from paper_1506_06140_gb300 import dg
    cases = [(dict(wl.mesh_uniform(2, [8, 8], [0.0, 0.0], [1.0, 1.0]), refine_boxes=[[2, 2, 3, 3]]), "fp64"),
             (wl.mesh_uniform(2, [8, 8], [0.0, 0.0], [1.0, 1.0]), "mixed"),
             (wl.mesh_uniform(2, [8, 8], [0.0, 0.0], [1.0, 1.0]), "fp32_tc"),
             (wl.mesh_uniform(3, [4, 4, 4], [0.0] * 3, [1.0] * 3), "fp64")]
    for mesh, prec in cases:
        s = dg.Solver(mesh, 1, 1.4, precision=prec)
        with pytest.raises(dg.DGError) as ei:
            s.set_tiles(32, 0)
        assert ei.value.code == dg.DG_ERR_UNSUPPORTED
