"""dg_advance as one persistent, cooperatively launched kernel.

The persistent kernel runs every phase of the steps (timestep, face fluxes,
cell updates, slope and positivity limiters) with the same block code as
the launch-by-launch path, separated by bounded grid barriers.  Its results
must therefore equal the CUDA-graph path bit for bit -- states, timestep
histories and limiter counts -- on every kind of step program: RK2 to RK4
(up to five stages), the characteristic limiter, the positivity limiter,
static two-level meshes, FP64 and FP32 states and ensembles.  The wave run
is also compared with the FP64 oracle.
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


def both_paths(make, ic, n_steps, limited=False, dtype=torch.float64):
    """states, timestep histories and limiter counts after n_steps of
    dg_advance, once per path, from the same initial state"""
    out = {}
    for mode in ("graph", "persistent"):
        s = make()
        s.set_advance_mode(mode)
        assert s.advance_mode() == mode
        W = s.project(torch.as_tensor(ic(s.quad_points().cpu().numpy())))
        if limited:
            s.limit(W)
        s.limiter_counts(reset=True)
        hist = s.dt_buffer(n_steps)
        s.advance(W, n_steps, hist)
        torch.cuda.synchronize()
        assert s.status() == 0, mode
        out[mode] = (W.cpu(), hist.cpu(), s.limiter_counts().cpu())
    return out


def assert_identical(out):
    (Wg, hg, cg), (Wp, hp, cp) = out["graph"], out["persistent"]
    assert torch.equal(Wg, Wp)
    assert torch.equal(hg, hp)
    assert torch.equal(cg, cp)


def test_wave_rk2_identical_and_matches_the_oracle():
    from paper_1506_06140_gb300 import dg
    m = wl.mesh_uniform(2, [32, 32], [0.0, 0.0], [1.0, 1.0])
    make = lambda: dg.Solver(m, 1, 1.4, rk_order=2, cfl=0.3)
    out = both_paths(make, wl.wave2d, 25)
    assert_identical(out)
    o = O.Oracle(2, m["n"], m["lo"], m["hi"], 1, 1.4, rk_order=2, cfl=0.3)
    W = o.project(wl.wave2d(o.quad_points()))
    dts = []
    for _ in range(25):
        W, dt = o.rk_step(W, 0.0)
        dts.append(dt)
    Wp, hp, _ = out["persistent"]
    np.testing.assert_allclose(hp.numpy(), dts, rtol=1e-13)
    err = np.abs(Wp.numpy() - W).max() / np.abs(W).max()
    assert err < 1e-12, err


def test_square_rk3_characteristic_limiter_identical():
    from paper_1506_06140_gb300 import dg
    m = wl.mesh_uniform(2, [64, 64], [0.0, 0.0], [1.0, 1.0])
    make = lambda: dg.Solver(m, 2, 1.4, rk_order=3, limiter="characteristic")
    out = both_paths(make, wl.square2d, 12, limited=True)
    assert_identical(out)
    assert out["persistent"][2][0].item() > 0  # the slope limiter acted


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_positivity_and_slope_limiters_identical(precision):
    # the cold disc without its field: near-vacuum background (rho = p = 1e-5)
    # around a rotating ring, both limiters active
    from paper_1506_06140_gb300 import dg
    m = wl.mesh_uniform(2, [48, 48], [0.0, 0.0], [6.0, 6.0])
    make = lambda: dg.Solver(m, 2, 5.0 / 3.0, rk_order=3, limiter="characteristic", positivity=True,
                             precision=precision)
    out = both_paths(make, lambda x: wl.keplerian_disc(x), 15, limited=True)
    assert_identical(out)
    assert out["persistent"][2][2].item() > 0  # cells went through the FP64 positivity pass


def test_rk4_five_stages_fp32_two_level_mesh_identical():
    from paper_1506_06140_gb300 import dg
    m = dict(wl.mesh_uniform(2, [24, 24], [-5.0, -5.0], [5.0, 5.0]), refine_boxes=[[8, 8, 15, 15]])
    make = lambda: dg.Solver(m, 3, 1.4, rk_order=4, precision="fp32")
    assert_identical(both_paths(make, wl.vortex, 10))


def test_ensemble_identical():
    from paper_1506_06140_gb300 import dg
    probs = [(16, 3.5), (24, 5.0), (12, 6.0)]
    meshes = [wl.mesh_uniform(2, [n, n], [-5.0, -5.0], [5.0, 5.0]) for n, _ in probs]

    def ic(xyz):
        U = np.empty((4, xyz.shape[1], xyz.shape[2]))
        a = 0
        for n, beta in probs:
            U[:, :, a:a + n * n] = wl.vortex(xyz[:, :, a:a + n * n], beta=beta)
            a += n * n
        return U

    make = lambda: dg.Solver(meshes, 2, 1.4, rk_order=3, precision="fp32")
    assert_identical(both_paths(make, ic, 8))


def test_advance_mode_rules():
    from paper_1506_06140_gb300 import dg
    m2 = wl.mesh_uniform(2, [16, 16], [0.0, 0.0], [1.0, 1.0])
    for prec in ("mixed", "fp32_tc"):
        s = dg.Solver(m2, 2, 1.4, precision=prec)
        assert s.advance_mode() == "graph"
        with pytest.raises(dg.DGError) as ei:
            s.set_advance_mode("persistent")
        assert ei.value.code == dg.DG_ERR_UNSUPPORTED
    s3 = dg.Solver(wl.mesh_uniform(3, [4, 4, 4], [0.0] * 3, [1.0] * 3), 1, 1.4)
    assert s3.advance_mode() == "graph"
    with pytest.raises(dg.DGError):
        s3.set_advance_mode("persistent")
    # the graph is the default; a supported handle may switch
    big = dg.Solver(wl.mesh_uniform(2, [160, 160], [0.0, 0.0], [1.0, 1.0]), 1, 1.4)
    assert big.advance_mode() == "graph"
    big.set_advance_mode("persistent")
    assert big.advance_mode() == "persistent"
    # a gravity field sends dg_advance back to the graph
    s = dg.Solver(m2, 2, 1.4)
    s.set_advance_mode("persistent")
    assert s.advance_mode() == "persistent"
    s.set_gravity(torch.zeros((2, s.nq, s.n_cells), dtype=torch.float64, device="cuda"))
    assert s.advance_mode() == "graph"
