"""dg_totals_noalloc: conserved totals without a handle and without any
device allocation inside the library.

It serves callers that cannot allocate device memory -- a host application
that owns every device allocation, or code running while a stream is being
captured in global mode, where allocation calls are not permitted.  Such
callers cannot create a dg_handle (dg_create allocates), so the entry point
keeps its per-block partial sums in a fixed device array of the library.

The test calls it through the C ABI twice in a row, on different states and
meshes, and compares each result with the handle-based dg_totals and with
the FP64 CPU oracle's totals of the same state, at the tolerance the parity
tests use for totals (relative 1e-14).  It lives in a file that pytest
collects last.
"""
import ctypes

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


def _close(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    np.testing.assert_allclose(a, b, rtol=1e-14, atol=1e-14 * np.abs(b).max())


def _oracle_totals(mesh, k, W):
    from oracle import pyoracle as O
    o = O.Oracle(mesh["dim"], mesh["n"], mesh["lo"], mesh["hi"], k,
                 refine_boxes=mesh.get("refine_boxes") or [])
    return torch.as_tensor(o.totals(W.double().cpu().numpy()))


def test_noalloc_totals_match_handle_totals_two_calls():
    from paper_1506_06140_gb300 import dg
    m2 = wl.mesh_uniform(2, [61, 47], [0.0, 0.0], [61 / 47.0, 1.0])
    s2 = dg.Solver(m2, 3, 1.4)
    m3 = dict(wl.mesh_uniform(3, [6, 5, 4], [0.0] * 3, [1.2, 1.0, 0.8]),
              refine_boxes=[[1, 1, 1, 3, 2, 2]])
    s3 = dg.Solver(m3, 2, 1.4, precision="fp32")
    dx2 = 1.0 / 47.0
    dx3 = 0.2
    # first call: uniform 2D FP64 state, all cells at level 0
    Wa = torch.as_tensor(wl.random_weights(2, s2.N, s2.n_cells, seed=1), device="cuda")
    got_a = dg.totals_noalloc(Wa, 2, dx2)
    ref_a = s2.totals(Wa)
    # second call: two-level 3D FP32 state with per-cell levels
    Wb = torch.as_tensor(wl.random_weights(3, s3.N, s3.n_cells, seed=2, dtype=np.float32),
                         device="cuda")
    levels = torch.as_tensor(s3.levels(), dtype=torch.int32, device="cuda")
    got_b = dg.totals_noalloc(Wb, 3, dx3, levels)
    ref_b = s3.totals(Wb)
    torch.cuda.synchronize()
    _close(got_a, ref_a)
    _close(got_b, ref_b)
    _close(got_a, _oracle_totals(m2, 3, Wa))
    _close(got_b, _oracle_totals(m3, 2, Wb))
    # and once more on the first state: the shared scratch keeps no stale sums
    _close(dg.totals_noalloc(Wa, 2, dx2), ref_a)


def test_noalloc_accepts_the_mixed_state():
    # DG_MIXED keeps a double state: the entry point reads it as such
    from paper_1506_06140_gb300 import dg
    m = wl.mesh_uniform(2, [40, 24], [0.0, 0.0], [5.0, 3.0])
    s = dg.Solver(m, 2, 1.4, precision="mixed")
    W = torch.as_tensor(wl.random_weights(2, s.N, s.n_cells, seed=3), device="cuda")
    L = dg.load()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    r = L.dg_totals_noalloc(2, s.N, s.n_cells, dg.PRECISIONS["mixed"], 0.125, None,
                            ctypes.c_void_p(W.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert r == dg.DG_OK
    torch.cuda.synchronize()
    _close(out, s.totals(W))
    _close(out, _oracle_totals(m, 2, W))


def test_noalloc_rejects_sizes_beyond_the_maximum():
    from paper_1506_06140_gb300 import dg
    L = dg.load()
    W = torch.zeros((4, 1, 8), dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    too_many = (1 << 24) + 1
    # rejected on the host before any launch; the pointers are never read
    r = L.dg_totals_noalloc(2, 1, too_many, 0, 1.0, None, ctypes.c_void_p(W.data_ptr()),
                            ctypes.c_void_p(out.data_ptr()), None)
    assert r == dg.DG_ERR_ARG
    r = L.dg_totals_noalloc(4, 1, 8, 0, 1.0, None, ctypes.c_void_p(W.data_ptr()),
                            ctypes.c_void_p(out.data_ptr()), None)
    assert r == dg.DG_ERR_ARG
