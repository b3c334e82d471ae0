"""The status path of the tensor-core cell kernel's bounded waits.

dg_test_force_timeout arms the next tensor-core cell launch so that its
first CTA issues neither its first multiply nor the commit that would
complete its barrier, and polls that barrier only 2^12 times.  The wait
gives up with no tensor-core work of the CTA in flight; the CTA frees its
tensor memory and latches DG_ERR_TIMEOUT.  The test checks that dg_status
reports it, and that the next launch on the same context runs normally and
matches the FP64 oracle.  No fault, trap or endless loop is involved: the
failure is a barrier that nothing completes, behind a bounded wait.
"""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O
from paper_1506_06140_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL32_MAX, TOL32_RMS = 2e-5, 2e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1506_06140_gb300 import build
    build.build()


def rel_err(got, ref):
    """max and RMS difference relative to max |ref| (the parity tests' measure)"""
    scale = max(np.max(np.abs(ref)), 1e-300)
    return np.max(np.abs(got - ref)) / scale, np.sqrt(np.mean((got - ref) ** 2)) / scale


@pytest.mark.parametrize("precision", ["fp32_tc", "mixed_tc"])
def test_forced_timeout_is_reported_and_the_context_stays_usable(precision):
    from paper_1506_06140_gb300 import dg
    m = wl.mesh_uniform(2, [150, 131], [0.0, 0.0], [1.5, 1.31])
    o = O.Oracle(2, m["n"], m["lo"], m["hi"], 3, 1.4, rk_order=3)
    s = dg.Solver(m, 3, 1.4, rk_order=3, precision=precision)
    dtype = np.float32 if precision == "fp32_tc" else np.float64
    W = wl.random_weights(2, o.N, o.n_cells, seed=2100).astype(dtype)
    Wd = torch.as_tensor(W, device="cuda").contiguous()
    ref = o.rhs(W.astype(np.float64))
    assert s.status() == dg.DG_OK
    s.force_timeout()
    s.rhs(Wd)  # the armed launch: its first CTA gives up its wait
    assert s.status() == dg.DG_ERR_TIMEOUT
    assert s.status() == dg.DG_OK  # dg_status clears the word
    # the same context, next launch: normal results
    got = s.rhs(Wd).double().cpu().numpy()
    assert s.status() == dg.DG_OK
    e, erms = rel_err(got, ref)
    assert e < TOL32_MAX and erms < TOL32_RMS, (e, erms)
    # and a whole SSP-RK3 step afterwards agrees with the oracle's
    dt = 0.5 * o.compute_dt(W.astype(np.float64))
    W1, _ = o.rk_step(W.astype(np.float64), dt)
    s.rk_step(Wd, dt)
    got = Wd.double().cpu().numpy()
    e, _ = rel_err(got - W, W1 - W)
    assert e < 1e-3, e
    assert s.status() == dg.DG_OK


def test_force_timeout_needs_the_tensor_core_kernel():
    from paper_1506_06140_gb300 import dg
    m = wl.mesh_uniform(2, [8, 8], [0.0, 0.0], [1.0, 1.0])
    s = dg.Solver(m, 2, 1.4, precision="fp32")
    with pytest.raises(dg.DGError) as ei:
        s.force_timeout()
    assert ei.value.code == dg.DG_ERR_UNSUPPORTED
