"""CPU checks of bench.py's host-side helpers: the equal-L1 comparison on a
synthetic ladder, the per-launch DRAM traffic table against the profile
summaries it cites, and the bookkeeping of the algorithmic work counts."""
import importlib.util
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def row(p, n, l1, ms, steps):
    return dict(precision=p, n=n, L1=l1, ms_per_stage=ms, steps=steps)


def test_equal_l1_picks_the_cheapest_resolution_that_reaches_the_target(bench):
    rows = [row("fp64", 64, 1e-6, 1.0, 100), row("fp64", 128, 1e-7, 4.0, 200),
            # reaches 1e-6 (within 5%) only at 128, and 1e-7 never
            row("mixed", 64, 1.2e-6, 0.2, 100), row("mixed", 128, 1.04e-6, 0.5, 200),
            # reaches both targets at 64
            row("fp32", 64, 1e-8, 0.1, 100), row("fp32", 128, 1e-9, 0.3, 200)]
    out = bench.equal_l1(rows, tol=1.05)
    assert [e["fp64_n"] for e in out] == [64, 128]
    m = out[0]["mixed"]
    assert m["n"] == 128 and m["stage_speedup_vs_fp64"] == pytest.approx(1.0 / 0.5)
    assert m["run_speedup_vs_fp64"] == pytest.approx((1.0 * 100) / (0.5 * 200))
    assert out[1]["mixed"] is None
    assert out[0]["fp32"]["n"] == 64 and out[1]["fp32"]["n"] == 64
    assert out[1]["fp32"]["stage_speedup_vs_fp64"] == pytest.approx(40.0)


def profile_bytes(fn, pattern):
    """read + write DRAM bytes of the kernel block matching pattern in a summary"""
    units = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    text = open(os.path.join(ROOT, "profiles", fn)).read()
    hits = []
    for block in text.split("Kernel: `")[1:]:
        name = block.split("`")[0]
        if not re.search(pattern, name):
            continue
        r = re.search(r"\| DRAM read \| ([\d.]+) (\w+) \|", block)
        w = re.search(r"\| DRAM write \| ([\d.]+) (\w+) \|", block)
        hits.append(float(r.group(1)) * units[r.group(2)] + float(w.group(1)) * units[w.group(2)])
    return hits


def test_traffic_table_matches_the_profiles_it_cites(bench):
    """Every entry of profiles/dram_traffic.txt equals the DRAM read + write
    of a kernel block in the summary it names (so the bench's roofline
    traffic comes from a committed capture), and bench.dram_traffic reads it."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    entries = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(entries) >= 10
    for kernel, workload, nbytes, src in entries:
        assert os.path.exists(os.path.join(ROOT, "profiles", src)), src
        hits = profile_bytes(src, re.escape(kernel) + r"\b")
        assert any(abs(h - float(nbytes)) <= 1.0 for h in hits), (kernel, workload, nbytes, hits)
        assert bench.dram_traffic(kernel, workload) == float(nbytes)
    assert bench.dram_traffic("no_such_kernel", "vortex256_k3_fp64") is None


def test_work_counts(bench):
    """The face moments move the face contraction out of the cell count
    (once per face instead of once per side) and never add work overall per
    cell (d faces per cell); the tensor basis has more coefficients; 3D
    counts exceed 2D ones at the same k."""
    for dim, k in ((2, 1), (2, 2), (2, 3), (3, 1), (3, 2)):
        c0, f0 = bench.kernel_flops(dim, k)
        c1, f1 = bench.kernel_flops(dim, k, moments=True)
        assert c1 < c0 and f1 > f0
        assert c1 + dim * f1 <= c0 + dim * f0
    assert bench.shape(2, 3, "tensor")[0] == 16 and bench.shape(2, 3)[0] == 10
    assert bench.kernel_flops(2, 3, "tensor")[0] > bench.kernel_flops(2, 3)[0]
    assert bench.kernel_flops(3, 2)[0] > bench.kernel_flops(2, 2)[0]
    # bytes per cell: nv N element-size
    assert bench.state_bytes_per_cell(2, 3, 8) == 4 * 10 * 8
    assert bench.state_bytes_per_cell(3, 2, 4) == 5 * 10 * 4
