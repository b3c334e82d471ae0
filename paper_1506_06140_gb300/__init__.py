"""GB300-native modal DG solver for the Euler equations (after Schaal et al. 2015).

The compute path is the C-ABI library ``libdg.so`` (hand-written sm_103a CUDA
kernels); :mod:`paper_1506_06140_gb300.dg` is its thin ctypes binding and
:mod:`paper_1506_06140_gb300.workloads` holds the seeded synthetic inputs.
"""
__all__ = ["dg", "workloads"]
