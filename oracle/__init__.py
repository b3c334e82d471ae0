"""Oracle: a plain, slow FP64 CPU implementation of the modal DG scheme.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import it.  It shares no code
with the CUDA library in ``paper_1506_06140_gb300``.
"""
