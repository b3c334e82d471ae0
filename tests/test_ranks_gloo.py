"""The multi-rank path of bench.py on CPU: two gloo ranks exchange only the
timing barrier and the maximum (and sum) of their values; the reference arm
runs on rank 0 alone."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r = bench.Ranks(world, backend="gloo", device="cpu")
    r.barrier()
    value = 10.0 * (rank + 1)
    out[rank] = (r.max(value), r.sum(value))
    # reference arm: ranks other than 0 return without output
    if rank != 0:
        buf = io.StringIO()
        with redirect_stdout(buf):
            rc = bench.reference_arm(None, rank, world)
        out[world + rank] = (rc, buf.getvalue())
    r.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_and_sum():
    ctx = mp.get_context("spawn")
    world, port = 2, _free_port()
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    assert res[0] == (20.0, 30.0) and res[1] == (20.0, 30.0)
    assert res[3] == (0, "")


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks(1, backend="gloo", device="cpu")
    r.barrier()
    assert r.max(3.5) == 3.5 and r.sum(2.0) == 2.0
