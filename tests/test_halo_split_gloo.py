"""The slab split a single problem would use across GPUs, simulated with two
gloo ranks on the CPU: each rank owns half of a periodic 2D mesh (columns),
keeps one ghost column on either side, and exchanges its boundary columns
with the other rank before evaluating the oracle on its slab.  A cell's DG
right-hand side and limiter need only the cell and its face neighbours, so
the owned columns reproduce the single-domain results: the limiter bit for
bit, the right-hand side to rounding (a cell's face contributions are summed
in another order at the periodic seam)."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NX, NY, K, SEED = 8, 6, 2, 2024
DX = 0.125  # small enough that the TVB bound Mtilde dx lets the limiter act


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _global_state(N):
    sys.path.insert(0, ROOT)
    from paper_1506_06140_gb300 import workloads as wl
    W = wl.random_weights(2, N, NX * NY, seed=SEED, slope=0.2)
    return W.reshape(4, N, NY, NX)  # [var][coef][y][x]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from oracle import pyoracle as O
    dist.init_process_group("gloo", rank=rank, world_size=world)
    half = NX // world
    probe = O.Oracle(2, [NX, NY], [0.0, 0.0], [NX * DX, NY * DX], K, 1.4)
    own = _global_state(probe.N)[:, :, :, rank * half:(rank + 1) * half].copy()  # this rank's columns
    # halo exchange: my first column goes to the left neighbour, my last to the right one
    left, right = (rank - 1) % world, (rank + 1) % world
    send_l = torch.from_numpy(own[:, :, :, 0].copy())
    send_r = torch.from_numpy(own[:, :, :, -1].copy())
    recv_l, recv_r = torch.empty_like(send_l), torch.empty_like(send_r)
    # tag 0: leftward messages (a rank's first column, received by its left
    # neighbour as that rank's right ghost); tag 1: rightward ones.  With two
    # ranks left == right, so the tags, not the posting order, pair them.
    reqs = [dist.isend(send_l, left, tag=0), dist.isend(send_r, right, tag=1),
            dist.irecv(recv_r, right, tag=0), dist.irecv(recv_l, left, tag=1)]
    for q in reqs:
        q.wait()
    slab = np.concatenate([recv_l.numpy()[..., None], own, recv_r.numpy()[..., None]], axis=3)
    nxl = half + 2
    o = O.Oracle(2, [nxl, NY], [0.0, 0.0], [nxl * DX, NY * DX], K, 1.4, bc=[O.BC_TRANSMISSIVE, O.BC_PERIODIC],
                 limiter=O.LIM_CHARACTERISTIC, positivity=True)
    Wl = slab.reshape(4, o.N, nxl * NY)
    rhs = o.rhs(Wl).reshape(4, o.N, NY, nxl)[:, :, :, 1:-1]
    lim = o.limit(Wl).reshape(4, o.N, NY, nxl)[:, :, :, 1:-1]
    out[rank] = (rhs.copy(), lim.copy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_slab_split_reproduces_single_domain():
    sys.path.insert(0, ROOT)
    from oracle import pyoracle as O
    o = O.Oracle(2, [NX, NY], [0.0, 0.0], [NX * DX, NY * DX], K, 1.4,
                 limiter=O.LIM_CHARACTERISTIC, positivity=True)
    W = _global_state(o.N).reshape(4, o.N, NX * NY)
    rhs_ref = o.rhs(W).reshape(4, o.N, NY, NX)
    lim_ref = o.limit(W).reshape(4, o.N, NY, NX)
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    rhs = np.concatenate([res[r][0] for r in range(world)], axis=3)
    lim = np.concatenate([res[r][1] for r in range(world)], axis=3)
    np.testing.assert_array_equal(lim, lim_ref)
    np.testing.assert_allclose(rhs, rhs_ref, rtol=0, atol=1e-13 * np.abs(rhs_ref).max())
    assert not np.array_equal(lim_ref, W.reshape(lim_ref.shape))  # the limiter acted somewhere
