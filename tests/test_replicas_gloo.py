"""N > 1 is replicas only (one independent solve per rank, no data-path
collective).  The host logic of that path runs here on CPU with two gloo
ranks: each rank draws its own seeded workload, and the reported time is the
maximum over ranks."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        import workloads as W
        prob = W.checkerboard_square(N=33, J=4, ncell=4, values=(1.0, 1e4), batch=1, seed=r)
        mine = [10.0 + r, 5.0 * (world - r), float(prob.f[0, 0])]
        agg = bench.max_over_ranks(mine, dist, torch.device("cpu"))
        out[rank] = (ws, r, local, mine, agg, float(prob.f.sum()))
    finally:
        dist.destroy_process_group()


def test_replica_timing_is_max_over_ranks():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    assert sorted(out.keys()) == [0, 1]
    mine = np.array([out[r][3] for r in range(world)])
    for r in range(world):
        ws, rr, local, _, agg, _ = out[r]
        assert (ws, rr, local) == (world, r, r)
        assert np.array_equal(agg, mine.max(axis=0))
    # each rank solves its own seeded problem (weak scaling: fixed work per rank)
    assert out[0][5] != out[1][5]
