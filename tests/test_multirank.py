"""The N>1 bench path on CPU with gloo (world size 2): each rank simulates its
own independent patterns and the job time is the slowest rank's."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    g, shapes = bench.rank_batch(rank, 4)
    sig = [round(float(s.alm[3]), 12) for s in shapes]
    # every rank reports its shard; gather on all ranks
    gathered = [None] * world
    dist.all_gather_object(gathered, sig)
    t = bench.max_over_ranks(1.0 + rank, dist, "cpu")
    out[rank] = (gathered, t)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    g0, t0 = res[0]
    g1, t1 = res[1]
    assert t0 == t1 == 2.0                                  # max over ranks
    assert g0 == g1                                         # both ranks see the same shards
    assert len(g0[0]) == len(g0[1]) == 4
    assert not set(g0[0]) & set(g0[1])                      # disjoint patterns


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
