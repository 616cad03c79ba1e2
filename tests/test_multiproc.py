"""The multi-GPU path is replicas only: each rank transforms its own maps and the job time is
the slowest rank's.  These world-size-2 gloo tests run that host logic on CPU processes."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    items = bench.replica_items(rank)
    # every rank reports a different time; all must agree on the maximum
    t = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    gathered = [None] * world
    dist.all_gather_object(gathered, items)
    out[rank] = (t, gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_disjoint_and_max_time():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    a, b = res[0][1]
    assert len(a) == len(b) == 16 and not set(a) & set(b)   # no rank shares maps


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.replica_items(0) == list(range(16))
