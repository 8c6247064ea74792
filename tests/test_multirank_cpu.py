"""Host-side multi-rank logic of the benchmark on CPU (gloo, world size 2):
instance sharding by rank and the max-over-ranks throughput aggregation."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    insts = bench.rank_instances(rank, nz=10, groups=((8, 2), (16, 1)))
    pts = sum(w.nx * w.ny * w.nz for w in insts)
    fake_seconds = 1.0 + rank            # rank 1 is the slowest
    value, t = bench.aggregate_rate(pts, fake_seconds, world)
    out[rank] = (value, t, pts, [w.p1 for w in insts])
    dist.destroy_process_group()


def test_sharding_and_aggregation_two_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()   # no fork of this multi-threaded process
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    (v0, t0, p0, pw0), (v1, t1, p1, pw1) = out[0], out[1]
    assert t0 == t1 == 2.0                       # max over ranks
    assert v0 == v1 == pytest.approx((p0 + p1) / 2.0)
    assert pw0 != pw1                            # independent instance sets
