"""Multi-process (replica) logic of bench.py on the CPU: world size 2 over gloo.

The path shards by problem: every rank runs its own replica and the job's throughput is the
steps of all ranks over the slowest rank's time.  This checks the rank bookkeeping (barrier,
max-over-ranks timing, aggregate value) without a GPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 100.0 + 50.0 * rank  # rank 1 is the slowest
        ms, value = bench.aggregate_replicas(ms_local, steps=10, world=world)
        out[rank] = (ms, value)
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_world_size_2():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, value = out[r]
        assert ms == pytest.approx(150.0)                 # max over ranks
        assert value == pytest.approx(world * 10 / 0.150)  # all ranks' steps / slowest time
