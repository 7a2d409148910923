"""The N > 1 path of bench.py on CPU: two gloo ranks run replicas, the whole-job value is all
ranks' digits over the slowest rank's time (the path does not shard, so there is no data-path
collective; only this max-reduction of the timing)."""
import os
import socket

import pytest
import torch
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
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 if rank == 0 else 250.0  # rank 1 is the slow one
    value, tot = bench.aggregate(local_ms, 1000, 10, world)
    out[rank] = (value, tot)
    dist.destroy_process_group()


def test_replica_aggregation_gloo():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    for r in range(world):
        value, tot = out[r]
        assert tot == pytest.approx(250.0)
        assert value == pytest.approx(1000 * 10 * 2 / 0.25)


def test_single_rank_aggregation():
    import bench
    v, t = bench.aggregate(50.0, 2 * 2**24, 4, 1)
    assert t == 50.0 and v == pytest.approx(2 * 2**24 * 4 / 0.05)
