"""The multi-GPU path is replicas only: each rank solves its own seeded batch and
the ranks meet only for timing (max of the times, sum of the work).  Tested with
two gloo processes on the CPU."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, u = bench.replica_aggregate(dist, "cpu", seconds=1.5 * (rank + 1), units=8 + rank)
    p = bench.rank_batch(rank, mesh=4, nrhs=2)
    out[rank] = (t, u, p.b.copy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_aggregate_max_time_and_total_work():
    world = 2
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        t, u, _ = out[r]
        assert t == 3.0 and u == 17.0
    # each rank solves its own batch: different seeded right-hand sides
    assert not np.array_equal(out[0][2], out[1][2])


def test_single_process_aggregate_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_aggregate(None, "cpu", 2.5, 8) == (2.5, 8.0)
