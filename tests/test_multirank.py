"""The N > 1 path of bench.py (replicas, no collective on the data path):
whole-job throughput = units of all ranks / slowest rank's time, computed
with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, root, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, root)
    import bench
    # rank 0 took 10 ms for 1000 units, rank 1 took 20 ms for 1000 units
    value, tmax = bench.job_value(1000, 10.0 * (rank + 1), world, torch.device("cpu"))
    out[rank] = (value, tmax)
    dist.barrier()
    dist.destroy_process_group()


def test_job_value_two_gloo_ranks(root_dir):
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), root_dir, out), nprocs=world, join=True)
    for r in range(world):
        value, tmax = out[r]
        assert tmax == pytest.approx(20.0)
        assert value == pytest.approx(2000 / 0.020)


def test_job_value_single_rank(root_dir):
    sys.path.insert(0, root_dir)
    import bench
    value, t = bench.job_value(500, 5.0, 1)
    assert value == pytest.approx(1e5) and t == 5.0
