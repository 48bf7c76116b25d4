"""The N > 1 path of bench.py is replicas: one independent solve stream per
rank, no collective on the data path; only the timing is reduced (max over
ranks) and rank 0 reports the whole job.  Checked here with two gloo ranks
on the CPU, through the same helpers bench.py calls."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.replica_barrier(world)
    t_local = 100.0 + 50.0 * rank          # rank 1 is the slower replica
    t_max = bench.replica_max(t_local, world, torch.device("cpu"))
    out[rank] = (t_max, bench.replica_value(world, 2 * 3, t_max))
    bench.replica_barrier(world)
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank():
    world = 2
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 150.0
    # 2 ranks x 6 solves in 150 ms
    assert res[0][1] == pytest.approx(2 * 6 / 0.150)


def test_single_process_needs_no_process_group():
    import bench
    assert bench.replica_max(7.0, 1, None) == 7.0
    assert bench.replica_value(1, 4, 2000.0) == 2.0
