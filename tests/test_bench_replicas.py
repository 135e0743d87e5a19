"""The replica job's accounting in bench.py (N > 1: one independent replica per
rank) on two gloo ranks on the CPU: the time is the slowest rank's, the work is
summed, and one rank alone reduces to its own figures."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    work = [1000.0, 3000.0][rank]
    secs = [2.0, 5.0][rank]
    out[rank] = (bench.rank_reduce(secs, "max", dist), bench.rank_reduce(work, "sum", dist),
                 bench.replica_value(work, secs, dist))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    for r in (0, 1):
        tmax, wsum, val = out[r]
        assert tmax == 5.0 and wsum == 4000.0
        assert val == pytest.approx(800.0)


def test_single_rank_is_its_own_figure():
    import bench
    assert bench.rank_reduce(3.5, "max") == 3.5
    assert bench.replica_value(100.0, 4.0) == 25.0
