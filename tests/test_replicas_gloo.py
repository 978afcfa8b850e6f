"""The multi-GPU path of the bench is replicas only (one lattice per rank,
weak scaling, no data-path collective): its timing takes the slowest rank's
time and counts every rank's node updates.  Checked here with two gloo ranks
on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world)  # rank 1 is the slower one
    out[rank] = (ms, bench.replica_throughput(1_000_000, world, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_time_by_slowest_rank_and_count_all_updates():
    world = 2
    with mp.get_context("spawn").Manager() as mgr:  # no fork of this multi-threaded process
        out = mgr.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    # 2 ranks x 1e6 updates in 15 ms
    assert res[0][1] == pytest.approx(2e6 / 15e-3 / 1e6)


def test_one_rank_is_the_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.replica_throughput(1e6, 1, 1000.0) == pytest.approx(1.0)
