"""Multi-process host logic of the replicas-only benchmark (no GPU): two gloo ranks on the CPU
each time their own replica; the job time is the slowest rank's and the value counts every
rank's cells. The reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.replica_time(1.0 + 0.5 * rank, dist, "cpu")
    out[rank] = (t, bench.replica_value(world, 1000, 10, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_every_replica():
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 1.5
    assert res[0][1] == pytest.approx(2 * 1000 * 10 / 1.5)


def test_single_process_run_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_time(0.25) == 0.25
    assert bench.replica_value(1, 100, 4, 0.5) == 800


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        grid, steps, warmup, gpus = 512, 1, 3, 2
    assert bench.reference_arm(Args(), 2, 1) is None
    assert capsys.readouterr().out == ""
