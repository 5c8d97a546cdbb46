"""The multi-process side of bench.py on the CPU (gloo, world size 2): each
rank runs its own replica, the job time is the slowest rank's, the value
counts the views of every rank, and the oracle arm runs on rank 0 only."""
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


def _rank_main(rank, world, port, times, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as tdist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        barrier, max_over_ranks = bench.rank_collectives(tdist, "cpu")
        barrier()
        t = max_over_ranks(times[rank])
        out[rank] = (t, bench.job_throughput(world, 100, 8, 5, t))
        barrier()
    finally:
        tdist.destroy_process_group()


def test_slowest_rank_sets_the_job_time():
    world = 2
    times = [0.75, 1.25]
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), times, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, v = res[r]
        assert t == max(times)
        assert v == pytest.approx(world * 100 * 8 * 5 / max(times))


def test_single_process_collectives_are_identities():
    sys.path.insert(0, ROOT)
    import bench
    barrier, max_over_ranks = bench.rank_collectives(None, "cpu")
    barrier()
    assert max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(1, 10, 2, 3, 2.0) == 30.0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        cpu_views = 6
        warmup = 0
        steps = 1
        gpus = 2

    bench.run_reference(Args, world=2, rank=1)
    assert capsys.readouterr().out == ""
