"""The whole-job aggregation of bench.py across ranks, on CPU with the gloo
backend (world size 2): every rank learns the slowest rank's time, and the
rate counts the units of all ranks over that time.  On the GPU the same
helpers run over NCCL with one independent replica per rank (no collective
on the data path)."""
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
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_max = bench.max_over_ranks(times[rank], world, "cpu")
        out[rank] = (ms_max, bench.whole_job_rate(10, world, ms_max))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    world, port = 2, _free_port()
    times = [120.0, 250.0]                      # rank 1 is the slowest
    with mp.get_context("spawn").Manager() as m:   # no fork of a process with threads
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, times, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 250.0
    # 10 units a rank, 2 ranks, 0.25 s: 80 units per second, the same on every rank
    assert res[0][1] == res[1][1] == pytest.approx(80.0)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, None) == 12.5
    assert bench.whole_job_rate(2 * 5, 1, 1000.0) == pytest.approx(10.0)
