"""The multi-rank host path of bench.py on CPU: two gloo ranks (127.0.0.1) with different
timed regions; both must see the slowest rank's time, and the whole-job rate counts the
units of every rank over that time (replicas: each rank runs the full workload)."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_s = [0.25, 0.40][rank]
        dist.barrier()
        t = bench.reduce_max(local_s, world, "cpu")
        out[rank] = (t, bench.whole_job_rate(3, world, t))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_and_whole_job_rate():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as mgr:   # no fork of this multi-threaded process
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == pytest.approx(0.40)
    assert res[0][1] == res[1][1] == pytest.approx(2 * 3 / 0.40)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(1.5, 1, None) == 1.5
    assert bench.whole_job_rate(4, 1, 2.0) == 2.0
