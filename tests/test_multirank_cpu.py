"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the step time of a run is the slowest rank's,
and the whole-job PID divides it by the DOF of all ranks (each rank advances its own copy of the workload)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        ms = 1.0 + rank  # rank 1 is the slow one
        slowest = bench.max_over_ranks(ms, torch.device("cpu"))
        out[rank] = (slowest, bench.whole_job_pid(slowest, 262144, world))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_and_whole_job_pid():
    import bench
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0][0] == out[1][0] == 2.0
    expected = 2.0 * 1e6 / (bench.STAGES * 262144 * 2)
    assert abs(out[0][1] - expected) < 1e-12 and abs(out[1][1] - expected) < 1e-12


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, torch.device("cpu")) == 3.5
    assert bench.whole_job_pid(1.0, 1000, 1) == 1e6 / (bench.STAGES * 1000)
