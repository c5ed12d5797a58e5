"""The multi-GPU reporting of bench.py runs independent replicas (the path
does not shard): the job value is every rank's work over the slowest rank's
time.  Checked here with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) seconds for 1e6 units
        value, seconds = bench.job_throughput(1.0 + rank, 1e6)
        out[rank] = (value, seconds)
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_total_work_over_slowest_rank():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        value, seconds = res[r]
        assert seconds == pytest.approx(2.0)
        assert value == pytest.approx(2e6 / 2.0)


def test_single_process_is_its_own_job():
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    assert bench.job_throughput(0.5, 1e6) == (2e6, 0.5)
