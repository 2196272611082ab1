"""The N > 1 path of bench.py on CPU: independent replicas, max-over-ranks time.

Two gloo ranks on 127.0.0.1 report different local times and units; both
must get the job time (the slower rank) and the summed throughput. No GPU.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [10.0, 25.0][rank]
        units = [1.0e9, 3.0e9][rank]
        job_ms, value = bench.aggregate_ranks(ms, units, dist, device="cpu")
        dist.barrier()
        out[rank] = (job_ms, value)
    finally:
        dist.destroy_process_group()


def test_replicas_take_max_time_and_sum_units():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        job_ms, value = res[r]
        assert job_ms == 25.0
        assert value == pytest.approx(4.0e9 / 0.025)


def test_single_rank_aggregate_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(20.0, 1.0e9) == (20.0, 1.0e9 / 0.02)
