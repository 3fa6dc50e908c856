"""The multi-process path of bench.py (replicas only: one independent run
per rank, the slowest rank's time, whole-job throughput) on world_size 2
with the gloo backend on the host."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r took 1 + r seconds for 3 steps
    value, t = bench.replica_throughput(3, 1.0 + rank, world)
    dist.barrier()
    out[rank] = (value, t)
    dist.destroy_process_group()


def test_replicas_report_whole_job_throughput_over_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        value, t = res[r]
        assert t == 2.0                     # the slowest rank's time on every rank
        assert value == pytest.approx(3.0)  # 2 ranks x 3 steps / 2 s


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.replica_throughput(5, 2.0, 1) == (2.5, 2.0)
