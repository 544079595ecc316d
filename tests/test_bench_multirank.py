"""Host logic of the multi-rank bench (one process per GPU, replicas): the
whole-job value is the units of all ranks over the slowest rank's time.
Runs as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 250.0][rank]
    out[rank] = bench.job_throughput(local_ms, steps=5, k=1000, world=world, device="cpu")
    dist.destroy_process_group()


def test_job_throughput_takes_the_slowest_rank():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn")
    for r in range(world):
        ms, value = out[r]
        assert ms == 250.0
        assert value == pytest.approx(world * 5 * 1000 / 0.25)


def test_job_throughput_single_rank():
    import bench
    ms, value = bench.job_throughput(100.0, steps=4, k=500, world=1, device="cpu")
    assert ms == 100.0 and value == pytest.approx(4 * 500 / 0.1)
