"""Host logic of the multi-GPU path, which is replicas only: every rank solves
its own instance and the job's time is the slowest rank's.  Two gloo ranks on
the CPU check the max-over-ranks reduction bench.py applies to the timed
region (no GPU, no data-path collective)."""
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


def _rank(rank, world, port, times, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        out[rank] = bench.max_over_ranks(dist, times[rank])
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("times", [[12.5, 30.25], [41.0, 7.0]])
def test_max_over_two_gloo_ranks(times):
    out = mp.Manager().dict()
    mp.start_processes(_rank, args=(2, _free_port(), times, out), nprocs=2, join=True, start_method="spawn")
    assert out[0] == out[1] == max(times)
