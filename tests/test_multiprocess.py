"""The N > 1 path of bench.py on CPU: two gloo ranks (world_size 2) aggregate their
timings with the max-over-ranks rule and compute the whole-job rate.  The
factorization itself does not shard (independent replicas); only this host-side
aggregation runs across ranks."""
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


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_seconds = 1.0 + rank          # rank 1 is the slower one
    mx = bench.reduce_max(local_seconds, world)
    rate = bench.whole_job_rate(10.0, mx, world)
    out[rank] = (mx, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_and_rate():
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    assert out[0] == out[1]
    mx, rate = out[0]
    assert mx == 2.0                     # the slowest rank's time
    assert rate == 2 * 10.0 / 2.0        # units of all ranks over that time


def test_single_process_identity():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.whole_job_rate(4.0, 2.0, 1) == 2.0
