"""Host logic of the multi-GPU batched and serving forms: the size-balanced partition
of independent matrices over ranks, checked for coverage, determinism and balance
against Graham's bound for the longest-processing-time rule, and used by two gloo
ranks that each take their share and gather the results."""
import os
import socket

import numpy as np
import pytest

from paper_2411_09859_gb300 import inputs, shard


def _exact_cover(bins, count):
    allidx = np.concatenate(bins) if bins else np.array([], dtype=np.int64)
    return sorted(allidx.tolist()) == list(range(count))


@pytest.mark.parametrize("parts", [1, 2, 3, 4, 8])
def test_batched_workload_partition(parts):
    sizes = inputs.batched_sizes(4096)
    bins = shard.balanced_bins(sizes, parts)
    assert len(bins) == parts
    assert _exact_cover(bins, len(sizes))
    assert all((np.diff(b) > 0).all() for b in bins)          # sorted, no repeats
    # Graham: LPT makespan <= (4/3 - 1/(3m)) OPT, OPT >= max(total/m, largest job)
    w = shard.work_of(sizes)
    lower = max(w.sum() / parts, w.max())
    assert max(w[b].sum() for b in bins) <= (4 / 3 - 1 / (3 * parts)) * lower + 1e-6
    # and on this many small jobs the shares are nearly equal
    assert shard.imbalance(sizes, bins) < 1.001


def test_deterministic_and_tie_rules():
    sizes = [64] * 6                      # equal work: round-robin by index
    bins = shard.balanced_bins(sizes, 3)
    assert [b.tolist() for b in bins] == [[0, 3], [1, 4], [2, 5]]
    assert [b.tolist() for b in shard.balanced_bins(sizes, 3)] == [b.tolist() for b in bins]


def test_one_big_job_and_more_parts_than_jobs():
    bins = shard.balanced_bins([4096, 32, 32, 32], 2)
    assert [b.tolist() for b in bins] == [[0], [1, 2, 3]]
    bins = shard.balanced_bins([16, 16], 4)
    assert _exact_cover(bins, 2) and sum(len(b) == 0 for b in bins) == 2
    with pytest.raises(ValueError):
        shard.balanced_bins([16], 0)


def test_lpt_worst_case_matches_graham_bound():
    # the classical tight instance for m = 2: jobs 3, 3, 2, 2, 2 (LPT 7, optimum 6)
    n = np.cbrt(np.array([3, 3, 2, 2, 2]) * 3.0)
    bins = shard.balanced_bins(n, 2)
    loads = sorted(float(shard.work_of(n)[b].sum()) for b in bins)
    assert loads == pytest.approx([5.0, 7.0])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    from paper_2411_09859_gb300 import inputs as inp, shard as sh
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = inp.batched_sizes(256)
    mine = sh.balanced_bins(sizes, world)[rank]
    # a stand-in per-matrix result (the order) for this rank's share, gathered at the end
    results = [(int(i), int(sizes[i])) for i in mine]
    gathered = [None] * world
    dist.all_gather_object(gathered, results)
    out[rank] = gathered
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_disjoint_shares_and_gather():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    assert out[0] == out[1]
    merged = sorted(x for part in out[0] for x in part)
    sizes = inputs.batched_sizes(256)
    assert merged == [(i, int(sizes[i])) for i in range(256)]
    assert torch is not None
