"""Host-side helpers of bench.py that need no GPU: the sysfs cpulist parser used to
place page-locked buffers near the GPU, the panel width the reference arm reports
(it must match what the library resolves for nb = 0), and the sizes of the serving
and batched workloads."""
import json
import os

import numpy as np

import bench
from paper_2411_09859_gb300 import inputs, shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parse_cpulist():
    assert bench.parse_cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench.parse_cpulist("5") == {5}
    assert bench.parse_cpulist("") == set()
    assert bench.parse_cpulist("0-0,2-2") == {0, 2}


def test_table_nb_matches_the_saved_table_and_the_builtin_rule():
    with open(os.path.join(ROOT, "paper_2411_09859_gb300", "nb_table.json")) as f:
        table = json.load(f)["table"]
    for entry in table:                            # (n_upper, nb[, look-ahead])
        hi, nb = entry[0], entry[1]
        assert bench.table_nb(hi) == nb            # the range's upper end
    assert bench.table_nb(table[-1][0] * 2) == table[-1][1]   # beyond: the last entry
    # orders of the at-scale configuration take the width the bench reports
    for n in (4096, 8192, 16384):
        assert bench.table_nb(n) in (32, 48, 64, 96)


def test_serving_and_batched_workload_shapes():
    # the serving orders: even, log-uniform in [32, 4096] (seed 6), as in bench.py
    rng = np.random.default_rng(inputs.SEED_SERVING)
    logn = rng.uniform(np.log(32), np.log(4096), size=20000)
    sizes = np.clip(2 * np.round(np.exp(logn) / 2), 32, 4096).astype(np.int64)
    assert (sizes % 2 == 0).all() and sizes.min() >= 32 and sizes.max() <= 4096
    # log-uniform: about a third of the requests in each factor-of-five band
    assert 0.2 < np.mean(sizes <= 160) < 0.45
    # the batched orders: even, uniform in [16, 256]
    b = inputs.batched_sizes(4096)
    assert (b % 2 == 0).all() and b.min() >= 16 and b.max() <= 256
    assert len(set(b.tolist())) > 100                 # nearly all 121 orders occur
    # every share of the batch is balanced for 2..8 ranks
    for parts in (2, 4, 8):
        assert shard.imbalance(b, shard.balanced_bins(b, parts)) < 1.001
