"""Panel-width autotuner: times the factorization on this device for candidate panel
widths at a set of orders, and installs the fastest width per order range as the
library's default (skew_set_nb_table).  The result is saved as JSON beside this file
(``nb_table.json``) and installed again by the package at import.

    python -m paper_2411_09859_gb300.autotune [--sizes 512,2048,4096,8192,16384]
                                              [--candidates 32,48,64,96] [--reps 2]

The inputs are the synthetic iid N(0,1) skew matrices of ``inputs.skew_gaussian``.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics

TABLE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "nb_table.json")


def measure(n: int, nb: int, reps: int, seed: int = 17) -> float:
    """Median milliseconds of skew_ltlt (FP64 update, with L) at order n, width nb."""
    import torch

    from . import _native as nat
    from . import inputs
    A = torch.from_numpy(inputs.skew_gaussian(n, seed)).cuda()
    work = nat.fortran_empty(n, n, A.device)
    L = nat.fortran_empty(n, n, A.device)
    t = torch.empty(max(n - 1, 1), dtype=torch.float64, device=A.device)
    piv = torch.empty(n, dtype=torch.int32, device=A.device)
    stream = torch.cuda.Stream()
    times = []
    for i in range(reps + 1):
        work.copy_(A)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        nat.ltlt(work, nb=nb, stream=stream, L=L, t=t, piv=piv)
        e1.record(stream)
        torch.cuda.synchronize()
        if i > 0:
            times.append(e0.elapsed_time(e1))
    return statistics.median(times)


TIE = 0.005   # widths within 0.5 % of the fastest count as equally fast


def pick(ms_by_nb: dict) -> int:
    """The smallest width whose time is within TIE of the fastest (smaller panels need
    less workspace and stay within the split-precision limit of 64)."""
    best = min(ms_by_nb.values())
    return min(int(nb) for nb, v in ms_by_nb.items() if v <= best * (1.0 + TIE))


def table_from_ms(ms: dict):
    """[(n, pick(ms[n])) ...] in increasing n: the range (previous n, n] takes the width
    picked at n."""
    return [(int(n), pick(d)) for n, d in sorted(ms.items(), key=lambda e: int(e[0]))]


def tune(sizes=(512, 2048, 4096, 8192, 16384), candidates=(32, 48, 64, 96), reps: int = 2):
    """Returns ``{"table": [(n_upper, nb), ...], "ms": {n: {nb: ms}}}``."""
    sizes = sorted(int(s) for s in sizes)
    ms = {n: {nb: measure(n, nb, reps) for nb in candidates if nb < n} for n in sizes}
    return {"table": table_from_ms(ms), "tie": TIE,
            "ms": {str(n): {str(b): v for b, v in d.items()} for n, d in ms.items()}}


def save(result, path: str = TABLE_PATH):
    import torch
    out = dict(result)
    out["device"] = torch.cuda.get_device_name()
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


def load(path: str = TABLE_PATH) -> bool:
    """Install a saved table if there is one; returns whether it did."""
    if not os.path.exists(path):
        return False
    with open(path) as f:
        table = [tuple(e) for e in json.load(f)["table"]]
    from . import _native as nat
    nat.set_nb_table(table)
    return True


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--sizes", default="512,2048,4096,8192,16384")
    ap.add_argument("--candidates", default="32,48,64,96")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--no-save", action="store_true")
    args = ap.parse_args()
    res = tune([int(x) for x in args.sizes.split(",")], [int(x) for x in args.candidates.split(",")],
               args.reps)
    from . import _native as nat
    nat.set_nb_table(res["table"])
    if not args.no_save:
        save(res)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
