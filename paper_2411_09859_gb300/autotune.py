"""Panel-width autotuner: times the factorization on this device for candidate panel
widths at a set of orders, and installs the fastest width per order range as the
library's default (skew_set_nb_table); likewise the batched kernels' panel width per
order bucket (skew_set_batched_nb_table), timed on batches of that bucket.  The result is saved as JSON beside this file
(``nb_table.json``) and installed again by the package at import.

    python -m paper_2411_09859_gb300.autotune [--sizes 512,2048,4096,8192,16384]
                                              [--candidates 32,48,64,96,128] [--reps 2]

Panel widths above 96 use the global-memory panel (the shared-memory one holds at most
96 columns per row); the candidates include 128 so that the table records what that
costs.  The batched kernels are tuned over two parameters per order bucket: the panel
width (8, 16, 32) and the trailing update's warp tile (16 or 32).

The inputs are the synthetic iid N(0,1) skew matrices of ``inputs.skew_gaussian``.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics

TABLE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "nb_table.json")


def measure(n: int, nb: int, reps: int, seed: int = 17, lookahead: bool = False) -> float:
    """Median milliseconds of skew_ltlt (FP64 update, with L) at order n, width nb, on
    the look-ahead path or the plain one."""
    import torch

    from . import _native as nat
    from . import inputs
    old = nat.set_lookahead(2 if lookahead else 0)
    try:
        return _measure(n, nb, reps, seed)
    finally:
        nat.set_lookahead(old)


def _measure(n: int, nb: int, reps: int, seed: int) -> float:
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


def pick_path(ms_by_key: dict):
    """(nb, lookahead) from timings keyed "nb" (plain path) and "nb+la" (look-ahead):
    among the choices within TIE of the fastest, the plain path first (it needs less
    workspace), then the smallest width."""
    best = min(ms_by_key.values())
    close = [k for k, v in ms_by_key.items() if v <= best * (1.0 + TIE)]
    key = min(close, key=lambda k: (k.endswith("+la"), int(str(k).split("+")[0])))
    return int(str(key).split("+")[0]), 1 if str(key).endswith("+la") else 0


def table_from_ms(ms: dict):
    """[(n, nb, lookahead) ...] in increasing n: the range (previous n, n] takes the
    width and path picked at n."""
    out = []
    for n, d in sorted(ms.items(), key=lambda e: int(e[0])):
        nb, la = pick_path({str(k): v for k, v in d.items()})
        out.append((int(n), nb, la))
    return out


def tune(sizes=(512, 2048, 4096, 8192, 16384), candidates=(32, 48, 64, 96, 128), reps: int = 2):
    """Returns ``{"table": [(n_upper, nb, lookahead), ...], "ms": {n: {key: ms}}}`` with
    key "nb" for the plain path and "nb+la" for the look-ahead (widths up to 64)."""
    from . import _native as nat
    sizes = sorted(int(s) for s in sizes)
    ms = {}
    for n in sizes:
        d = {}
        for nb in candidates:
            if nb >= n:
                continue
            d[str(nb)] = measure(n, nb, reps)
            old = nat.set_lookahead(2)
            try:
                la_ok = nat.lookahead_used(n, nb)
            finally:
                nat.set_lookahead(old)
            if la_ok:
                d[f"{nb}+la"] = measure(n, nb, reps, lookahead=True)
        ms[n] = d
    return {"table": table_from_ms(ms), "tie": TIE,
            "ms": {str(n): d for n, d in ms.items()}}


BUCKETS = (64, 128, 256, 512)      # order buckets of the batched kernels
BATCHED_NB = (8, 16, 32)
BATCHED_WT = (16, 32)


def _batch(sizes, seed_base: int):
    """Device buffers of one batch of iid skew matrices of the given orders."""
    import numpy as np
    import torch

    from . import _native as nat
    from . import inputs
    mats = [inputs.skew_gaussian(int(n), seed_base + i) for i, n in enumerate(sizes)]
    offs = np.concatenate([[0], np.cumsum(np.asarray(sizes, dtype=np.int64) ** 2)])
    flat = np.empty(int(offs[-1]))
    for i, A in enumerate(mats):
        flat[offs[i]:offs[i + 1]] = A.ravel(order="F")
    pristine = torch.from_numpy(flat).cuda()
    work = torch.empty_like(pristine)
    views = [work[int(offs[i]):int(offs[i + 1])].view(int(n), int(n)).t()
             for i, n in enumerate(sizes)]
    ts = [torch.empty(max(int(n) - 1, 1), dtype=torch.float64, device="cuda") for n in sizes]
    pivs = [torch.empty(max(int(n), 1), dtype=torch.int32, device="cuda") for n in sizes]
    table = nat.problem_table(views, [None] * len(views), ts, pivs, "cuda")
    return pristine, work, views, ts, pivs, table


def measure_batched_mix(sizes, table_nb, reps: int = 2, batch=None) -> float:
    """Median milliseconds of skew_ltlt_batched plus skew_pfaffian_batched on one batch
    of the given orders, with the bucket table `table_nb` installed."""
    import torch

    from . import _native as nat
    pristine, work, views, ts, pivs, table = batch or _batch(sizes, 50000)
    mx = int(max(sizes))
    nat.set_batched_nb_table(table_nb)
    stream = torch.cuda.Stream()
    total = 0.0
    for fn in (lambda: nat.ltlt_batched(views, stream=stream, max_n=mx, table=table,
                                        outs=(ts, pivs, [None] * len(views))),
               lambda: nat.pfaffian_batched(views, stream=stream, max_n=mx, table=table,
                                            outs=(ts, pivs))):
        times = []
        for i in range(reps + 1):
            work.copy_(pristine)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            if i > 0:
                times.append(e0.elapsed_time(e1))
        total += statistics.median(times)
    return total


def tune_batched(sizes=None, buckets=BUCKETS, candidates=BATCHED_NB, tiles=BATCHED_WT,
                 reps: int = 2):
    """The batched kernels' panel width and update warp tile per order bucket, and the
    CTA size of the blocked kernels, chosen on a workload mix (default: the batched
    workload, 4096 orders even in [16, 256]).  For each CTA size (256, then 128
    threads): every combination of widths over the buckets the mix populates is timed
    with warp tile 32 (both batched kernels, summed), then, with those widths, every
    combination of warp tiles.  The fastest CTA size wins (256 unless 128 is faster by
    more than the tie margin).  A bucket the mix does not reach takes the fastest
    (width, tile) on a batch of its own orders."""
    import itertools

    from . import _native as nat
    from . import inputs
    if sizes is None:
        sizes = inputs.batched_sizes(4096)
    sizes = [int(n) for n in sizes]
    batch = _batch(sizes, 50000)
    lows = [16] + [b + 2 for b in buckets[:-1]]
    used = [hi for lo, hi in zip(lows, buckets) if any(lo <= n <= hi for n in sizes)]
    per_thr = {}
    for thr in (256, 128):
        old_thr = nat.set_batched_threads(thr)
        try:
            mix_ms = {}
            for combo in itertools.product(candidates, repeat=len(used)):
                tab = [(hi, nb, 32) for hi, nb in zip(used, combo)]
                mix_ms[combo] = measure_batched_mix(sizes, tab, reps, batch)
            best_nb = dict(zip(used, min(mix_ms, key=mix_ms.get)))
            wt_ms = {}
            for combo in itertools.product(tiles, repeat=len(used)):
                tab = [(hi, best_nb[hi], wt) for hi, wt in zip(used, combo)]
                wt_ms[combo] = measure_batched_mix(sizes, tab, reps, batch)
            best_wt = dict(zip(used, min(wt_ms, key=wt_ms.get)))
        finally:
            nat.set_batched_threads(old_thr)
        per_thr[thr] = (min(wt_ms.values()), best_nb, best_wt, mix_ms, wt_ms)
    best_thr = 128 if per_thr[128][0] < per_thr[256][0] * (1.0 - TIE) else 256
    _, best_nb, best_wt, mix_ms, wt_ms = per_thr[best_thr]
    del batch
    extra = {}
    old_thr = nat.set_batched_threads(best_thr)
    try:
        for lo, hi in zip(lows, buckets):
            if hi in best_nb:
                continue
            own = [lo + 2 * ((hi - lo) // 4)] * 256
            extra[hi] = {(nb, wt): measure_batched_mix(own, [(hi, nb, wt)], reps)
                         for nb in candidates for wt in tiles}
            fastest = min(extra[hi].values())
            nb, wt = min(k for k, v in extra[hi].items() if v <= fastest * (1.0 + TIE))
            best_nb[hi], best_wt[hi] = nb, wt
    finally:
        nat.set_batched_threads(old_thr)
    return {"batched_table": [(hi, best_nb[hi], best_wt[hi]) for hi in buckets],
            "batched_threads": best_thr,
            "batched_threads_best_ms": {str(t): v[0] for t, v in per_thr.items()},
            "batched_mix_ms": {",".join(map(str, k)): v for k, v in mix_ms.items()},
            "batched_mix_warp_tile_ms": {",".join(map(str, k)): v for k, v in wt_ms.items()},
            "batched_mix_buckets": used,
            "batched_own_ms": {str(h): {f"{a},{b}": v for (a, b), v in d.items()}
                               for h, d in extra.items()}}


def save(result, path: str = TABLE_PATH):
    import torch
    out = dict(result)
    out["device"] = torch.cuda.get_device_name()
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


def load(path: str = TABLE_PATH) -> bool:
    """Install saved tables if there are any; returns whether it did."""
    if not os.path.exists(path):
        return False
    with open(path) as f:
        saved = json.load(f)
    from . import _native as nat
    nat.set_nb_table([tuple(e) for e in saved.get("table", [])])
    nat.set_batched_nb_table([tuple(e) for e in saved.get("batched_table", [])])
    nat.set_batched_threads(int(saved.get("batched_threads", 256)))
    return True


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--sizes", default="512,2048,4096,8192,16384")
    ap.add_argument("--candidates", default="32,48,64,96,128")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--no-save", action="store_true")
    ap.add_argument("--batched-only", action="store_true",
                    help="tune only the batched kernels' widths (keep the saved panel table)")
    args = ap.parse_args()
    from . import _native as nat
    res = {}
    if os.path.exists(TABLE_PATH):
        with open(TABLE_PATH) as f:
            res = json.load(f)
    for stale in ("batched_note", "command"):
        res.pop(stale, None)
    if not args.batched_only:
        res.update(tune([int(x) for x in args.sizes.split(",")],
                        [int(x) for x in args.candidates.split(",")], args.reps))
        nat.set_nb_table(res["table"])
    res.update(tune_batched(reps=args.reps))
    nat.set_batched_nb_table(res["batched_table"])
    nat.set_batched_threads(res["batched_threads"])
    res["command"] = ("python -m paper_2411_09859_gb300.autotune "
                      + ("--batched-only " if args.batched_only else
                         f"--sizes {args.sizes} --candidates {args.candidates} ")
                      + f"--reps {args.reps} (the smallest width within {TIE * 100:.1f} % "
                      "of the fastest is kept; batched: widths over the mix's buckets with "
                      "warp tile 32, then warp tiles with those widths, then 256 or 128 threads per CTA)")
    if not args.no_save:
        save(res)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
