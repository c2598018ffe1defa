#!/usr/bin/env python
"""Benchmark of the pivoted skew-symmetric LTL^T factorization (FP64) on GB300.

One step = one whole factorization P A P^T = L T L^T (panel, pivot_rows, skew
rank-2k update, Pfaffian read-off) of an n = 16384 skew matrix with iid N(0, 1)
strictly lower entries (seed 3), counted as n^3 / 3 flops.  Inputs are resident in
HBM before the timed region: one fresh copy per step (2.1 GB each, larger than the
129 MB L2, so no flush is needed).  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank factors its own copy of the matrix (independent
replicas, no collective on the data path); the barrier and the max over ranks of
the timed region give the whole-job throughput.  The batched and serving legs split
their matrices / requests into size-balanced shares instead (one per rank), and
report all units over the slowest rank's time.

The same line carries the other forms: `e2e` (the host-buffer call, copies
included), `precision` (split-precision update; QDQ^T accuracy at n = 2048 against
the oracle and at n = 16384 against the closed form), `pfaffian_only` (the two-step
elimination), `batched` (4096 matrices of order 16..256 in one launch, LTL^T and
Pfaffian-only, with a CUDA graph replay), `serving` (Pfaffian-only requests of order
32..4096 against serial calls, saturation and Poisson streams; the factor-keeping
mode alongside), `cpu_baseline` (the oracle on the whole factorization, all host
cores, timed once) and `oracle_parity` (the timed GPU factors against the oracle's).
`--skip-<leg>` drops a leg; `--impl reference` times the oracle alone: the whole
factorization in W + K consecutive pieces of equal update work, K of them timed.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import queue
import re
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "skew LTLt FP64 TFLOP/s at n=16384 (% peak); batched Pfaffians/s, p99 latency"
UNIT = "TFLOP/s"
FP64_NOMINAL_TFLOPS = 1.25       # GB300 dense FP64 (nominal)
BF16_NOMINAL_TFLOPS = 2250.0     # GB300 dense bf16 (nominal)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--nb", type=int, default=0)
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--path", choices=["auto", "plain", "lookahead"], default="auto",
                    help="factorization path of the timed steps (auto: the library's choice "
                         "for the order)")
    ap.add_argument("--grid-panels", action="store_true",
                    help="grid-wide panels for every trailing block (skew_set_cluster_panel(0))")
    ap.add_argument("--la-switch", type=int, default=-1,
                    help="trailing order below which a look-ahead factorization goes on "
                         "without it (skew_set_lookahead_switch; -1: the library's default)")
    ap.add_argument("--skip-plain", action="store_true",
                    help="skip timing the other path (plain / look-ahead) beside the headline")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-batched", action="store_true")
    ap.add_argument("--skip-serving", action="store_true")
    ap.add_argument("--skip-precision", action="store_true")
    ap.add_argument("--qdq-full-n", type=int, default=16384,
                    help="order of the device-generated QDQ^T check (0: skip)")
    ap.add_argument("--skip-twostep", action="store_true",
                    help="skip the Pfaffian-only (two-step and one-step) leg")
    ap.add_argument("--qdq-n", type=int, default=2048)
    ap.add_argument("--serve-requests", type=int, default=20000,
                    help="requests of the serving stream (all of them at saturation)")
    ap.add_argument("--serve-poisson", type=int, default=2000,
                    help="first requests of the stream replayed as each Poisson stream")
    ap.add_argument("--serve-serial", type=int, default=2000,
                    help="first requests of the stream timed as serial calls")
    ap.add_argument("--serve-factors", type=int, default=1000,
                    help="first requests of the stream run with their factors kept")
    ap.add_argument("--plain-calls", type=int, default=1024,
                    help="matrices of the batched workload timed as back-to-back plain calls")
    return ap.parse_args()


def factorization_flops(n: int) -> float:
    return n ** 3 / 3.0


def workload_config(n: int, nb: int, seed: int) -> dict:
    return {"workload": f"plain pivoted LTL^T, n={n}, iid N(0,1) skew, seed {seed}",
            "n": n, "nb": nb, "seed": seed, "flops_per_step": "n^3/3",
            "l2": (f"inputs larger than L2: a fresh {n * n * 8 / 1e9:.2f} GB HBM-resident "
                   "copy per step"),
            "parallelism": "independent replicas (one matrix per GPU)"}


def table_nb(n: int) -> int:
    """The panel width the library picks for order n (nb = 0): from the saved tuned
    table when there is one, else its built-in rule (16 up to 256, 32 up to 2048, 64).
    Read from the file here so that the reference arm, which runs no GPU code, reports
    the same configuration as the GPU arm."""
    path = os.path.join(ROOT, "paper_2411_09859_gb300", "nb_table.json")
    try:
        with open(path) as f:
            table = json.load(f).get("table", [])
    except (OSError, ValueError):
        table = []
    for entry in table:                       # (n_upper, nb[, look-ahead])
        if n <= entry[0]:
            return int(entry[1])
    if table:
        return int(table[-1][1])
    return 16 if n <= 256 else (32 if n <= 2048 else 64)


# ----------------------------------------------------------------------------- peaks
def fp64_peak():
    """FP64 tensor peak per the measured bf16 figure x the nominal FP64:bf16 ratio."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    ratio = FP64_NOMINAL_TFLOPS / BF16_NOMINAL_TFLOPS
    try:
        with open(path) as f:
            mp = json.load(f)
        bf16 = float(mp["bf16_tflops_sustained"])
        return bf16 * ratio, (f"of measured: bf16_tflops_sustained {bf16} x FP64:bf16 "
                              f"nominal {FP64_NOMINAL_TFLOPS}/{BF16_NOMINAL_TFLOPS}")
    except (OSError, KeyError, ValueError):
        return 1700.0 * ratio, "of fallback: 1.7 PFLOP/s bf16 sustained x 1.25/2250"


def recorded_traffic():
    """DRAM bytes per algorithmic byte of the skr2k kernel from the committed ncu
    summary, if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "skr2k_fused_n8192.md")
    src = os.path.join(ROOT, "paper_2411_09859_gb300", "csrc", "skr2k.cu")
    try:
        text = open(path).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    m_sha = re.search(r"source_sha256[^:\n]*:\s*([0-9a-f]{64})", text)
    m_ratio = re.search(r"dram_bytes_per_algorithmic_byte:\s*([0-9.eE+-]+)", text)
    if not m_sha or not m_ratio or m_sha.group(1) != sha:
        return None
    return float(m_ratio.group(1))


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "note": "nvidia-smi unavailable"}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(self.NAMES, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- kernels
SIDE_STREAM_KERNELS = ("pivot_rows",)


def kernel_table(prof: dict, steps: int, total_ms: float, concurrent_panel: bool = False) -> dict:
    """Per-kernel time from the library's event pairs (recorded on each launch's own
    stream).  Kernels on the critical stream get ms per step and their share of the
    step.  A side-stream kernel (pivot_rows; with the look-ahead also the panel) runs
    beside the trailing update: its event span includes the time it waits for
    multiprocessors the update holds, so it is reported as a span only, with no share
    (its device time per launch is in the ncu launch list)."""
    out = {}
    side = SIDE_STREAM_KERNELS + (("panel",) if concurrent_panel else ())
    for k, v in prof.items():
        if not v["launches"]:
            continue
        row = {"launches_per_step": v["launches"] / steps}
        if k in side:
            row.update({"ms_per_step": None, "event_span_ms_per_step": v["ms"] / steps,
                        "share": None,
                        "note": "side stream, overlaps the trailing update; span, not "
                                "device time"})
        else:
            row.update({"ms_per_step": v["ms"] / steps,
                        "share": v["ms"] / total_ms if total_ms > 0 else None})
        out[k] = row
    return out


# ----------------------------------------------------------------------------- oracle
def update_work(n: int) -> np.ndarray:
    """Entries the rank-2 update of elimination step k touches, (n-k-2)(n-k-3)/2, for
    k = 0 .. n-2: the unit by which a piece of the oracle's factorization is credited
    with its share of the n^3/3 flops of the whole one."""
    k = np.arange(n - 1, dtype=np.float64)
    return np.maximum(n - k - 2, 0) * np.maximum(n - k - 3, 0) / 2.0


def oracle_full(A_host: np.ndarray) -> dict:
    """The CPU oracle (as it stands, all host cores) on the whole factorization of
    A_host, timed once from its set-up to its last elimination step.  Returns the
    baseline figures and the oracle's factors (for the parity check of the GPU run on
    the same matrix)."""
    import oracle
    n = A_host.shape[0]
    t0 = time.perf_counter()
    st = oracle.ltlt_begin(A_host)
    oracle.ltlt_continue(st, n - 1)
    sec = time.perf_counter() - t0
    return {"value": factorization_flops(n) / sec / 1e12, "unit": UNIT,
            "cores": oracle.threads(), "kind": "oracle",
            "sample": (f"full: the whole n={n} factorization (set-up and all {n - 1} "
                       f"elimination steps), timed once: {sec:.1f} s"),
            "seconds": sec, "L": st["L"], "t": st["t"], "piv": st["piv"],
            "info": st["info"]}


def oracle_parity(orc: dict, L_dev, t: np.ndarray, piv: np.ndarray, n: int) -> dict:
    """The GPU factors of the timed matrix against the oracle's: pivots, t and L
    element by element, and log|Pf| and sign read off each side's own factors."""
    import oracle
    eps = 2.0 ** -52
    tol = 2000.0 * n * eps
    dL = 0.0
    for j in range(0, n, 1024):
        blk = L_dev[:, j:j + 1024].cpu().numpy()
        dL = max(dL, float(np.max(np.abs(blk - orc["L"][:, j:j + 1024]))))
    t0, p0 = orc["t"], orc["piv"]
    dt = float(np.max(np.abs(t - t0))) / max(1.0, float(np.max(np.abs(t0))))
    la0, sg0 = oracle.pfaffian_from_factors(n, t0, p0)
    la1, sg1 = oracle.pfaffian_from_factors(n, t, piv)
    return {"pivots_identical": bool(np.array_equal(piv, p0)),
            "first_pivot_difference": (None if np.array_equal(piv, p0)
                                       else int(np.argmax(piv != p0))),
            "max_abs_dL": dL, "max_abs_dt_over_max_t": dt, "tol_L_t": tol,
            "log_abs_pf_oracle": la0, "log_abs_pf_gpu": la1,
            "rel_dlog_abs_pf": abs(la1 - la0) / max(1.0, abs(la0)),
            "signs_equal": sg0 == sg1,
            "within_bars": bool(np.array_equal(piv, p0) and dL <= tol and dt <= tol
                                and sg0 == sg1
                                and abs(la1 - la0) <= 1e-10 * max(1.0, abs(la0)))}


# ----------------------------------------------------------------------------- dist
# ----------------------------------------------------------------------------- batched
def run_batched_leg(skew, inputs, torch, dev, steps: int, warmup: int, plain_count: int,
                    rank: int = 0, world: int = 1, cpu_baseline: bool = True):
    """The batched workload: 4096 skew matrices, orders even in [16, 256] (seed 4),
    matrix i from seed 1000+i, all factored in one skew_ltlt_batched launch per step
    (Pfaffian-only: L not stored).  Compared with back-to-back skew_pfaffian calls on
    the same matrices.  Inputs are HBM-resident: a pristine copy is restored before
    every step outside the timed events.  With several ranks the 4096 matrices are
    split into size-balanced shares (one per rank, no exchange on the data path) and
    the rates are the whole batch over the slowest rank's time."""
    from paper_2411_09859_gb300 import shard
    all_sizes = inputs.batched_sizes(4096)
    total = len(all_sizes)
    idx = shard.balanced_bins(all_sizes, world)[rank] if world > 1 else np.arange(total)
    sizes = all_sizes[idx]
    mats = [inputs.skew_gaussian(int(all_sizes[i]), inputs.SEED_BATCH_BASE + int(i)) for i in idx]
    offs = np.concatenate([[0], np.cumsum(sizes.astype(np.int64) ** 2)])
    flat = np.empty(int(offs[-1]), dtype=np.float64)
    for i, A in enumerate(mats):
        flat[offs[i]:offs[i + 1]] = A.ravel(order="F")
    pristine = torch.from_numpy(flat).to(dev)
    work = torch.empty_like(pristine)
    views = [work[int(offs[i]):int(offs[i + 1])].view(int(n), int(n)).t()
             for i, n in enumerate(sizes)]
    ts = [torch.empty(int(n) - 1, dtype=torch.float64, device=dev) for n in sizes]
    pivs = [torch.empty(int(n), dtype=torch.int32, device=dev) for n in sizes]
    table = skew.problem_table(views, [None] * len(views), ts, pivs, dev)
    stream = torch.cuda.Stream(device=dev)
    flops = float(np.sum(sizes.astype(np.float64) ** 3) / 3.0)

    def one():
        work.copy_(pristine)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        la, sg, info, *_ = skew.ltlt_batched(views, stream=stream, max_n=256, table=table,
                                             outs=(ts, pivs, [None] * len(views)))
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), la, sg, info

    for _ in range(warmup):
        one()
    times = []
    for _ in range(steps):
        ms, la, sg, info = one()
        times.append(ms)
    if int((info != 0).sum().item()) != 0:
        raise RuntimeError("batched factorization reported a nonzero info")
    ms = reduce_max(statistics.median(times), world, dev)
    # the Pfaffian-only form of the same batch: two-step elimination, no T/L output
    as_ = [torch.empty(max(int(n) // 2, 1), dtype=torch.float64, device=dev) for n in sizes]
    pivs2 = [torch.empty(int(n), dtype=torch.int32, device=dev) for n in sizes]
    table2 = skew.problem_table(views, [None] * len(views), as_, pivs2, dev)
    times2 = []
    for i in range(warmup + steps):
        work.copy_(pristine)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        la2, sg2, info2, *_ = skew.pfaffian_batched(views, stream=stream, max_n=256, table=table2,
                                                     outs=(as_, pivs2))
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= warmup:
            times2.append(e0.elapsed_time(e1))
    if int((info2 != 0).sum().item()) != 0:
        raise RuntimeError("two-step batched Pfaffians reported a nonzero info")
    ms2 = reduce_max(statistics.median(times2), world, dev)
    agree = reduce_max(float(torch.max(torch.abs(la2 - la) / torch.clamp(torch.abs(la), min=1.0)).item()),
                       world, dev)
    signs_equal = reduce_max(0.0 if torch.equal(sg2, sg) else 1.0, world, dev) == 0.0
    # the same launch captured once in a CUDA graph (caller-supplied workspace and
    # result buffers), replayed per batch; the inputs are restored outside the graph
    ws = torch.empty(skew.batched_workspace_bytes(len(views), 256), dtype=torch.uint8, device=dev)
    res = (torch.empty(len(views), dtype=torch.float64, device=dev),
           torch.empty(len(views), dtype=torch.int32, device=dev),
           torch.empty(len(views), dtype=torch.int32, device=dev))
    work.copy_(pristine)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        skew.pfaffian_batched(views, stream=stream, max_n=256, table=table2, outs=(as_, pivs2),
                              workspace=ws, results=res)
    times3 = []
    for i in range(warmup + steps):
        work.copy_(pristine)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with torch.cuda.stream(stream):
            graph.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= warmup:
            times3.append(e0.elapsed_time(e1))
    ms3 = reduce_max(statistics.median(times3), world, dev)
    graph_equal = reduce_max(0.0 if (torch.equal(res[0], la2) and torch.equal(res[1], sg2)) else 1.0,
                             world, dev) == 0.0
    del graph
    # back-to-back plain calls on the same matrices (first plain_count of them)
    work.copy_(pristine)
    la1 = torch.empty(1, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    m = min(plain_count, len(views))
    e0.record(stream)
    for i in range(m):
        skew.pfaffian(views[i], stream=stream, t=ts[i], piv=pivs[i])
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = reduce_max(e0.elapsed_time(e1), world, dev)
    plain_rate = world * m / (plain_ms / 1e3)
    flops = reduce_sum(flops, world, dev)
    rate = total / (ms / 1e3)
    # CPU baseline: the oracle on the whole batch, one matrix per host thread, largest
    # first; its log|Pf| and signs are also the reference for every GPU result
    cpu = None
    oracle_check = None
    if world == 1 and cpu_baseline:
        import oracle
        order = np.argsort(-sizes, kind="stable")
        la_o, sg_o, inf_o, _, _, sec = oracle.ltlt_many([mats[i] for i in order])
        la_c = np.empty(len(sizes))
        sg_c = np.empty(len(sizes), dtype=np.int64)
        la_c[order] = la_o
        sg_c[order] = sg_o
        la_g = la.cpu().numpy()
        sg_g = sg.cpu().numpy()
        la_t = la2.cpu().numpy()
        cpu = {"value": total / sec, "unit": "Pfaffians/s", "cores": oracle.threads(),
               "kind": "oracle",
               "sample": (f"full: all {total} matrices, one matrix per host thread, "
                          f"largest first, {sec:.2f} s")}
        oracle_check = {
            "matrices": int(total),
            "signs_equal": bool(np.array_equal(sg_g, sg_c)),
            "max_rel_dlog_abs_pf": float(np.max(np.abs(la_g - la_c) / np.maximum(1.0, np.abs(la_c)))),
            "twostep_signs_equal": bool(np.array_equal(sg2.cpu().numpy(), sg_c)),
            "twostep_max_rel_dlog_abs_pf": float(np.max(np.abs(la_t - la_c) / np.maximum(1.0, np.abs(la_c)))),
            "oracle_info_nonzero": int(np.count_nonzero(inf_o))}
    return {"metric": "batched Pfaffians/s", "value": rate, "unit": "Pfaffians/s",
            "workload": "4096 skew matrices, n even uniform in [16, 256] (seed 4), "
                        "matrix i seed 1000+i, FP64, one persistent launch"
                        + (f" per rank on {world} size-balanced shares" if world > 1 else ""),
            "scaling": "strong" if world > 1 else None,
            "ms_per_batch": ms, "tflops": flops / (ms / 1e3) / 1e12,
            "plain_calls": {"value": plain_rate, "unit": "Pfaffians/s", "matrices": m * world,
                            "api": "skew_pfaffian, one call per matrix, back to back"},
            "speedup_vs_plain_calls": rate / plain_rate,
            "cpu_baseline": cpu,
            "oracle_check": oracle_check,
            "accuracy": "same algorithm in FP64; every log|Pf| and sign against the "
                        "oracle in oracle_check",
            "pfaffian_only_twostep": {
                "value": total / (ms2 / 1e3), "unit": "Pfaffians/s", "ms_per_batch": ms2,
                "api": "skew_pfaffian_batched (two-step elimination; no T, L output)",
                "max_rel_logabs_diff_vs_ltlt_batched": agree, "signs_equal": signs_equal,
                "speedup_vs_plain_calls": (total / (ms2 / 1e3)) / plain_rate,
                "cuda_graph_replay": {"value": total / (ms3 / 1e3), "unit": "Pfaffians/s",
                                      "ms_per_batch": ms3, "results_equal_direct_call": graph_equal}}}


# ----------------------------------------------------------------------------- precision
def run_precision_leg(skew, inputs, torch, dev, A_host, nb_fp64, fp64_ms, fp64_t, fp64_piv,
                      steps: int, warmup: int, n_qdq: int, n_full: int = 0):
    """The precision form: the same n = 16384 matrix with the trailing update run as
    split-precision bf16 tensor-core products (panel, pivots, division, t and
    log|Pf| in FP64), timed like the FP64 run, compared with it (pivots, log|Pf|);
    and A = Q D Q^T (Q Haar in SO(n), D blocks [[0,s],[-s,0]], s log-spaced in
    [1, 1e6], seed 5) at a reduced order n_qdq, against its closed form
    log|Pf| = sum ln s and against the CPU oracle, for both precisions."""
    import oracle
    n = A_host.shape[0]
    split = skew.PRECISION_SPLIT_BF16
    nb = min(nb_fp64, 64)
    pristine = torch.from_numpy(A_host).to(dev)
    L = skew.fortran_empty(n, n, dev)
    t = torch.empty(n - 1, dtype=torch.float64, device=dev)
    piv = torch.empty(n, dtype=torch.int32, device=dev)
    info = torch.empty(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    work = skew.fortran_empty(n, n, dev)
    times = []
    for i in range(warmup + steps):
        work.copy_(pristine)
        torch.cuda.synchronize()
        if i == warmup:
            skew.profile_read()
            skew.profile_enable(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        skew.ltlt(work, nb=nb, stream=stream, L=L, t=t, piv=piv, info=info, precision=split)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= warmup:
            times.append(e0.elapsed_time(e1))
    prof = skew.profile_read()
    skew.profile_enable(False)
    ms = statistics.median(times)
    kernels = kernel_table(prof, steps, ms * steps)
    sk = prof["skr2k"]
    split_tflops = (sk["flops"] / (sk["ms"] / 1e3) / 1e12) if sk["ms"] > 0 else None
    t_s, piv_s = t.cpu().numpy(), piv.cpu().numpy()
    la_f, sg_f = skew.pfaffian_from_factors(torch.from_numpy(fp64_t).to(dev),
                                            torch.from_numpy(fp64_piv).to(dev), n)
    la_s, sg_s = skew.pfaffian_from_factors(t, piv, n)
    torch.cuda.synchronize()
    la_f, la_s = float(la_f.item()), float(la_s.item())
    first_diff = int(np.argmax(piv_s != fp64_piv)) if not np.array_equal(piv_s, fp64_piv) else None
    del pristine, work, L
    torch.cuda.empty_cache()

    # QDQ^T accuracy at a reduced order
    Aq, s_vals = inputs.qdq_skew(n_qdq, inputs.SEED_PRECISION, smax=1e6)
    closed = float(np.sum(np.log(s_vals)))
    L0, t0, p0, _ = oracle.ltlt(Aq)
    la_o, sg_o = oracle.pfaffian_from_factors(n_qdq, t0, p0)
    acc = {}
    for name, prec in (("fp64_dmma", skew.PRECISION_FP64), ("split_bf16", split)):
        la, sg, tq, pq, iq = skew.pfaffian(torch.from_numpy(Aq).to(dev), nb=min(64, nb_fp64),
                                           precision=prec)
        torch.cuda.synchronize()
        la = float(la.item())
        acc[name] = {"log_abs_pf": la, "sign": int(sg.item()),
                     "rel_err_vs_closed_form": abs(la - closed) / abs(closed),
                     "rel_err_vs_oracle": abs(la - la_o) / abs(la_o),
                     "pivots_equal_oracle": bool(np.array_equal(pq.cpu().numpy(), p0))}
    # the precision workload at full order: QDQ^T generated on the device
    full = None
    if n_full > 0:
        tg0 = time.perf_counter()
        Af, s_full, detQ = inputs.qdq_skew_device(n_full, inputs.SEED_PRECISION, smax=1e6,
                                                  device=dev)
        torch.cuda.synchronize()
        gen_s = time.perf_counter() - tg0
        closed_f = float(np.sum(np.log(s_full)))
        full = {"n": n_full, "closed_form_log_abs_pf": closed_f, "closed_form_sign": detQ,
                "generation_s": gen_s,
                "generator": "device QR of a seeded Gaussian (torch), sign(diag R) correction; "
                             "Pf = det(Q) prod s"}
        work_f = skew.fortran_empty(n_full, n_full, dev)
        for name, prec in (("fp64_dmma", skew.PRECISION_FP64), ("split_bf16", split)):
            for algo in ("one_step", "twostep"):
                work_f.copy_(Af)
                torch.cuda.synchronize()
                if algo == "one_step":
                    la, sg, *_ = skew.pfaffian(work_f, nb=64, precision=prec)
                else:
                    la, sg, *_ = skew.pfaffian_twostep(work_f, nb=64, precision=prec)
                torch.cuda.synchronize()
                la = float(la.item())
                full[f"{name}_{algo}"] = {"log_abs_pf": la, "sign": int(sg.item()),
                                          "sign_ok": int(sg.item()) == detQ,
                                          "rel_err_vs_closed_form": abs(la - closed_f) / abs(closed_f)}
        del Af, work_f
        torch.cuda.empty_cache()
    flops = factorization_flops(n)
    return {"metric": "skew LTLt TFLOP/s (n^3/3) with the split-precision trailing update",
            "value": flops / (ms / 1e3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms,
            "speedup_vs_fp64": fp64_ms / ms, "nb": nb, "kernels": kernels,
            "update_fp64_equivalent_tflops": split_tflops,
            "vs_fp64_run": {"pivots_equal": first_diff is None, "first_pivot_difference": first_diff,
                            "log_abs_pf_fp64": la_f, "log_abs_pf_split": la_s,
                            "rel_diff": abs(la_s - la_f) / abs(la_f), "sign_equal": int(sg_f.item()) == int(sg_s.item()),
                            "max_rel_t_diff": float(np.max(np.abs(t_s - fp64_t)) / np.max(np.abs(fp64_t)))},
            "qdq_full_order": full,
            "qdq": {"n": n_qdq, "closed_form_log_abs_pf": closed, "oracle_log_abs_pf": la_o,
                    "oracle_rel_err_vs_closed_form": abs(la_o - closed) / abs(closed), **acc,
                    "note": "QDQ^T at a reduced order against the CPU oracle (host generation); "
                            "qdq_full_order: the same workload at full order, generated on the "
                            "device, against its closed form"}}


# ----------------------------------------------------------------------------- serving
def latency_summary(res) -> dict:
    """p50/p99 of the latency and of its three parts (waiting for the memory budget,
    for a stream, then running), and the mean parts of the requests at or above the
    p99 latency, in milliseconds."""
    lat = np.array([r["latency_s"] for r in res]) * 1e3
    out = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))}
    if res and all("queued_s" in r for r in res):
        parts = {k: np.array([r[k] for r in res]) * 1e3
                 for k in ("queued_s", "waiting_s", "running_s")}
        tail = lat >= np.percentile(lat, 99)
        out["breakdown"] = {
            k.replace("_s", ""): {"p50_ms": float(np.percentile(v, 50)),
                                  "p99_ms": float(np.percentile(v, 99)),
                                  "mean_ms_of_p99_requests": float(np.mean(v[tail]))}
            for k, v in parts.items()}
        out["breakdown"]["what"] = ("queued: submission to admission (memory budget); "
                                    "waiting: admission to launch (free stream or batch); "
                                    "running: launch to observed completion")
    return out


def run_serving_leg(skew, inputs, torch, dev, n_requests: int, n_poisson: int,
                    n_serial: int, n_factors: int, rank: int = 0, world: int = 1):
    """The serving workload: a stream of n_requests requests with even orders
    log-uniform in [32, 4096] (seed 6); request i is the leading n_i x n_i block of one
    seeded 4096 x 4096 skew matrix (every principal block of an iid N(0,1) skew matrix
    is one of order n_i).  The requests ask for the Pfaffian only (SKEW_SERVE_PFAFFIAN:
    the two-step elimination).  Measured:
      - saturation: the continuous-batching server (64 GB budget, 4 streams, batched
        kernel up to n = 512) with the whole stream submitted at once;
      - serial: back-to-back skew_pfaffian_twostep calls (the same algorithm, so the
        same accuracy) on the first n_serial requests, as a rate;
      - Poisson streams of the first n_poisson requests at 0.5x, 0.8x and 1.2x that
        serial rate (seeded gaps), p50/p99 latency from submission to completion and
        where it went (budget, stream, running); `poisson` is the 0.8x stream;
      - factors_kept: serial and saturation runs on the first n_factors requests with
        requests that keep their LTL^T factors (SKEW_SERVE_FACTORS; serial skew_pfaffian
        calls).
    Results are consumed in submission order and released at once, so a stream longer
    than the memory budget holds keeps flowing.  With several ranks each runs its own
    server on a size-balanced share of the requests (at their arrival times in the one
    global stream); rates are all requests over the slowest rank's time and the latency
    percentiles are taken over the gathered latencies."""
    from paper_2411_09859_gb300 import shard
    rng = np.random.default_rng(inputs.SEED_SERVING)
    logn = rng.uniform(np.log(32), np.log(4096), size=n_requests)
    sizes = np.clip(2 * np.round(np.exp(logn) / 2), 32, 4096).astype(np.int64)
    mine = shard.balanced_bins(sizes, world)[rank] if world > 1 else np.arange(n_requests)
    n_serial = min(n_serial, n_requests)
    n_poisson = min(n_poisson, n_requests)
    n_factors = min(n_factors, n_requests)

    def gather(values):
        if world <= 1:
            return list(values)
        import torch.distributed as dist
        parts = [None] * world
        dist.all_gather_object(parts, list(values))
        return [v for part in parts for v in part]
    master = torch.from_numpy(inputs.skew_gaussian(4096, inputs.SEED_SERVING)).to(dev)
    views = [master[:int(n), :int(n)] for n in sizes]
    flops_of = lambda count: float(np.sum(sizes[:count].astype(np.float64) ** 3) / 3.0)
    stream = torch.cuda.Stream(device=dev)
    work = skew.fortran_empty(4096, 4096, dev)

    def serial(idx, pf_only):
        for i in idx:
            n = int(sizes[i])
            w = work[:n, :n]
            w.copy_(views[i])
            if pf_only:
                skew.pfaffian_twostep(w, stream=stream)
            else:
                skew.pfaffian(w, stream=stream)

    def time_serial(count, pf_only):
        idx = [int(i) for i in mine if i < count]
        with torch.cuda.stream(stream):
            serial(idx[:8], pf_only)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            serial(idx, pf_only)
            e1.record(stream)
        torch.cuda.synchronize()
        return reduce_max(e0.elapsed_time(e1) / 1e3, world, dev)

    serial_s = time_serial(n_serial, True)
    serial_rate = n_serial / serial_s
    serial_f_s = time_serial(n_factors, False)

    srv = skew.Server(64 << 30, n_streams=4, small_n_max=512)
    for pf in (True, False):
        for tk in [srv.submit(views[i], pfaffian_only=pf) for i in mine[:16]]:
            srv.wait(tk)
            srv.release(tk)

    def consume(tickets):
        # results are read in submission order and released at once, as a client
        # would: the factors of a long stream do not all fit the budget together
        out = []
        for tk in tickets:
            out.append(srv.wait(tk))
            srv.release(tk)
        return out

    def saturation(count, pf_only):
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        t0 = time.perf_counter()
        tickets = [srv.submit(views[i], pfaffian_only=pf_only) for i in mine if i < count]
        res = consume(tickets)
        sec = reduce_max(time.perf_counter() - t0, world, dev)
        return sec, gather(res), sum(1 for r in res if r["info"] != 0)

    sat_s, sat_res, bad = saturation(n_requests, True)
    sat_f_s, sat_f_res, bad_f = saturation(n_factors, False)
    bad += bad_f

    def poisson_stream(factor, seed):
        """Requests 0 .. n_poisson-1 arriving as a Poisson stream at `factor` x the
        serial rate (seeded gaps); a client thread consumes results while the stream is
        still being submitted."""
        lam = factor * serial_rate
        arrive = np.cumsum(np.random.default_rng(seed).exponential(1.0 / lam, size=n_poisson))
        todo = [int(i) for i in mine if i < n_poisson]
        pending = queue.Queue()
        out = []
        client = threading.Thread(target=lambda: out.extend(consume(iter(pending.get, None))))
        client.start()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        t0 = time.perf_counter()
        for i in todo:
            delay = t0 + arrive[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            pending.put(srv.submit(views[i], pfaffian_only=True))
        pending.put(None)
        client.join()
        seconds = reduce_max(time.perf_counter() - t0, world, dev)
        if len(out) != len(todo):
            raise RuntimeError("the serving client thread did not consume every result")
        summary = {"rate_factor": factor, "rate_per_s": lam, "requests": n_poisson,
                   "value": n_poisson / seconds}
        summary.update(latency_summary(gather(out)))
        return out, summary

    rates = []
    # gap seeds: 0.8x (the headline stream) seed 7, 0.5x seed 8, 1.2x seed 9
    for factor, off in ((0.5, 2), (0.8, 1), (1.2, 3)):
        out, summary = poisson_stream(factor, inputs.SEED_SERVING + off)
        bad += sum(1 for r in out if r["info"] != 0)
        rates.append(summary)
    srv.close()
    bad = int(reduce_sum(bad, world, dev))
    if bad:
        raise RuntimeError(f"{bad} served requests reported a nonzero info")
    sat = {"value": n_requests / sat_s, "requests": n_requests, "seconds": sat_s,
           "tflops": flops_of(n_requests) / sat_s / 1e12,
           "speedup_vs_serial": serial_rate and (n_requests / sat_s) / serial_rate}
    sat.update(latency_summary(sat_res))
    sat_f = {"value": n_factors / sat_f_s, "requests": n_factors, "seconds": sat_f_s,
             "speedup_vs_serial": (n_factors / sat_f_s) / (n_factors / serial_f_s)}
    sat_f.update(latency_summary(sat_f_res))
    return {"metric": "served Pfaffians/s and latency", "unit": "Pfaffians/s",
            "value": n_requests / sat_s,
            "workload": (f"{n_requests} requests, even n log-uniform in [32, 4096] (seed 6), "
                         "leading blocks of one seeded 4096^2 iid N(0,1) skew matrix; "
                         f"saturation on all {n_requests}; serial rate on the first "
                         f"{n_serial}; Poisson streams on the first {n_poisson}; factor-"
                         f"keeping runs on the first {n_factors}"),
            "requests": "Pfaffian only (SKEW_SERVE_PFAFFIAN, two-step elimination)",
            "serial_plain_calls": {"value": serial_rate, "requests": n_serial,
                                   "seconds": serial_s,
                                   "tflops": flops_of(n_serial) / serial_s / 1e12,
                                   "api": "skew_pfaffian_twostep, one call per request, back to back"},
            "saturation": sat,
            "poisson": rates[1],
            "poisson_rates": rates,
            "factors_kept": {
                "requests": "SKEW_SERVE_FACTORS (pivoted LTL^T, t and piv kept)",
                "serial_plain_calls": {"value": n_factors / serial_f_s, "requests": n_factors,
                                       "seconds": serial_f_s,
                                       "api": "skew_pfaffian, one call per request, back to back"},
                "saturation": sat_f},
            "server": "budget 64 GB, 4 streams, batched kernel for n <= 512"
                      + (f"; one server per rank on {world} size-balanced shares" if world > 1 else "")}


def reduce_max(value: float, world: int, device=None) -> float:
    """Max of `value` over the ranks of the default process group (the timing rule:
    the slowest rank defines the whole-job time).  Identity for a single process."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, world: int, device=None) -> float:
    """Sum of `value` over the ranks (identity for a single process)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units_per_rank: float, seconds_max: float, world: int) -> float:
    """Units processed by all ranks divided by the slowest rank's time (replicas:
    every rank processes the same number of units)."""
    return world * units_per_rank / seconds_max


def parse_cpulist(text: str) -> set:
    """CPU numbers of a sysfs cpulist ("0-3,8,10-11")."""
    cpus = set()
    for part in text.strip().split(","):
        if not part:
            continue
        lo, _, hi = part.partition("-")
        cpus.update(range(int(lo), int(hi or lo) + 1))
    return cpus


def gpu_local_cpus(torch, local: int):
    """The CPUs next to GPU `local` (its PCI device's local_cpulist) that this process
    may run on, or None when that cannot be read."""
    try:
        pr = torch.cuda.get_device_properties(local)
        bus = f"{pr.pci_domain_id:04x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
        with open(f"/sys/bus/pci/devices/{bus}/local_cpulist") as f:
            near = parse_cpulist(f.read())
        mine = os.sched_getaffinity(0) & near
        return mine or None
    except (OSError, ValueError, AttributeError):
        return None


def pinned_near_gpu(torch, local: int, make):
    """Calls make() (which allocates and fills page-locked host buffers) with this
    process bound to the CPUs next to the GPU, so that the pages are placed in the
    memory nearest to it (first touch); the previous affinity is restored after.  On
    a two-socket host, buffers on the far node are copied at a fraction of the link's
    rate (measured on a GB300 node: 2 x 2 GB per factorization took about 100 ms
    longer from the far node)."""
    near = gpu_local_cpus(torch, local)
    if near is None:
        return make(), None
    before = os.sched_getaffinity(0)
    os.sched_setaffinity(0, near)
    try:
        return make(), len(near)
    finally:
        os.sched_setaffinity(0, before)


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    """The reference arm: the CPU oracle (this paper has no code to install; the oracle
    is its algorithm A1 written out) on the same n = 16384 matrix.  The whole
    factorization is run once, in W + K consecutive pieces of equal rank-2 update work;
    the first W pieces are the warm-up and each of the K timed steps is one piece,
    credited with its share of the n^3/3 flops.  Every timed piece is measured, none is
    extrapolated."""
    world, rank, local = dist_setup(args)
    if rank != 0:
        return 0
    import oracle
    from paper_2411_09859_gb300 import inputs
    n = args.n
    seed = inputs.SEED_SCALE.get(n, 3)
    A_host = inputs.skew_gaussian(n, seed)
    pieces = args.warmup + args.steps
    work = update_work(n)
    cum = np.concatenate([[0.0], np.cumsum(work)])
    bounds = [0] + [int(np.searchsorted(cum, cum[-1] * (i + 1) / pieces)) for i in range(pieces)]
    bounds[-1] = n - 1
    t0 = time.perf_counter()
    st = oracle.ltlt_begin(A_host)
    t_setup = time.perf_counter() - t0
    times, credit = [], []
    for i in range(pieces):
        t0 = time.perf_counter()
        oracle.ltlt_continue(st, bounds[i + 1])
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            credit.append(float(cum[bounds[i + 1]] - cum[bounds[i]]) / cum[-1])
    sec = sum(times)
    value = factorization_flops(n) * sum(credit) / sec / 1e12
    sample = (f"the whole n={n} factorization in {pieces} consecutive pieces of equal "
              f"rank-2 update work (set-up {t_setup:.1f} s, then the {args.warmup} warm-up "
              f"pieces, elimination steps 0..{bounds[args.warmup] - 1}); timed: the "
              f"{args.steps} pieces of steps {bounds[args.warmup]}..{n - 2}, "
              f"{100 * sum(credit):.1f}% of the update work in {sec:.1f} s, credited with "
              "that share of n^3/3")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sec / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(n, args.nb if args.nb > 0 else table_nb(n), seed),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "timed_pieces": [{"steps": [bounds[args.warmup + i], bounds[args.warmup + i + 1] - 1],
                              "seconds": times[i], "share_of_work": credit[i]}
                             for i in range(args.steps)]}
    print(json.dumps(line), flush=True)
    return 0


def run_twostep_leg(skew, inputs, torch, dev, A_host, steps: int, warmup: int):
    """The Pfaffian-only forms on the same n x n matrix: skew_pfaffian_twostep (the
    two-step elimination, pivot searches at even steps only) and skew_pfaffian (the
    one-step factorization without L), each with the FP64 and the split-precision
    trailing update; timed like the main leg, with the per-kernel split and the
    agreement of their log|Pf| (the two eliminations pivot differently)."""
    n = A_host.shape[0]
    pristine = torch.from_numpy(A_host).to(dev)
    work = skew.fortran_empty(n, n, dev)
    stream = torch.cuda.Stream(device=dev)
    flops = factorization_flops(n)
    out = {"metric": "Pfaffian TFLOP/s (n^3/3 counted) by the two-step elimination",
           "unit": "TFLOP/s", "nb": 64}
    vals = {}
    for algo in ("twostep", "one_step"):
        for pname, prec in (("fp64", skew.PRECISION_FP64), ("split", skew.PRECISION_SPLIT_BF16)):
            times = []
            for i in range(warmup + steps):
                work.copy_(pristine)
                torch.cuda.synchronize()
                if i == warmup:
                    skew.profile_read()
                    skew.profile_enable(True)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if algo == "twostep":
                    la, sg, *_ = skew.pfaffian_twostep(work, nb=64, stream=stream, precision=prec)
                else:
                    la, sg, *_ = skew.pfaffian(work, nb=64, stream=stream, precision=prec)
                e1.record(stream)
                torch.cuda.synchronize()
                if i >= warmup:
                    times.append(e0.elapsed_time(e1))
            prof = skew.profile_read()
            skew.profile_enable(False)
            ms = statistics.median(times)
            vals[(algo, pname)] = (float(la.item()), int(sg.item()))
            out.setdefault(algo, {})[pname] = {
                "ms_per_step": ms, "value": flops / (ms / 1e3) / 1e12,
                "kernels": {k: {"ms_per_step": v["ms"] / steps, "launches_per_step": v["launches"] / steps}
                            for k, v in prof.items() if v["launches"]}}
    ref = vals[("one_step", "fp64")]
    out["value"] = out["twostep"]["fp64"]["value"]
    out["log_abs_pf"] = {f"{a}_{p}": v[0] for (a, p), v in vals.items()}
    out["max_rel_diff_vs_one_step_fp64"] = max(abs(v[0] - ref[0]) / abs(ref[0]) for v in vals.values())
    out["signs_equal"] = all(v[1] == ref[1] for v in vals.values())
    out["speedup_vs_one_step"] = {p: out["one_step"][p]["ms_per_step"] / out["twostep"][p]["ms_per_step"]
                                  for p in ("fp64", "split")}
    del pristine, work
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2411_09859_gb300 as skew
    from paper_2411_09859_gb300 import build as skew_build
    from paper_2411_09859_gb300 import inputs

    world, rank, local = dist_setup(args)
    # one process per GPU; the modulo only matters when fewer GPUs than ranks are
    # visible (a functional run of the N > 1 code path on one GPU, with the gloo backend
    # chosen by SKEW_BENCH_DIST_BACKEND)
    local = local % max(1, torch.cuda.device_count())
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group(os.environ.get("SKEW_BENCH_DIST_BACKEND", "nccl"))
    # the library is built once per node, before any rank loads it
    if int(os.environ.get("LOCAL_RANK", "0")) == 0:
        skew_build.build()
    if world > 1:
        dist.barrier()
    dev = torch.device("cuda", local)

    n = args.n
    seed = inputs.SEED_SCALE.get(n, 3)
    nb = args.nb if args.nb > 0 else skew.default_nb(n)
    A_host = inputs.skew_gaussian(n, seed)
    W, K = args.warmup, args.steps
    stream = torch.cuda.Stream(device=dev)

    # one fresh HBM-resident copy of A per step, made before the timed region
    pristine = torch.from_numpy(A_host).to(dev)
    copies = []
    for _ in range(W + K):
        c = skew.fortran_empty(n, n, dev)
        c.copy_(pristine)
        copies.append(c)
    del pristine
    L = skew.fortran_empty(n, n, dev)
    t = torch.empty(n - 1, dtype=torch.float64, device=dev)
    piv = torch.empty(n, dtype=torch.int32, device=dev)
    info = torch.empty(1, dtype=torch.int32, device=dev)
    if args.path != "auto":
        skew.set_lookahead(2 if args.path == "lookahead" else 0)
    skew.set_lookahead_switch(args.la_switch)
    skew.set_cluster_panel(not args.grid_panels)
    lookahead = skew.lookahead_used(n, nb)
    ws = torch.empty(skew.workspace_bytes(n, nb, True, lookahead=True), dtype=torch.uint8,
                     device=dev)
    torch.cuda.synchronize()

    def step(A):
        skew.ltlt(A, nb=nb, stream=stream, L=L, t=t, piv=piv, info=info, workspace=ws)

    for i in range(W):
        step(copies[i])
    torch.cuda.synchronize()
    if int(info.item()) != 0:
        raise RuntimeError(f"warm-up factorization reported info={int(info.item())}")

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    skew.profile_read()
    skew.profile_enable(True)
    launches0 = skew.kernel_launches()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(K):
        step(copies[W + i])
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = skew.kernel_launches() - launches0
    prof = skew.profile_read()
    skew.profile_enable(False)
    if world > 1:
        dist.barrier()
    ms = reduce_max(e0.elapsed_time(e1), world, dev)
    if int(info.item()) != 0:
        raise RuntimeError(f"timed factorization reported info={int(info.item())}")
    del copies
    torch.cuda.empty_cache()
    t_host, piv_host = t.cpu().numpy(), piv.cpu().numpy()

    value = whole_job_rate(K * factorization_flops(n), ms / 1e3, world) / 1e12
    peak, peak_note = fp64_peak()
    sk = prof["skr2k"]
    achieved = sk["flops"] / (sk["ms"] / 1e3) / 1e12 if sk["ms"] > 0 else None
    ratio = recorded_traffic()
    traffic = (ratio * sk["bytes"] / sk["launches"]) if (ratio and sk["launches"]) else None
    kernels = kernel_table(prof, K, ms, concurrent_panel=lookahead)
    panel = prof["panel"]
    kernels["panel"]["achieved_gbs"] = (panel["bytes"] / (panel["ms"] / 1e3) / 1e9
                                        if panel["ms"] > 0 else None)
    kernels["panel"]["us_per_column_step"] = panel["ms"] / K * 1e3 / max(n - 1, 1)
    kernels["panel"]["path"] = ("look-ahead: beside the previous block's update, on its own "
                                "stream (us per column step is its span)" if lookahead else
                                "plain: between the updates, on the launch stream")

    # ---- the same factorization on the other path (plain <-> look-ahead), for comparison
    other = None
    old_la = skew.set_lookahead(2)
    la_possible = skew.lookahead_used(n, nb)
    skew.set_lookahead(old_la)
    if la_possible and not args.skip_plain:
        old_la = skew.set_lookahead(0 if lookahead else 2)
        try:
            ws_p = torch.empty(skew.workspace_bytes(n, nb, True, lookahead=not lookahead),
                               dtype=torch.uint8, device=dev)
            A_p = skew.fortran_empty(n, n, dev)
            L_p = skew.fortran_empty(n, n, dev)
            t_p = torch.empty_like(t)
            piv_p = torch.empty_like(piv)
            info_p = torch.empty_like(info)
            pt = []
            for i in range(3):
                A_p.copy_(torch.from_numpy(A_host).to(dev))
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                skew.ltlt(A_p, nb=nb, stream=stream, L=L_p, t=t_p, piv=piv_p, info=info_p,
                          workspace=ws_p)
                e1.record(stream)
                torch.cuda.synchronize()
                if i:
                    pt.append(e0.elapsed_time(e1))
            other_ms = statistics.median(pt)
            same = bool(np.array_equal(piv_p.cpu().numpy(), piv_host))
            other = {"path": "plain" if lookahead else "look-ahead",
                     "ms_per_step": other_ms,
                     "value": factorization_flops(n) / (other_ms / 1e3) / 1e12,
                     "unit": UNIT, "steps": len(pt), "pivots_equal": same,
                     "headline_speedup_over_it": other_ms / (ms / K)}
            del ws_p, A_p, L_p, t_p, piv_p, info_p
            torch.cuda.empty_cache()
        finally:
            skew.set_lookahead(old_la)

    # ---- end to end through the host-buffer C-ABI call (pinned host buffers)
    e2e = None
    if not args.skip_e2e:
        def make_pinned():
            a = torch.empty((n, n), dtype=torch.float64).pin_memory().t()
            a.copy_(torch.from_numpy(A_host))
            lo = torch.empty((n, n), dtype=torch.float64).pin_memory().t()
            lo.zero_()
            return (a, lo, torch.zeros(n - 1, dtype=torch.float64).pin_memory(),
                    torch.zeros(n, dtype=torch.int32).pin_memory())
        (A_pin, L_pin, t_pin, p_pin), near_cpus = pinned_near_gpu(torch, local, make_pinned)
        A_np, L_np, t_np, p_np = A_pin.numpy(), L_pin.numpy(), t_pin.numpy(), p_pin.numpy()
        skew.ltlt_host(A_np, True, nb, L_out=L_np, t_out=t_np, piv_out=p_np)
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        step_ends = []
        phases = []
        for _ in range(K):
            res = skew.ltlt_host(A_np, True, nb, L_out=L_np, t_out=t_np, piv_out=p_np)
            step_ends.append(time.perf_counter())
            phases.append(skew.ltlt_host_timing())
            if res[5] != 0:
                raise RuntimeError(f"host-buffer factorization reported info={res[5]}")
        el = reduce_max(step_ends[-1] - t0, world, dev)
        step_ms = list(np.diff([t0] + step_ends) * 1e3)
        ph = np.array([p for p in phases if p is not None]).reshape(-1, 3)
        med = np.median(ph, axis=0) if len(ph) else [None] * 3
        # the library copies A's lower triangle only, in blocks of 256 columns
        h2d_b = sum((n - c0) * min(256, n - c0) for c0 in range(0, n, 256)) * 8
        e2e = {"value": whole_job_rate(K * factorization_flops(n), el, world) / 1e12, "unit": UNIT,
               "h2d_bytes_per_step": h2d_b,
               "d2h_bytes_per_step": n * n * 8 + (n - 1) * 8 + n * 4 + 8 + 4 + 4,
               "ms_per_step": el / K * 1e3, "step_ms_rank0": [float(x) for x in step_ms],
               "phases_ms_median_rank0": {
                   "h2d_ms": float(med[0]) if len(ph) else None,
                   "device_ms": float(med[1]) if len(ph) else None,
                   "d2h_ms": float(med[2]) if len(ph) else None,
                   "host_side_ms": (float(np.median(np.array(step_ms) - ph.sum(axis=1)))
                                    if len(ph) == len(step_ms) and len(ph) else None),
                   "h2d_gbs": float(h2d_b / (med[0] / 1e3) / 1e9) if len(ph) else None,
                   "what": ("CUDA events on the call's stream around the copy of A, the "
                            "factorization and the copies back; with a page-locked L the "
                            "library sends each panel's final rows of L back while later "
                            "panels run, so d2h_ms is only what remains after the "
                            "factorization (the last rows, t, piv); host_side_ms = median "
                            "over steps of the step's wall time minus its three phases")},
               "host_buffers": ("page-locked, allocated while bound to the "
                                f"{near_cpus} CPUs next to the GPU" if near_cpus else
                                "page-locked (GPU-local CPUs unknown: not bound)"),
               "api": "skew_ltlt_host (page-locked host A in, L, t, piv, log|Pf|, sign out)"}

    precision = None
    if not args.skip_precision:
        precision = run_precision_leg(skew, inputs, torch, dev, A_host, nb, ms / K,
                                      t_host, piv_host, steps=2, warmup=1,
                                      n_qdq=args.qdq_n, n_full=args.qdq_full_n)

    twostep = None
    if not args.skip_twostep:
        twostep = run_twostep_leg(skew, inputs, torch, dev, A_host, steps=2, warmup=1)

    batched = None
    if not args.skip_batched:
        batched = run_batched_leg(skew, inputs, torch, dev, steps=3, warmup=1,
                                  plain_count=args.plain_calls, rank=rank, world=world,
                                  cpu_baseline=not args.skip_cpu_baseline)

    serving = None
    if not args.skip_serving:
        serving = run_serving_leg(skew, inputs, torch, dev, args.serve_requests,
                                  args.serve_poisson, args.serve_serial, args.serve_factors,
                                  rank=rank, world=world)

    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.skip_cpu_baseline:
        r = oracle_full(A_host)
        cpu = {k: r[k] for k in ("value", "unit", "cores", "kind", "sample")}
        parity = oracle_parity(r, L, t_host, piv_host, n)
        parity["what"] = ("the timed GPU factorization (last timed step) against the "
                          "oracle's on the same matrix")
        del r

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(n, nb, seed),
                           **({"serving_workload": serving["workload"]} if serving else {}),
                           **({"batched_workload": batched["workload"]} if batched else {})),
            "pct_of_fp64_peak": 100.0 * (value / world) / peak,
            "roofline": {"kernel": "skr2k (fused skew rank-2k trailing update, DMMA)",
                         "bound": "tensor", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s",
                         "frac": (achieved / peak) if achieved else None,
                         "traffic": traffic, "peak_source": peak_note,
                         "algorithmic_bytes_per_launch": sk["bytes"] / max(sk["launches"], 1),
                         "algorithmic_flops_per_launch": sk["flops"] / max(sk["launches"], 1)},
            "kernels": kernels,
            "path": "look-ahead" if lookahead else "plain",
            "other_path": other,
            "e2e": e2e,
            "precision": precision,
            "pfaffian_only": twostep,
            "batched": batched,
            "serving": serving,
            "cpu_baseline": cpu,
            "oracle_parity": parity,
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
