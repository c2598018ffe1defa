"""Serving form (skew_server_*): continuous batching under a device-memory budget.

Each result must be the same alone and in the mix (pivots identical, log|Pf| within
1e-10 relative, same sign), agree with the oracle, and admission must follow the
budget.  Failure handling is exercised on the host: a request that cannot be
admitted makes a bounded wait time out, without any device-side fault.
"""
import math
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle  # noqa: E402
import paper_2411_09859_gb300 as skew  # noqa: E402
from paper_2411_09859_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def dev(A):
    return torch.from_numpy(np.asfortranarray(A, dtype=np.float64)).cuda()


def close(a, b):
    return abs(a - b) <= 1e-10 * max(1.0, abs(b))


SIZES = [32, 64, 100, 256, 300, 512, 600, 1000, 2, 1, 0, 48, 777]


def run_alone(A, want_L):
    srv = skew.Server(8 << 30, n_streams=1, small_n_max=512)
    tk = srv.submit(dev(A), want_L=want_L)
    res = srv.wait(tk, 60.0)
    t, piv, L = srv.factors(tk, A.shape[0], want_L)
    srv.release(tk)
    srv.close()
    return res, t, piv, L


def test_alone_equals_in_the_mix_and_oracle():
    mats = [inputs.skew_gaussian(n, 7000 + n) for n in SIZES]
    srv = skew.Server(8 << 30, n_streams=4, small_n_max=512)
    devs = [dev(A) for A in mats]
    torch.cuda.synchronize()
    tickets = [srv.submit(d, want_L=(i % 2 == 0)) for i, d in enumerate(devs)]
    mixed = [srv.wait(tk, 120.0) for tk in tickets]
    for i, (A, tk, res) in enumerate(zip(mats, tickets, mixed)):
        n = A.shape[0]
        want_L = (i % 2 == 0)
        t, piv, L = srv.factors(tk, n, want_L)
        alone, t1, piv1, L1 = run_alone(A, want_L)
        assert res["info"] == alone["info"]
        assert np.array_equal(piv, piv1)
        assert res["sign"] == alone["sign"]
        if res["sign"] != 0:
            assert close(res["logabs"], alone["logabs"])
        L0, t0, p0, i0 = oracle.ltlt(A)
        assert np.array_equal(piv, p0) and res["info"] == i0
        la0, sg0 = oracle.pfaffian_from_factors(n, t0, p0)
        assert res["sign"] == sg0
        if sg0 != 0:
            assert close(res["logabs"], la0)
        if n > 1:
            assert np.max(np.abs(t - t0)) <= 2000 * n * 2.0 ** -52 * np.max(np.abs(t0))
        if want_L and n > 1:
            assert np.max(np.abs(L - L0)) <= 2000 * n * 2.0 ** -52
        assert res["latency_s"] >= 0
        srv.release(tk)
    assert srv.stats() == {"used_bytes": 0, "queued": 0, "in_flight": 0}
    srv.close()


def test_pfaffian_only_requests_alone_in_the_mix_and_oracle():
    """SKEW_SERVE_PFAFFIAN: small orders go to the batched two-step kernel, larger ones
    to the two-step call; interleaved with factor requests of the same matrices, each
    result equals the request run alone, agrees with the oracle's two-step elimination
    and with the factor request's Pfaffian, and keeps no factors."""
    sizes = [32, 100, 256, 300, 512, 600, 1000, 2, 1, 0, 48, 777]
    mats = [inputs.skew_gaussian(n, 7100 + n) for n in sizes]
    devs = [dev(A) for A in mats]
    torch.cuda.synchronize()
    srv = skew.Server(8 << 30, n_streams=4, small_n_max=512)
    pairs = [(srv.submit(d, pfaffian_only=True), srv.submit(d)) for d in devs]
    for A, d, (tp, tf) in zip(mats, devs, pairs):
        n = A.shape[0]
        rp, rf = srv.wait(tp, 120.0), srv.wait(tf, 120.0)
        assert rp["t_ptr"] is None and rp["piv_ptr"] is None and rp["L_ptr"] is None
        with pytest.raises(skew.SkewError):
            srv.factors(tp, n)
        la0, sg0, _, _, info0 = oracle.pfaffian_twostep(A)
        assert rp["sign"] == sg0 == rf["sign"]
        if sg0 != 0:
            assert close(rp["logabs"], la0) and close(rp["logabs"], rf["logabs"])
        if n % 2 == 0:
            assert rp["info"] == info0
        alone = skew.Server(8 << 30, n_streams=1, small_n_max=512)
        ta = alone.submit(d, pfaffian_only=True)
        ra = alone.wait(ta, 60.0)
        assert ra["sign"] == rp["sign"] and ra["logabs"] == rp["logabs"]
        alone.release(ta)
        alone.close()
        srv.release(tp)
        srv.release(tf)
    with pytest.raises(ValueError):
        srv.submit(devs[0], want_L=True, pfaffian_only=True)
    assert srv.stats() == {"used_bytes": 0, "queued": 0, "in_flight": 0}
    srv.close()


def test_admission_follows_budget():
    """Admission keeps what the server's requests hold within the budget: the resident
    buffers and the workspaces their launches allocate.  Checked both on the server's
    own count and on the library's device allocations (their high-water mark over the
    run, less what was held before the server started)."""
    n = 400
    A = dev(inputs.skew_gaussian(n, 11))
    per = 8 * n * n + 8 * n + 4 * n + 4096                 # about one request's buffers
    budget = int(2.5 * per) + skew.workspace_bytes(n, 0, False, lookahead=True)
    torch.cuda.synchronize()
    base, _ = skew.pool_usage(reset_high=True)
    srv = skew.Server(budget, n_streams=4, small_n_max=256)
    tickets = [srv.submit(A) for _ in range(12)]
    seen_queue = srv.stats()["queued"] > 0
    res = []
    for tk in tickets:                       # results stay resident until released, so
        res.append(srv.wait(tk, 60.0))       # each is released once read to let the
        srv.release(tk)                      # next queued request in
        assert srv.stats()["used_bytes"] <= budget
    assert seen_queue
    ref = res[0]
    assert all(r["sign"] == ref["sign"] and r["logabs"] == ref["logabs"] for r in res)
    srv.close()
    _, high = skew.pool_usage()
    assert high - base <= budget


def test_wait_times_out_until_memory_is_released():
    n = 300
    A = dev(inputs.skew_gaussian(n, 12))
    per = 8 * n * n + 8 * n + 4 * n + 4096
    srv = skew.Server(int(1.5 * per), n_streams=2, small_n_max=512)
    t1 = srv.submit(A)
    srv.wait(t1, 60.0)                      # done, still holding its memory
    t2 = srv.submit(A)
    with pytest.raises(skew.SkewError) as ei:
        srv.wait(t2, 0.3)
    assert ei.value.status == -103          # SKEW_ERR_TIMEOUT: not admitted
    assert srv.stats()["queued"] == 1
    srv.release(t1)
    r2 = srv.wait(t2, 60.0)
    assert r2["info"] == 0
    srv.release(t2)
    srv.close()


def test_refuses_request_larger_than_budget():
    srv = skew.Server(1 << 20, n_streams=1)
    A = dev(inputs.skew_gaussian(600, 1))
    with pytest.raises(skew.SkewError) as ei:
        srv.submit(A)
    assert ei.value.status == -101
    srv.close()


def test_destroy_with_pending_requests():
    srv = skew.Server(4 << 30, n_streams=2)
    A = dev(inputs.skew_gaussian(200, 3))
    for _ in range(20):
        srv.submit(A)
    srv.close()                              # finishes admitted work, drops the rest


def test_cancel_and_malformed_requests():
    import ctypes
    lib = skew.lib()
    n = 300
    A = dev(inputs.skew_gaussian(n, 13))
    per = 8 * n * n + 8 * n + 4 * n + 4096
    srv = skew.Server(int(1.5 * per), n_streams=1, small_n_max=512)
    tk = ctypes.c_uint64()
    ptr = ctypes.c_void_p(A.data_ptr())
    assert lib.skew_server_submit(srv._h, -1, ptr, n, 0, ctypes.byref(tk)) == -2   # order
    assert lib.skew_server_submit(srv._h, n, None, n, 0, ctypes.byref(tk)) == -3   # no matrix
    assert lib.skew_server_submit(srv._h, n, ptr, n - 1, 0, ctypes.byref(tk)) == -4  # lda
    assert lib.skew_server_submit(srv._h, n, ptr, n, 7, ctypes.byref(tk)) == -5    # kind
    assert lib.skew_server_release(srv._h, 10 ** 9) == -2                         # unknown
    # a request that cannot be admitted yet is cancelled before it runs
    t1 = srv.submit(A)
    srv.wait(t1, 60.0)                       # done, still holding its memory
    t2 = srv.submit(A)
    assert srv.stats()["queued"] == 1
    srv.release(t2)                          # cancel: dropped from the queue
    assert srv.stats()["queued"] == 0
    with pytest.raises(skew.SkewError):
        srv.wait(t2, 0.1)                    # the ticket is gone
    srv.release(t1)
    assert srv.stats() == {"used_bytes": 0, "queued": 0, "in_flight": 0}
    srv.close()


def test_latency_breakdown_sums_to_latency():
    """Each finished request reports where its latency went (waiting for the budget,
    for a stream, then running); the three parts are non-negative and add up to the
    latency skew_server_wait reports."""
    n = 300
    A = dev(inputs.skew_gaussian(n, 13))
    per = 8 * n * n + 8 * n + 4 * n + 4096
    budget = int(2.5 * per) + skew.workspace_bytes(n, 0, False, lookahead=True)
    srv = skew.Server(budget, n_streams=2, small_n_max=128)
    tickets = [srv.submit(A, pfaffian_only=(i % 2 == 0)) for i in range(8)]
    queued_any = False
    for tk in tickets:
        r = srv.wait(tk, 60.0)
        parts = (r["queued_s"], r["waiting_s"], r["running_s"])
        assert all(x >= 0.0 for x in parts)
        assert abs(sum(parts) - r["latency_s"]) <= 1e-6 + 1e-9 * r["latency_s"]
        queued_any |= r["queued_s"] > 0.0
        srv.release(tk)
    assert queued_any                      # the budget held some requests back
    srv.close()
