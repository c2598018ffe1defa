"""Batched persistent form (skew_ltlt_batched) against the oracle and the single
matrix path: identical pivots, factors within the element-wise tolerance of the
single-matrix tests, log|Pf| within 1e-10 relative with the same sign."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle  # noqa: E402
import paper_2411_09859_gb300 as skew  # noqa: E402
from paper_2411_09859_gb300 import inputs  # noqa: E402
from skewcheck import EPS, check_structure  # noqa: E402

pytestmark = pytest.mark.gpu
TOL_C = 2000.0


def dev(A):
    return torch.from_numpy(np.asfortranarray(A, dtype=np.float64)).cuda()


def run_batch(mats, want_L):
    As = [dev(A) for A in mats]
    la, sg, info, ts, pivs, Ls = skew.ltlt_batched(As, want_L=want_L)
    torch.cuda.synchronize()
    return (la.cpu().numpy(), sg.cpu().numpy(), info.cpu().numpy(),
            [t.cpu().numpy() for t in ts], [p.cpu().numpy() for p in pivs],
            [None if L is None else L.cpu().numpy() for L in Ls])


def check_against_oracle(A, la, sg, info, t, piv, L):
    n = A.shape[0]
    L0, t0, p0, i0 = oracle.ltlt(A)
    assert np.array_equal(piv, p0)
    assert info == i0
    tol = TOL_C * max(n, 1) * EPS
    if n > 1:
        assert np.max(np.abs(t - t0)) <= tol * max(1.0, np.max(np.abs(t0)))
    if L is not None:
        if n > 1:
            assert np.max(np.abs(L - L0)) <= tol
        check_structure(L, t, piv, n)
    la0, sg0 = oracle.pfaffian_from_factors(n, t0, p0)
    assert sg == sg0
    if sg0 != 0:
        assert abs(la - la0) <= 1e-10 * max(1.0, abs(la0))


@pytest.mark.parametrize("want_L", [False, True])
def test_mixed_orders_against_oracle(want_L):
    sizes = [0, 1, 2, 3, 4, 5, 16, 17, 31, 64, 100, 127, 128, 200, 255, 256, 257, 300, 513]
    mats = [inputs.skew_gaussian(n, 5000 + n) for n in sizes]
    la, sg, info, ts, pivs, Ls = run_batch(mats, want_L)
    for b, A in enumerate(mats):
        check_against_oracle(A, la[b], sg[b], info[b], ts[b], pivs[b], Ls[b])


def test_batched_workload_sample():
    """The 4096-matrix workload (orders even in [16, 256], matrix i from seed 1000+i):
    all of it in one launch; every 32nd matrix checked against the oracle, all of
    them for the invariants."""
    sizes = inputs.batched_sizes(4096)
    mats = [inputs.skew_gaussian(int(n), inputs.SEED_BATCH_BASE + i) for i, n in enumerate(sizes)]
    la, sg, info, ts, pivs, Ls = run_batch(mats, False)
    assert np.all(info == 0)
    assert np.all(sg != 0)
    for b in range(0, 4096, 32):
        check_against_oracle(mats[b], la[b], sg[b], info[b], ts[b], pivs[b], None)
    for b in range(4096):
        n = int(sizes[b])
        assert pivs[b][0] == 0 and np.all(pivs[b] >= np.arange(n))


def test_batched_equals_single_calls():
    mats = [inputs.skew_gaussian(n, 6000 + n) for n in (40, 96, 180, 256)]
    la, sg, info, ts, pivs, Ls = run_batch(mats, True)
    for b, A in enumerate(mats):
        L1, t1, p1, i1 = skew.ltlt(dev(A), nb=16)
        torch.cuda.synchronize()
        assert np.array_equal(pivs[b], p1.cpu().numpy())
        n = A.shape[0]
        assert np.max(np.abs(ts[b] - t1.cpu().numpy())) <= TOL_C * n * EPS * np.max(np.abs(ts[b]))
        assert np.max(np.abs(Ls[b] - L1.cpu().numpy())) <= TOL_C * n * EPS


def test_zero_pivots_block_diagonal():
    D = inputs.block_diag_skew([1.0, 3.0, 5.0])
    la, sg, info, ts, pivs, Ls = run_batch([D, D.copy()], True)
    for b in range(2):
        assert np.array_equal(ts[b], [-1.0, 0.0, -3.0, 0.0, -5.0])
        assert info[b] == 2 and sg[b] == 1 and math.isclose(la[b], math.log(15.0), rel_tol=1e-15)
        assert np.array_equal(Ls[b], np.eye(6))


def test_bad_descriptor_and_nonfinite():
    good = inputs.skew_gaussian(20, 1)
    bad = inputs.skew_gaussian(20, 2)
    bad[10, 3] = np.nan
    As = [dev(good), dev(bad), dev(good)]
    ts = [torch.empty(19, dtype=torch.float64, device="cuda") for _ in range(3)]
    pivs = [torch.empty(20, dtype=torch.int32, device="cuda") for _ in range(3)]
    table = skew.problem_table(As, [None] * 3, ts, pivs, "cuda")
    table[2, 2] = 5                     # lda < n: an invalid descriptor
    la, sg, info, *_ = skew.ltlt_batched(As, table=table, outs=(ts, pivs, [None] * 3))
    torch.cuda.synchronize()
    info = info.cpu().numpy()
    assert info[0] == 0 and info[1] == -100 and info[2] == -2


def test_rejects_bad_arguments():
    st = skew.lib().skew_ltlt_batched(-1, None, None, None, None, 16, None, 0, None)
    assert st == -1
    st = skew.lib().skew_ltlt_batched(3, None, None, None, None, 16, None, 0, None)
    assert st == -2
    st = skew.lib().skew_ltlt_batched(0, None, None, None, None, 99999, None, 0, None)
    assert st == -6


@pytest.mark.parametrize("want_L", [False, True])
def test_blocked_kernel_orders_against_oracle(want_L):
    """Batches with every order <= 512 take the blocked (panel + DMMA) kernel."""
    sizes = [0, 1, 2, 3, 5, 16, 17, 18, 31, 32, 33, 47, 64, 100, 129, 255, 256, 300, 511, 512]
    mats = [inputs.skew_gaussian(n, 9000 + n) for n in sizes]
    la, sg, info, ts, pivs, Ls = run_batch(mats, want_L)
    for b, A in enumerate(mats):
        check_against_oracle(A, la[b], sg[b], info[b], ts[b], pivs[b], Ls[b])


def test_blocked_kernel_zero_pivots_and_ties():
    D = inputs.block_diag_skew(np.arange(1.0, 21.0))          # n = 40, zero columns
    rng = np.random.default_rng(3)
    Mi = np.triu(rng.integers(-2, 3, size=(70, 70)).astype(float), 1)
    I = np.asfortranarray(Mi - Mi.T)                           # many ties
    la, sg, info, ts, pivs, Ls = run_batch([D, I], True)
    check_against_oracle(D, la[0], sg[0], info[0], ts[0], pivs[0], Ls[0])
    check_against_oracle(I, la[1], sg[1], info[1], ts[1], pivs[1], Ls[1])


# ------------------------------------------------ Pfaffian-only (two-step) batched form
def run_pf_batch(mats):
    As = [dev(A) for A in mats]
    la, sg, info, as_, pivs = skew.pfaffian_batched(As)
    torch.cuda.synchronize()
    return (la.cpu().numpy(), sg.cpu().numpy(), info.cpu().numpy(),
            [a.cpu().numpy() for a in as_], [p.cpu().numpy() for p in pivs])


def check_twostep(A, la, sg, info, a, piv):
    n = A.shape[0]
    la0, sg0, a0, p0, i0 = oracle.pfaffian_twostep(A)
    assert np.array_equal(piv[:n], p0)
    assert info == i0 and sg == sg0
    if n >= 2:
        assert np.max(np.abs(a[: n // 2] - a0)) <= TOL_C * n * EPS * max(1e-300, np.max(np.abs(a0)))
    if sg0 != 0:
        assert abs(la - la0) <= 1e-10 * max(1.0, abs(la0))


def test_pfaffian_batched_mixed_orders_against_oracle():
    rng = np.random.default_rng(77)
    sizes = [0, 1, 2, 3, 5, 16, 17, 31, 33, 64, 100, 129, 255, 256, 300, 511, 512] + \
        [int(x) for x in rng.integers(2, 257, size=40)]
    mats = [inputs.skew_gaussian(n, 2000 + i) for i, n in enumerate(sizes)]
    la, sg, info, as_, pivs = run_pf_batch(mats)
    for b, A in enumerate(mats):
        if A.shape[0] == 0:
            assert sg[b] == 1 and la[b] == 0.0
            continue
        check_twostep(A, la[b], sg[b], info[b], as_[b], pivs[b])


def test_pfaffian_batched_equals_single_two_step_and_one_step():
    mats = [inputs.skew_gaussian(n, 3100 + n) for n in (40, 96, 200, 256)]
    la, sg, info, as_, pivs = run_pf_batch(mats)
    for b, A in enumerate(mats):
        l1, s1, a1, p1, i1 = skew.pfaffian_twostep(dev(A), nb=16)
        l2, s2, *_ = skew.pfaffian(dev(A))
        torch.cuda.synchronize()
        assert np.array_equal(pivs[b], p1.cpu().numpy())
        assert int(s1.item()) == sg[b] == int(s2.item())
        assert abs(la[b] - float(l1.item())) <= 1e-12 * max(1.0, abs(la[b]))
        assert abs(la[b] - float(l2.item())) <= 1e-10 * max(1.0, abs(la[b]))


def test_pfaffian_batched_zero_pivots_nonfinite_and_bad_descriptor():
    D = inputs.block_diag_skew([2.0, -1.0, 4.0])
    Z = np.zeros((6, 6))
    B = inputs.skew_gaussian(20, 4)
    B[13, 2] = np.nan
    la, sg, info, as_, pivs = run_pf_batch([D, Z, B])
    assert sg[0] == -1 and math.isclose(la[0], math.log(8.0), rel_tol=1e-15)
    assert np.array_equal(as_[0][:3], [-2.0, 1.0, -4.0])
    assert sg[1] == 0 and info[1] == 1
    assert info[2] == -100
    As = [dev(inputs.skew_gaussian(8, 1))]
    with pytest.raises(skew.SkewError):
        skew.pfaffian_batched(As, max_n=513)


# ------------------------------------------------------------------ CUDA graph capture
def test_pfaffian_batched_replays_from_a_cuda_graph():
    """The batched launch (ordering kernel + persistent kernel) captured once in a CUDA
    graph, with a caller-supplied workspace and result buffers, and replayed on fresh
    inputs: the results equal those of direct calls."""
    sizes = [16, 30, 64, 100, 130, 200, 256, 98]
    mats = [inputs.skew_gaussian(n, 6000 + i) for i, n in enumerate(sizes)]
    pristine = [dev(A) for A in mats]
    work = [skew.fortran_empty(A.shape[0], A.shape[0], "cuda") for A in pristine]
    as_ = [torch.empty(max(n // 2, 1), dtype=torch.float64, device="cuda") for n in sizes]
    pivs = [torch.empty(n, dtype=torch.int32, device="cuda") for n in sizes]
    table = skew.problem_table(work, [None] * len(work), as_, pivs, "cuda")
    ws = torch.empty(skew.batched_workspace_bytes(len(work), 256), dtype=torch.uint8, device="cuda")
    res = (torch.empty(len(work), dtype=torch.float64, device="cuda"),
           torch.empty(len(work), dtype=torch.int32, device="cuda"),
           torch.empty(len(work), dtype=torch.int32, device="cuda"))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):                    # warm up outside the capture
        for w, p in zip(work, pristine):
            w.copy_(p)
        skew.pfaffian_batched(work, stream=s, max_n=256, table=table, outs=(as_, pivs),
                              workspace=ws, results=res)
    torch.cuda.synchronize()
    direct = [r.clone() for r in res]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for w, p in zip(work, pristine):
            w.copy_(p)
        skew.pfaffian_batched(work, stream=s, max_n=256, table=table, outs=(as_, pivs),
                              workspace=ws, results=res)
    for _ in range(3):
        for r in res:
            r.fill_(0)
        g.replay()
        torch.cuda.synchronize()
        for r, d in zip(res, direct):
            assert torch.equal(r, d)
    for b, A in enumerate(mats):
        check_twostep(A, float(res[0][b]), int(res[1][b]), int(res[2][b]),
                      as_[b].cpu().numpy(), pivs[b].cpu().numpy())


@pytest.mark.parametrize("nb", [8, 16, 32])
@pytest.mark.parametrize("wt", [16, 32])
@pytest.mark.parametrize("threads", [256, 128])
def test_batched_panel_widths_against_oracle(nb, wt, threads):
    """Every (panel width, update warp tile, CTA size) the batched tuner can choose,
    forced for all orders, in both batched kernels."""
    from paper_2411_09859_gb300 import autotune
    sizes = [2, 9, 16, 33, 70, 128, 200, 256, 300, 512]
    mats = [inputs.skew_gaussian(n, 7100 + n) for n in sizes]
    old_threads = skew.set_batched_threads(threads)
    try:
        skew.set_batched_nb_table([(512, nb, wt)])
        assert skew.batched_nb(100) == nb and skew.batched_warp_tile(100) == wt
        la, sg, info, ts, pivs, Ls = run_batch(mats, want_L=True)
        for b, A in enumerate(mats):
            check_against_oracle(A, la[b], sg[b], info[b], ts[b], pivs[b], Ls[b])
        la, sg, info, as_, pivs = run_pf_batch(mats)
        for b, A in enumerate(mats):
            check_twostep(A, la[b], sg[b], info[b], as_[b], pivs[b])
    finally:
        skew.set_batched_threads(old_threads)
        if not autotune.load():
            skew.set_batched_nb_table([])
