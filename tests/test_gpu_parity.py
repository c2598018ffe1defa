"""GPU path (through the C ABI) against the CPU oracle on the same seeded inputs.

Bars:
  - pivots: identical (integer work, bit-exact);
  - t and L element by element: |dL| <= TOL_C * n * eps (|L| <= 1) and
    |dt| <= TOL_C * n * eps * max|t|; both implementations are backward stable
    (error ~ n eps ||A||) and differ only in rounding order, and a wrong sign, index
    or dropped term gives O(1) differences;
  - reconstruction ||P A P^T - L T L^T||_F / (n eps ||A||_F) <= 10;
  - log|Pf| within 1e-10 * max(1, |log|Pf||) and the same sign.
"""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle  # noqa: E402
import paper_2411_09859_gb300 as skew  # noqa: E402
from paper_2411_09859_gb300 import inputs  # noqa: E402
from skewcheck import (EPS, backward_error, check_structure, perm_from_piv,  # noqa: E402
                       tridiag_from_t)

pytestmark = pytest.mark.gpu
TOL_C = 2000.0


def to_dev(A_np):
    return torch.from_numpy(np.asfortranarray(A_np, dtype=np.float64)).cuda()


def gpu_ltlt(A_np, nb):
    L, t, piv, info = skew.ltlt(to_dev(A_np), nb=nb)
    torch.cuda.synchronize()
    return (L.cpu().numpy(), t.cpu().numpy(), piv.cpu().numpy(), int(info.item()))


def gpu_pf(A_np, nb):
    la, sg, t, piv, info = skew.pfaffian(to_dev(A_np), nb=nb)
    torch.cuda.synchronize()
    return (float(la.item()), int(sg.item()), t.cpu().numpy(), piv.cpu().numpy(),
            int(info.item()))


def assert_pf_close(la, sg, la_ref, sg_ref):
    assert sg == sg_ref
    if sg_ref != 0:
        assert abs(la - la_ref) <= 1e-10 * max(1.0, abs(la_ref)), (la, la_ref)


def assert_parity(A, nb, check_backward=True):
    n = A.shape[0]
    L0, t0, p0, i0 = oracle.ltlt(A)
    L1, t1, p1, i1 = gpu_ltlt(A, nb)
    if not np.array_equal(p0, p1):
        k = int(np.argmax(p0 != p1))
        raise AssertionError(f"pivots differ first at {k}: oracle {p0[k]} gpu {p1[k]}")
    assert i1 == i0
    tol = TOL_C * max(n, 1) * EPS
    if n > 1:
        assert np.max(np.abs(L1 - L0)) <= tol
        assert np.max(np.abs(t1 - t0)) <= tol * max(1.0, np.max(np.abs(t0)))
    check_structure(L1, t1, p1, n)
    if check_backward and n <= 2048:
        assert backward_error(A, L1, t1, p1) <= 10
    la0, sg0 = oracle.pfaffian_from_factors(n, t0, p0)
    la1, sg1 = skew.pfaffian_from_factors(torch.from_numpy(t1).cuda(),
                                          torch.from_numpy(p1).cuda(), n)
    assert_pf_close(float(la1.item()), int(sg1.item()), la0, sg0)
    return L1, t1, p1


# ----------------------------------------------------------------------- factorization
@pytest.mark.parametrize("n", [2, 3, 4, 5, 8, 17, 33, 64, 65, 100])
@pytest.mark.parametrize("nb", [1, 2, 3, 8, 16])
def test_small_orders_all_panel_widths(n, nb):
    assert_parity(inputs.skew_gaussian(n, 1000 + n), nb)


@pytest.mark.parametrize("n,nb", [(127, 32), (128, 64), (129, 64), (200, 7), (255, 32),
                                  (256, 64), (257, 64), (300, 128), (333, 256), (384, 0)])
def test_ragged_orders(n, nb):
    """Orders that span several 64 x 64 update tiles and leave ragged tails."""
    assert_parity(inputs.skew_gaussian(n, 2000 + n), nb)


@pytest.mark.parametrize("nb", [1, 32])
def test_plain_n512_seed0(nb):
    """The n = 512, seed 0 workload, unblocked (nb = 1) and blocked (nb = 32)."""
    A = inputs.skew_gaussian(512, inputs.SEED_SMALL)
    assert_parity(A, nb)


def test_n4096_seed1_full_parity():
    """The n = 4096 at-scale workload (seed 1) in the default launch configuration,
    compared element by element with the oracle."""
    A = inputs.skew_gaussian(4096, inputs.SEED_SCALE[4096])
    assert_parity(A, 0, check_backward=False)


def test_trivial_orders():
    L, t, piv, info = gpu_ltlt(np.zeros((1, 1)), 0)
    assert L.tolist() == [[1.0]] and piv.tolist() == [0] and t.size == 0 and info == 0
    la, sg, _, _, info = gpu_pf(np.zeros((1, 1)), 0)
    assert sg == 0 and la == -math.inf
    A0 = torch.zeros((0, 0), dtype=torch.float64, device="cuda")
    la, sg, t, piv, info = skew.pfaffian(A0)
    torch.cuda.synchronize()
    assert float(la.item()) == 0.0 and int(sg.item()) == 1 and int(info.item()) == 0


def test_block_diagonal_zero_pivots():
    D = inputs.block_diag_skew([1.0, 3.0, 5.0, 0.5, 2.0])
    L, t, piv, info = gpu_ltlt(D, 4)
    assert np.array_equal(t, [-1.0, 0.0, -3.0, 0.0, -5.0, 0.0, -0.5, 0.0, -2.0])
    assert np.array_equal(piv, np.arange(10)) and np.array_equal(L, np.eye(10))
    assert info == 2
    la, sg, *_ = gpu_pf(D, 4)
    assert sg == 1 and math.isclose(la, math.log(1 * 3 * 5 * 0.5 * 2), rel_tol=1e-14)


@pytest.mark.parametrize("seed", range(3))
def test_permuted_block_diagonal(seed):
    rng = np.random.default_rng(seed)
    s = rng.uniform(0.5, 4.0, size=40) * rng.choice([-1, 1], size=40)
    P = inputs.permutation_matrix(rng.permutation(80))
    A = np.asfortranarray(P @ inputs.block_diag_skew(s) @ P.T)
    ref = round(np.linalg.det(P)) * np.prod(s)
    la, sg, *_ = gpu_pf(A, 16)
    assert sg == (1 if ref > 0 else -1)
    assert math.isclose(la, math.log(abs(ref)), rel_tol=1e-12)
    assert_parity(A, 16)


def test_ties_and_integer_matrix():
    n = 6
    M = np.zeros((n, n))
    M[1:, 0] = [1.0, -2.0, 2.0, -2.0, 0.5]
    M[2:, 1] = 0.25
    A = np.asfortranarray(np.tril(M, -1) - np.tril(M, -1).T)
    L, t, piv, info = gpu_ltlt(A, 2)
    assert piv[1] == 2 and t[0] == -2.0
    rng = np.random.default_rng(5)
    Mi = np.triu(rng.integers(-2, 3, size=(40, 40)).astype(float), 1)
    assert_parity(np.asfortranarray(Mi - Mi.T), 8)


@pytest.mark.parametrize("n,nb", [(6, 2), (50, 8), (300, 32), (1000, 64), (1001, 0)])
def test_pfaffian_only_path(n, nb):
    """skew_pfaffian keeps only the current panel of L: same t, piv and Pf."""
    A = inputs.skew_gaussian(n, 3000 + n)
    L0, t0, p0, _ = oracle.ltlt(A)
    la0, sg0 = oracle.pfaffian_from_factors(n, t0, p0)
    la, sg, t, piv, info = gpu_pf(A, nb)
    assert np.array_equal(piv, p0)
    assert np.max(np.abs(t - t0)) <= TOL_C * n * EPS * max(1.0, np.max(np.abs(t0)))
    assert_pf_close(la, sg, la0, sg0)
    assert info == 0


@pytest.mark.parametrize("n", [8, 64])
def test_qdq_closed_form_on_gpu(n):
    A, s = inputs.qdq_skew(n, inputs.SEED_PRECISION, smax=1e3)
    la, sg, *_ = gpu_pf(A, 16)
    assert sg == 1
    assert abs(la - float(np.sum(np.log(s)))) <= 1e-9 * max(1.0, abs(la))


def test_nonfinite_input_reported():
    A = inputs.skew_gaussian(100, 4)
    A[70, 30] = np.nan
    A[30, 70] = np.nan
    _, _, _, info = gpu_ltlt(A, 16)
    assert info == -100
    A[70, 30] = np.inf
    la, sg, t, piv, info = gpu_pf(A, 16)
    assert info == -100


def test_upper_triangle_never_read():
    A = inputs.skew_gaussian(150, 6)
    B = A.copy(order="F")
    B[np.triu_indices(150)] = np.nan
    r1, r2 = gpu_ltlt(A, 16), gpu_ltlt(B, 16)
    assert np.array_equal(r1[2], r2[2])
    assert np.array_equal(r1[1], r2[1]) and np.array_equal(r1[0], r2[0])


def test_host_entry_point_matches_device_path():
    A = inputs.skew_gaussian(300, 7)
    L, t, piv, la, sg, info = skew.ltlt_host(A, want_L=True, nb=32)
    L1, t1, p1, i1 = gpu_ltlt(A, 32)
    assert np.array_equal(piv, p1) and np.array_equal(t, t1) and np.array_equal(L, L1)
    la0, sg0 = oracle.pfaffian_from_factors(300, t, piv)
    assert_pf_close(la, sg, la0, sg0)
    _, t2, p2, la2, sg2, info2 = skew.ltlt_host(A, want_L=False, nb=32)
    assert np.array_equal(p2, p1) and info2 == 0
    assert_pf_close(la2, sg2, la0, sg0)


@pytest.mark.parametrize("n", [255, 256, 700])
def test_host_entry_point_upper_triangles(n):
    """skew_ltlt_host: NaN in A's upper triangle (and diagonal) changes nothing, and L's
    upper triangle comes back exactly zero in an output buffer that held NaN."""
    A = inputs.skew_gaussian(n, 11 + n)
    Apoison = np.asfortranarray(A.copy())
    Apoison[np.triu_indices(n)] = np.nan
    Lout = np.full((n, n), np.nan, order="F")
    L, t, piv, la, sg, info = skew.ltlt_host(Apoison, want_L=True, nb=32, L_out=Lout)
    L1, t1, p1, i1 = gpu_ltlt(A, 32)
    assert info == 0 and np.array_equal(piv, p1) and np.array_equal(t, t1)
    assert np.array_equal(L, L1)
    assert np.all(L[np.triu_indices(n, 1)] == 0.0) and np.all(np.diag(L) == 1.0)
    # padded host matrices (leading dimension n + 3) take the pitched copies
    Apad = np.full((n + 3, n), np.nan, order="F")
    Apad[:n, :] = A
    L2 = np.full((n + 3, n), np.nan, order="F")
    t2, p2 = np.zeros(n - 1), np.zeros(n, dtype=np.int32)
    la2, sg2, inf2 = ctypes.c_double(), ctypes.c_int32(), ctypes.c_int32()
    vp = ctypes.c_void_p
    st = skew.lib().skew_ltlt_host(n, vp(Apad.ctypes.data), n + 3, vp(L2.ctypes.data), n + 3,
                                   vp(t2.ctypes.data), vp(p2.ctypes.data), ctypes.byref(la2),
                                   ctypes.byref(sg2), ctypes.byref(inf2), 32)
    assert st == 0 and inf2.value == 0
    assert np.array_equal(L2[:n], L1) and np.array_equal(p2, p1) and np.array_equal(t2, t1)
    assert np.all(np.isnan(L2[n:]))                  # the padding rows are not written


@pytest.mark.parametrize("n,nb", [(700, 32), (33, 32), (300, 64), (1, 8), (2, 8)])
def test_host_entry_point_page_locked_rows_during_factorization(n, nb):
    """With a page-locked L the final rows of L reach it panel by panel while the
    factorization runs; the result equals the device path's, rows past n untouched."""
    A = inputs.skew_gaussian(n, 21 + n)
    Lpin = torch.empty((n, n), dtype=torch.float64).pin_memory().t()   # Fortran order
    Lpin.fill_(float("nan"))
    L, t, piv, la, sg, info = skew.ltlt_host(A, want_L=True, nb=nb, L_out=Lpin.numpy())
    L1, t1, p1, i1 = gpu_ltlt(A, nb)
    assert info == 0 and np.array_equal(piv, p1) and np.array_equal(t, t1)
    assert np.array_equal(L, L1)
    ph = skew.ltlt_host_timing()
    assert ph is not None and all(x >= 0 for x in ph)


def test_host_entry_point_keeps_buffers_and_reports_phases():
    """Repeated host calls of one order reuse the library's buffers (no change in free
    device memory after the first) and report their three phases."""
    A = inputs.skew_gaussian(1000, 8)
    r0 = skew.ltlt_host(A, want_L=True, nb=32)
    ph = skew.ltlt_host_timing()
    assert ph is not None and all(x > 0 for x in ph)
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        r1 = skew.ltlt_host(A, want_L=True, nb=32)
        assert np.array_equal(r1[0], r0[0]) and np.array_equal(r1[2], r0[2])
    assert torch.cuda.mem_get_info()[0] == free0
    small = skew.ltlt_host(inputs.skew_gaussian(40, 9), want_L=True, nb=8)
    assert small[5] == 0
    assert torch.cuda.mem_get_info()[0] == free0        # a smaller order fits the same buffers
    skew.trim_memory()


def test_input_sizes_rejected():
    with pytest.raises(skew.SkewError):
        skew.ltlt(to_dev(inputs.skew_gaussian(8, 0)), nb=300)
    A = to_dev(inputs.skew_gaussian(8, 0))
    st = skew.lib().skew_ltlt(8, A.data_ptr(), 4, A.data_ptr(), 8, None, None, None, 0,
                              None, 0, None)
    assert st == -3


def test_full_size_n16384_sampled():
    """n = 16384 (seed 3), default launch configuration: properties that hold at any
    size, and the reconstruction (P A P^T)[i, j] = (L T L^T)[i, j] on sampled entries,
    each computed on the CPU from two rows of L and t."""
    n = 16384
    A = inputs.skew_gaussian(n, inputs.SEED_SCALE[n])
    L, t, piv, info = gpu_ltlt(A, 0)
    assert info == 0
    assert piv[0] == 0 and np.all(piv >= np.arange(n)) and np.all(piv < n)
    assert np.all(np.isfinite(t)) and np.all(t != 0)
    assert np.all(np.abs(L) <= 1.0)
    assert np.all(np.diag(L) == 1.0) and np.all(L[1:, 0] == 0.0)
    rng = np.random.default_rng(0)
    perm = np.arange(n)
    for i in range(n):
        r = int(piv[i])
        perm[i], perm[r] = perm[r], perm[i]
    idx_i = rng.integers(0, n, 3000)
    idx_j = rng.integers(0, n, 3000)
    nrm = np.linalg.norm(A)
    worst = 0.0
    for i, j in zip(idx_i, idx_j):
        # (L T L^T)[i, j] = sum_a t[a] (L[i, a+1] L[j, a] - L[i, a] L[j, a+1])
        li, lj = L[i], L[j]
        val = float(np.dot(t, li[1:] * lj[:-1] - li[:-1] * lj[1:]))
        ref = A[perm[i], perm[j]]
        worst = max(worst, abs(val - ref))
    # entrywise residuals are bounded by the normwise one
    assert worst / (n * EPS * nrm) <= 10
    # read-off restated: sign = (-1)^(#exchanges) prod sign(-t[2i]), log = sum log|t[2i]|
    la, sg = skew.pfaffian_from_factors(torch.from_numpy(t).cuda(),
                                        torch.from_numpy(piv).cuda(), n)
    even = t[0::2][: n // 2]
    sg_ref = (-1) ** int(np.sum(piv != np.arange(n))) * int(np.prod(np.sign(-even)))
    la_ref = math.fsum(np.log(np.abs(even)))
    assert_pf_close(float(la.item()), int(sg.item()), la_ref, sg_ref)


# ----------------------------------------------------------------------- level-3 ops
@pytest.mark.parametrize("m,k", [(2, 1), (63, 5), (64, 16), (65, 17), (130, 33), (200, 64),
                                 (257, 3)])
@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (-0.5, 2.0), (1.5, 0.0)])
def test_skew_rank2k_vs_oracle(m, k, alpha, beta):
    rng = np.random.default_rng(m * 100 + k)
    X = np.asfortranarray(rng.standard_normal((m, k)))
    Y = np.asfortranarray(rng.standard_normal((m, k)))
    C = np.asfortranarray(rng.standard_normal((m, m)))
    if beta == 0.0:
        C[np.tril_indices(m, -1)] = np.nan          # beta = 0: C is not read
    ref = oracle.skew_rank2k(alpha, X, Y, beta, np.nan_to_num(C) if beta == 0.0 else C)
    Cd = to_dev(C)
    skew.rank2k(alpha, to_dev(X), to_dev(Y), beta, Cd)
    got = Cd.cpu().numpy()
    il = np.tril_indices(m, -1)
    scale = max(1.0, np.max(np.abs(ref[il])))
    assert np.max(np.abs(got[il] - ref[il])) <= 64 * k * EPS * scale * 10
    iu = np.triu_indices(m)
    assert np.array_equal(got[iu], C[iu], equal_nan=True)


@pytest.mark.parametrize("m,b", [(5, 2), (64, 8), (100, 33), (129, 64), (300, 128), (70, 1)])
def test_skew_tridiag_rankk_vs_oracle(m, b):
    rng = np.random.default_rng(m + 7 * b)
    Am = np.asfortranarray(rng.standard_normal((m, b)))
    t = rng.standard_normal(max(b - 1, 0))
    C = np.asfortranarray(rng.standard_normal((m, m)))
    ref = oracle.skew_tridiag_rankk(-1.0, Am, t, 1.0, C)
    Cd = to_dev(C)
    skew.tridiag_rankk(-1.0, to_dev(Am), torch.from_numpy(t).cuda(), 1.0, Cd)
    got = Cd.cpu().numpy()
    il = np.tril_indices(m, -1)
    assert np.max(np.abs(got[il] - ref[il])) <= 1e-12 * max(1.0, np.max(np.abs(ref[il])))
    dense = C - Am @ tridiag_from_t(t, b) @ Am.T
    assert np.allclose(got[il], dense[il], atol=1e-11)
    iu = np.triu_indices(m)
    assert np.array_equal(got[iu], C[iu])


def test_launch_counter_moves():
    before = skew.kernel_launches()
    gpu_ltlt(inputs.skew_gaussian(100, 1), 16)
    assert skew.kernel_launches() > before


def test_order_beyond_one_row_per_panel_thread():
    """n = 39000: the first panels have more rows than 256 x (multiprocessors), so they
    run the global-memory panel, the later ones the shared-memory panel.  The oracle
    would take minutes, so the factors are checked by properties that hold at any
    order: randomized residuals of P A P^T = L T L^T (O(n^2) per vector), |L| <= 1,
    L e_0 = e_0, the pivot vector, and log|Pf| against the Pfaffian-only path."""
    n = 39000
    props = torch.cuda.get_device_properties(0)
    if n - 1 <= props.multi_processor_count * 256:
        pytest.skip("this device's panel keeps one row per thread at n = 39000")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(123)
    A = torch.tril(torch.randn((n, n), generator=gen, dtype=torch.float64, device="cuda"), -1)
    A = A - A.t()                                   # skew; element (i, j) is A[i, j]
    work = skew.fortran_empty(n, n, "cuda")
    work.copy_(A)
    L, t, piv, info = skew.ltlt(work, nb=64)
    torch.cuda.synchronize()
    del work
    assert int(info.item()) == 0
    p = piv.cpu().numpy()
    assert p[0] == 0 and np.all(p[1:] >= np.arange(1, n))
    perm = torch.from_numpy(perm_from_piv(p)).cuda()
    assert float(torch.max(torch.abs(torch.tril(L, -1)))) <= 1.0
    assert bool(torch.all(L[:, 0] == torch.eye(n, 1, dtype=torch.float64, device="cuda")[:, 0]))
    normA = float(torch.linalg.norm(A))
    for _ in range(3):
        x = torch.randn(n, generator=gen, dtype=torch.float64, device="cuda")
        xp = torch.zeros_like(x)
        xp[perm] = x
        y = (A @ xp)[perm]                          # (P A P^T) x, (P A P^T)[a, b] = A[perm a, perm b]
        z = L.t() @ x                               # L T L^T x, T[i+1, i] = t[i] = -T[i, i+1]
        Tz = torch.zeros_like(z)
        Tz[1:] += t * z[:-1]
        Tz[:-1] -= t * z[1:]
        w = L @ Tz
        rel = float(torch.linalg.norm(y - w)) / (normA * float(torch.linalg.norm(x)))
        assert rel <= 10 * n * EPS, rel
    la1, sg1 = skew.pfaffian_from_factors(t, piv, n)
    del L
    w2 = skew.fortran_empty(n, n, "cuda")
    w2.copy_(A)
    del A
    la2, sg2, *_ = skew.pfaffian(w2, nb=64)
    torch.cuda.synchronize()
    assert int(sg1.item()) == int(sg2.item())
    assert abs(float(la1.item()) - float(la2.item())) <= 1e-10 * abs(float(la2.item()))


@pytest.mark.parametrize("n,nb", [(2, 1), (40, 8), (257, 32), (1000, 64), (2050, 96), (4097, 64)])
def test_cluster_panel_on_and_off_match_the_oracle(n, nb):
    """The plain path's panels of trailing blocks up to 4096 rows run as one thread-block
    cluster (candidates exchanged through distributed shared memory); with the cluster
    panel turned off they run as the grid-wide panel.  Both reach the oracle's
    factorization.  (The look-ahead is off here, so that every panel is a plain one.)"""
    A = inputs.skew_gaussian(n, 13000 + n)
    old_la = skew.set_lookahead(0)
    try:
        for on in (True, False):
            old = skew.set_cluster_panel(on)
            try:
                assert_parity(A, nb, check_backward=(n <= 1100))
            finally:
                skew.set_cluster_panel(old)
    finally:
        skew.set_lookahead(old_la)


def test_cluster_panel_nonfinite_leaves_together():
    """A recorded error (here the prologue's flag for a NaN in the input) reaches every
    CTA of a cluster panel through the first exchange, and they all leave at the same
    point: the call returns info = -100 and the context stays usable."""
    A = inputs.skew_gaussian(600, 14)
    A[500, 300] = np.nan
    A[300, 500] = np.nan
    old_la = skew.set_lookahead(0)
    try:
        _, _, _, info = gpu_ltlt(A, 32)
        assert info == -100
        la, sg, t, piv, info = gpu_pf(A, 32)
        assert info == -100
        # the context is still usable
        B = inputs.skew_gaussian(300, 15)
        assert_parity(B, 32)
    finally:
        skew.set_lookahead(old_la)
