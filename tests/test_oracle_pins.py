"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: every expected value comes from the
Pfaffian's definition, a determinant by LAPACK LU, a closed form, a structural
invariant of the factors, or an independent restatement (full-storage blocked
algorithm, dense numpy products).
"""
import math

import numpy as np
import pytest

from paper_2411_09859_gb300 import inputs
from skewcheck import (backward_error, check_structure, full_skew_from_lower,
                       ltlt_blocked, ltlt_blocked_delayed, perm_from_piv, pf4_closed_form,
                       pfaffian_by_definition, pfaffian_by_matchings,
                       pfaffian_from_t_piv, tridiag_from_t)


def signed_pf(logabs, sign):
    return sign * math.exp(logabs) if sign != 0 else 0.0


# ---------------------------------------------------------------- Pfaffian value
@pytest.mark.parametrize("n", [2, 4, 6, 8])
@pytest.mark.parametrize("seed", range(4))
def test_pfaffian_matches_definition(orc, n, seed):
    """Pf by the permutation sum of Section 1, n <= 8."""
    A = inputs.skew_gaussian(n, 100 + seed)
    ref = pfaffian_by_definition(A)
    la, sg = orc.pfaffian(A)
    assert sg == (1 if ref > 0 else -1)
    assert math.isclose(la, math.log(abs(ref)), rel_tol=1e-12, abs_tol=1e-12)


@pytest.mark.parametrize("n", [10, 12])
def test_pfaffian_matches_matching_expansion(orc, n):
    A = inputs.skew_gaussian(n, 7)
    ref = pfaffian_by_matchings(A)
    la, sg = orc.pfaffian(A)
    assert sg == (1 if ref > 0 else -1)
    assert math.isclose(la, math.log(abs(ref)), rel_tol=1e-11, abs_tol=1e-11)


def test_definition_and_matchings_agree():
    for seed in range(3):
        A = inputs.skew_gaussian(6, seed)
        assert math.isclose(pfaffian_by_definition(A), pfaffian_by_matchings(A),
                            rel_tol=1e-12)


def test_integer_matrices_exact(orc):
    """Small integer skew matrices: the Pfaffian is an integer; compare exactly
    after rounding the oracle's value."""
    rng = np.random.default_rng(11)
    for n in (2, 4, 6, 8):
        for _ in range(5):
            M = np.triu(rng.integers(-3, 4, size=(n, n)).astype(float), 1)
            A = np.asfortranarray(M - M.T)
            ref = pfaffian_by_definition(A)
            la, sg = orc.pfaffian(A)
            got = signed_pf(la, sg)
            assert round(got) == round(ref)
            assert abs(got - ref) <= 1e-9 * max(1.0, abs(ref))


def test_pf_2x2_and_4x4_closed_forms(orc):
    for seed in range(10):
        A2 = inputs.skew_gaussian(2, 200 + seed)
        la, sg = orc.pfaffian(A2)
        assert math.isclose(signed_pf(la, sg), A2[0, 1], rel_tol=1e-14)
        A4 = inputs.skew_gaussian(4, 300 + seed)
        la, sg = orc.pfaffian(A4)
        assert math.isclose(signed_pf(la, sg), pf4_closed_form(A4), rel_tol=1e-12)


@pytest.mark.parametrize("n", [2, 10, 16, 32, 64])
def test_pf_squared_is_det(orc, n):
    """Pf(X)^2 = det(X) (Section 1), det by LAPACK LU via numpy.slogdet."""
    A = inputs.skew_gaussian(n, 400 + n)
    la, sg = orc.pfaffian(A)
    s, ld = np.linalg.slogdet(A)
    assert s > 0            # det of a real skew matrix of even order is >= 0
    assert math.isclose(2 * la, ld, rel_tol=1e-11, abs_tol=1e-10)


# ---------------------------------------------------------------- closed forms
def test_block_diagonal_closed_form(orc):
    """D = blockdiag([[0, s_k], [-s_k, 0]]): Pf(D) = prod s_k, and every odd step
    meets an all-zero column (the zero-pivot path): t = (-1, 0, -3, 0, -5)."""
    D = inputs.block_diag_skew([1.0, 3.0, 5.0])
    L, t, piv, info = orc.ltlt(D)
    assert np.array_equal(t, [-1.0, 0.0, -3.0, 0.0, -5.0])
    assert np.array_equal(piv, np.arange(6))
    assert np.array_equal(L, np.eye(6))
    assert info == 2                      # 1 + first k with t[k] == 0
    la, sg = orc.pfaffian_from_factors(6, t, piv)
    assert sg == 1 and math.isclose(la, math.log(15.0), rel_tol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_permuted_block_diagonal(orc, seed):
    """Pf(P D P^T) = det(P) Pf(D) = det(P) prod s (Section 2.2 with B = P)."""
    rng = np.random.default_rng(seed)
    m = 5
    s = rng.uniform(0.5, 4.0, size=m) * rng.choice([-1, 1], size=m)
    D = inputs.block_diag_skew(s)
    perm = rng.permutation(2 * m)
    P = inputs.permutation_matrix(perm)
    A = np.asfortranarray(P @ D @ P.T)
    detP = round(np.linalg.det(P))
    ref = detP * np.prod(s)
    la, sg = orc.pfaffian(A)
    assert sg == (1 if ref > 0 else -1)
    assert math.isclose(la, math.log(abs(ref)), rel_tol=1e-13)
    L, t, piv, info = orc.ltlt(A)
    assert backward_error(A, L, t, piv) <= 10


@pytest.mark.parametrize("n", [8, 40])
def test_qdq_closed_form(orc, n):
    """A = Q D Q^T with Q in SO(n): Pf(A) = det(Q) Pf(D) = prod s (> 0)."""
    A, s = inputs.qdq_skew(n, 5, smax=1e3)
    la, sg = orc.pfaffian(A)
    assert sg == 1
    assert math.isclose(la, float(np.sum(np.log(s))), rel_tol=1e-9, abs_tol=1e-9)


# ---------------------------------------------------------------- factors
@pytest.mark.parametrize("n", [3, 5, 8, 17, 50, 128, 301])
def test_reconstruction_and_invariants(orc, n):
    A = inputs.skew_gaussian(n, 500 + n)
    L, t, piv, info = orc.ltlt(A)
    assert info == 0
    check_structure(L, t, piv, n)
    assert backward_error(A, L, t, piv) <= 10


def test_pfaffian_readoff_agrees_with_t_piv(orc):
    for n in (2, 6, 12, 30):
        A = inputs.skew_gaussian(n, 600 + n)
        L, t, piv, _ = orc.ltlt(A)
        la, sg = orc.pfaffian_from_factors(n, t, piv)
        ref = pfaffian_from_t_piv(t, piv, n)
        assert sg == (1 if ref > 0 else -1)
        assert math.isclose(la, math.log(abs(ref)), rel_tol=1e-12)


def test_input_upper_triangle_ignored(orc):
    A = inputs.skew_gaussian(20, 9)
    B = A.copy(order="F")
    B[np.triu_indices(20)] = 123.0           # garbage above and on the diagonal
    r1, r2 = orc.ltlt(A), orc.ltlt(B)
    for a, b in zip(r1[:3], r2[:3]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("n,nb", [(50, 1), (50, 4), (61, 8), (64, 32), (7, 3),
                                  (33, 2), (40, 5), (100, 16), (130, 64)])
def test_blocked_equals_unblocked(orc, n, nb):
    """The pivoted blocked right-looking algorithm (Sections 4.2 and 5.2) gives the
    same pivots as the unblocked one, and the same factors up to rounding; block
    size one is the unblocked right-looking algorithm (Section 4.2 notes)."""
    A = inputs.skew_gaussian(n, 700 + n + nb)
    L0, t0, p0, _ = orc.ltlt(A)
    for fused in (False, True):
        L1, t1, p1 = ltlt_blocked(A, nb, fused_w=fused)
        assert np.array_equal(p0, p1)
        assert np.max(np.abs(L0 - L1)) <= 1e-12
        assert np.max(np.abs(t0 - t1)) <= 1e-12 * max(1.0, np.max(np.abs(t0)))


@pytest.mark.parametrize("n,nb", [(50, 1), (50, 4), (61, 8), (64, 32), (7, 3),
                                  (33, 2), (40, 5), (100, 16), (130, 64)])
def test_delayed_transform_ordering_reaches_the_same_factorization(orc, n, nb):
    """The fused ordering of Invariant 2a (the last Gauss transform of each panel
    applied with the next panel, Section 4.2) reaches the oracle's factorization:
    identical pivots, factors equal up to rounding.  The GPU path keeps Variant 1 and
    fuses that last transform into the same trailing-update launch instead."""
    A = inputs.skew_gaussian(n, 900 + n + nb)
    L0, t0, p0, _ = orc.ltlt(A)
    L1, t1, p1 = ltlt_blocked_delayed(A, nb)
    assert np.array_equal(p0, p1)
    assert np.max(np.abs(L0 - L1)) <= 1e-12
    assert np.max(np.abs(t0 - t1)) <= 1e-12 * max(1.0, np.max(np.abs(t0)))


def test_w_identity_and_tridiag_rankk(orc):
    """Theorem (T = S - S^T): A T A^T = W A^T - A W^T with W = A S; and the oracle's
    skew_tridiag_rankk / skew_rank2k match dense numpy products."""
    rng = np.random.default_rng(3)
    for m, b in ((9, 4), (17, 7), (30, 8)):
        A = rng.standard_normal((m, b))
        t = rng.standard_normal(b - 1)
        T = tridiag_from_t(t, b)
        S = np.zeros((b, b))
        for j in range(1, b, 2):
            S[j - 1, j] = -t[j - 1]
            if j + 1 < b:
                S[j + 1, j] = t[j]
        assert np.allclose(S - S.T, T, atol=0)
        W = A @ S
        assert np.all(W[:, 0::2] == 0)
        assert np.allclose(W @ A.T - A @ W.T, A @ T @ A.T, atol=1e-12)
        C = rng.standard_normal((m, m))
        ref = 0.5 * C + (-1.0) * (A @ T @ A.T)
        got = orc.skew_tridiag_rankk(-1.0, A, t, 0.5, C)
        il = np.tril_indices(m, -1)
        assert np.allclose(got[il], ref[il], atol=1e-12)
        assert np.array_equal(np.triu(got), np.triu(C))       # untouched
        Y = rng.standard_normal((m, b))
        ref2 = 2.0 * C + 0.75 * (A @ Y.T - Y @ A.T)
        got2 = orc.skew_rank2k(0.75, A, Y, 2.0, C)
        assert np.allclose(got2[il], ref2[il], atol=1e-12)
        assert np.array_equal(np.triu(got2), np.triu(C))


# ---------------------------------------------------------------- special cases
def test_trivial_sizes(orc):
    L, t, piv, info = orc.ltlt(np.zeros((0, 0)))
    assert L.shape == (0, 0) and t.size == 0 and piv.size == 0 and info == 0
    assert orc.pfaffian_from_factors(0, t, piv) == (0.0, 1)        # Pf(empty) = 1
    L, t, piv, info = orc.ltlt(np.zeros((1, 1)))
    assert np.array_equal(L, [[1.0]]) and t.size == 0 and list(piv) == [0]
    la, sg = orc.pfaffian_from_factors(1, t, piv)
    assert sg == 0 and la == -math.inf


@pytest.mark.parametrize("n", [3, 7, 21])
def test_odd_order_has_zero_pfaffian(orc, n):
    A = inputs.skew_gaussian(n, n)
    L, t, piv, info = orc.ltlt(A)
    la, sg = orc.pfaffian_from_factors(n, t, piv)
    assert sg == 0 and la == -math.inf
    assert backward_error(A, L, t, piv) <= 10
    assert abs(np.linalg.det(A)) < 1e-9 * np.linalg.norm(A) ** n


def test_zero_matrix(orc):
    L, t, piv, info = orc.ltlt(np.zeros((6, 6)))
    assert info == 1 and np.all(t == 0) and np.array_equal(piv, np.arange(6))
    assert np.array_equal(L, np.eye(6))
    assert orc.pfaffian_from_factors(6, t, piv)[1] == 0


def test_nonfinite_rejected(orc):
    A = inputs.skew_gaussian(6, 1)
    A[4, 2] = np.nan
    assert orc.ltlt(A)[3] == -100
    A[4, 2] = np.inf
    assert orc.ltlt(A)[3] == -100
    A[4, 2] = 1.0
    A[2, 4] = np.nan                     # upper triangle is never read
    assert orc.ltlt(A)[3] == 0


def test_ties_take_lowest_index(orc):
    """Equal magnitudes in the pivot column: the first (lowest) index is chosen."""
    n = 6
    M = np.zeros((n, n))
    M[1:, 0] = [1.0, -2.0, 2.0, -2.0, 0.5]      # max |.| = 2 first at row 2
    M[2:, 1] = 0.25
    A = np.asfortranarray(np.tril(M, -1) - np.tril(M, -1).T)
    L, t, piv, info = orc.ltlt(A)
    assert piv[1] == 2
    assert t[0] == -2.0
    check_structure(L, t, piv, n)
    assert backward_error(A, L, t, piv) <= 10


def test_perm_helper_matches_permutation_matrix():
    piv = [0, 3, 2, 4, 4]
    perm = perm_from_piv(piv)
    P = np.eye(5)
    for i, r in enumerate(piv):
        P[[i, r]] = P[[r, i]]
    A = np.arange(25.0).reshape(5, 5)
    assert np.array_equal((P @ A @ P.T), A[np.ix_(perm, perm)])


def test_generator_is_skew_and_seeded():
    A = inputs.skew_gaussian(9, 4)
    assert A.flags.f_contiguous
    assert np.array_equal(A, -A.T)
    assert np.array_equal(A, inputs.skew_gaussian(9, 4))
    assert not np.array_equal(A, inputs.skew_gaussian(9, 5))
    Q = inputs.haar_orthogonal(12, 1)
    assert np.allclose(Q.T @ Q, np.eye(12), atol=1e-13)
    assert np.linalg.det(Q) > 0
    sz = inputs.batched_sizes(1000)
    assert sz.min() >= 16 and sz.max() <= 256 and np.all(sz % 2 == 0)
    assert full_skew_from_lower(A).tolist() == A.tolist()


def test_device_qdq_generator_closed_form_on_cpu(orc):
    """The device QDQ^T generator (used at n = 16384), run on the CPU: exactly skew,
    Pf = det(Q) prod s with det(Q) read off the Householder reflectors; with Q forced
    into SO(n) (the default) the sign is +1 for every seed, including the seeds whose
    QR factor had det(Q) = -1."""
    torch = pytest.importorskip("torch")
    raw_dets = []
    for n, seed in ((12, 3), (40, 5), (64, 9), (12, 1), (12, 2), (12, 4), (12, 6)):
        A, s, detQ = inputs.qdq_skew_device(n, seed, smax=1e3, device="cpu", special=False)
        A = A.numpy()
        assert np.array_equal(A, -A.T)
        la, sg = orc.pfaffian(np.asfortranarray(A))
        assert sg == detQ
        assert math.isclose(la, float(np.sum(np.log(s))), rel_tol=1e-10)
        raw_dets.append(detQ)
        A, s, detQ = inputs.qdq_skew_device(n, seed, smax=1e3, device="cpu")
        la, sg = orc.pfaffian(np.asfortranarray(A.numpy()))
        assert detQ == 1 and sg == 1
        assert math.isclose(la, float(np.sum(np.log(s))), rel_tol=1e-10)
    assert -1 in raw_dets and 1 in raw_dets

def test_oracle_in_pieces_and_batched_equal_single_calls(orc):
    """The oracle run in consecutive pieces of elimination steps (how the CPU baseline
    times a long factorization) and the one-matrix-per-thread batch driver give
    results bitwise equal to one whole call per matrix."""
    A = inputs.skew_gaussian(300, 5)
    L, t, piv, info = orc.ltlt(A)
    st = orc.ltlt_begin(A)
    for kend in (7, 50, 51, 200, 400):
        orc.ltlt_continue(st, kend)
    assert np.array_equal(st["L"], L) and np.array_equal(st["t"], t)
    assert np.array_equal(st["piv"], piv) and st["info"] == info
    D = inputs.block_diag_skew([2.0, 3.0, 5.0])              # zero pivots at odd steps
    st = orc.ltlt_begin(D)
    orc.ltlt_continue(st, 2)
    orc.ltlt_continue(st, 5)
    assert st["info"] == orc.ltlt(D)[3] == 2
    As = [inputs.skew_gaussian(n, 10 + n) for n in (0, 1, 2, 5, 16, 40, 33, 64)] + [D]
    la, sg, inf, ts, pivs, _ = orc.ltlt_many(As)
    for A, l1, s1, i1, t1, p1 in zip(As, la, sg, inf, ts, pivs):
        n = A.shape[0]
        L0, t0, p0, i0 = orc.ltlt(A)
        l0, s0 = orc.pfaffian_from_factors(n, t0, p0)
        assert i1 == i0 and s1 == s0
        assert np.array_equal(t1, t0) and np.array_equal(p1, p0)
        assert l1 == l0 or (math.isinf(l1) and math.isinf(l0))


@pytest.mark.parametrize("n,nb", [(5, 2), (17, 4), (40, 8), (100, 16), (131, 32), (64, 64),
                                  (200, 10), (97, 3)])
def test_lookahead_data_flow_reaches_the_oracle(orc, n, nb):
    """The look-ahead factorization's data flow (panel of block j+1 formed from the
    state before block j's update, left-looking over both blocks, its exchanges kept
    as a map and applied by the next out-of-place update), restated in numpy, reaches
    the oracle's factorization: identical pivots, factors equal up to rounding."""
    from skewcheck import ltlt_lookahead
    A = inputs.skew_gaussian(n, 300 + n)
    L0, t0, p0, _ = orc.ltlt(A)
    L, t, p = ltlt_lookahead(A, nb)
    assert np.array_equal(p, p0)
    assert np.max(np.abs(L - L0)) <= 1e-12
    assert np.max(np.abs(t - t0)) <= 1e-12 * np.max(np.abs(t0))
    D = inputs.block_diag_skew([2.0, 3.0, 5.0, 7.0])       # zero pivots at odd steps
    L1, t1, p1 = ltlt_lookahead(D, 2)
    L2, t2, p2, _ = orc.ltlt(D)
    assert np.array_equal(p1, p2) and np.array_equal(t1, t2)
