"""Pins of the two-step (Pfaffian-only) oracle, oracle_pfaffian_twostep.

The two-step elimination keeps only the even-step Gauss transforms (Wimmer's
algorithm, notes to the two-step right-looking algorithm of Section 4.1).  Its
Pfaffian is pinned to the permutation-sum definition, Pf^2 = det, closed forms and
the full LTL^T read-off; its pivot order to an independent blocked left-looking
restatement (the order the GPU path takes).
"""
import math

import numpy as np
import pytest

from paper_2411_09859_gb300 import inputs
from skewcheck import pfaffian_by_definition, twostep_blocked


def signed(la, sg):
    return sg * math.exp(la) if sg != 0 else 0.0


@pytest.mark.parametrize("n", [2, 4, 6, 8])
@pytest.mark.parametrize("seed", range(3))
def test_twostep_matches_definition(orc, n, seed):
    A = inputs.skew_gaussian(n, 300 + 10 * n + seed)
    ref = pfaffian_by_definition(A)
    la, sg, a, piv, info = orc.pfaffian_twostep(A)
    assert info == 0
    assert sg == (1 if ref > 0 else -1)
    assert math.isclose(signed(la, sg), ref, rel_tol=1e-12)


@pytest.mark.parametrize("n", [3, 5, 7, 11])
def test_twostep_odd_order_is_zero(orc, n):
    la, sg, *_ = orc.pfaffian_twostep(inputs.skew_gaussian(n, n))
    assert sg == 0 and la == -math.inf


@pytest.mark.parametrize("n", [10, 24, 64])
def test_twostep_squared_is_det(orc, n):
    A = inputs.skew_gaussian(n, 40 + n)
    la, sg, *_ = orc.pfaffian_twostep(A)
    sgn, logdet = np.linalg.slogdet(A)
    assert sgn > 0
    assert math.isclose(2 * la, logdet, rel_tol=1e-11, abs_tol=1e-10)


def test_twostep_block_diagonal_and_permuted(orc):
    s = [1.0, -3.0, 5.0, 0.5]
    D = inputs.block_diag_skew(s)
    la, sg, a, piv, info = orc.pfaffian_twostep(D)
    assert np.array_equal(piv, np.arange(8)) and info == 0
    assert np.array_equal(a, -np.asarray(s))        # a[j] = D[2j+1, 2j] = -s_j
    assert math.isclose(signed(la, sg), float(np.prod(s)), rel_tol=1e-15)
    rng = np.random.default_rng(3)
    perm = rng.permutation(8)
    P = inputs.permutation_matrix(perm)
    A = np.asfortranarray(P @ D @ P.T)
    ref = round(np.linalg.det(P)) * float(np.prod(s))
    la, sg, *_ = orc.pfaffian_twostep(A)
    assert math.isclose(signed(la, sg), ref, rel_tol=1e-13)


@pytest.mark.parametrize("n", [8, 40])
def test_twostep_qdq_closed_form(orc, n):
    A, s = inputs.qdq_skew(n, 5, smax=1e3)
    la, sg, *_ = orc.pfaffian_twostep(A)
    assert sg == 1
    assert math.isclose(la, float(np.sum(np.log(s))), rel_tol=1e-9, abs_tol=1e-9)


@pytest.mark.parametrize("n", [50, 200, 301])
def test_twostep_agrees_with_full_ltlt(orc, n):
    """Two different eliminations (different pivots after the first) of the same
    Pfaffian: they agree to rounding."""
    A = inputs.skew_gaussian(n, 500 + n)
    la, sg, *_ = orc.pfaffian_twostep(A)
    la2, sg2 = orc.pfaffian(A)
    assert sg == sg2
    if sg != 0:
        assert abs(la - la2) <= 1e-11 * max(1.0, abs(la2))


@pytest.mark.parametrize("n,nb", [(7, 2), (8, 4), (50, 2), (50, 8), (61, 16), (64, 32),
                                  (200, 64), (301, 32)])
def test_twostep_blocked_left_looking_same_pivots(orc, n, nb):
    A = inputs.skew_gaussian(n, 31 + n)
    la, sg, a0, p0, info = orc.pfaffian_twostep(A)
    a1, p1 = twostep_blocked(A, nb)
    assert np.array_equal(p0, p1)
    assert np.max(np.abs(a0 - a1)) <= 1e-12 * np.max(np.abs(a0))


def test_twostep_pivots_only_at_even_steps(orc):
    n = 40
    la, sg, a, piv, info = orc.pfaffian_twostep(inputs.skew_gaussian(n, 9))
    assert piv[0] == 0
    for i in range(2, n, 2):
        assert piv[i] == i                     # odd steps are never pivoted
    for k in range(0, n - 1, 2):
        assert piv[k + 1] >= k + 1


def test_twostep_zero_column_and_nonfinite(orc):
    D = np.zeros((6, 6))
    la, sg, a, piv, info = orc.pfaffian_twostep(D)
    assert sg == 0 and info == 1
    B = inputs.skew_gaussian(6, 1)
    B[4, 1] = np.nan
    assert orc.pfaffian_twostep(np.asfortranarray(B))[4] == -100


def test_twostep_trivial_sizes(orc):
    la, sg, a, piv, info = orc.pfaffian_twostep(np.zeros((0, 0)))
    assert sg == 1 and la == 0.0 and info == 0
    la, sg, *_ = orc.pfaffian_twostep(np.zeros((1, 1)))
    assert sg == 0
