"""The split-precision update's arithmetic, modelled exactly on the CPU.

The split-precision trailing update (SKEW_PRECISION_SPLIT_BF16) is documented as: each
row i of the pair columns gets the exponent E_i of its largest entry; each entry x
becomes X = trunc(x 2^(54-E_i)) (|X| < 2^55), cut into seven base-256 digits (d_7 ..
d_2 balanced in [-128, 127], d_1 the rest); with U = [a | -w], V = [w | a], the digit
group sums P_d = sum_{s+t=d} U_s V_t^T (d = 2 .. 9) are exact FP32 tensor-core sums,
recombined as acc = (256 P_2 + P_3) 2^34 + (256 P_4 + P_5) 2^18 + (256 P_6 + P_7) 2^2
+ floor(fl32(256 P_8 + P_9) 2^-14), and the update is acc 2^(E_i + E_j - 54).  The
stated bound: with k column pairs the update differs from the exact one by at most
(2.02 k + 0.5) 2^-53 (row max of U)(row max of V).

This file restates that description in exact integer arithmetic (Python integers and
fractions, independent of the GPU code) and checks, on random and adversarial rows,
that every group sum stays below 2^24 (so the FP32 sums are exact) and that the
error stays within the stated bound -- a check of the scheme as documented, while the
GPU tests check the kernels against the oracle."""
import math
from fractions import Fraction

import numpy as np
import pytest


def row_exponent(row):
    """Exponent E of the row's largest |entry| (|x| < 2^(E+1)); -1022 for a zero row."""
    e = -1022
    for x in row:
        if x != 0.0:
            e = max(e, math.frexp(abs(x))[1] - 1)
    return e


def fixed55(x, E):
    """trunc(x 2^(54-E)) as an exact integer."""
    return int(Fraction(x) * Fraction(2) ** (54 - E))   # int() truncates toward zero


def digits(X):
    """[d_1, .., d_7] with X = sum_s d_s 256^(7-s), d_7 .. d_2 in [-128, 127]."""
    d = [0] * 7
    for s in range(6, 0, -1):
        d[s] = ((X + 128) & 255) - 128
        X = (X - d[s]) >> 8
    d[0] = X
    return d


def model_product(u, v):
    """The scheme's value of sum_k u_k v_k for one row i of U and one row j of V
    (both given as lists of floats), and the group sums it used."""
    Eu, Ev = row_exponent(u), row_exponent(v)
    du = [digits(fixed55(x, Eu)) for x in u]
    dv = [digits(fixed55(x, Ev)) for x in v]
    P = {}
    for d in range(2, 10):
        P[d] = sum(du[k][s - 1] * dv[k][d - s - 1]
                   for k in range(len(u)) for s in range(1, 8) if 1 <= d - s <= 7)
    q89 = float(np.float32(256.0 * P[8] + P[9]))      # one FP32 rounding of the fma
    acc = ((256 * P[2] + P[3]) << 34) + ((256 * P[4] + P[5]) << 18) + \
          ((256 * P[6] + P[7]) << 2) + math.floor(q89 / 2 ** 14)
    return Fraction(acc) * Fraction(2) ** (Eu + Ev - 54), P, du, dv


def check_rows(a_i, w_i, a_j, w_j):
    """U row i = [a_i | -w_i], V row j = [w_j | a_j] (k pairs each): the model's value
    of (U V^T)[i, j] against the exact one and the bound."""
    u = list(a_i) + [-x for x in w_i]
    v = list(w_j) + list(a_j)
    k = len(a_i)
    got, P, du, dv = model_product(u, v)
    exact = sum(Fraction(x) * Fraction(y) for x, y in zip(u, v))
    for dig in du + dv:
        assert all(-128 <= x <= 127 for x in dig[1:]) and abs(dig[0]) <= 128
    assert all(abs(p) < 2 ** 24 for p in P.values())          # exact FP32 sums
    assert all(abs(P[d]) <= 2 ** 22 for d in (2, 3, 4, 5))     # the add-based conversion
    Ru = max(abs(x) for x in u)
    Rv = max(abs(x) for x in v)
    bound = Fraction(2.02 * k + 0.5) * Fraction(2) ** -53 * Fraction(Ru) * Fraction(Rv)
    assert abs(got - exact) <= bound, (float(abs(got - exact) / bound))
    return float(abs(got - exact) / bound) if bound else 0.0


@pytest.mark.parametrize("k", [1, 7, 32])
def test_gaussian_rows(k):
    rng = np.random.default_rng(100 + k)
    worst = 0.0
    for _ in range(40):
        a_i, w_i, a_j, w_j = (rng.standard_normal(k) for _ in range(4))
        worst = max(worst, check_rows(a_i, w_i, a_j, w_j))
    assert worst < 1.0


@pytest.mark.parametrize("k", [4, 32])
def test_rows_spanning_many_binades(k):
    # entries from 2^-60 to 1 in one row: the small ones lose their low bits to the
    # row's fixed point, which is what the bound accounts for
    rng = np.random.default_rng(200 + k)
    for _ in range(30):
        rows = [rng.standard_normal(k) * 2.0 ** rng.integers(-60, 1, k) for _ in range(4)]
        check_rows(*rows)


def test_largest_digits_and_sums():
    # every entry just below the row's power of two: all digit magnitudes near their
    # limits, the group sums at their largest
    k = 32
    top = math.nextafter(2.0, 0.0)
    for sgn in (1.0, -1.0):
        a = [sgn * top] * k
        w = [-sgn * top] * k
        check_rows(a, w, a, w)
        check_rows(a, [top] * k, [top] * k, a)


def test_digit_recomposition_and_range():
    rng = np.random.default_rng(5)
    for _ in range(2000):
        X = int(rng.integers(-(2 ** 55) + 1, 2 ** 55))
        d = digits(X)
        assert sum(d[s] * 256 ** (6 - s) for s in range(7)) == X
        assert abs(d[0]) <= 128 and all(-128 <= x <= 127 for x in d[1:])


def test_add_based_conversion_of_small_group_sums():
    """The epilogue turns the group sums P_2 .. P_5 (integers, |P_d| <= 2^22) into int32
    by one FP32 add of 1.5 2^23 and a subtraction of bit patterns; in IEEE single
    precision with rounding to nearest that is exact on the whole range, ends included."""
    magic = np.float32(12582912.0)
    vals = np.concatenate([np.arange(-2 ** 22, -2 ** 22 + 5000), np.arange(-3000, 3000),
                           np.arange(2 ** 22 - 5000, 2 ** 22 + 1),
                           np.random.default_rng(9).integers(-2 ** 22, 2 ** 22 + 1, 20000)])
    f = vals.astype(np.float32)
    assert np.array_equal(f.astype(np.int64), vals)                 # exact FP32 integers
    got = (f + magic).view(np.int32).astype(np.int64) - 0x4B400000
    assert np.array_equal(got, vals)
    # just outside the range the trick is no longer exact
    assert ((np.float32(2 ** 22 + 1) + magic).view(np.int32) - 0x4B400000) != 2 ** 22 + 1
