"""Planted mistakes in the CPU oracle must be caught by its pins.

Each case copies the oracle's C source, plants one plausible mistake (a dropped
term, a wrong sign, a wrong index, a transposed operand), compiles the copy into a
temporary library and runs a quick battery of the same pins as test_oracle_pins.
The mistake lives only in the temporary copy; nothing here touches a GPU.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2411_09859_gb300 import inputs
from skewcheck import (backward_error, check_structure, pf4_closed_form,
                       pfaffian_by_definition, tridiag_from_t)

MUTANTS = {
    "signed_argmax": ("double a = fabs(X_(i, k));", "double a = X_(i, k);"),
    "argmax_ties_last": ("if (a > best) { best = a; r = i; }",
                         "if (a >= best) { best = a; r = i; }"),
    "swap_no_sign_flip": ("X_(i, p) = -X_(q, i);", "X_(i, p) = X_(q, i);"),
    "swap_corner_no_flip": ("X_(q, p) = -X_(q, p);", "X_(q, p) = X_(q, p);"),
    "swap_tail_dropped": ("tmp = X_(i, p); X_(i, p) = X_(i, q); X_(i, q) = tmp;",
                          "tmp = X_(i, p);"),
    "no_L_row_swap": ("tmp = L_(p, c); L_(p, c) = L_(q, c); L_(q, c) = tmp;",
                      "tmp = L_(p, c);"),
    "update_sign": ("(L_(i, c1) * xj - X_(i, c1) * lj)",
                    "(X_(i, c1) * lj - L_(i, c1) * xj)"),
    "update_term_dropped": ("(L_(i, c1) * xj - X_(i, c1) * lj)", "(L_(i, c1) * xj)"),
    "update_wrong_column": ("const int64_t c1 = k + 1;", "const int64_t c1 = k + 2 < n ? k + 2 : k + 1;"),
    "gauss_multiply": ("X_(i, k) / tau", "X_(i, k) * tau"),
    "pf_no_detP": ("if (piv[i] != i) sg = -sg;", "if (piv[i] < 0) sg = -sg;"),
    "pf_sign_T": ("double v = -t[2 * i];", "double v = t[2 * i];"),
    "pf_odd_entries": ("double v = -t[2 * i];", "double v = -t[i];"),
    "r2k_transposed": ("A[i + p * lda] * B[j + p * ldb] - B[i + p * ldb] * A[j + p * lda]",
                       "A[i + p * lda] * B[j + p * ldb] - A[i + p * lda] * B[j + p * ldb]"),
    "rankk_index": ("s -= A[i + a * lda] * t[a] * A[j + (a + 1) * lda];",
                    "s -= A[j + a * lda] * t[a] * A[i + (a + 1) * lda];"),
    "rankk_sign": ("s -= A[i + a * lda] * t[a] * A[j + (a + 1) * lda];",
                   "s += A[i + a * lda] * t[a] * A[j + (a + 1) * lda];"),
    "twostep_update_sign": ("(X_(i, k) * yj - X_(i, k + 1) * lj)",
                            "(X_(i, k + 1) * lj - X_(i, k) * yj)"),
    "twostep_update_term_dropped": ("(X_(i, k) * yj - X_(i, k + 1) * lj)", "(X_(i, k) * yj)"),
    "twostep_multiply": ("(ak != 0.0) ? X_(i, k) / ak : 0.0", "(ak != 0.0) ? X_(i, k) * ak : 0.0"),
    "twostep_swap_no_flip": ("X_(i, u) = -X_(w, i);", "X_(i, u) = X_(w, i);"),
    "twostep_pf_sign": ("const double v = -a[j];", "const double v = a[j];"),
    "twostep_no_detP": ("if (piv[i] != (int32_t)i) sg = -sg;", "if (piv[i] < 0) sg = -sg;"),
}


def battery(orc) -> list:
    """Run the quick pins; return the names of those that fail."""
    failed = []

    def check(name, fn):
        try:
            ok = fn()
        except Exception:
            ok = False
        if not ok:
            failed.append(name)

    def pf_def():
        for n in (2, 4, 6):
            for seed in range(3):
                A = inputs.skew_gaussian(n, 10 * n + seed)
                ref = pfaffian_by_definition(A)
                la, sg = orc.pfaffian(A)
                if sg != (1 if ref > 0 else -1):
                    return False
                if not math.isclose(la, math.log(abs(ref)), rel_tol=1e-11, abs_tol=1e-11):
                    return False
        A = inputs.skew_gaussian(4, 77)
        la, sg = orc.pfaffian(A)
        return math.isclose(sg * math.exp(la), pf4_closed_form(A), rel_tol=1e-12)

    def factors():
        for n in (5, 17, 50):
            A = inputs.skew_gaussian(n, 900 + n)
            L, t, piv, info = orc.ltlt(A)
            check_structure(L, t, piv, n)
            if backward_error(A, L, t, piv) > 10:
                return False
        return True

    def ties():
        n = 6
        M = np.zeros((n, n))
        M[1:, 0] = [1.0, -2.0, 2.0, -2.0, 0.5]
        M[2:, 1] = 0.25
        A = np.asfortranarray(np.tril(M, -1) - np.tril(M, -1).T)
        return orc.ltlt(A)[2][1] == 2

    def dense_ops():
        rng = np.random.default_rng(5)
        m, b = 11, 6
        A = rng.standard_normal((m, b))
        Y = rng.standard_normal((m, b))
        t = rng.standard_normal(b - 1)
        C = rng.standard_normal((m, m))
        il = np.tril_indices(m, -1)
        r1 = orc.skew_tridiag_rankk(-1.0, A, t, 1.0, C)
        ok1 = np.allclose(r1[il], (C - A @ tridiag_from_t(t, b) @ A.T)[il], atol=1e-12)
        r2 = orc.skew_rank2k(1.0, A, Y, 1.0, C)
        ok2 = np.allclose(r2[il], (C + A @ Y.T - Y @ A.T)[il], atol=1e-12)
        return ok1 and ok2

    def twostep():
        for n in (4, 6, 8):
            for seed in range(2):
                A = inputs.skew_gaussian(n, 700 + 10 * n + seed)
                ref = pfaffian_by_definition(A)
                la, sg, *_ = orc.pfaffian_twostep(A)
                if sg != (1 if ref > 0 else -1):
                    return False
                if not math.isclose(la, math.log(abs(ref)), rel_tol=1e-11, abs_tol=1e-11):
                    return False
        A = inputs.skew_gaussian(30, 5)
        la, sg, *_ = orc.pfaffian_twostep(A)
        return math.isclose(2 * la, np.linalg.slogdet(A)[1], rel_tol=1e-10)

    check("pfaffian_definition", pf_def)
    check("twostep", twostep)
    check("factors", factors)
    check("ties", ties)
    check("dense_ops", dense_ops)
    return failed


def test_unmutated_oracle_passes_battery(orc):
    assert battery(orc) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(oracle.SOURCE).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    mpath = os.path.join(tmp_path, "mutant.c")
    with open(mpath, "w") as f:
        f.write(src.replace(old, new))
    lib = oracle.compile_source(mpath, os.path.join(tmp_path, f"libmut_{name}.so"))
    failed = battery(oracle.OracleLib(lib))
    assert failed, f"planted mistake {name} was not caught by any pin"
