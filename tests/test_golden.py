"""Hand-worked examples (tests/golden/worked_examples.json) against the oracle.

Every expected value in the fixture was derived by hand from the paper's
definitions and is exact in binary floating point, so the comparison is exact.
"""
import json
import math
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "worked_examples.json")) as f:
    CASES = json.load(f)["cases"]


def matrix_of(case):
    n = case["n"]
    A = np.zeros((n, n), order="F")
    for i, j, v in case["lower"]:
        A[i, j] = v
        A[j, i] = -v
    return A


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_worked_example(orc, case):
    A = matrix_of(case)
    L, t, piv, info = orc.ltlt(A)
    assert np.array_equal(t, np.array(case["t"]))
    assert np.array_equal(piv, np.array(case["piv"]))
    assert np.array_equal(L, np.array(case["L"], dtype=float))
    assert info == case["info"]
    la, sg = orc.pfaffian_from_factors(case["n"], t, piv)
    pf = case["pfaffian"]
    assert sg == (1 if pf > 0 else -1)
    assert math.isclose(la, math.log(abs(pf)), rel_tol=1e-15)
