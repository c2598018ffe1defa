"""Split-precision trailing update (bf16 digit slices on tcgen05 tensor cores,
Ozaki-type error-free splitting) against the oracle.

The update's error bound follows from the splitting: every operand entry is held as
a 55-bit integer relative to its row's largest entry (truncation below 2^(E_i-54),
i.e. at most 2^-54 R_i) and the digit products that are dropped (s + t >= 10) are
below 2^-60 R_i R_j per column, so with k pairs (K = 2k columns)
|dC[i,j]| <= (2.02 k + 0.5) 2^-53 R_i R_j (R_i the largest |entry| of row i of
[X, Y]) plus the rounding of the final FP64 add.  The factorization in this mode must
still give the oracle's pivots, a backward error <= 10 and log|Pf| within 1e-10.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle  # noqa: E402
import paper_2411_09859_gb300 as skew  # noqa: E402
from paper_2411_09859_gb300 import inputs  # noqa: E402
from skewcheck import EPS, backward_error, check_structure  # noqa: E402

pytestmark = pytest.mark.gpu
SPLIT = skew.PRECISION_SPLIT_BF16


def dev(A):
    return torch.from_numpy(np.asfortranarray(A, dtype=np.float64)).cuda()


# (3001, 32) and (2500, 5) give several tiles per persistent CTA: the U block reuse,
# both V buffers and both parities of every accumulator barrier are exercised.
@pytest.mark.parametrize("m,k", [(2, 1), (65, 7), (130, 16), (200, 32), (513, 31), (2500, 5),
                                 (3001, 32)])
@pytest.mark.parametrize("scale", ["unit", "wide"])
def test_split_rank2k_error_bound(m, k, scale):
    rng = np.random.default_rng(m + k)
    X = rng.standard_normal((m, k))
    Y = rng.standard_normal((m, k))
    if scale == "wide":                      # rows and columns of very different size
        X *= np.exp2(rng.integers(-30, 30, size=(m, 1))) * np.exp2(rng.integers(-5, 5, size=(1, k)))
        Y *= np.exp2(rng.integers(-30, 30, size=(m, 1)))
    C = rng.standard_normal((m, m))
    ref = oracle.skew_rank2k(1.0, X, Y, 1.0, C)
    Cd = dev(C)
    skew.rank2k(1.0, dev(X), dev(Y), 1.0, Cd, precision=SPLIT)
    got = Cd.cpu().numpy()
    R = np.maximum(np.max(np.abs(X), axis=1), np.max(np.abs(Y), axis=1))
    tol = (2 * k + 1) * EPS * np.outer(R, R) + 2 * EPS * np.abs(ref)   # EPS = 2^-52
    il = np.tril_indices(m, -1)
    err = np.abs(got - ref)
    assert np.all(err[il] <= tol[il]), float(np.max((err / np.maximum(tol, 1e-300))[il]))
    iu = np.triu_indices(m)
    assert np.array_equal(got[iu], C[iu])


def test_split_rank2k_zero_rows_and_k_limit():
    m, k = 70, 5
    X = np.zeros((m, k))
    Y = np.zeros((m, k))
    X[10] = 1.0
    Y[20] = -2.0
    C = np.ones((m, m))
    ref = oracle.skew_rank2k(1.0, X, Y, 1.0, C)
    Cd = dev(C)
    skew.rank2k(1.0, dev(X), dev(Y), 1.0, Cd, precision=SPLIT)
    il = np.tril_indices(m, -1)
    assert np.array_equal(Cd.cpu().numpy()[il], ref[il])
    with pytest.raises(skew.SkewError):
        skew.rank2k(1.0, dev(np.zeros((8, 33))), dev(np.zeros((8, 33))), 1.0, dev(np.zeros((8, 8))),
                    precision=SPLIT)


@pytest.mark.parametrize("n,nb", [(64, 16), (257, 32), (500, 64), (1000, 64), (1023, 0)])
def test_split_factorization_matches_oracle(n, nb):
    A = inputs.skew_gaussian(n, 8000 + n)
    L0, t0, p0, i0 = oracle.ltlt(A)
    L, t, piv, info = skew.ltlt(dev(A), nb=nb, precision=SPLIT)
    torch.cuda.synchronize()
    L, t, piv, info = L.cpu().numpy(), t.cpu().numpy(), piv.cpu().numpy(), int(info.item())
    assert np.array_equal(piv, p0) and info == i0
    tol = 2000 * n * EPS
    assert np.max(np.abs(L - L0)) <= tol
    assert np.max(np.abs(t - t0)) <= tol * np.max(np.abs(t0))
    check_structure(L, t, piv, n)
    assert backward_error(A, L, t, piv) <= 10
    la0, sg0 = oracle.pfaffian_from_factors(n, t0, p0)
    la, sg = skew.pfaffian_from_factors(torch.from_numpy(t).cuda(), torch.from_numpy(piv).cuda(), n)
    assert int(sg.item()) == sg0
    if sg0:
        assert abs(float(la.item()) - la0) <= 1e-10 * max(1.0, abs(la0))


def test_split_pfaffian_only_and_qdq_closed_form():
    n = 256
    A, s = inputs.qdq_skew(n, inputs.SEED_PRECISION, smax=1e6)
    la, sg, t, piv, info = skew.pfaffian(dev(A), nb=32, precision=SPLIT)
    torch.cuda.synchronize()
    closed = float(np.sum(np.log(s)))
    la_f, sg_f, *_ = skew.pfaffian(dev(A), nb=32)
    torch.cuda.synchronize()
    assert int(sg.item()) == 1 == int(sg_f.item())
    # both paths agree with the closed form to the conditioning of the problem
    assert abs(float(la.item()) - closed) <= 1e-7 * abs(closed)
    assert abs(float(la.item()) - float(la_f.item())) <= 1e-8 * abs(closed)


def test_split_rejects_wide_panels():
    A = dev(inputs.skew_gaussian(100, 1))
    with pytest.raises(skew.SkewError):
        skew.ltlt(A, nb=128, precision=SPLIT)
