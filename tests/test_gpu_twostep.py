"""Two-step (Pfaffian-only) elimination on the GPU against the two-step oracle.

Pivots are exact integers and must equal the oracle's; the pivot-block entries a_j
agree to the rounding of two backward-stable eliminations that sum in different
orders (left-looking panel and blocked update on the GPU, right-looking in the
oracle); log|Pf| within 1e-10 relative and the same sign.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle  # noqa: E402
import paper_2411_09859_gb300 as skew  # noqa: E402
from paper_2411_09859_gb300 import inputs  # noqa: E402
from skewcheck import EPS  # noqa: E402

pytestmark = pytest.mark.gpu


def dev(A):
    return torch.from_numpy(np.asfortranarray(A, dtype=np.float64)).cuda()


def run(A, nb=0, precision=skew.PRECISION_FP64):
    la, sg, a, piv, info = skew.pfaffian_twostep(dev(A), nb=nb, precision=precision)
    torch.cuda.synchronize()
    return (float(la.item()), int(sg.item()), a.cpu().numpy(), piv.cpu().numpy(),
            int(info.item()))


def check_against_oracle(A, la, sg, a, piv, info, rel_a=None):
    n = A.shape[0]
    la0, sg0, a0, p0, i0 = oracle.pfaffian_twostep(A)
    assert np.array_equal(piv, p0), np.nonzero(piv != p0)[0][:5]
    assert info == i0 and sg == sg0
    if n >= 2:
        tol = (2000 * n * EPS if rel_a is None else rel_a) * max(np.max(np.abs(a0)), 1e-300)
        assert np.max(np.abs(a - a0)) <= tol
    if sg0 != 0:
        assert abs(la - la0) <= 1e-10 * max(1.0, abs(la0))


@pytest.mark.parametrize("n,nb", [(2, 2), (3, 2), (4, 2), (17, 4), (64, 16), (257, 32),
                                  (500, 64), (1000, 64), (1001, 64), (1024, 96), (2050, 0),
                                  (3001, 32)])
def test_twostep_matches_oracle(n, nb):
    A = inputs.skew_gaussian(n, 4000 + n)
    la, sg, a, piv, info = run(A, nb)
    check_against_oracle(A, la, sg, a, piv, info)


@pytest.mark.parametrize("seed", range(6))
def test_twostep_many_seeds(seed):
    """Several matrices per size: every pair step exchanges entries that other CTAs
    read in the same step, so a wrong ordering shows up as a pivot difference."""
    for n in (1001, 1503):
        A = inputs.skew_gaussian(n, 9000 + 17 * seed + n)
        la, sg, a, piv, info = run(A, 64)
        check_against_oracle(A, la, sg, a, piv, info)


@pytest.mark.parametrize("n", [300, 1000])
def test_twostep_agrees_with_full_factorization(n):
    A = inputs.skew_gaussian(n, 70 + n)
    la, sg, *_ = run(A)
    la1, sg1, *_ = skew.pfaffian(dev(A))
    assert sg == int(sg1.item())
    assert abs(la - float(la1.item())) <= 1e-10 * max(1.0, abs(la))


def test_twostep_closed_forms():
    s = np.array([1.0, -3.0, 5.0, 0.5, 2.0, -7.0])
    D = inputs.block_diag_skew(s)
    la, sg, a, piv, info = run(D, nb=4)
    assert np.array_equal(piv, np.arange(12)) and info == 0
    assert np.array_equal(a, -s)
    assert sg == (1 if np.prod(s) > 0 else -1)
    assert math.isclose(la, float(np.sum(np.log(np.abs(s)))), rel_tol=1e-15)
    rng = np.random.default_rng(11)
    P = inputs.permutation_matrix(rng.permutation(12))
    A = np.asfortranarray(P @ D @ P.T)
    ref = round(np.linalg.det(P)) * float(np.prod(s))
    la, sg, a, piv, info = run(A, nb=4)
    check_against_oracle(A, la, sg, a, piv, info)
    assert sg == (1 if ref > 0 else -1)
    assert math.isclose(la, math.log(abs(ref)), rel_tol=1e-13)
    A, sv = inputs.qdq_skew(256, inputs.SEED_PRECISION, smax=1e6)
    la, sg, *_ = run(A, nb=32)
    assert sg == 1
    assert abs(la - float(np.sum(np.log(sv)))) <= 1e-9 * abs(la)


def test_twostep_zero_pivot_and_odd_and_nonfinite():
    Z = np.zeros((10, 10))
    Z[5, 4], Z[4, 5] = 2.0, -2.0
    la, sg, a, piv, info = run(Z, nb=4)
    assert sg == 0 and la == -math.inf and info == 1
    la, sg, a, piv, info = run(inputs.skew_gaussian(9, 1), nb=4)
    assert sg == 0 and la == -math.inf
    B = inputs.skew_gaussian(40, 2)
    B[30, 7] = np.inf
    assert run(B, nb=8)[4] == -100          # SKEW_ERR_NONFINITE


def test_twostep_split_precision():
    n = 1000
    A = inputs.skew_gaussian(n, 91)
    la, sg, a, piv, info = run(A, nb=64, precision=skew.PRECISION_SPLIT_BF16)
    check_against_oracle(A, la, sg, a, piv, info)


def test_twostep_argument_checks():
    A = dev(inputs.skew_gaussian(16, 3))
    for nb in (3, 98, -2):
        with pytest.raises(skew.SkewError):
            skew.pfaffian_twostep(A, nb=nb)
    with pytest.raises(skew.SkewError):
        skew.pfaffian_twostep(A, nb=96, precision=skew.PRECISION_SPLIT_BF16)


def test_twostep_trivial_sizes():
    la, sg, *_ = skew.pfaffian_twostep(torch.zeros((0, 0), dtype=torch.float64, device="cuda"))
    assert int(sg.item()) == 1 and float(la.item()) == 0.0
    la, sg, *_ = skew.pfaffian_twostep(torch.zeros((1, 1), dtype=torch.float64, device="cuda"))
    assert int(sg.item()) == 0


def test_twostep_from_two_host_threads():
    """Two host threads call skew_pfaffian_twostep at once, each on its own stream and
    matrix, with the widest panel (its launch needs the raised shared-memory limit);
    both results equal the oracle's."""
    import threading
    mats = [inputs.skew_gaussian(900 + 2 * i, 5100 + i) for i in range(2)]
    out = [None, None]
    err = []

    def work(i):
        try:
            s = torch.cuda.Stream()
            res = []
            for _ in range(3):
                # the input stays referenced until the stream is done with it: torch's
                # caching allocator would otherwise hand its memory to the other thread
                Ad = dev(mats[i])
                la, sg, a, piv, info = skew.pfaffian_twostep(Ad, nb=96, stream=s)
                s.synchronize()
                del Ad
                res.append((float(la.item()), int(sg.item()), a.cpu().numpy(),
                            piv.cpu().numpy(), int(info.item())))
            out[i] = res
        except Exception as e:                      # reported on the main thread
            err.append(e)

    th = [threading.Thread(target=work, args=(i,)) for i in range(2)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert not err, err
    for i in range(2):
        for la, sg, a, piv, info in out[i]:
            check_against_oracle(mats[i], la, sg, a, piv, info)
