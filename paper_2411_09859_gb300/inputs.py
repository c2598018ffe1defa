"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only draws random numbers and lays them out; it holds none of the
factorization's arithmetic.  Matrices are returned as float64 numpy arrays in
Fortran (column-major) order holding BOTH triangles of the skew matrix, so a
caller can hand the same memory to the column-major GPU library and to a CPU
implementation, and can also form dense products for checks.

Recipe for the iid Gaussian skew matrices (the paper's experiments use
"skew-symmetric matrices" of a stated order without a value distribution):
numpy ``default_rng(seed)`` (PCG64); for column j = 0 .. n-1 in turn, one call
``standard_normal(n - j - 1)`` fills rows j+1 .. n-1 of the strictly lower
triangle; the upper triangle is the negated transpose and the diagonal is zero.
"""
from __future__ import annotations

import numpy as np

# seeds of the workload configurations
SEED_SMALL = 0                       # n = 512 plain-method case
SEED_SCALE = {4096: 1, 8192: 2, 16384: 3}
SEED_BATCH_SIZES = 4                 # sizes of the batched workload
SEED_BATCH_BASE = 1000               # matrix i of the batched workload uses 1000 + i
SEED_PRECISION = 5
SEED_SERVING = 6


def skew_gaussian(n: int, seed: int) -> np.ndarray:
    """n x n skew matrix, strictly lower entries iid N(0, 1) (recipe above)."""
    rng = np.random.default_rng(seed)
    # At is A^T stored row-major, i.e. the memory of A stored column-major
    At = np.zeros((n, n), dtype=np.float64)
    for j in range(n - 1):
        At[j, j + 1:] = rng.standard_normal(n - j - 1)    # A[j+1:, j]
    # the lower part of At is still zero, so At - At^T keeps the upper part and
    # writes At[i, j] = -At[j, i] below the diagonal
    At = At - At.T
    return At.T                                             # Fortran-ordered view


def block_diag_skew(s) -> np.ndarray:
    """blockdiag([[0, s_k], [-s_k, 0]]): the 2x2 skew blocks with upper entry s_k."""
    s = np.asarray(s, dtype=np.float64)
    n = 2 * len(s)
    D = np.zeros((n, n), dtype=np.float64, order="F")
    for k, sk in enumerate(s):
        D[2 * k, 2 * k + 1] = sk
        D[2 * k + 1, 2 * k] = -sk
    return D


def permutation_matrix(perm) -> np.ndarray:
    """P with (P x)[i] = x[perm[i]]."""
    perm = np.asarray(perm)
    n = len(perm)
    P = np.zeros((n, n), dtype=np.float64, order="F")
    P[np.arange(n), perm] = 1.0
    return P


def haar_orthogonal(n: int, seed: int) -> np.ndarray:
    """Haar-distributed Q in SO(n): QR of a Gaussian matrix with the columns scaled
    by sign(diag R) (Mezzadri 2007), then column 0 negated if det Q < 0."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    Q = Q * np.sign(np.diag(R))[None, :]
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return np.asfortranarray(Q)


def log_spaced_s(n: int, smax: float = 1e6) -> np.ndarray:
    """s_k = smax^(k / (n/2 - 1)) for k = 0 .. n/2 - 1 (log-spaced in [1, smax])."""
    h = n // 2
    if h == 1:
        return np.ones(1)
    return smax ** (np.arange(h) / (h - 1))


def qdq_skew(n: int, seed: int, smax: float = 1e6):
    """A = Q D Q^T with Q Haar in SO(n) and D = block_diag_skew(log_spaced_s(n)),
    made exactly skew as (M - M^T)/2.  Returns (A, s)."""
    Q = haar_orthogonal(n, seed)
    s = log_spaced_s(n, smax)
    M = Q @ block_diag_skew(s) @ Q.T
    return np.asfortranarray((M - M.T) / 2.0), s


def qdq_skew_device(n: int, seed: int, smax: float = 1e6, device="cuda",
                    special: bool = True):
    """A = Q D Q^T generated on the device, for orders whose host generation would take
    minutes (n = 16384).  G: n x n standard normal from a torch generator seeded with
    `seed` (not the numpy stream of `qdq_skew`); Q: the Householder QR of G with the
    sign(diag R) correction (Haar in O(n)); with `special` (the default) column 0 of Q
    is negated when det(Q) = -1, so that Q is Haar in SO(n).  det(Q) before that is
    (-1)^(number of nonzero reflectors) * prod sign(R_ii).
    D = block_diag_skew(log_spaced_s(n, smax)); A = U V^T - V U^T with
    U = Q[:, 0::2] * s and V = Q[:, 1::2] (= Q D Q^T, exactly skew).

    Returns (A, s, detQ): A a column-major float64 CUDA tensor, s (numpy), detQ the
    determinant of the Q used (+1 with `special`); Pf(A) = detQ * prod(s)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    G = torch.randn((n, n), generator=gen, dtype=torch.float64, device=device)
    H, tau = torch.geqrf(G)
    del G
    dR = torch.diagonal(H).clone()
    Q = torch.linalg.householder_product(H, tau)
    sgn = torch.where(dR < 0, -1.0, 1.0).to(torch.float64)
    Q *= sgn.unsqueeze(0)
    nneg = int((dR < 0).sum().item())
    nref = int((tau != 0).sum().item())
    detQ = -1 if (nneg + nref) % 2 else 1
    if special and detQ < 0:
        Q[:, 0] = -Q[:, 0]
        detQ = 1
    del H, tau
    s = log_spaced_s(n, smax)
    st = torch.from_numpy(s).to(device)
    U = Q[:, 0::2] * st.unsqueeze(0)
    V = Q[:, 1::2].contiguous()
    del Q
    M = U @ V.t()
    del U, V
    A = torch.empty((n, n), dtype=torch.float64, device=device).t()   # column-major
    A.copy_(M - M.t())
    del M
    return A, s, detQ


def batched_sizes(count: int = 4096, seed: int = SEED_BATCH_SIZES, lo: int = 16,
                  hi: int = 256) -> np.ndarray:
    """count even orders drawn uniformly from {lo, lo+2, ..., hi}."""
    rng = np.random.default_rng(seed)
    return lo + 2 * rng.integers(0, (hi - lo) // 2 + 1, size=count)
