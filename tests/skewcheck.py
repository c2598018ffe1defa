"""Checks used by the tests: the Pfaffian by its definition, the factor properties,
and a numpy restatement of the pivoted blocked right-looking algorithm.

Nothing here calls the GPU library.  Section and equation numbers refer to
"Performant Tridiagonal Factorization of Skew-Symmetric Matrices" (arXiv 2411.09859).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

EPS = 2.0 ** -52


# ----------------------------------------------------------------------------------
# the Pfaffian from its definition (Section 1)
# ----------------------------------------------------------------------------------
def _perm_sign(p) -> int:
    p = list(p)
    s = 1
    for i in range(len(p)):
        while p[i] != i:
            j = p[i]
            p[i], p[j] = p[j], p[i]
            s = -s
    return s


def pfaffian_by_definition(X: np.ndarray) -> float:
    """Pf(X) = 1/(2^m m!) sum over all permutations sigma of the 2m indices of
    sgn(sigma) prod_{i=1..m} x[sigma(2i-1), sigma(2i)]  (Section 1), summed literally.
    Feasible for n <= 8 (40320 permutations).  Odd n gives 0; n = 0 gives 1."""
    n = X.shape[0]
    if n % 2:
        return 0.0
    if n == 0:
        return 1.0
    m = n // 2
    total = 0.0
    for sigma in itertools.permutations(range(n)):
        prod = 1.0
        for i in range(m):
            prod *= X[sigma[2 * i], sigma[2 * i + 1]]
        total += _perm_sign(sigma) * prod
    return total / (2 ** m * math.factorial(m))


def pfaffian_by_matchings(X: np.ndarray) -> float:
    """The same sum grouped by perfect matchings (each matching appears 2^m m! times
    with one sign): expansion along the first index, recursively.  n <= 14."""
    n = X.shape[0]
    if n % 2:
        return 0.0

    def rec(idx):
        if not idx:
            return 1.0
        a = idx[0]
        total = 0.0
        for pos in range(1, len(idx)):
            b = idx[pos]
            rest = idx[1:pos] + idx[pos + 1:]
            total += (-1) ** (pos - 1) * X[a, b] * rec(rest)
        return total

    return rec(list(range(n)))


def pf4_closed_form(X: np.ndarray) -> float:
    """Pf of a 4x4 skew matrix: x01 x23 - x02 x13 + x03 x12."""
    return X[0, 1] * X[2, 3] - X[0, 2] * X[1, 3] + X[0, 3] * X[1, 2]


# ----------------------------------------------------------------------------------
# factor properties
# ----------------------------------------------------------------------------------
def perm_from_piv(piv) -> np.ndarray:
    """perm with (P A P^T)[a, b] = A[perm[a], perm[b]] for P = P(p) of Section 5.1
    (the row exchanges i <-> piv[i] applied in order i = 0, 1, ...)."""
    n = len(piv)
    perm = np.arange(n)
    for i in range(n):
        r = int(piv[i])
        perm[i], perm[r] = perm[r], perm[i]
    return perm


def tridiag_from_t(t, n: int) -> np.ndarray:
    """T with T[i+1, i] = t[i] and T[i, i+1] = -t[i] (Eq. (T))."""
    T = np.zeros((n, n))
    for i in range(n - 1):
        T[i + 1, i] = t[i]
        T[i, i + 1] = -t[i]
    return T


def full_skew_from_lower(X: np.ndarray) -> np.ndarray:
    """Full skew matrix from the strictly lower triangle of X."""
    Lw = np.tril(X, -1)
    return Lw - Lw.T


def backward_error(A: np.ndarray, L: np.ndarray, t, piv) -> float:
    """||P A P^T - L T L^T||_F / (n eps ||A||_F) with eps = 2^-52."""
    n = A.shape[0]
    if n <= 1:
        return 0.0
    Af = full_skew_from_lower(A)
    perm = perm_from_piv(piv)
    PAPt = Af[np.ix_(perm, perm)]
    T = tridiag_from_t(t, n)
    R = PAPt - L @ T @ L.T
    nrm = np.linalg.norm(Af)
    if nrm == 0:
        return float(np.linalg.norm(R))
    return float(np.linalg.norm(R) / (n * EPS * nrm))


def check_structure(L: np.ndarray, t, piv, n: int):
    """Invariants of the pivoted factorization: L unit lower triangular, L e_0 = e_0,
    |L_ij| <= 1 (the pivot is the entry of largest magnitude), piv[0] = 0 and
    piv[i] >= i."""
    assert L.shape == (n, n)
    if n == 0:
        return
    assert np.all(np.diag(L) == 1.0)
    assert np.all(np.triu(L, 1) == 0.0)
    e0 = np.zeros(n)
    e0[0] = 1.0
    assert np.array_equal(L[:, 0], e0)
    assert np.all(np.abs(L) <= 1.0)
    assert piv[0] == 0
    assert all(int(piv[i]) >= i and int(piv[i]) < n for i in range(n))
    assert len(t) == n - 1


def pfaffian_from_t_piv(t, piv, n):
    """Independent restatement of the read-off: Pf = det(P) prod_i T[2i, 2i+1]."""
    if n % 2:
        return 0.0
    swaps = sum(1 for i in range(n) if int(piv[i]) != i)
    val = 1.0
    for i in range(n // 2):
        val *= -t[2 * i]
    return (-1) ** swaps * val


# ----------------------------------------------------------------------------------
# the pivoted blocked right-looking algorithm (Section 4.2 Variant 1 with the
# pivoted panel of Section 5.2), restated in numpy on FULL storage
# ----------------------------------------------------------------------------------
def ltlt_blocked(A: np.ndarray, nb: int, fused_w: bool = False):
    """Blocked right-looking pivoted LTL^T.

    Each panel of nb columns k0 .. k0+nb-1 is factored with the left-looking
    (modified Aasen) algorithm: the column to eliminate is formed on the fly as
    v = X[k+1:, k] - L[k+1:, k0+1:k+1] h with h = T L[k, :]^T restricted to the
    panel (skew_tridiag_gemv); the pivot exchanges rows and columns of the whole
    unfactored matrix and rows of the panel's L columns; L columns left of the panel
    get the panel's exchanges afterwards (pivot_rows).  The trailing matrix then
    receives X[s:, s:] -= A T_p A^T with A = L[s:, k0+1:s+1] (s = k0+nb) and T_p the
    panel's skew tridiagonal block, followed by the last Gauss transform as a skew
    rank-2 update X[s+1:, s+1:] += l x^T - x l^T.

    With ``fused_w`` the trailing update is instead done the way the GPU path does
    it: W = A S (Theorem on T = S - S^T), the updated column x = X[s+1:, s] is
    formed first by the same left-looking formula, and one skew rank-2(k+1) update
    C += X' Y'^T - Y' X'^T with X' = [odd columns of A, l], Y' = [odd columns of W, x]
    covers both parts.
    """
    n = A.shape[0]
    X = full_skew_from_lower(np.asarray(A, dtype=np.float64))
    L = np.eye(n)
    t = np.zeros(max(n - 1, 0))
    piv = np.arange(n)

    def h_vector(k, k0):
        # h_q for q = k0+1 .. k, with L[k, k] = 1
        h = np.zeros(k - k0)
        for q in range(k0 + 1, k + 1):
            val = 0.0
            if q - 1 >= k0 + 1:
                val += t[q - 1] * L[k, q - 1]
            if q + 1 <= k:
                val -= t[q] * L[k, q + 1]
            h[q - k0 - 1] = val
        return h

    k0 = 0
    while k0 < n - 1:
        kend = min(k0 + nb, n - 1)
        for k in range(k0, kend):
            h = h_vector(k, k0)
            v = X[k + 1:, k] - L[k + 1:, k0 + 1:k + 1] @ h
            r = k + 1 + int(np.argmax(np.abs(v)))       # first index of the maximum
            piv[k + 1] = r
            if r != k + 1:
                v[[0, r - k - 1]] = v[[r - k - 1, 0]]
                X[[k + 1, r], :] = X[[r, k + 1], :]
                X[:, [k + 1, r]] = X[:, [r, k + 1]]
                L[[k + 1, r], k0 + 1:k + 1] = L[[r, k + 1], k0 + 1:k + 1]
            t[k] = v[0]
            L[k + 2:, k + 1] = v[1:] / t[k] if t[k] != 0.0 else 0.0
        for k in range(k0, kend):                         # pivot_rows
            r = piv[k + 1]
            if r != k + 1:
                L[[k + 1, r], 1:k0 + 1] = L[[r, k + 1], 1:k0 + 1]
        s = kend
        if s < n - 1:
            Ap = L[s:, k0 + 1:s + 1]
            b = Ap.shape[1]
            if not fused_w:
                Tp = tridiag_from_t(t[k0 + 1:s], b)
                X[s:, s:] -= Ap @ Tp @ Ap.T
                l = L[s + 1:, s]
                x = X[s + 1:, s].copy()
                X[s + 1:, s + 1:] += np.outer(l, x) - np.outer(x, l)
            else:
                # updated column s by the left-looking formula (step k = s)
                h = h_vector(s, k0)
                x = X[s + 1:, s] - L[s + 1:, k0 + 1:s + 1] @ h
                X[s + 1:, s] = x
                X[s, s + 1:] = -x
                tp = t[k0 + 1:s]                          # T_p sub-diagonal, b-1 values
                a = L[s + 1:, k0 + 1:s + 1]               # rows s+1.. of A
                cols_x, cols_y = [], []
                for j in range(1, b, 2):                   # odd columns of W = A S
                    w = -tp[j - 1] * a[:, j - 1]
                    if j + 1 < b:
                        w = w + tp[j] * a[:, j + 1]
                    cols_x.append(a[:, j])
                    cols_y.append(w)
                cols_x.append(L[s + 1:, s])
                cols_y.append(x)
                Xp = np.stack(cols_x, axis=1)
                Yp = np.stack(cols_y, axis=1)
                X[s + 1:, s + 1:] += Xp @ Yp.T - Yp @ Xp.T
        k0 = kend
    return L, t, piv


def ltlt_blocked_delayed(A: np.ndarray, nb: int):
    """The fused right-looking ordering of Invariant 2a (Section 4.2 "Fused
    right-looking algorithms"): the last Gauss transform of a panel is not applied at
    the end of that panel but fused with the next one.  Its coupling t[k0] between L
    columns k0 and k0+1 (k0 = the panel's first column) is then part of the next
    panel: the left-looking column uses L[:, k0 .. k] with its real entries (column k0
    is no longer the unit vector e_f, so the panel also exchanges its rows), and the
    trailing update after the panel is X[s:, s:] -= A' T' A'^T with A' = L[s:, k0 .. s]
    (one column more) and T' the tridiagonal block of t[k0 .. s-1].  No updated column
    x and no separate skew rank-2 pass are needed.  The factorization reached is the
    same as Variant 1's (same pivots, factors up to rounding)."""
    n = A.shape[0]
    X = full_skew_from_lower(np.asarray(A, dtype=np.float64))
    L = np.eye(n)
    t = np.zeros(max(n - 1, 0))
    piv = np.arange(n)

    def h_vector(k, k0):
        # h_q for q = k0 .. k (L[k, k] = 1): the coupling t[q-1] enters only for
        # q - 1 >= k0, i.e. the couplings t[k0] .. t[k-1] not yet applied to X
        h = np.zeros(k - k0 + 1)
        for q in range(k0, k + 1):
            val = 0.0
            if q - 1 >= k0:
                val += t[q - 1] * L[k, q - 1]
            if q + 1 <= k:
                val -= t[q] * L[k, q + 1]
            h[q - k0] = val
        return h

    k0 = 0
    while k0 < n - 1:
        kend = min(k0 + nb, n - 1)
        for k in range(k0, kend):
            h = h_vector(k, k0)
            v = X[k + 1:, k] - L[k + 1:, k0:k + 1] @ h
            r = k + 1 + int(np.argmax(np.abs(v)))
            piv[k + 1] = r
            if r != k + 1:
                v[[0, r - k - 1]] = v[[r - k - 1, 0]]
                X[[k + 1, r], :] = X[[r, k + 1], :]
                X[:, [k + 1, r]] = X[:, [r, k + 1]]
                L[[k + 1, r], k0:k + 1] = L[[r, k + 1], k0:k + 1]
            t[k] = v[0]
            L[k + 2:, k + 1] = v[1:] / t[k] if t[k] != 0.0 else 0.0
        for k in range(k0, kend):                         # pivot_rows: columns < k0
            r = piv[k + 1]
            if r != k + 1:
                L[[k + 1, r], 1:k0] = L[[r, k + 1], 1:k0]
        s = kend
        if s < n - 1:
            Ap = L[s:, k0:s + 1]
            Tp = tridiag_from_t(t[k0:s], Ap.shape[1])
            X[s:, s:] -= Ap @ Tp @ Ap.T
        k0 = kend
    return L, t, piv


def ltlt_lookahead(A: np.ndarray, nb: int):
    """The data flow of the look-ahead factorization, restated in numpy: the panel of
    block j+1 is formed from S_{j-1}, the state BEFORE block j's trailing update,
    left-looking over the L columns of blocks j and j+1 (h = T L[k, :]^T over columns
    kb+1 .. k with kb = block j's first column); it never writes S: its exchanges only
    update a map from positions to rows/columns of S (starting from block j's map), and
    the trailing update of block j+1 reads S_j through that map and writes S_{j+1} to
    another buffer.  Block j's L rows are exchanged in the panel's working copy only;
    pivot_rows applies each panel's exchanges to the earlier L columns after the update
    that reads them.  Returns ``(L, t, piv)``; must equal the oracle's factorization."""
    n = A.shape[0]
    src0 = full_skew_from_lower(np.asarray(A, dtype=np.float64))
    L = np.eye(n)
    t = np.zeros(max(n - 1, 0))
    piv = np.arange(n)
    if n < 2:
        return L, t, piv

    def panel(S, map_prev, xprev, kb, k0, kend, with_x):
        rows = np.arange(k0 + 1, n)
        phs = np.array(map_prev[k0 + 1:], copy=True)          # source index by position
        pho = np.arange(k0 + 1, n)                            # panel-start position
        # working copy of L columns kb+1 .. kend for rows k0+1 .. n-1 (by position)
        W = np.zeros((n, kend - kb))
        W[k0 + 1:, :k0 - kb] = L[k0 + 1:, kb + 1:k0 + 1]
        v = np.zeros(n)
        if xprev is not None:
            v[k0 + 1:] = xprev[k0 + 1:]
        else:
            v[k0 + 1:] = S[phs, map_prev[k0]]
        xout = None
        for k in range(k0, kend):
            p = k + 1
            r = p + int(np.argmax(np.abs(v[p:])))
            tau = v[r]
            t[k] = tau
            piv[p] = r
            if r != p:
                for arr in (v,):
                    arr[[p, r]] = arr[[r, p]]
                W[[p, r], :] = W[[r, p], :]
                a, b = p - (k0 + 1), r - (k0 + 1)
                phs[[a, b]] = phs[[b, a]]
                pho[[a, b]] = pho[[b, a]]
                L[[p, r], k0 + 1:k + 1] = L[[r, p], k0 + 1:k + 1]
            c = k + 1 - kb - 1                                # W column of L column k+1
            W[p, c] = 1.0
            W[p + 1:, c] = v[p + 1:] / tau if tau != 0.0 else 0.0
            L[p:, k + 1] = W[p:, c]
            if k + 1 < kend or with_x:
                h = np.zeros(k + 1 - kb)
                for q in range(kb + 1, k + 2):
                    val = 0.0
                    if q - 1 >= kb + 1:
                        tq1 = t[q - 1]
                        val += tq1 * W[p, q - 1 - kb - 1]
                    if q + 1 <= k + 1:
                        lq1 = 1.0 if q + 1 == k + 1 else W[p, q + 1 - kb - 1]
                        val -= t[q] * lq1
                    h[q - kb - 1] = val
                idx = phs[p + 1 - (k0 + 1):]
                xnew = S[idx, phs[p - (k0 + 1)]]
                vn = xnew - W[p + 1:, :k + 1 - kb] @ h
                v[:] = 0.0
                v[p + 1:] = vn
                if k + 1 == kend:
                    xout = np.zeros(n)
                    xout[p + 1:] = vn
        map_out = np.arange(n)
        map_out[k0 + 1:] = pho
        return map_out, xout

    def update(S_in, map_j, k0, kend, x):
        s = kend
        S_out = np.zeros_like(S_in)
        idx = map_j[s + 1:]
        C = S_in[np.ix_(idx, idx)]
        Ap = L[s + 1:, k0 + 1:kend + 1]
        Tp = tridiag_from_t(t[k0 + 1:kend], Ap.shape[1])
        l = L[s + 1:, kend]
        xv = x[s + 1:]
        C = C - Ap @ Tp @ Ap.T + (np.outer(l, xv) - np.outer(xv, l))
        S_out[s + 1:, s + 1:] = C
        return S_out

    def pivot_rows(k0, kend):
        for k in range(k0, kend):
            r = piv[k + 1]
            if r != k + 1:
                L[[k + 1, r], 1:k0 + 1] = L[[r, k + 1], 1:k0 + 1]

    ident = np.arange(n)
    k0, kend = 0, min(nb, n - 1)
    maps, xs = {}, {}
    maps[0], xs[0] = panel(src0, ident, None, 0, 0, kend, kend < n - 1)
    states = {-1: src0}
    blocks = {0: (0, kend)}
    j = 0
    while True:
        k0, kend = blocks[j]
        s = kend
        if j >= 1:
            pivot_rows(k0, kend)          # after panel j and update j-1
        if s >= n - 1:
            break
        k0n, kendn = kend, min(kend + nb, n - 1)
        blocks[j + 1] = (k0n, kendn)
        # panel j+1 beside update j: both read S_{j-1}
        maps[j + 1], xs[j + 1] = panel(states[j - 1], maps[j][np.arange(n)] if j >= 0 else ident,
                                       xs[j], k0, k0n, kendn, kendn < n - 1)
        states[j] = update(states[j - 1], maps[j], k0, kend, xs[j])
        j += 1
    return L, t, piv


def twostep_blocked(A, nb):
    """Blocked left-looking restatement of the two-step (Pfaffian-only) elimination,
    in the order the GPU path takes it.  Returns ``(a, piv)``.

    Within a panel of ``nb`` columns (nb/2 pairs), the current matrix is the matrix at
    the start of the panel plus the panel's rank-2 terms, X + sum_q (l_q y_q^T -
    y_q l_q^T), so a column is formed left-looking: v = X[:, k] + sum_q (l_q y_q[k] -
    y_q l_q[k]).  Pair at column k: r = argmax |v[k+1:]| (lowest index on ties),
    exchange k+1 <-> r in X, in the stored vectors and in v; a = v[k+1];
    l = v[k+2:] / a; y = column k+1 formed left-looking.  After the panel the trailing
    block takes sum_q (l_q y_q^T - y_q l_q^T) (one skew rank-2k update)."""
    n = A.shape[0]
    X = np.array(A, dtype=np.float64)
    piv = np.arange(n, dtype=np.int32)
    a = np.zeros(n // 2)
    k = 0
    while k + 1 < n:
        kend = k + nb
        ls, ys = [], []
        while k < kend and k + 1 < n:
            v = X[:, k].copy()
            for lq, yq in zip(ls, ys):
                v += lq * yq[k] - yq * lq[k]
            r = k + 1 + int(np.argmax(np.abs(v[k + 1:])))
            piv[k + 1] = r
            if r != k + 1:
                sw = [r, k + 1]
                X[[k + 1, r], :] = X[sw, :]
                X[:, [k + 1, r]] = X[:, sw]
                for w in ls + ys + [v]:
                    w[[k + 1, r]] = w[sw]
            ak = v[k + 1]
            a[k // 2] = ak
            l = np.zeros(n)
            if ak != 0.0:
                l[k + 2:] = v[k + 2:] / ak
            yy = X[:, k + 1].copy()
            for lq, yq in zip(ls, ys):
                yy += lq * yq[k + 1] - yq * lq[k + 1]
            y = np.zeros(n)
            y[k + 2:] = yy[k + 2:]
            ls.append(l)
            ys.append(y)
            k += 2
        for lq, yq in zip(ls, ys):
            X[k:, k:] += np.outer(lq[k:], yq[k:]) - np.outer(yq[k:], lq[k:])
    return a, piv
