/*
 * skew_oracle.c -- plain, slow, obviously correct FP64 CPU oracle for the pivoted
 * skew-symmetric triangular tridiagonalization  P X P^T = L T L^T  and the Pfaffian.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  The GPU library shares no code, header,
 * table or helper with this file, and this file includes nothing from it.
 *
 * Source: "Performant Tridiagonal Factorization of Skew-Symmetric Matrices"
 * (arXiv 2411.09859).  Each function names the passage it follows.
 *
 * Conventions (0-based, Section 2.1):
 *   - matrices are column-major, element (i,j) of M at M[i + j*ldm];
 *   - only the strictly lower triangle of the skew matrix X is stored or referenced
 *     (Section 3.1: the upper triangle and the zero diagonal are implicit);
 *   - t[j] = tau_{j+1,j}, the sub-diagonal of T (Eq. (T) in Section 1);
 *   - L is unit lower triangular with L e_0 = e_0 (Section 4.1: the first column of L
 *     is chosen as the first standard basis vector);
 *   - piv[i] is the absolute 0-based row exchanged with row i before the Gauss
 *     transform that produces column i of L; piv[0] = 0, since the pivoted blocked
 *     algorithm of Section 5.2 never searches for a first pivot and fixes it at zero.
 *     The relative pivot pi_i of Definition P(pi) equals piv[i] - i.
 *
 * Compile with -O2 -ffp-contract=off so every product and sum is rounded separately.
 * Where the paper is silent the readings are:
 *   - iamax returns the lowest index among entries of maximal magnitude;
 *   - a zero pivot column gives t[k] = 0 and a zero column of L (the Gauss transform
 *     is the identity); the factorization continues and the return value reports it;
 *   - a non-finite entry in the input is an error (returned before any work).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define X_(i, j) X[(size_t)(i) + (size_t)(j) * (size_t)ldx]
#define L_(i, j) L[(size_t)(i) + (size_t)(j) * (size_t)ldl]

/* Error codes shared in value (not in code) with the public library header. */
#define ORACLE_ERR_NONFINITE (-100)

/*
 * oracle_ltlt_steps: the unblocked right-looking (modified Parlett-Reid) algorithm
 * with partial pivoting, Section 4.1 ("Modifying the Parlett-Reid algorithm",
 * Eq. (1)) and Section 5.2 ("Adding pivoting to unblocked algorithms").
 *
 *   n        order of X (n >= 0)
 *   X, ldx   strictly lower triangle of X, overwritten (destroyed) as workspace
 *   L, ldl   n x n output, fully written: unit lower triangular, L e_0 = e_0
 *   t        n-1 outputs t[k] = tau_{k+1,k}
 *   piv      n outputs (absolute pivots, piv[0] = 0)
 *   nsteps   number of elimination steps k = 0 .. nsteps-1 to perform; pass n-1 (or
 *            any value >= n-1) for the whole factorization.  A smaller value stops
 *            early (used only to time a bounded sample of a large factorization);
 *            outputs beyond the last step are then left as initialised.
 *
 * Returns 0 on success, 1 + the first k with t[k] == 0 when a zero pivot occurred
 * (the factorization is still complete and valid), ORACLE_ERR_NONFINITE (nothing
 * written) if the strictly lower triangle holds a NaN or infinity, and -1 for a bad
 * argument.
 *
 * It is oracle_ltlt_setup followed by oracle_ltlt_range over steps 0 .. nsteps-1.
 */
int oracle_ltlt_range(int64_t n, double *X, int64_t ldx, double *L, int64_t ldl,
                      double *t, int32_t *piv, int64_t kbegin, int64_t kend);

/*
 * oracle_ltlt_setup: the checks and the initial state of oracle_ltlt_steps (same
 * arguments and error returns): L := I, piv := identity, t := 0.  Returns 0 when the
 * elimination steps may start.
 */
int oracle_ltlt_setup(int64_t n, double *X, int64_t ldx, double *L, int64_t ldl,
                      double *t, int32_t *piv)
{
    if (n < 0) return -1;
    if (n == 0) return 0;
    if (ldx < n || ldl < n) return -1;

    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = j + 1; i < n; ++i)
            if (!isfinite(X_(i, j))) return ORACLE_ERR_NONFINITE;

    /* L := I and piv := identity; piv[0] stays 0 (no first pivot, Section 5.2). */
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i)
            L_(i, j) = (i == j) ? 1.0 : 0.0;
    for (int64_t i = 0; i < n; ++i) piv[i] = (int32_t)i;
    for (int64_t k = 0; k + 1 < n; ++k) t[k] = 0.0;
    return 0;
}

int oracle_ltlt_steps(int64_t n, double *X, int64_t ldx, double *L, int64_t ldl,
                      double *t, int32_t *piv, int64_t nsteps)
{
    const int st = oracle_ltlt_setup(n, X, ldx, L, ldl, t, piv);
    if (st != 0 || n == 0) return st;
    return oracle_ltlt_range(n, X, ldx, L, ldl, t, piv, 0, nsteps);
}

/*
 * oracle_ltlt_range: elimination steps k = kbegin .. min(kend, n-1) - 1 of
 * oracle_ltlt_steps, on the state that oracle_ltlt_setup and the steps before kbegin
 * left in X, L, t and piv (so that a long factorization can be run, and timed, in
 * consecutive pieces with results identical to one call).  Returns 0, or 1 + the
 * first k of this range with t[k] == 0.
 */
int oracle_ltlt_range(int64_t n, double *X, int64_t ldx, double *L, int64_t ldl,
                      double *t, int32_t *piv, int64_t kbegin, int64_t kend)
{
    int info = 0;
    int64_t last = n - 1;                 /* steps k = 0 .. n-2 */
    if (kend < last) last = kend;

    for (int64_t k = kbegin; k < last; ++k) {
        /* ---- pivot: r = (k+1) + iamax(X[k+1:, k])  (Definition of iamax) ---- */
        int64_t r = k + 1;
        double best = fabs(X_(k + 1, k));
        for (int64_t i = k + 2; i < n; ++i) {
            double a = fabs(X_(i, k));
            if (a > best) { best = a; r = i; }   /* strict: lowest index wins ties */
        }
        piv[k + 1] = (int32_t)r;

        if (r != k + 1) {
            const int64_t p = k + 1, q = r;
            /* the pivot column itself */
            double tmp = X_(p, k); X_(p, k) = X_(q, k); X_(q, k) = tmp;
            /* rows p and q of the part of L already computed, columns 1..k */
            for (int64_t c = 1; c <= k; ++c) {
                tmp = L_(p, c); L_(p, c) = L_(q, c); L_(q, c) = tmp;
            }
            /* symmetric exchange of indices p and q of the trailing skew block
             * X[p:, p:], using only its strictly lower triangle (Section 5.2:
             * rows and columns are swapped; an entry that moves across the
             * diagonal changes sign because X = -X^T). */
            for (int64_t i = p + 1; i < q; ++i) {
                tmp = X_(i, p);
                X_(i, p) = -X_(q, i);
                X_(q, i) = -tmp;
            }
            X_(q, p) = -X_(q, p);
            for (int64_t i = q + 1; i < n; ++i) {
                tmp = X_(i, p); X_(i, p) = X_(i, q); X_(i, q) = tmp;
            }
        }

        /* ---- Gauss transform: tau := chi_21, l_32 := x_31 / chi_21 (Eq. (1)) ---- */
        const double tau = X_(k + 1, k);
        t[k] = tau;
        if (tau == 0.0 && info == 0) info = (int)(k + 1);
        for (int64_t i = k + 2; i < n; ++i) {
            L_(i, k + 1) = (tau != 0.0) ? X_(i, k) / tau : 0.0;
            X_(i, k) = 0.0;                       /* x_31 := 0 */
        }

        /* ---- X_33 := X_33 + (l_32 x_32^T - x_32 l_32^T), strictly lower part.
         * Column k+1 (x_32) is unchanged because chi_22 = 0 (Section 4.1). ---- */
        const int64_t c1 = k + 1;
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t j = k + 2; j < n; ++j) {
            const double xj = X_(j, c1), lj = L_(j, c1);
            for (int64_t i = j + 1; i < n; ++i)
                X_(i, j) = X_(i, j) + (L_(i, c1) * xj - X_(i, c1) * lj);
        }
    }
    return info;
}

/* The whole factorization. */
int oracle_ltlt(int64_t n, double *X, int64_t ldx, double *L, int64_t ldl,
                double *t, int32_t *piv)
{
    return oracle_ltlt_steps(n, X, ldx, L, ldl, t, piv, n);
}

/*
 * oracle_pfaffian: Pf(X) read off the factors.
 *
 * Pf(B X B^T) = det(B) Pf(X); with P X P^T = L T L^T and det L = 1 this gives
 * Pf(X) = det(P) Pf(T).  T is skew tridiagonal with T[i+1,i] = tau_{i+1,i} and
 * T[i,i+1] = -tau_{i+1,i} (Eq. (T)); by the definition in Section 1,
 * Pf([[0, a], [-a, 0]]) = a, so Pf(T) = prod_i T[2i, 2i+1] = prod_i (-t[2i]).
 * det(P) = (-1)^(number of i with piv[i] != i).
 *
 * Outputs log|Pf(X)| and sign(Pf(X)) in {-1, 0, +1}.  Odd n, or any t[2i] == 0,
 * gives Pf = 0: *logabs = -inf, *sign = 0.  n == 0 gives Pf = 1.
 * The sum of logarithms is taken left to right.
 */
void oracle_pfaffian(int64_t n, const double *t, const int32_t *piv,
                     double *logabs, int *sign)
{
    if (n % 2 != 0) { *logabs = -INFINITY; *sign = 0; return; }
    double s = 0.0;
    int sg = 1;
    for (int64_t i = 0; i < n / 2; ++i) {
        double v = -t[2 * i];                   /* T[2i, 2i+1] */
        if (v == 0.0) { *logabs = -INFINITY; *sign = 0; return; }
        if (v < 0.0) sg = -sg;
        s += log(fabs(v));
    }
    for (int64_t i = 0; i < n; ++i)
        if (piv[i] != i) sg = -sg;
    *logabs = s;
    *sign = sg;
}

/*
 * oracle_skew_rank2k: C := beta C + alpha (A B^T - B A^T), strictly lower triangle of
 * the m x m skew matrix C only (operation skew_rank2k in the table of BLAS-like
 * operations, Section 4.2; the diagonal of a skew matrix is zero and not stored).
 * A and B are m x k column-major.
 */
void oracle_skew_rank2k(int64_t m, int64_t k, double alpha,
                        const double *A, int64_t lda, const double *B, int64_t ldb,
                        double beta, double *C, int64_t ldc)
{
    for (int64_t j = 0; j < m; ++j)
        for (int64_t i = j + 1; i < m; ++i) {
            double s = 0.0;
            for (int64_t p = 0; p < k; ++p)
                s += A[i + p * lda] * B[j + p * ldb] - B[i + p * ldb] * A[j + p * lda];
            C[i + j * ldc] = beta * C[i + j * ldc] + alpha * s;
        }
}

/*
 * oracle_skew_tridiag_rankk: C := beta C + alpha A T A^T, strictly lower triangle of
 * the m x m skew matrix C only (operation skew_tridiag_rankk, Section 4.2).  A is
 * m x b column-major and T is the b x b skew tridiagonal matrix with sub-diagonal
 * t[0 .. b-2] (T[a+1,a] = t[a], T[a,a+1] = -t[a]).  Written directly from the
 * definition: (A T A^T)[i,j] = sum_{a,c} A[i,a] T[a,c] A[j,c].
 */
void oracle_skew_tridiag_rankk(int64_t m, int64_t b, double alpha,
                               const double *A, int64_t lda, const double *t,
                               double beta, double *C, int64_t ldc)
{
    for (int64_t j = 0; j < m; ++j)
        for (int64_t i = j + 1; i < m; ++i) {
            double s = 0.0;
            for (int64_t a = 0; a + 1 < b; ++a) {
                /* T[a+1,a] = t[a] contributes A[i,a+1] t[a] A[j,a];
                 * T[a,a+1] = -t[a] contributes -A[i,a] t[a] A[j,a+1]. */
                s += A[i + (a + 1) * lda] * t[a] * A[j + a * lda];
                s -= A[i + a * lda] * t[a] * A[j + (a + 1) * lda];
            }
            C[i + j * ldc] = beta * C[i + j * ldc] + alpha * s;
        }
}

/*
 * oracle_pfaffian_twostep: Pf(X) by the two-step elimination that keeps only what
 * the Pfaffian needs -- Wimmer's algorithm, as described in the notes to the two-step
 * right-looking algorithm of Section 4.1: the second Gauss transform of each step
 * (l_43) and tau_32 are skipped, since only every other sub-diagonal element of T
 * enters the Pfaffian.  Pivoting as in Section 5.2, at the even steps only.
 *
 * For k = 0, 2, 4, ... while k + 1 < n:
 *   r = (k+1) + iamax(X[k+1:, k]) (lowest index on ties); piv[k+1] = r; exchange
 *   of indices k+1 and r in X[k:, k:] (as in oracle_ltlt_steps);
 *   a[k/2] = X[k+1, k];
 *   with x0 = X[k+2:, k], y = X[k+2:, k+1] and l = x0 / a[k/2] (0 when a[k/2] = 0):
 *   X[k+2:, k+2:] := X[k+2:, k+2:] + (l y^T - y l^T).
 * The last statement is the Schur complement S = D + B^T A^{-1} B of the leading
 * 2 x 2 skew block A = [[0, -a], [a, 0]] in M = [[A, B], [-B^T, D]] (here B^T = -X21,
 * A^{-1} = [[0, 1/a], [-1/a, 0]], so B^T A^{-1} B = (x0 y^T - y x0^T) / a), and
 * Pf(M) = Pf(A) Pf(S) = (-a) Pf(S).  With the exchanges, Pf(X) = det(P) prod (-a[j]).
 *
 *   n        order of X (n >= 0)
 *   X, ldx   strictly lower triangle of X, overwritten (destroyed)
 *   a        floor(n/2) outputs a[j] = tau_{2j+1,2j} of the two-step elimination
 *   piv      n outputs: piv[k+1] at even k as above, piv[i] = i elsewhere
 *   logabs, sign   log|Pf(X)| and sign(Pf(X)) (odd n or a zero a[j]: -inf and 0)
 *
 * Returns 0, 1 + the first even k with a[k/2] == 0 (Pf = 0; the elimination still
 * runs to the end with l = 0), ORACLE_ERR_NONFINITE if the strictly lower triangle
 * holds a NaN or infinity (nothing written), or -1 for a bad argument.
 */
int oracle_pfaffian_twostep(int64_t n, double *X, int64_t ldx, double *a, int32_t *piv,
                            double *logabs, int *sign)
{
    if (n < 0 || ldx < (n > 0 ? n : 1)) return -1;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = j + 1; i < n; ++i)
            if (!isfinite(X_(i, j))) return ORACLE_ERR_NONFINITE;
    for (int64_t i = 0; i < n; ++i) piv[i] = (int32_t)i;
    for (int64_t j = 0; j < n / 2; ++j) a[j] = 0.0;

    int info = 0;
    for (int64_t k = 0; k + 1 < n; k += 2) {
        int64_t r = k + 1;
        double best = fabs(X_(k + 1, k));
        for (int64_t i = k + 2; i < n; ++i) {
            double v = fabs(X_(i, k));
            if (v > best) { best = v; r = i; }   /* strict: lowest index wins ties */
        }
        piv[k + 1] = (int32_t)r;
        if (r != k + 1) {
            const int64_t u = k + 1, w = r;   /* exchange indices u and w */
            double sv = X_(u, k); X_(u, k) = X_(w, k); X_(w, k) = sv;
            for (int64_t i = u + 1; i < w; ++i) {
                sv = X_(i, u);
                X_(i, u) = -X_(w, i);
                X_(w, i) = -sv;
            }
            X_(w, u) = -X_(w, u);
            for (int64_t i = w + 1; i < n; ++i) {
                sv = X_(i, u); X_(i, u) = X_(i, w); X_(i, w) = sv;
            }
        }
        const double ak = X_(k + 1, k);
        a[k / 2] = ak;
        if (ak == 0.0 && info == 0) info = (int)(k + 1);
        /* l := X[k+2:, k] / a (stored over x0), y = X[k+2:, k+1] */
        for (int64_t i = k + 2; i < n; ++i)
            X_(i, k) = (ak != 0.0) ? X_(i, k) / ak : 0.0;
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t j = k + 2; j < n; ++j) {
            const double lj = X_(j, k), yj = X_(j, k + 1);
            for (int64_t i = j + 1; i < n; ++i)
                X_(i, j) = X_(i, j) + (X_(i, k) * yj - X_(i, k + 1) * lj);
        }
    }

    if (n % 2 != 0) { *logabs = -INFINITY; *sign = 0; return info; }
    double s = 0.0;
    int sg = 1;
    for (int64_t j = 0; j < n / 2; ++j) {
        const double v = -a[j];
        if (v == 0.0) { *logabs = -INFINITY; *sign = 0; return info; }
        if (v < 0.0) sg = -sg;
        s += log(fabs(v));
    }
    for (int64_t i = 0; i < n; ++i)
        if (piv[i] != (int32_t)i) sg = -sg;   /* det(P) */
    *logabs = s;
    *sign = sg;
    return info;
}

/* Number of host threads the rank-2 update of oracle_ltlt_steps may use. */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * oracle_ltlt_many: oracle_ltlt_steps (whole factorizations) and oracle_pfaffian on
 * `count` independent matrices, one matrix per host thread (OpenMP, dynamic schedule
 * in the order given; the update loop inside each factorization runs on its own
 * thread).  Matrix b has order n[b], leading dimensions max(n[b], 1), and its own X,
 * L, t and piv arrays as for oracle_ltlt_steps; info[b], logabs[b] and sign[b] are
 * its results.  This is the CPU baseline of a batch of small factorizations.
 */
void oracle_ltlt_many(int64_t count, const int64_t *n, double *const *X,
                      double *const *L, double *const *t, int32_t *const *piv,
                      int *info, double *logabs, int *sign)
{
#ifdef _OPENMP
    const int levels = omp_get_max_active_levels();
    omp_set_max_active_levels(1);
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < count; ++b) {
        const int64_t nn = n[b], ld = nn > 0 ? nn : 1;
        info[b] = oracle_ltlt_steps(nn, X[b], ld, L[b], ld, t[b], piv[b], nn);
        if (info[b] >= 0)
            oracle_pfaffian(nn, t[b], piv[b], &logabs[b], &sign[b]);
        else {
            logabs[b] = NAN;
            sign[b] = 0;
        }
    }
#ifdef _OPENMP
    omp_set_max_active_levels(levels);
#endif
}
