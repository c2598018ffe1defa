/*
 * skewltlt.h -- C ABI of the GB300 (sm_103a) skew-symmetric LTL^T library.
 *
 * Operation (arXiv 2411.09859, Section 1 and Section 5): for a real skew-symmetric
 * n x n matrix X (X = -X^T), compute the pivoted triangular tridiagonalization
 *
 *     P X P^T = L T L^T,
 *
 * with P a permutation, L unit lower triangular with L e_0 = e_0 (Section 4.1), and T
 * skew-symmetric tridiagonal with sub-diagonal tau_{i+1,i} (Eq. (T)); and the
 * Pfaffian Pf(X) = det(P) Pf(T) read off the factors.  The method is the pivoted
 * blocked right-looking algorithm (Section 4.2 "Blocked algorithms", Variant 1, with
 * the pivoted left-looking panel of Section 5.2), whose trailing update is a
 * skew-symmetric rank-2k update obtained from A T A^T through W = A S (Theorem on
 * T = S - S^T, Section 2.2).
 *
 * Conventions shared by every entry point:
 *   - Matrices are FP64, column-major: element (i, j) of M is M[i + j * ldm].
 *   - Only the strictly lower triangle of a skew input is read; its upper triangle
 *     and diagonal are never referenced (Section 4.1: the skew structure is implicit).
 *   - Indices are 0-based.  t[j] = tau_{j+1,j}, j = 0 .. n-2.
 *   - piv[i] (i = 0 .. n-1) is the absolute row exchanged with row i just before
 *     column i of L is formed; piv[0] = 0 and piv[i] >= i.  The relative pivot
 *     pi_i of Section 5.1 is piv[i] - i, and P = P(p) of Section 5.1.
 *   - Pivot search: the entry of largest magnitude; among equal magnitudes the
 *     lowest row index (the paper leaves ties open).
 *   - Pointers named "device" must point to memory of the current CUDA device.  The
 *     caller owns every buffer it passes.  The library owns only the workspace it
 *     allocates itself (stream-ordered, freed before the call's work completes).
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Device work is
 *     enqueued on it and the call returns without waiting; outputs are valid once
 *     the stream has reached the call's end.
 *   - Return value: SKEW_OK, or a negative status.  A value -i with 1 <= i <= 99
 *     means argument i (1-based) is invalid; nothing is enqueued then.
 *   - `info` (device int32, may be NULL) receives, in stream order: 0 on success;
 *     1 + the first j with t[j] == 0 (a zero pivot column: the factorization is
 *     still complete and valid, its Gauss transform is the identity); or a negative
 *     status detected on the device (SKEW_ERR_NONFINITE, SKEW_ERR_TIMEOUT), in which
 *     case the outputs are unspecified.
 */
#ifndef SKEWLTLT_H
#define SKEWLTLT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SKEW_OK = 0,
    SKEW_ERR_NONFINITE = -100,  /* a NaN or infinity in the strictly lower input */
    SKEW_ERR_NOMEM = -101,      /* device workspace could not be allocated */
    SKEW_ERR_CUDA = -102,       /* a CUDA runtime call failed (see skew_last_error) */
    SKEW_ERR_TIMEOUT = -103,    /* a bounded device-side wait gave up */
    SKEW_ERR_NODEVICE = -104,   /* no usable sm_103 device is current */
    SKEW_ERR_SCRATCH_LIMIT = -105, /* skew_pfaffian_noalloc: the problem needs more
                                      than its fixed scratch (see there) */
    SKEW_ERR_BUSY = -106           /* skew_server_release: the request is in flight */
} skew_status;

/* Library version as 10000*major + 100*minor + patch. */
int skew_version(void);

/* Text of the last CUDA error seen by this thread's calls ("" if none).  The
 * returned string is owned by the library and valid until the next call. */
const char *skew_last_error(void);

/* Number of device kernels this process has launched through the library so far
 * (every entry point counts its own launches; never reset). */
uint64_t skew_kernel_launches(void);

/* Return the device memory that the library keeps in its private stream-ordered
 * pool (freed blocks stay reserved for reuse by later calls) to the system.  Call
 * only when no library work is in flight on the current device. */
int skew_trim_memory(void);

/* Device memory the library's allocations hold on the current device: used_now in
 * use right now, used_high the most held at once since the last reset (reset_high != 0
 * resets it after reading).  Counts what the library allocates itself (workspaces,
 * server buffers, host-call buffers), not the caller's buffers.  No counterpart in the
 * paper. */
int skew_pool_usage(size_t *used_now, size_t *used_high, int reset_high);

/*
 * Per-kernel timing.  While enabled, every kernel launch made by skew_ltlt,
 * skew_pfaffian, skew_pfaffian_twostep, the batched calls, skew_rank2k and
 * skew_tridiag_rankk is bracketed by two CUDA events recorded on the launch's stream,
 * tagged with the launch's algorithmic work.  (Whether enabled or not, each such
 * launch is also enclosed in an NVTX range named for its kind -- "prologue",
 * "panel", "pivot_rows", "skr2k", "finish", "batched" -- for profilers.)
 * skew_profile_read waits for the recorded events, adds up the elapsed times per
 * kernel kind, and clears the record.  Kinds: 0 prologue, 1 panel, 2 pivot_rows,
 * 3 skr2k (the skew rank-2k update), 4 finish, 5 batched (the whole batched call).
 *   flops: skr2k counts 4 * (number of pairs) per strictly lower entry of C, i.e.
 *          2 * npairs * m * (m - 1); panel counts 2 * rows * (columns already formed)
 *          per step for its skew_tridiag_gemv.
 *   bytes: skr2k counts reading and writing the strictly lower triangle of C once;
 *          panel counts, per step, the column read, the L column written and the
 *          exchanged entries read and written.
 */
typedef struct {
    double ms;          /* summed event time of this kind's launches */
    double flops;       /* summed algorithmic flops */
    double bytes;       /* summed algorithmic DRAM bytes */
    uint64_t launches;  /* number of launches */
} skew_kernel_stat;

#define SKEW_KIND_COUNT 6
int skew_profile_enable(int on);
int skew_profile_read(skew_kernel_stat *stats /* SKEW_KIND_COUNT entries */);

/* Self-test of the device-side bounded waits (failure detection without a fault):
 * launches two CTAs into a grid barrier that waits for a third one, which never
 * comes; after timeout_s seconds (0 < timeout_s <= 10) the wait gives up, records
 * SKEW_ERR_TIMEOUT and the kernel returns normally.  Synchronous; *status receives
 * the recorded status (SKEW_ERR_TIMEOUT when the mechanism works).  The device stays
 * usable afterwards. */
int skew_selftest_bounded_wait(double timeout_s, int32_t *status);

/* The same check for the bounded mbarrier wait of the tensor-core (tcgen05) kernels: one
 * thread waits for the completion of an mbarrier phase that no thread ever arrives on;
 * after timeout_s seconds (0 < timeout_s <= 10) the wait gives up and records
 * SKEW_ERR_TIMEOUT in *status.  Synchronous; the device stays usable afterwards.
 * Returns 0, -1 / -2 for a bad argument, or a host-side status. */
int skew_selftest_mbarrier_wait(double timeout_s, int32_t *status);

/* Panel width used when `nb` is 0 for a matrix of order n: from the table installed
 * by skew_set_nb_table, else 16 (n <= 256), 32 (n <= 2048), 64. */
int skew_default_nb(int64_t n);

/* Installs a panel-width table (typically an autotuner's measurements on this device):
 * orders n <= n_upper[i] (the first such i; n_upper strictly increasing) take nb[i]
 * (1 .. 256), larger orders the last entry.  count = 0 restores the built-in rule.
 * The paper has no counterpart (its block size is a parameter of the C++ routine,
 * Section 5.2); here it only chooses the default of `nb = 0`.  Thread safe.
 * Returns 0, or -1 / -2 / -3 for a bad count / n_upper / nb. */
int skew_set_nb_table(int count, const int64_t *n_upper, const int32_t *nb);
/* The same with, per entry, lookahead[i] = 1 / 0 / -1: that order range takes the
 * look-ahead path / the plain path / the built-in choice (see skew_set_lookahead);
 * lookahead may be NULL (all -1).  Returns as skew_set_nb_table, or -4 for a bad
 * lookahead entry.  No counterpart in the paper. */
int skew_set_nb_table_ex(int count, const int64_t *n_upper, const int32_t *nb,
                         const int32_t *lookahead);

/* Panel width (8, 16 or 32) of the CTA-local batched kernels (skew_ltlt_batched for
 * orders <= 512, skew_pfaffian_batched) per order bucket: a matrix of order
 * n <= n_upper[i] (first such i; strictly increasing, count <= 8) takes nb[i], larger
 * ones the last entry; count = 0 restores 16 for every order.  Typically the batched
 * autotuner's result.  No counterpart in the paper.  Thread safe; returns 0, or -1 /
 * -2 / -3 for a bad count / n_upper / nb.  skew_get_batched_nb(n) reports the width an
 * order takes. */
int skew_set_batched_nb_table(int count, const int32_t *n_upper, const int32_t *nb);
int skew_get_batched_nb(int n);

/* The same table with the trailing update's warp tile per bucket as well: a matrix of
 * order n <= n_upper[i] also takes warp_tile[i] (16 or 32; NULL: 32 for every bucket),
 * the side of the square tile of the lower triangle that one warp of the CTA updates
 * with 8 x 8 FP64 DMMA sub-tiles (16 wastes less on the ragged edge of small orders,
 * 32 reuses each staged operand over more sub-tiles).  No counterpart in the paper.
 * Returns 0, or -1 / -2 / -3 / -4 for a bad count / n_upper / nb / warp_tile;
 * skew_get_batched_warp_tile(n) reports the tile an order takes. */
int skew_set_batched_tiles(int count, const int32_t *n_upper, const int32_t *nb,
                           const int32_t *warp_tile);
int skew_get_batched_warp_tile(int n);

/* Threads per CTA of the blocked batched kernels (skew_ltlt_batched up to n = 512,
 * skew_pfaffian_batched): 256 (the default) or 128.  Returns the previous value, or -1
 * for another value.  With 128, a multiprocessor can hold more matrices at once (when
 * the panel width keeps shared memory small enough), each factored by fewer warps.
 * Typically the batched autotuner's choice.  No counterpart in the paper. */
int skew_set_batched_threads(int threads);

/*
 * Device workspace, in bytes, that skew_ltlt / skew_pfaffian need for order n and
 * panel width nb (0 = default).  `with_L` = 0 gives the figure for skew_pfaffian,
 * which keeps only the current panel of L.  Pass a buffer of at least this size to
 * avoid the library's own stream-ordered allocation.
 */
size_t skew_workspace_bytes(int64_t n, int nb, int with_L);

/*
 * Workspace for the look-ahead path of skew_ltlt / skew_pfaffian (FP64 update, panel
 * width 2 .. 64, n - 1 <= 128 x the multiprocessors of the device): the panel of each
 * block runs on a second stream beside the trailing update of the block before it
 * (Section 5.2's panel, left-looking over both blocks, with its exchanges deferred to
 * the next update), which then reads and writes two matrix buffers: A and an n x n
 * copy in this workspace.  A call given at least this many bytes (or no workspace)
 * takes the look-ahead path; one given only skew_workspace_bytes takes the plain
 * path.  Both give the same pivots and factors up to rounding.  Where the look-ahead
 * does not apply this equals skew_workspace_bytes.  No counterpart in the paper (its
 * blocked algorithm updates in place, Section 5.2).
 */
size_t skew_workspace_bytes_lookahead(int64_t n, int nb, int with_L);

/* Chooses the path of later calls of this process; returns the previous setting.
 * Both paths compute the factorization of Section 5.2; the look-ahead is a schedule of
 * this library with no counterpart in the paper.
 *   0  plain path always;
 *   1  (the default) the look-ahead where the panel-width table says so for the order
 *      (skew_set_nb_table_ex); without a table entry, for 3072 <= n <= 5120 with
 *      cluster panels (skew_set_cluster_panel) and 3072 <= n <= 10240 without;
 *   2  the look-ahead wherever it applies;
 *   32, 64  as 2, with that many rows per CTA in the look-ahead panel instead of 128
 *      (a tuning knob). */
int skew_set_lookahead(int mode);

/* Sets the trailing order below which a look-ahead factorization goes on without the
 * look-ahead: once the next trailing update is smaller than `rows`, that update is the
 * last out-of-place one and the remaining blocks are factored as on the plain path, in
 * place on its result (the panel of such a block costs more than the update it would
 * hide).  Returns the previous value; -1 (the default) means 2560 rows (where an
 * update stops hiding a look-ahead panel on GB300, whatever the width), 0 keeps the
 * look-ahead to the end.  A schedule of this library, no counterpart in the
 * paper; results as on the plain path. */
long long skew_set_lookahead_switch(long long rows);

/* Turns the cluster panel on (1, the default) or off (0) for later calls of this
 * process; returns the previous setting.  On, the plain path factors each panel whose
 * trailing block has at most 4096 rows (and width <= 96) with one thread-block cluster
 * of at most 16 CTAs, exchanging each column step's pivot candidates through
 * distributed shared memory instead of global memory.  Same steps and results as the
 * grid-wide panel (Section 5.2); the exchange is this library's. */
int skew_set_cluster_panel(int on);

/* 1 if skew_ltlt / skew_pfaffian_ex at order n, width nb (0 = default) and this
 * trailing-update precision take the look-ahead path on the current device when given
 * skew_workspace_bytes_lookahead bytes (or no workspace), else 0.  No counterpart in
 * the paper. */
int skew_lookahead_used(int64_t n, int nb, int precision);

/*
 * skew_ltlt -- pivoted blocked right-looking P A P^T = L T L^T
 * (Section 4.2, Variant 1; Section 5.2 pivoted blocked right-looking algorithm).
 *
 *   1  n          order, n >= 0
 *   2  A          device, lda x n; strictly lower triangle = the skew input.
 *                 DESTROYED: used as the trailing-matrix workspace.
 *   3  lda        >= max(1, n)
 *   4  L          device, ldl x n output, fully written: unit lower triangular,
 *                 zero above the diagonal, L[:, 0] = e_0
 *   5  ldl        >= max(1, n)
 *   6  t          device, n-1 outputs t[j] = tau_{j+1,j} (may be NULL when n <= 1)
 *   7  piv        device, n int32 outputs (absolute pivots, piv[0] = 0)
 *   8  info       device int32 or NULL (see above)
 *   9  nb         panel width 1 .. 256, or 0 for skew_default_nb(n)
 *  10  workspace  device buffer or NULL (library allocates on `stream`)
 *  11  workspace_bytes  size of `workspace` (ignored when it is NULL)
 *  12  stream     cudaStream_t
 * A, L, t, piv must not overlap.
 */
int skew_ltlt(int64_t n, double *A, int64_t lda, double *L, int64_t ldl, double *t,
              int32_t *piv, int32_t *info, int nb, void *workspace,
              size_t workspace_bytes, void *stream);

/*
 * skew_pfaffian -- Pf(A) through the same factorization, keeping only the current
 * panel of L (Pf(X) = det(P) Pf(T) = det(P) prod_i T[2i, 2i+1], Section 1 with
 * Pf(B X B^T) = det(B) Pf(X)).
 *
 *   1  n        order, n >= 0
 *   2  A        device, lda x n, strictly lower triangle read; DESTROYED
 *   3  lda      >= max(1, n)
 *   4  logabs   device double: log |Pf(A)| (-inf when Pf = 0; 0 for n = 0)
 *   5  sign     device int32: sign of Pf(A) in {-1, 0, +1} (0 for odd n or a zero
 *               t[2i]; +1 for n = 0)
 *   6  t        device, n-1 outputs, or NULL (then kept in the workspace)
 *   7  piv      device, n outputs, or NULL (then kept in the workspace)
 *   8  info     device int32 or NULL
 *   9  nb, 10 workspace, 11 workspace_bytes, 12 stream: as for skew_ltlt
 */
int skew_pfaffian(int64_t n, double *A, int64_t lda, double *logabs, int32_t *sign,
                  double *t, int32_t *piv, int32_t *info, int nb, void *workspace,
                  size_t workspace_bytes, void *stream);

/*
 * skew_pfaffian_from_factors -- the read-off alone: log|Pf| and sign from t and piv
 * of an order-n factorization (all device pointers; t has n-1 entries).
 *   1 n, 2 t, 3 piv, 4 logabs, 5 sign, 6 stream
 * The sum of logarithms uses a fixed (deterministic) reduction order.
 */
int skew_pfaffian_from_factors(int64_t n, const double *t, const int32_t *piv,
                               double *logabs, int32_t *sign, void *stream);

/*
 * skew_pfaffian_noalloc -- skew_pfaffian for callers that must not have the library
 * allocate device memory.  The paper has no counterpart: this is a deployment
 * variant.  It serves programs whose device memory belongs to another allocator (for
 * example a framework that reserves nearly all of HBM for its own caching pool, so a
 * library allocation would fail or fragment that pool) and latency-bound loops that
 * cannot take an allocation on their critical path, when they cannot pass a
 * workspace to skew_pfaffian either.
 *
 * The workspace is a fixed 16 MiB device array inside the library, present on every
 * device that loads the library until the process exits.  The call itself allocates
 * nothing (no cudaMalloc, cudaFree, pool or library allocation).  Problems whose
 * workspace, skew_workspace_bytes(n, nb, 0), exceeds 16 MiB are rejected with
 * SKEW_ERR_SCRATCH_LIMIT before any device work (at nb = 64 this admits n up to about
 * 29990; a smaller nb admits larger n).
 *
 * The first call on a device looks up the array's device address (with that device
 * current); make that first call before any stream capture begins.  All calls share
 * the one array, which keeps the previous call's contents; the call clears, in
 * stream order, what must start at zero.  Calls whose device work overlaps (on
 * different streams, or from different threads) race on the array: serialise them.
 *
 *   1 n, 2 A (device, DESTROYED), 3 lda, 4 logabs (device), 5 sign (device),
 *   6 info (device or NULL), 7 nb (0 = default), 8 stream -- as for skew_pfaffian;
 *   t and piv are kept in the fixed array.
 */
int skew_pfaffian_noalloc(int64_t n, double *A, int64_t lda, double *logabs,
                          int32_t *sign, int32_t *info, int nb, void *stream);

/*
 * Precision of the trailing (skew rank-2k) update.  The panel, the pivot search,
 * the Gauss-transform division, t and the log-Pfaffian stay FP64 in both.
 *   SKEW_PRECISION_FP64       FP64 tensor-core (DMMA) products: rounding as in an FP64
 *                             dot product, entry by entry.
 *   SKEW_PRECISION_SPLIT_BF16 the FP64 operands held as 55-bit integers relative to
 *                             their row's largest entry, cut into seven 8-bit digit
 *                             slices and multiplied on the fifth-generation tensor
 *                             cores (tcgen05, bf16 inputs, exact FP32 sums per digit
 *                             group), recombined exactly in 64-bit integers
 *                             (Ozaki-type error-free splitting); with k column pairs
 *                             the update differs from the exact one by at most about
 *                             (2.02 k + 0.5) 2^-53 (row max of U)(row max of V), plus
 *                             the rounding of the final FP64 add.  In the
 *                             factorization's trailing updates each pair (a_p, w_p)
 *                             is first balanced to (2^e a_p, 2^-e w_p) with
 *                             2^(2e) about the size of the T entries in w_p (its
 *                             term a_p w_p^T - w_p a_p^T is unchanged, exactly), so
 *                             that large T entries do not raise the row maxima.
 *                             At most 32 column pairs per update (panel width
 *                             nb <= 64).
 */
#define SKEW_PRECISION_FP64 0
#define SKEW_PRECISION_SPLIT_BF16 1

/* skew_ltlt / skew_pfaffian with the trailing-update precision chosen by argument 10
 * (`precision`; for SKEW_PRECISION_SPLIT_BF16, nb must be at most 64 and 0 picks
 * min(default, 64)).  Other arguments as there; workspace (argument 11) of
 * skew_workspace_bytes_ex bytes, or NULL. */
int skew_ltlt_ex(int64_t n, double *A, int64_t lda, double *L, int64_t ldl, double *t,
                 int32_t *piv, int32_t *info, int nb, int precision, void *workspace,
                 size_t workspace_bytes, void *stream);
int skew_pfaffian_ex(int64_t n, double *A, int64_t lda, double *logabs, int32_t *sign,
                     double *t, int32_t *piv, int32_t *info, int nb, int precision,
                     void *workspace, size_t workspace_bytes, void *stream);
size_t skew_workspace_bytes_ex(int64_t n, int nb, int with_L, int precision);

/*
 * skew_pfaffian_twostep -- Pf(A) by the two-step (Pfaffian-only) elimination: Wimmer's
 * algorithm as described in the notes to the two-step right-looking algorithm of
 * Section 4.1, i.e. the factorization of skew_pfaffian with the second Gauss transform
 * of every two-step iteration (l_43) and tau_32 skipped, since only every other
 * sub-diagonal element of T enters the Pfaffian.  Partial pivoting (Section 5.2) at
 * the even steps only: for k = 0, 2, 4, ...  r = (k+1) + iamax(X[k+1:, k]), exchange
 * of k+1 and r, a_(k/2) = X[k+1, k], and the Schur complement of the 2 x 2 pivot block,
 *     X[k+2:, k+2:] += l y^T - y l^T,  l = X[k+2:, k] / a_(k/2),  y = X[k+2:, k+1];
 * Pf(A) = det(P) prod_j (-a_j).  The same n^3/3 flops as skew_pfaffian, but half the
 * pivot searches (n/2 grid-wide exchanges instead of n) and no L.  Blocked: a
 * left-looking panel of nb columns (nb/2 pairs), then one skew rank-2k update of the
 * trailing block per panel (precision as for skew_pfaffian_ex).
 *   1  n          order, 0 <= n - 1 <= 256 x (multiprocessors of the device)
 *   2  A          device, lda x n, column-major; strictly lower triangle read, and
 *                 overwritten (destroyed) as workspace
 *   3  lda        >= max(1, n)
 *   4  logabs     device, 1 double: log|Pf(A)| (-inf when Pf = 0), or NULL
 *   5  sign       device, 1 int32: sign of Pf(A) in {-1, 0, 1}, or NULL
 *   6  a          device, n/2 doubles: the pivot-block entries a_j, or NULL
 *   7  piv        device, n int32: piv[k+1] = r at even k, piv[i] = i elsewhere, or NULL
 *   8  info       device, 1 int32: 0; 1 + the first even k with a_(k/2) = 0 (Pf = 0);
 *                 or a negative device error (SKEW_ERR_NONFINITE, SKEW_ERR_TIMEOUT);
 *                 or NULL
 *   9  nb         panel width: even, 2 .. 96 (at most 64 with split precision), 0 = 64
 *   10 precision  SKEW_PRECISION_FP64 or SKEW_PRECISION_SPLIT_BF16
 *   11 workspace  device, skew_workspace_bytes_twostep(n, nb, precision) bytes, or NULL
 *   12 workspace_bytes
 *   13 stream     cudaStream_t (NULL: legacy default stream)
 * Returns 0 (asynchronous on the stream), -i for a bad argument i (-1 also when n is
 * too large for one row per thread of the panel: use skew_pfaffian), or a host-side
 * status (SKEW_ERR_NOMEM, SKEW_ERR_CUDA, SKEW_ERR_NODEVICE).
 */
int skew_pfaffian_twostep(int64_t n, double *A, int64_t lda, double *logabs, int32_t *sign,
                          double *a, int32_t *piv, int32_t *info, int nb, int precision,
                          void *workspace, size_t workspace_bytes, void *stream);
size_t skew_workspace_bytes_twostep(int64_t n, int nb, int precision);

/* skew_rank2k with the precision of argument 11 (split: k <= 32). */
int skew_rank2k_ex(int64_t m, int64_t k, double alpha, const double *X, int64_t ldx,
                   const double *Y, int64_t ldy, double beta, double *C, int64_t ldc,
                   int precision, void *stream);

/*
 * skew_rank2k -- C := beta C + alpha (X Y^T - Y X^T) on the strictly lower
 * triangle of the m x m skew matrix C (operation skew_rank2k of the table of
 * BLAS-like operations in Section 4.2).  FP64 tensor-core (DMMA) tiles.
 *   1 m, 2 k, 3 alpha, 4 X (device, ldx x k), 5 ldx, 6 Y (device, ldy x k), 7 ldy,
 *   8 beta, 9 C (device, ldc x m), 10 ldc, 11 stream
 * The upper triangle and diagonal of C are not touched.
 */
int skew_rank2k(int64_t m, int64_t k, double alpha, const double *X, int64_t ldx,
                const double *Y, int64_t ldy, double beta, double *C, int64_t ldc,
                void *stream);

/*
 * skew_tridiag_rankk -- C := beta C + alpha A T A^T on the strictly lower triangle
 * of the m x m skew matrix C, where A is m x b and T is the b x b skew tridiagonal
 * matrix with sub-diagonal t[0 .. b-2] (operation skew_tridiag_rankk, Section 4.2).
 * Evaluated as the rank-2*floor(b/2) update W A^T - A W^T with W = A S, where
 * T = S - S^T and only the odd columns of W are nonzero (Section 2.2); W is formed
 * while the operand tiles are staged, never stored.
 *   1 m, 2 b, 3 alpha, 4 A (device, lda x b), 5 lda, 6 t (device, b-1 values),
 *   7 beta, 8 C (device, ldc x m), 9 ldc, 10 stream
 */
int skew_tridiag_rankk(int64_t m, int64_t b, double alpha, const double *A,
                       int64_t lda, const double *t, double beta, double *C,
                       int64_t ldc, void *stream);

/*
 * One problem of a batched call: an order-n skew matrix and where its factors go.
 * All pointers are device pointers; the array of descriptors itself is in device
 * memory too.  A is DESTROYED.  L may be NULL: the factorization is then computed
 * without storing L (Pfaffian-only use).  t has n-1 entries, piv n.
 */
typedef struct {
    int64_t n;
    double *A;
    int64_t lda;
    double *L;
    int64_t ldl;
    double *t;
    int32_t *piv;
} skew_problem;

/* Largest order skew_ltlt_batched accepts. */
#define SKEW_BATCH_MAX_N 8192

/* Device workspace of skew_ltlt_batched for `count` problems of order <= max_n. */
size_t skew_batched_workspace_bytes(int count, int max_n);

/*
 * skew_ltlt_batched -- `count` independent pivoted factorizations P A P^T = L T L^T
 * and their Pfaffians in one persistent launch: each CTA factors whole matrices
 * (the unblocked right-looking algorithm of Section 4.1, Eq. (1), with the pivoting
 * of Section 5.2), taking them largest first from a device queue.  Meant for many
 * small and medium matrices (a few hundred); results are the same as skew_ltlt's up
 * to rounding, with identical pivots.
 *
 *   1 count      number of problems, >= 0
 *   2 problems   device array of `count` descriptors
 *   3 logabs     device array [count] or NULL: log|Pf| per problem
 *   4 sign       device array [count] or NULL: sign of Pf per problem
 *   5 info       device array [count] or NULL: per problem as for skew_ltlt, or -2
 *                when its descriptor is invalid (negative or too large n, NULL
 *                pointers, short leading dimensions); that problem is skipped
 *   6 max_n      an upper bound of every n, 0 <= max_n <= SKEW_BATCH_MAX_N
 *   7 workspace  device buffer of skew_batched_workspace_bytes(count, max_n) bytes,
 *                or NULL (allocated stream-ordered by the library)
 *   8 workspace_bytes
 *   9 stream
 */
int skew_ltlt_batched(int count, const skew_problem *problems, double *logabs,
                      int32_t *sign, int32_t *info, int max_n, void *workspace,
                      size_t workspace_bytes, void *stream);

/*
 * skew_pfaffian_batched -- the Pfaffians of `count` independent skew matrices by the
 * two-step elimination of skew_pfaffian_twostep, each matrix factored in place by one
 * CTA of a persistent kernel (largest orders first): panels (8, 16 or 32 columns, per
 * order bucket from the table of skew_set_batched_nb_table) formed left-looking in
 * shared memory, one skew rank-2k update per panel on FP64 tensor cores.  Arguments as for skew_ltlt_batched, with these differences: max_n
 * <= 512; problem j's `t` (n/2 doubles, required for n >= 2) receives the pivot-block
 * entries a_i and its `piv` (n int32) the even-step exchanges; its `L` is not used;
 * info[j] = 1 + the first even k with a_(k/2) = 0 (Pf = 0), -100 for a non-finite
 * entry, -2 for a bad descriptor.
 */
int skew_pfaffian_batched(int count, const skew_problem *problems, double *logabs,
                          int32_t *sign, int32_t *info, int max_n, void *workspace,
                          size_t workspace_bytes, void *stream);


/*
 * Serving form: a continuous-batching server of factorizations / Pfaffians.
 *
 * skew_server_submit queues a request (an order-n skew matrix in device memory) and
 * returns at once with a ticket.  A worker thread of the server admits queued
 * requests in arrival order as soon as their device memory (a copy of the matrix, t,
 * piv, and L if asked for) fits in the budget; it launches admitted work on the first
 * free stream -- all admitted small requests of one kind together in one batched
 * launch, larger ones one at a time (the kinds and the calls they use are listed at
 * SKEW_SERVE_FACTORS below) -- so that requests arriving while others are on the GPU
 * are batched and run beside them on other streams.  Results (log|Pf|, sign, info,
 * and the factors t, piv, L in device memory when the request keeps them) stay
 * resident until skew_server_release.
 * The matrix a request points to must be fully written when it is submitted (its
 * producing work complete), and is read before the request completes: keep it
 * unchanged until skew_server_poll reports it done.  A request whose buffers exceed
 * the whole budget is refused with SKEW_ERR_NOMEM.  Admitted requests keep their
 * buffers until skew_server_release, so a client that submits more than the budget
 * holds must release results as it reads them: requests queued behind a full budget
 * are admitted only as memory is released (skew_server_wait on one of them times out
 * otherwise).  All calls are thread-safe.
 */
typedef struct skew_server skew_server;

/*   1 device_budget_bytes  device memory the requests' buffers may hold at once
 *   2 n_streams            concurrent launches (1 .. 64)
 *   3 small_n_max          largest order sent to the batched kernel (0 .. 8192)
 *   4 out                  the new server (on the current device) */
int skew_server_create(size_t device_budget_bytes, int n_streams, int small_n_max,
                       skew_server **out);

/* What a request asks for (argument 5 of skew_server_submit):
 *   SKEW_SERVE_FACTORS    log|Pf|, sign, and the factors t, piv kept on the device
 *                         (the pivoted LTL^T: skew_ltlt_batched, skew_pfaffian)
 *   SKEW_SERVE_FACTORS_L  the same with L kept too (skew_ltlt_batched, skew_ltlt)
 *   SKEW_SERVE_PFAFFIAN   log|Pf| and sign only, by the two-step elimination
 *                         (skew_pfaffian_batched for orders up to min(small_n_max, 512),
 *                         else skew_pfaffian_twostep, or skew_pfaffian above its order
 *                         limit); no factors are kept: skew_server_wait returns NULL t
 *                         and piv, skew_server_copy_factors returns -3.
 * Requests of different kinds are never batched together. */
#define SKEW_SERVE_FACTORS 0
#define SKEW_SERVE_FACTORS_L 1
#define SKEW_SERVE_PFAFFIAN 2

/*   1 server, 2 n, 3 A (device, lda x n, strictly lower triangle read, not modified),
 *   4 lda, 5 mode (SKEW_SERVE_*; -5 for another value), 6 ticket (out) */
int skew_server_submit(skew_server *server, int64_t n, const double *A, int64_t lda,
                       int mode, uint64_t *ticket);

/* done = 1 once the request has completed (or failed), else 0.  -2: unknown ticket. */
int skew_server_poll(skew_server *server, uint64_t ticket, int *done);

/*
 * Wait up to timeout_s seconds (negative: no limit) for a request; then return its
 * status and, through the non-NULL pointers, log|Pf|, its sign and the info word
 * (host values), the device pointers of t, piv and L (L NULL unless kept) and the
 * latency from submission to completion in seconds.  SKEW_ERR_TIMEOUT if it has not
 * completed in time (it keeps running).
 */
int skew_server_wait(skew_server *server, uint64_t ticket, double timeout_s, double *logabs,
                     int32_t *sign, int32_t *info, const double **t, const int32_t **piv,
                     const double **L, double *latency_s);

/* Free a completed (or still queued) request's device buffers and forget the ticket.
 * SKEW_ERR_BUSY while it is admitted or running. */
int skew_server_release(skew_server *server, uint64_t ticket);

/* Copy a completed request's factors to host buffers (any of them NULL to skip):
 * t_host (n-1 values), piv_host (n), L_host (ldl x n; the request must have kept L,
 * else -5).  Synchronous.  SKEW_ERR_BUSY if the request has not completed; -3 for a
 * SKEW_SERVE_PFAFFIAN request (it keeps no factors). */
int skew_server_copy_factors(skew_server *server, uint64_t ticket, double *t_host,
                             int32_t *piv_host, double *L_host, int64_t ldl);

/* Where the latency of a finished request (not yet released) went, in seconds:
 * queued_s from submission to admission (waiting for the memory budget), waiting_s from
 * admission to the launch of its work (waiting for a free stream, or for the batch it
 * joined), running_s from that launch to the worker's observing its completion (device
 * time of its launch, which it may share with a batch, plus the worker's polling).
 * Their sum is the latency skew_server_wait reports.  Any pointer may be NULL.  Returns
 * 0, -1 / -2 for a bad server / ticket, SKEW_ERR_BUSY while the request has not
 * finished (or failed before its launch).  No counterpart in the paper. */
int skew_server_timing(skew_server *server, uint64_t ticket, double *queued_s,
                       double *waiting_s, double *running_s);

/* Budget bytes in use, requests waiting for admission, requests admitted or running. */
int skew_server_stats(skew_server *server, size_t *used_bytes, int *queued, int *in_flight);

/* Finish admitted work, drop requests never admitted, free everything. */
int skew_server_destroy(skew_server *server);

/*
 * skew_ltlt_host -- convenience form of skew_ltlt + skew_pfaffian_from_factors on
 * HOST buffers, for callers without device memory of their own.  Copies A to the
 * device, factors it on the current device, copies the results back and returns
 * when they are in host memory (synchronous).  A is not modified.  The library keeps,
 * per device, one stream and the device buffers of the largest order seen so far
 * (an n x n matrix for A, another for L when L_host is given, and O(n) more) between
 * calls; skew_trim_memory releases them.  Calls on one device are serialised.
 *   1  n
 *   2  A_host    lda x n host input (strictly lower triangle read)
 *   3  lda
 *   4  L_host    ldl x n host output, or NULL (then L is not formed on the device:
 *                the Pfaffian-only path)
 *   5  ldl
 *   6  t_host    n-1 host outputs or NULL
 *   7  piv_host  n host outputs or NULL
 *   8  logabs    host double or NULL
 *   9  sign      host int32 or NULL
 *  10  info      host int32 or NULL
 *  11  nb
 * Host buffers may be pageable or page-locked (page-locked copies are faster).  Only
 * A's lower triangle crosses the host link (in blocks of 256 columns).  A
 * page-locked L_host receives each panel's rows of L as soon as they are final (the
 * panel of their step and its row exchanges done), while later panels are factored;
 * a pageable L_host receives L after the factorization.
 */
int skew_ltlt_host(int64_t n, const double *A_host, int64_t lda, double *L_host,
                   int64_t ldl, double *t_host, int32_t *piv_host, double *logabs,
                   int32_t *sign, int32_t *info, int nb);

/*
 * skew_ltlt_host_timing -- where the time of the last completed skew_ltlt_host call
 * on the current device went, from CUDA events on its stream: the host-to-device copy
 * of A (h2d_ms), the factorization and read-off (device_ms), and the copies of the
 * results back to host memory (d2h_ms).  Any pointer may be NULL.  Returns SKEW_OK,
 * or -1 when no call has completed on this device since its buffers were created.
 * No counterpart in the paper: an instrument of the host-buffer call.
 */
int skew_ltlt_host_timing(float *h2d_ms, float *device_ms, float *d2h_ms);

#ifdef __cplusplus
}
#endif

#endif /* SKEWLTLT_H */
