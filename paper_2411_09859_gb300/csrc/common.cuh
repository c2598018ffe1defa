// common.cuh -- internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "skewltlt.h"

namespace skew {

// ------------------------------------------------------------------ host bookkeeping
void note_launches(uint64_t count);           // adds to skew_kernel_launches()
void set_last_error(cudaError_t e);           // records for skew_last_error()
int check_launch();                           // cudaGetLastError -> SKEW_OK / ERR_CUDA

#define SKEW_TRY(call)                                     \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) {                           \
            ::skew::set_last_error(e_);                    \
            return SKEW_ERR_CUDA;                          \
        }                                                  \
    } while (0)

#define SKEW_TRY_STATUS(expr)                              \
    do {                                                   \
        int s_ = (expr);                                   \
        if (s_ != SKEW_OK) return s_;                      \
    } while (0)

struct DeviceInfo {
    int device;
    int sms;              // multiprocessors
    int panel_grid_max;   // co-resident CTAs of the panel kernel (cooperative limit)
    int cluster_ok;       // clusters of 16 panel CTAs can be resident (cluster panel)
    int cluster_la_ok;    // the same for the look-ahead cluster panel
};
// Properties of the current device; SKEW_ERR_NODEVICE unless it is an sm_103 part.
int current_device_info(DeviceInfo *out);

// Stream-ordered allocation from the library's private pool of the current device
// (freed blocks stay reserved for reuse); release with cudaFreeAsync.
int pool_alloc(void **p, size_t bytes, cudaStream_t st);

// ------------------------------------------------------------------ device control block
// Lives at the start of every workspace.  Zeroed (cudaMemsetAsync) at the start of
// each factorization.
constexpr int kPanelThreads = 256;
constexpr int kMaxPanelGrid = 256;      // >= SMs of the part (152 on GB300)
constexpr int kMaxNb = 256;

struct Ctrl {
    unsigned int bar_count;   // grid barrier: CTAs arrived in the current round
    unsigned int bar_gen;     // grid barrier: completed rounds
    int err;                  // first device-detected error status (0 = none)
    int pad0;
    double vtop[2];           // panel: v[k+1] of step k (slot k & 1), before the exchange
    double pad1[4];
    double rowp[2][kMaxNb];   // panel: L[k+1, k0+1..k] of step k (slot k & 1)
    int physp[2][4];          // look-ahead panel: source index and panel-start position
                              // of row k+1 of step k (slot k & 1)
    double vnext[2];          // two-step panel: v[k+2] of pair step j (slot j & 1)
    double rowq[2][kMaxNb];   // two-step panel: stored row k+2 of pair step j (slot j & 1)
};

// One per panel CTA and step parity: the CTA's best candidate row of the step and
// that row's L values in the panel columns formed so far.
struct __align__(16) ArgmaxPartial {
    double val;               // signed v at the CTA's best row
    int idx;                  // that row (INT32_MAX if none)
    unsigned int tag;         // shared-memory panels: step tag; val, idx, tag are written
                              // and read together as one 128-bit access
    int aux[4];               // look-ahead panel: aux[0] = panel-start position of idx
    double row[kMaxNb];       // L[idx, k0+1 .. k]
};
constexpr int64_t kMaxOrder = int64_t(1) << 22;   // keeps every tile count below 2^31

// Workspace layout (byte offsets), see workspace_layout().
struct WsLayout {
    size_t ctrl, partials, tbuf, pivbuf, lbuf, split, total;
};
WsLayout workspace_layout(int64_t n, int nb, bool with_L, int precision = 0);
// The look-ahead factorization's workspace: the plain layout, then a second n x n
// matrix (ld n), two position maps (n int32 each), two updated columns (n doubles
// each) and, without L, a second panel buffer (n x nb).
struct LaLayout {
    WsLayout base;
    size_t mat2, maps, xs, lbuf2, total;
};
LaLayout workspace_layout_la(int64_t n, int nb, bool with_L);
// Whether skew_ltlt / skew_pfaffian take the look-ahead path for this order and width.
bool lookahead_applies(int64_t n, int nb, int precision, const DeviceInfo &di);
// The panel-width table's (or the built-in) choice of the look-ahead for order n;
// cluster_panel: the plain path's panels run as thread-block clusters.
bool lookahead_wanted(int64_t n, bool cluster_panel);

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_acq_rel_gpu() {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

__device__ __forceinline__ void st_release_u32(unsigned int *p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_i32(const int *p) {
    return *reinterpret_cast<const volatile int *>(p);
}

// Record the first device-side error (later ones are dropped).
__device__ __forceinline__ void raise_error(Ctrl *c, int status) {
    atomicCAS(&c->err, 0, status);
}

// Grid-wide barrier for a cooperative launch of `nblocks` CTAs.  `gen` is the
// caller's copy of the barrier generation (read once at kernel entry).  Every wait
// is bounded: after kBarrierTimeoutNs the CTA records SKEW_ERR_TIMEOUT and returns
// false; a CTA also returns false as soon as any error has been recorded, so all
// CTAs leave promptly.  Returns true when the barrier completed normally.
constexpr uint64_t kBarrierTimeoutNs = 2000000000ull;   // 2 s

__device__ __forceinline__ bool grid_barrier(Ctrl *c, unsigned int nblocks,
                                             unsigned int &gen,
                                             uint64_t timeout_ns = kBarrierTimeoutNs) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned int target = gen + 1;
        __threadfence();
        unsigned int arrived = atomicAdd(&c->bar_count, 1u) + 1u;
        if (arrived == nblocks) {
            atomicExch(&c->bar_count, 0u);
            __threadfence();
            st_release_u32(&c->bar_gen, target);
        } else {
            uint64_t t0 = 0;
            unsigned int polls = 0;
            while (ld_acquire_u32(&c->bar_gen) != target) {
                if (ld_volatile_i32(&c->err) != 0) { ok = 0; break; }
                if ((++polls & 255u) == 0u) {
                    uint64_t now = global_ns();
                    if (t0 == 0) t0 = now;
                    else if (now - t0 > timeout_ns) {
                        raise_error(c, SKEW_ERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        __threadfence();
        gen = target;
        if (ld_volatile_i32(&c->err) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ------------------------------------------------------------------ kernel launchers
// (each returns SKEW_OK or a negative status; they count their own launches)

// Sets L := identity (when L != nullptr), piv := 0..n-1, and flags a non-finite
// strictly-lower entry of A in ctrl->err.
int launch_prologue(int64_t n, const double *A, int64_t lda, double *L, int64_t ldl,
                    int32_t *piv, Ctrl *ctrl, cudaStream_t stream);

// One pivoted left-looking panel: steps k = k0 .. kend-1; with `with_x`, also forms
// the updated column X[kend+1:, kend].  Lp points at L column k0+1 (stride ldl).
struct PanelArgs {
    double *X;
    int64_t ldx;
    double *Lp;
    int64_t ldl;
    double *t;
    int32_t *piv;
    Ctrl *ctrl;
    ArgmaxPartial *part;
    int n, k0, kend, with_x;
};
// Picks the shared-memory panel kernel when every panel row gets its own thread on
// `sms` CTAs and the panel is at most 96 columns wide, else the global-memory one.
int launch_panel(const PanelArgs &a, int sms, cudaStream_t stream);

// CTAs of a shared-memory panel.  One CTA per 128 rows (four warps of rows: the CTA's
// FP64 gemv runs on all four schedulers of its SM, as fast as one warp per CTA on one
// scheduler, with a quarter of the CTAs in each grid-wide exchange), at most 96 CTAs
// unless more are needed for one row per thread.  Fewer CTAs mean fewer participants
// in each step's exchange (and a shorter wait for the slowest) at the price of more
// rows per CTA for the gemv.  Measured at n = 16384 (panel ms, FP64 update): 96 / 128
// / 160 / 256 rows per CTA with caps of 48 / 64 / 96 CTAs gave 110.8 / 107.5 / 107.0,
// 110.5 / 107.5 / 106.4, 111.1 / 108.1 / 106.7, 119.2 / 119.2 / 119.5 (n = 4096:
// 24.4 - 24.7 ms for 96 to 160 rows, 28.3 for 256); one CTA per 32 rows and at most
// 152 had given 117.2 ms.
constexpr int64_t kPanelGridCap = 96;
constexpr int64_t kPanelRowsPerCta = 128;
inline int64_t panel_grid(int64_t rows, int sms) {
    int64_t g = (rows + kPanelRowsPerCta - 1) / kPanelRowsPerCta;
    if (g > kPanelGridCap) g = kPanelGridCap;
    const int64_t need = (rows + kPanelThreads - 1) / kPanelThreads;
    if (g < need) g = need;
    if (g > sms) g = sms;
    if (g < 1) g = 1;
    return g;
}
int panel_max_blocks_per_sm(int *out);

// Look-ahead panel (panel_la.cu): the same steps k = k0 .. kend-1 as launch_panel, but
// run beside the trailing update of the previous panel.  It reads the unfactored block
// from S, the state BEFORE that update (left-looking over the previous panel's L
// columns kb+1 .. k0 as well as its own), never writes S, and defers its exchanges:
// position i of the current order is row/column idx(i) of S, where idx starts as
// map_prev (the previous panel's exchanges; nullptr: identity) and follows this
// panel's exchanges.  Outputs: L columns k0+1 .. kend (rows by position), t, piv,
// map_out[i] (i > k0: the position at this panel's start of what is now at i), and,
// with `with_x`, the updated column kend in xout (positions kend+1 .. n-1).
struct PanelLAArgs {
    const double *S;          // source state, lds x n, strictly lower triangle read
    int64_t lds;
    const int32_t *map_prev;  // n entries or nullptr
    const double *xprev;      // updated column k0 by position (k0+1 .. n-1), or nullptr:
                              // column k0 is read from S
    const double *Lprev;      // L columns kb+1 .. k0 (k0 - kb <= 64 of them), by position
    int64_t ldlp;
    double *Lp;               // L columns k0+1 .. kend
    int64_t ldl;
    double *t;
    int32_t *piv;
    int32_t *map_out;
    double *xout;
    Ctrl *ctrl;
    ArgmaxPartial *part;
    int n, kb, k0, kend, with_x;
    int rows_per_cta;         // 0: the rule of la_rows_per_cta; 32, 64, 128: forced
};
constexpr int kLaThreads = 128;   // at most one row per thread, at most 128 per CTA
constexpr int kLaMaxCols = 128;   // (k0 - kb) + (kend - k0) L columns in shared memory
// Whether the rows of a look-ahead panel at k0 fit one per thread on `sms` CTAs.
inline bool panel_la_fits(int64_t n, int64_t k0, int sms) {
    return n - k0 - 1 <= (int64_t)sms * kLaThreads && n < 65535;
}
int launch_panel_la(const PanelLAArgs &a, int sms, cudaStream_t stream);

// Cluster panel (panel_cluster.cu): the same panel for trailing blocks of at most
// 16 x 256 rows and width <= 96, run by one thread-block cluster of at most 16 CTAs
// that exchanges each step's candidates through distributed shared memory.
bool panel_cluster_fits(int64_t rows, int width);
int launch_panel_cluster(const PanelArgs &a, cudaStream_t stream);
int panel_cluster_supported(int *ok);
// Look-ahead panel as one cluster (panel_la_cluster.cu): trailing blocks of at most
// 16 x 256 rows and at most 96 L columns over both blocks.
bool panel_la_cluster_fits(int64_t rows, int cols);
int launch_panel_la_cluster(const PanelLAArgs &a, cudaStream_t stream);
int panel_la_cluster_supported(int *ok);
// Whether the plain path uses the cluster panel where it fits (skew_set_cluster_panel).
bool cluster_panel_enabled();

// Row exchanges piv[k+1] <-> k+1, k = k0 .. kend-1 in order, on L columns 1 .. k0.
int launch_pivot_rows(int64_t n, double *L, int64_t ldl, const int32_t *piv, int k0,
                      int kend, cudaStream_t stream);

// Trailing update kinds of the skew rank-2k tile kernel.
enum class PairKind { Rank2k = 0, Tridiag = 1, Fused = 2 };
struct Skr2kArgs {
    int64_t m;             // order of the updated skew block C
    double *C;
    int64_t ldc;
    // Out of place (Cin != nullptr): the old C is read from the skew matrix Cin
    // (ldcin), entry (i, j) of C being entry (map[i], map[j]) of Cin (lower storage,
    // negated when map[i] < map[j]); C is only written.
    const double *Cin = nullptr;
    int64_t ldcin = 0;
    const int32_t *map = nullptr;
    int64_t nin = 0;       // order of Cin: map entries outside [0, nin) read as 0
    int balance = 0;       // split precision: balance each pair by powers of two first
    double alpha, beta;    // C := beta C + alpha * sum_p (a_p w_p^T - w_p a_p^T)
    const double *P;       // Rank2k: the a columns; Tridiag/Fused: the A columns
    int64_t ldp;
    const double *Q;       // Rank2k: the w columns
    int64_t ldq;
    const double *tt;      // Tridiag/Fused: sub-diagonal of T (b-1 values)
    const double *x;       // Fused: the updated column x (m values)
    int64_t b;             // Rank2k: k; Tridiag/Fused: number of A columns
};
int launch_skr2k(PairKind kind, const Skr2kArgs &a, cudaStream_t stream);

// Split-precision variant (skr2k_split.cu): at most 32 pairs; `scratch` holds
// split_scratch_bytes(m) bytes (digit slices and row exponents); a timed-out wait is
// recorded in *err (may be null); `sms` = multiprocessors of the device.
size_t split_scratch_bytes(int64_t m);
int launch_skr2k_split(PairKind kind, const Skr2kArgs &a, void *scratch, int *err, int sms,
                       cudaStream_t stream);

// Two-step (Pfaffian-only) panel (twostep.cu): pairs at columns k = k0, k0+2, ... <
// kend (and k + 1 < n).  V (ldv x (kend-k0)) receives l_j (column 2j) and y_j
// (column 2j+1) of pair j for rows k+2 .. n-1; a[k/2] and piv[k+1] are written.
struct TwoStepArgs {
    double *X;
    int64_t ldx;
    double *V;
    int64_t ldv;
    double *a;
    int32_t *piv;
    Ctrl *ctrl;
    ArgmaxPartial *part;
    int n, k0, kend;
};
// Returns SKEW_ERR_CUDA if the rows do not fit the shared-memory organisation
// (n - k0 - 1 > sms * kPanelThreads or kend - k0 > 96); callers check first.
int launch_twostep_panel(const TwoStepArgs &a, int sms, cudaStream_t stream);
bool twostep_fits(int64_t n, int nb, int sms);
// log|Pf| = sum log|a_j|, sign = det(P) prod sign(-a_j); info as for the one-step path
// but over the a_j (1 + the first even k with a[k/2] == 0).
int launch_finish_twostep(int64_t n, const double *a, const int32_t *piv, const Ctrl *ctrl,
                          double *logabs, int32_t *sign, int32_t *info, cudaStream_t stream);

// Panel width and update warp tile of the CTA-local batched kernels per order bucket:
// n <= n_upper[i] takes nb[i] (8, 16 or 32) and wt[i] (16 or 32: each warp of the
// trailing update owns a wt x wt tile of the lower triangle; first match), larger
// orders the last entry; count 0: width 16, warp tile 32.  `threads` (one value for a
// launch) is the CTA size of the blocked kernels, 256 or 128: with 128 a
// multiprocessor holds more matrices at once when shared memory allows it.
struct BatchedNb {
    int count;
    int n_upper[8];
    int nb[8];
    int wt[8];
    int threads;          // threads per CTA of the blocked batched kernels: 256 or 128
};
__host__ __device__ inline int batched_nb_for(const BatchedNb &t, int n) {
    for (int i = 0; i < t.count; ++i)
        if (n <= t.n_upper[i]) return t.nb[i];
    return t.count > 0 ? t.nb[t.count - 1] : 16;
}
__host__ __device__ inline int batched_wt_for(const BatchedNb &t, int n) {
    for (int i = 0; i < t.count; ++i)
        if (n <= t.n_upper[i]) return t.wt[i];
    return t.count > 0 ? t.wt[t.count - 1] : 32;
}
BatchedNb batched_nb_table();     // the table installed by skew_set_batched_nb_table

// Batched persistent factorization (batched.cu).
size_t batched_workspace_bytes(int count, int max_n);
int launch_batched(int count, const skew_problem *problems, double *logabs, int32_t *sign,
                   int32_t *info, int max_n, void *ws, cudaStream_t stream, int sms);
// Pfaffian-only batched variant (two-step elimination), max_n <= 512.
int launch_batched_twostep(int count, const skew_problem *problems, double *logabs,
                           int32_t *sign, int32_t *info, int max_n, void *ws,
                           cudaStream_t stream, int sms);

// Self-test of the bounded waits: `blocks` CTAs enter a grid barrier that expects one
// more CTA than launched, so it can only end by its time limit.
int launch_selftest_wait(Ctrl *ctrl, int blocks, uint64_t timeout_ns, cudaStream_t stream);
// Self-test of the bounded mbarrier wait of the tensor-core kernels (no arrival ever).
int launch_selftest_mbar(int *err, uint64_t timeout_ns, cudaStream_t stream);

// log|Pf|, sign (either may be null), and the final info word (may be null).
int launch_finish(int64_t n, const double *t, const int32_t *piv, const Ctrl *ctrl,
                  double *logabs, int32_t *sign, int32_t *info, cudaStream_t stream);

}  // namespace skew
