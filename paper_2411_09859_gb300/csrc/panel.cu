// panel.cu -- pivoted left-looking panel factorization (one cooperative launch).
//
// Section 5.2 (pivoted blocked right-looking algorithm): the panel of a blocked
// right-looking factorization must be factored with the left-looking (modified
// Aasen, Section 4.2 "Left-looking") algorithm so that pivoting can bring in any
// column of the not yet updated trailing matrix.  For a panel starting at column
// k0, step k (k0 <= k < kend) forms the current column on the fly,
//
//     v = X[k+1:, k] - L[k+1:, k0+1 .. k] h,     h = T L[k, :]^T  (skew_tridiag_gemv)
//     h_q = t[q-1] L[k, q-1] [q-1 > k0] - t[q] L[k, q+1] [q+1 <= k],  L[k, k] = 1,
//
// picks r = argmax |v| (lowest index on ties), exchanges indices k+1 and r of the
// whole unfactored skew matrix (lower storage: column k+1, row r, column r, with a
// sign change for entries that cross the diagonal) and rows k+1, r of the panel's
// L columns, then sets t[k] = v[k+1] and L[k+2:, k+1] = v[k+2:] / t[k].
// Columns of L left of the panel are exchanged later (pivot_rows).
//
// GPU organisation: one cooperative launch per panel (its CTAs wait on each other at
// every step).  Every row of the unfactored block has one owner thread for the whole
// panel, so everything a step does to row i -- its exchange, its scaled L entry, and
// the next step's v_i -- is done by one thread without synchronisation.  What crosses
// rows is published at each step: every CTA writes its best candidate (|v|, index)
// together with that row's L values in the panel columns, and the owner of row k+1
// writes v[k+1] and its L row.  Once every CTA has published, each knows the pivot r,
// t[k], the new row k+1 of L (old row r) and so the next h, and goes straight on.
// The published data are double-buffered by step parity: a CTA can be at most one
// step ahead of another.  Data written inside this launch are read with ld.global.cg.
// Two variants: the shared-memory panel (the panel's L rows in shared memory, one
// thread per row, the grid sized by panel_grid) for panels of at most 96 columns whose
// rows fit one per thread, and the global-memory panel (L in global memory, rows
// strided over all threads, a grid barrier per step) for the rest.
#include <cfloat>
#include <climits>

#include "argmax.cuh"
#include "common.cuh"

namespace skew {
namespace {

__global__ void __launch_bounds__(kPanelThreads)
panel_global_kernel(PanelArgs a) {
    __shared__ double s_h[kMaxNb + 1];   // h of the next step, index q - k0 - 1
    __shared__ double s_t[kMaxNb + 1];   // t[k] of this panel, index k - k0
    __shared__ double s_w[kMaxNb + 1];   // new L row k+1 (old row r), index c - k0 - 1
    __shared__ double s_rp[kMaxNb + 1];  // new L row r (old row k+1), index c - k0 - 1
    __shared__ double s_tau, s_vtop;
    __shared__ int s_r, s_win;

    Ctrl *ctrl = a.ctrl;
    const int n = a.n, k0 = a.k0, kend = a.kend;
    const unsigned int G = gridDim.x;
    const int64_t nthreads = (int64_t)G * blockDim.x;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned int gen = 0;
    if (threadIdx.x == 0) gen = ld_acquire_u32(&ctrl->bar_gen);
    if (ld_volatile_i32(&ctrl->err) != 0) return;

    double *X = a.X;
    const int64_t ldx = a.ldx, ldl = a.ldl;
    // panel column q (k0+1 <= q <= kend) of L
    auto Lcol = [&](int q) -> double * { return a.Lp + (int64_t)(q - k0 - 1) * ldl; };
    // first row >= lo owned by this thread (rows i with i mod nthreads == gtid)
    auto first_row = [&](int64_t lo) -> int64_t {
        int64_t rem = (gtid - lo) % nthreads;
        if (rem < 0) rem += nthreads;
        return lo + rem;
    };
    auto slot = [&](int k, unsigned int cta) -> ArgmaxPartial * {
        return a.part + (k & 1) * kMaxPanelGrid + cta;
    };
    // Publish this CTA's best candidate of step k and its L row (columns k0+1..k);
    // the CTA owning row k+1 also publishes that row.  The rows are copied by all
    // threads of the CTA in parallel.
    auto publish = [&](int k, Best best, bool nonfinite) {
        if (nonfinite) raise_error(ctrl, SKEW_ERR_NONFINITE);
        best = block_best(best);
        ArgmaxPartial *sp = slot(k, blockIdx.x);
        if (threadIdx.x == 0) {
            sp->val = as_double(best.raw);
            sp->idx = best.i;
        }
        if (best.i != INT_MAX)
            for (int q = threadIdx.x; q < k - k0; q += blockDim.x)
                sp->row[q] = __ldcg(Lcol(k0 + 1 + q) + best.i);
        const int64_t pn = k + 1;
        if (pn < n && (pn % nthreads) / blockDim.x == blockIdx.x)
            for (int q = threadIdx.x; q < k - k0; q += blockDim.x)
                ctrl->rowp[k & 1][q] = __ldcg(Lcol(k0 + 1 + q) + pn);
    };

    // ---------------- step k0: v = X[k0+1:, k0] (no panel column formed yet)
    {
        const int k = k0;
        double *vcol = Lcol(k + 1);
        const double *xk = X + (int64_t)k * ldx;
        Best best = no_candidate();
        bool nonfinite = false;
        for (int64_t i = first_row(k + 1); i < n; i += nthreads) {
            const double v = __ldcg(xk + i);
            vcol[i] = v;
            if (i == k + 1) ctrl->vtop[k & 1] = v;
            if (!isfinite(v)) nonfinite = true;
            offer(best, v, (int)i);
        }
        best.c = blockIdx.x;
        publish(k, best, nonfinite);
    }

    for (int k = k0; k < kend; ++k) {
        if (!grid_barrier(ctrl, G, gen)) return;

        // ---------------- pivot of step k: global argmax over the published partials
        if (threadIdx.x < 32) {
            Best b = no_candidate();
            for (unsigned int c = threadIdx.x; c < G; c += 32) {
                const ArgmaxPartial *sp = slot(k, c);
                const unsigned long long pr = (unsigned long long)__double_as_longlong(__ldcg(&sp->val));
                const int pi = __ldcg(&sp->idx);
                if (better(pr, pi, b.raw, b.i)) { b.raw = pr; b.i = pi; b.c = (int)c; }
            }
            b = warp_best(b);
            if (threadIdx.x == 0) {
                const double vt = __ldcg(&ctrl->vtop[k & 1]);
                s_vtop = vt;
                s_r = (b.i == INT_MAX) ? k + 1 : b.i;    // all NaN: keep the diagonal
                s_tau = (b.i == INT_MAX) ? vt : as_double(b.raw);
                s_win = (b.i == INT_MAX) ? -1 : b.c;
            }
        }
        __syncthreads();
        const int r = s_r, p = k + 1, nq = k - k0;
        const double tau = s_tau, vtop = s_vtop;
        // exchanged rows of L in the formed panel columns: new row p = old row r (the
        // winner's published row), new row r = old row p (published by its owner)
        if (s_win >= 0)
            for (int q = threadIdx.x; q < nq; q += blockDim.x) {
                s_w[q] = __ldcg(&slot(k, s_win)->row[q]);
                s_rp[q] = __ldcg(&ctrl->rowp[k & 1][q]);
            }
        if (threadIdx.x == 0) s_t[k - k0] = tau;
        if (gtid == 0) {
            a.t[k] = tau;
            a.piv[p] = r;
        }
        __syncthreads();

        const bool next = (k + 1 < kend);          // another step of this panel follows
        const bool form_x = (!next && a.with_x);   // last step: form column kend instead
        const int nqn = nq + 1;                     // panel columns k0+1 .. k+1
        if (next || form_x) {
            // h for step k+1 from the new row k+1 of L: L[k+1, c] = s_w[c-k0-1] for
            // c <= k and L[k+1, k+1] = 1
            for (int q = k0 + 1 + threadIdx.x; q <= k + 1; q += blockDim.x) {
                double hq = 0.0;
                if (q - 1 >= k0 + 1) hq = s_t[q - 1 - k0] * s_w[q - 2 - k0];
                if (q + 1 <= k + 1) {
                    const double lq1 = (q + 1 == k + 1) ? 1.0 : s_w[q - k0];
                    hq -= s_t[q - k0] * lq1;
                }
                s_h[q - k0 - 1] = hq;
            }
        }
        __syncthreads();

        double *vcol = Lcol(k + 1);                 // v of step k, parked in L column k+1
        double *vnext = next ? Lcol(k + 2) : nullptr;
        double *colp = X + (int64_t)p * ldx;
        Best best = no_candidate();
        bool nonfinite = false;
        for (int64_t i = first_row(p); i < n; i += nthreads) {
            // ---- finish step k for row i
            if (i == p) {
                vcol[i] = 1.0;
                if (r != p)
                    for (int q = 0; q < nq; ++q) Lcol(k0 + 1 + q)[i] = s_w[q];
            } else {
                const double v = (i == r) ? vtop : __ldcg(vcol + i);
                vcol[i] = (tau != 0.0) ? v / tau : 0.0;
                if (i == r)
                    for (int q = 0; q < nq; ++q) Lcol(k0 + 1 + q)[i] = s_rp[q];
            }
            if (r != p && i > p) {
                // symmetric exchange of indices p and r in the strictly lower storage
                if (i < r) {
                    double *xri = X + i * ldx + r;          // X[r, i]
                    const double tmp = __ldcg(colp + i);
                    colp[i] = -__ldcg(xri);
                    *xri = -tmp;
                } else if (i == r) {
                    colp[i] = -__ldcg(colp + i);
                } else {
                    double *colr = X + (int64_t)r * ldx;
                    const double tmp = __ldcg(colp + i);
                    colp[i] = __ldcg(colr + i);
                    colr[i] = tmp;
                }
            }
            // ---- step k+1 for row i (or the updated column kend at the last step)
            if ((next || form_x) && i > p) {
                double acc0 = 0.0, acc1 = 0.0;
                int q = 0;
#pragma unroll 4
                for (; q + 1 < nqn; q += 2) {
                    acc0 += __ldcg(a.Lp + (int64_t)q * ldl + i) * s_h[q];
                    acc1 += __ldcg(a.Lp + (int64_t)(q + 1) * ldl + i) * s_h[q + 1];
                }
                if (q < nqn) acc0 += __ldcg(a.Lp + (int64_t)q * ldl + i) * s_h[q];
                const double v = __ldcg(colp + i) - (acc0 + acc1);
                if (!isfinite(v)) nonfinite = true;
                if (form_x) {
                    colp[i] = v;
                } else {
                    vnext[i] = v;
                    if (i == p + 1) ctrl->vtop[(k + 1) & 1] = v;
                    offer(best, v, (int)i);
                }
            }
        }
        if (next) {
            best.c = blockIdx.x;
            publish(k + 1, best, nonfinite);
        } else if (nonfinite) {
            raise_error(ctrl, SKEW_ERR_NONFINITE);
        }
    }
}


// ------------------------------------------------------------------------------------
// Shared-memory panel: used when every row of the panel has its own thread
// (n - k0 - 1 <= #CTAs x 256) and the panel is at most kSmemMaxNb wide.  Each thread
// keeps its row of the panel's L columns in shared memory, so the per-step
// skew_tridiag_gemv reads no global memory, and the v of its row in a register.
// There is no separate grid barrier: each CTA publishes its step-k partial with a
// release store of a step tag, and every CTA's warp 0 acquires all G tags -- the
// gather of the argmax candidates is the barrier.  Rows are dealt to CTAs in chunks
// of 32 (one warp) round-robin, so the rows of a step are spread over all the panel's
// CTAs and each warp's accesses to a column are coalesced.
// ------------------------------------------------------------------------------------
constexpr int kSmemMaxNb = 96;
constexpr int kSmemLds = kPanelThreads + 1;   // s_L column stride: a row's entries in distinct banks

__global__ void __launch_bounds__(kPanelThreads)
panel_smem_kernel(PanelArgs a) {
    extern __shared__ double s_L[];          // [q * kSmemLds + threadIdx.x], q < kend - k0
    __shared__ double s_h[kSmemMaxNb + 1];   // h of the next step, index q - k0 - 1
    __shared__ double s_t[kSmemMaxNb + 1];   // t[k] of this panel, index k - k0
    __shared__ double s_w[kSmemMaxNb + 1];   // new L row k+1 (old row r), index c - k0 - 1
    __shared__ double s_rp[kSmemMaxNb + 1];  // new L row r (old row k+1)
    __shared__ unsigned long long s_wraw[kPanelThreads / 32];   // per-warp candidates
    __shared__ int s_wi[kPanelThreads / 32];
    __shared__ double s_tau, s_vtop;
    __shared__ int s_r, s_win, s_fail;
    __shared__ unsigned int s_base;

    Ctrl *ctrl = a.ctrl;
    const int n = a.n, k0 = a.k0, kend = a.kend;
    const int G = (int)gridDim.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double *X = a.X;
    const int64_t ldx = a.ldx, ldl = a.ldl;
    auto Lcol = [&](int q) -> double * { return a.Lp + (int64_t)(q - k0 - 1) * ldl; };
    auto slot = [&](int k, int cta) -> ArgmaxPartial * {
        return a.part + (k & 1) * kMaxPanelGrid + cta;
    };
    auto sL = [&](int q) -> double & { return s_L[q * kSmemLds + tid]; };

    // this thread's row: chunk (tid / 32) * G + cta, lane tid % 32
    const int64_t i = (int64_t)k0 + 1 + ((int64_t)((tid >> 5) * G + (int)blockIdx.x) << 5) + (tid & 31);
    const bool own = i < n;

    if (tid == 0) {
        s_base = ld_acquire_u32(&ctrl->bar_gen);
        s_fail = ld_volatile_i32(&ctrl->err) != 0;
    }
    __syncthreads();
    if (s_fail) return;
    const unsigned int base = s_base;

    // CTA and thread that own row `row` (k0 < row < n; 32-bit index arithmetic)
    auto owner_cta = [&](int row) -> int { return ((row - k0 - 1) >> 5) % G; };
    auto owner_tid = [&](int row) -> int {
        const int j = row - k0 - 1;
        return (((j >> 5) / G) << 5) + (j & 31);
    };

    // Publish this CTA's step-k candidate (and its L row), the row k+1 of L if this
    // CTA owns row k+1, then release the step tag.  One CTA barrier: every warp leaves
    // its best candidate in shared memory, then warp 0 alone finishes the reduction,
    // copies the rows from shared memory and releases, while the other warps go on to
    // wait for the next step's gather.
    auto publish = [&](int k, Best best, bool nonfinite) {
        if (nonfinite) raise_error(ctrl, SKEW_ERR_NONFINITE);
        best = warp_best_all(best);
        if (lane == 0) {
            s_wraw[warp] = best.raw;
            s_wi[warp] = best.i;
        }
        __syncthreads();
        if (warp != 0) return;
        Best y = no_candidate();
        if (lane < kPanelThreads / 32) {
            y.raw = s_wraw[lane];
            y.i = s_wi[lane];
        }
        y = warp_best_all(y);
        ArgmaxPartial *sp = slot(k, blockIdx.x);
        const int nq = k - k0;
        if (y.i != INT_MAX) {
            const int ot = owner_tid(y.i);
            for (int q = lane; q < nq; q += 32) sp->row[q] = s_L[q * kSmemLds + ot];
        }
        if (k + 1 < n && owner_cta(k + 1) == (int)blockIdx.x) {
            const int ot = owner_tid(k + 1);
            for (int q = lane; q < nq; q += 32) ctrl->rowp[k & 1][q] = s_L[q * kSmemLds + ot];
        }
        // release: the CTA's writes before the barrier and warp 0's copies (ordered by
        // __syncwarp) become visible to any CTA that sees the tag; candidate and tag
        // in one 128-bit store
        __syncwarp();
        if (lane == 0) record_release(sp, y.raw, y.i, base + (unsigned int)(k - k0) + 1u);
    };

    // ---------------- step k0: v = X[k0+1:, k0]
    double v = 0.0;
    {
        const int k = k0;
        Best best = no_candidate();
        bool nonfinite = false;
        if (own) {
            v = __ldcg(X + (int64_t)k * ldx + i);
            if (i == k + 1) ctrl->vtop[k & 1] = v;
            if (!finite_bits((unsigned long long)__double_as_longlong(v))) nonfinite = true;
            offer(best, v, (int)i);
        }
        best.c = blockIdx.x;
        publish(k, best, nonfinite);
    }

    for (int k = k0; k < kend; ++k) {
        // ---------------- gather the step-k candidates of all CTAs (the barrier).
        // Lane l of warp 0 watches slots l, l+32, ...: one 128-bit relaxed load per
        // slot returns candidate and tag together, all slots of a pass in flight at once.
        if (warp == 0) {
            constexpr int kPer = kMaxPanelGrid / 32;
            const unsigned int want = base + (unsigned int)(k - k0) + 1u;
            unsigned int pending = 0;
#pragma unroll
            for (int j = 0; j < kPer; ++j)
                if (lane + 32 * j < G) pending |= 1u << j;
            int fail = 0;
            uint64_t t0 = 0;
            unsigned int polls = 0;
            // relaxed loads (acquire loads would serialise); the fence after the loop
            // turns the observed tags into an acquire
            unsigned long long pv[kPer];
            unsigned int pi[kPer];
            while (pending != 0u) {
#pragma unroll
                for (int j = 0; j < kPer; ++j)
                    if ((pending >> j) & 1u) {
                        unsigned long long rv;
                        unsigned int ri, rt;
                        record_poll(slot(k, lane + 32 * j), rv, ri, rt);
                        if (rt == want) {
                            pending &= ~(1u << j);
                            pv[j] = rv;
                            pi[j] = ri;
                        }
                    }
                if (pending == 0u) break;
                // the error word and the clock are looked at every 16th pass only, so
                // that a pass is one round of loads
                if ((++polls & 15u) == 0u) {
                    if (ld_volatile_i32(&ctrl->err) != 0) { fail = 1; break; }
                    const uint64_t now = global_ns();
                    if (t0 == 0) t0 = now;
                    else if (now - t0 > kBarrierTimeoutNs) {
                        raise_error(ctrl, SKEW_ERR_TIMEOUT);
                        fail = 1;
                        break;
                    }
                }
            }
            fence_acq_rel_gpu();
            Best b = no_candidate();
            if (!fail) {
#pragma unroll
                for (int j = 0; j < kPer; ++j) {
                    const int c = lane + 32 * j;
                    if (c < G && better(pv[j], (int)pi[j], b.raw, b.i)) {
                        b.raw = pv[j];
                        b.i = (int)pi[j];
                        b.c = c;
                    }
                }
            }
            fail = __any_sync(0xffffffffu, fail);
            b = warp_best_all(b);
            if (lane == 0) {
                s_fail = fail;
                s_r = (b.i == INT_MAX) ? k + 1 : b.i;    // all NaN: keep the diagonal
                s_tau = as_double(b.raw);
                s_win = (b.i == INT_MAX) ? -1 : b.c;
            }
        }
        __syncthreads();
        if (s_fail) return;
        const int r = s_r, p = k + 1, nq = k - k0;

        // ---------------- one round of loads: exchanged L rows, v[k+1], own X entries
        if (s_win >= 0)
            for (int q = tid; q < nq; q += blockDim.x) {
                s_w[q] = __ldcg(&slot(k, s_win)->row[q]);
                s_rp[q] = __ldcg(&ctrl->rowp[k & 1][q]);
            }
        if (tid == 0) {
            const double vt = __ldcg(&ctrl->vtop[k & 1]);
            s_vtop = vt;
            if (s_win < 0) s_tau = vt;
        }
        double *colp = X + (int64_t)p * ldx;
        double x_old = 0.0, xe = 0.0;
        if (own && i > p) {
            x_old = __ldcg(colp + i);
            if (r != p) {
                if (i < r) xe = __ldcg(X + i * ldx + r);                 // X[r, i]
                else if (i > r) xe = __ldcg(X + (int64_t)r * ldx + i);   // X[i, r]
            }
        }
        __syncthreads();
        const double tau = s_tau, vtop = s_vtop;
        // s_t[k - k0] is first read at the next step (after more barriers); this
        // step's h takes tau from the register
        if (tid == 0) s_t[k - k0] = tau;
        if (blockIdx.x == 0 && tid == 0) {
            a.t[k] = tau;
            a.piv[p] = r;
        }

        // exchanged rows of the panel's L columns k0+1..k: new row p = old row r (s_w)
        // in the CTA owning p, new row r = old row p (s_rp) in the CTA owning r
        if (r != p && s_win >= 0) {
            if (owner_cta(p) == (int)blockIdx.x) {
                const int ot = owner_tid(p);
                for (int q = tid; q < nq; q += blockDim.x) {
                    s_L[q * kSmemLds + ot] = s_w[q];
                    Lcol(k0 + 1 + q)[p] = s_w[q];
                }
            }
            if (owner_cta(r) == (int)blockIdx.x) {
                const int ot = owner_tid(r);
                for (int q = tid; q < nq; q += blockDim.x) {
                    s_L[q * kSmemLds + ot] = s_rp[q];
                    Lcol(k0 + 1 + q)[r] = s_rp[q];
                }
            }
        }
        const bool next = (k + 1 < kend);
        const bool form_x = (!next && a.with_x);
        if (next || form_x) {
            auto tq = [&](int q) -> double { return q == k ? tau : s_t[q - k0]; };
            for (int q = k0 + 1 + tid; q <= k + 1; q += blockDim.x) {
                double hq = 0.0;
                if (q - 1 >= k0 + 1) hq = tq(q - 1) * s_w[q - 2 - k0];
                if (q + 1 <= k + 1) {
                    const double lq1 = (q + 1 == k + 1) ? 1.0 : s_w[q - k0];
                    hq -= tq(q) * lq1;
                }
                s_h[q - k0 - 1] = hq;
            }
        }
        __syncthreads();

        Best best = no_candidate();
        bool nonfinite = false;
        if (own && i >= p) {
            // ---- finish step k for this row: L column k+1 and the exchanged rows
            double *lk1 = Lcol(k + 1) + i;
            if (i == p) {
                sL(nq) = 1.0;
                *lk1 = 1.0;
            } else {
                const double val = (i == r) ? vtop : v;
                const double l = (tau != 0.0) ? val / tau : 0.0;
                sL(nq) = l;
                *lk1 = l;
            }
            if (i > p) {
                // ---- the gemv of step k+1 first: it needs no global data, so the
                // loads of x_old and xe are still in flight while it runs
                double acc0 = 0.0, acc1 = 0.0;
                if (next || form_x) {
                    int q = 0;
#pragma unroll 4
                    for (; q + 1 <= nq; q += 2) {
                        acc0 += sL(q) * s_h[q];
                        acc1 += sL(q + 1) * s_h[q + 1];
                    }
                    if (q <= nq) acc0 += sL(q) * s_h[q];
                }
                // ---- symmetric exchange of p and r in the strictly lower storage
                // (the new column p itself is not stored: it only enters v below, and
                // no later step of the panel reads column p)
                double xn = x_old;                        // new X[i, p]
                if (r != p) {
                    if (i < r) {
                        xn = -xe;
                        X[i * ldx + r] = -x_old;          // X[r, i]
                    } else if (i == r) {
                        xn = -x_old;
                    } else {
                        xn = xe;
                        X[(int64_t)r * ldx + i] = x_old;  // X[i, r]
                    }
                }
                // ---- step k+1 for this row (or the updated column kend)
                if (next || form_x) {
                    const double vn = xn - (acc0 + acc1);
                    if (!finite_bits((unsigned long long)__double_as_longlong(vn))) nonfinite = true;
                    if (form_x) {
                        colp[i] = vn;
                    } else {
                        v = vn;
                        if (i == p + 1) ctrl->vtop[(k + 1) & 1] = vn;
                        offer(best, vn, (int)i);
                    }
                }
            }
        }
        if (next) {
            best.c = blockIdx.x;
            publish(k + 1, best, nonfinite);
        } else if (nonfinite) {
            raise_error(ctrl, SKEW_ERR_NONFINITE);
        }
    }
    // tags of this launch were base+1 .. base+(kend-k0); the next launch starts above
    if (blockIdx.x == 0 && tid == 0) st_release_u32(&ctrl->bar_gen, base + (unsigned int)(kend - k0) + 1u);
}

}  // namespace

int launch_panel(const PanelArgs &a, int sms, cudaStream_t stream) {
    PanelArgs args = a;
    void *params[] = {&args};
    const int64_t rows = (int64_t)a.n - a.k0 - 1;
    const int width = a.kend - a.k0;
    cudaError_t e;
    if (width <= kSmemMaxNb && rows <= (int64_t)sms * kPanelThreads) {
        const int64_t g = panel_grid(rows, sms);
        // (the dynamic shared-memory limit was raised when the device was first used,
        // in panel_max_blocks_per_sm)
        const size_t smem = (size_t)width * kSmemLds * sizeof(double);
        e = cudaLaunchCooperativeKernel((const void *)panel_smem_kernel, dim3((unsigned)g),
                                        dim3(kPanelThreads), params, smem, stream);
    } else {
        int64_t g = (a.n + 127) / 128;
        if (g > sms) g = sms;
        if (g < 1) g = 1;
        e = cudaLaunchCooperativeKernel((const void *)panel_global_kernel, dim3((unsigned)g),
                                        dim3(kPanelThreads), params, 0, stream);
    }
    if (e != cudaSuccess) {
        set_last_error(e);
        return SKEW_ERR_CUDA;
    }
    note_launches(1);
    return SKEW_OK;
}

int panel_max_blocks_per_sm(int *out) {
    int a = 0, b = 0;
    cudaError_t e = cudaFuncSetAttribute((const void *)panel_smem_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kSmemMaxNb * kSmemLds * sizeof(double)));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, panel_global_kernel,
                                                          kPanelThreads, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &b, panel_smem_kernel, kPanelThreads, kSmemMaxNb * kSmemLds * sizeof(double));
    if (e != cudaSuccess) {
        set_last_error(e);
        return SKEW_ERR_CUDA;
    }
    *out = a < b ? a : b;
    return SKEW_OK;
}

}  // namespace skew
