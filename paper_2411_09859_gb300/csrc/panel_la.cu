// panel_la.cu -- the pivoted left-looking panel run beside the previous panel's
// trailing update (look-ahead).
//
// Section 5.2: the panel of the pivoted blocked right-looking algorithm must be
// left-looking, since pivoting can bring any column of the unfactored matrix into it.
// The left-looking column of step k,
//
//     v = X[k+1:, k] - L[k+1:, kb+1 .. k] h,   h_q = t[q-1] L[k, q-1] [q-1 > kb]
//                                                    - t[q] L[k, q+1] [q+1 <= k]
//
// (h = T L[k, :]^T, skew_tridiag_gemv, Section 4.2 "Left-looking"), holds for any kb
// at which X is the state after the Gauss transforms of columns <= kb.  The ordinary
// panel takes kb = k0, the state after the previous panel's trailing update.  This
// kernel takes kb = the previous panel's k0, i.e. the state S BEFORE the previous
// trailing update, and adds the previous panel's L columns to the gemv.  Nothing it
// reads is written by that update, which runs at the same time on another stream and
// writes its result into a second buffer.
//
// With pivoting the panel also exchanges indices k+1 and r of the unfactored matrix at
// every step.  Here S is never written: the exchanges are kept as a map from the
// current position i to the row/column idx(i) of S (the previous panel's map, then
// this panel's exchanges), and X[i, j] is read as S[idx(i), idx(j)] (lower storage,
// negated above the diagonal).  The exchanges reach the matrix when the next trailing
// update reads S through the combined map (skr2k, out of place).
//
// Organisation as in the shared-memory panel of panel.cu: one row per thread for the
// whole panel (rows dealt to CTAs in 32-row chunks), the row's L values over both
// panels in shared memory, v in a register, and one grid-wide exchange per step in
// which every CTA publishes its best candidate with a release-stored step tag.  The
// candidate record also carries the source index of the candidate row (16 bits, with
// 16 bits of position), so that every CTA knows which column of S the next step reads
// as soon as the exchange completes.
#include <cfloat>
#include <climits>

#include "argmax.cuh"
#include "common.cuh"

namespace skew {
namespace {

constexpr unsigned int kNoIdx = 0xffffu;

// X[a, c] of the skew matrix held in the strictly lower triangle of S (a != c)
__device__ __forceinline__ double skew_at(const double *S, int64_t lds, int a, int c) {
    return a > c ? __ldg(S + a + (int64_t)c * lds) : -__ldg(S + c + (int64_t)a * lds);
}

__global__ void __launch_bounds__(kLaThreads)
panel_la_kernel(PanelLAArgs a) {
    extern __shared__ double s_L[];          // [c][tid]: L column kb+1+c of this thread's row
    __shared__ double s_h[kLaMaxCols + 1];   // h of the next step, index q - kb - 1
    __shared__ double s_t[kLaMaxCols + 1];   // t[c], index c - kb
    __shared__ double s_w[kLaMaxCols + 1];   // new row k+1 of L (old row r), index c - kb - 1
    __shared__ double s_rp[kLaMaxCols + 1];  // new row r of L (old row k+1)
    __shared__ unsigned long long s_wraw[kLaThreads / 32];
    __shared__ int s_wi[kLaThreads / 32];
    __shared__ unsigned int s_wc[kLaThreads / 32];
    __shared__ double s_tau, s_vtop;
    __shared__ int s_r, s_win, s_fail, s_psr, s_psp, s_por, s_pop;
    __shared__ unsigned int s_base;

    Ctrl *ctrl = a.ctrl;
    const int n = a.n, kb = a.kb, k0 = a.k0, kend = a.kend;
    const int nbj = k0 - kb;                 // L columns of the previous panel
    const int G = (int)gridDim.x;
    const int nthr = (int)blockDim.x;        // rows per CTA: 32, 64 or 128
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double *S = a.S;
    const int64_t lds = a.lds, ldl = a.ldl;
    auto Lcol = [&](int q) -> double * { return a.Lp + (int64_t)(q - k0 - 1) * ldl; };
    auto slot = [&](int k, int cta) -> ArgmaxPartial * {
        return a.part + (k & 1) * kMaxPanelGrid + cta;
    };
    auto sL = [&](int c) -> double & { return s_L[c * nthr + tid]; };

    // this thread's row: chunk warp * G + cta, lane tid % 32
    const int i = k0 + 1 + ((warp * G + (int)blockIdx.x) << 5) + lane;
    const bool own = i < n;
    auto owner_cta = [&](int row) -> int { return ((row - k0 - 1) >> 5) % G; };
    auto owner_tid = [&](int row) -> int {
        const int j = row - k0 - 1;
        return (((j >> 5) / G) << 5) + (j & 31);
    };

    if (tid == 0) {
        s_base = ld_acquire_u32(&ctrl->bar_gen);
        s_fail = ld_volatile_i32(&ctrl->err) != 0;
    }
    // source index (phs) and panel-start position (pho) of this thread's row
    int phs = 0, pho = i;
    if (own) phs = a.map_prev ? __ldg(a.map_prev + i) : i;
    for (int c = 0; c < nbj; ++c) sL(c) = own ? __ldg(a.Lprev + i + (int64_t)c * a.ldlp) : 0.0;
    for (int c = tid; c < nbj; c += nthr) s_t[c] = __ldcg(a.t + kb + c);
    __syncthreads();
    if (s_fail) {
        // an earlier stage failed: leave a valid map (the identity) for the update that
        // follows, which reads through it
        if (own && a.map_out) a.map_out[i] = i;
        return;
    }
    const unsigned int base = s_base;

    // Publish this CTA's step-k candidate (value, position, source index; its L row
    // over columns kb+1 .. k and its panel-start position), the row k+1 of L if this
    // CTA owns it, then release the step tag (one CTA barrier; warp 0 finishes).
    auto publish = [&](int k, Best best, bool nonfinite) {
        if (nonfinite) raise_error(ctrl, SKEW_ERR_NONFINITE);
        // a thread offers only its own row: the candidate's source index and
        // panel-start position (both below 2^16) ride in the CTA field of the reduction
        best.c = (int)(((unsigned int)phs << 16) | ((unsigned int)pho & 0xffffu));
        best = warp_best_all(best);
        if (lane == 0) {
            s_wraw[warp] = best.raw;
            s_wi[warp] = best.i;
            s_wc[warp] = (unsigned int)best.c;
        }
        __syncthreads();
        if (warp != 0) return;
        Best y = no_candidate();
        if (lane < nthr / 32) {
            y.raw = s_wraw[lane];
            y.i = s_wi[lane];
            y.c = (int)s_wc[lane];
        }
        y = warp_best_all(y);
        ArgmaxPartial *sp = slot(k, blockIdx.x);
        const int nq = k - kb;
        unsigned int packed = kNoIdx;
        if (y.i != INT_MAX) {
            const int ot = owner_tid(y.i);
            for (int q = lane; q < nq; q += 32) sp->row[q] = s_L[q * nthr + ot];
            if (lane == 0) sp->aux[0] = (int)((unsigned int)y.c & 0xffffu);
            packed = ((unsigned int)y.c & 0xffff0000u) | (unsigned int)y.i;
        }
        if (k + 1 < n && owner_cta(k + 1) == (int)blockIdx.x) {
            const int ot = owner_tid(k + 1);
            for (int q = lane; q < nq; q += 32) ctrl->rowp[k & 1][q] = s_L[q * nthr + ot];
        }
        __syncwarp();
        if (lane == 0) record_release(sp, y.raw, (int)packed, base + (unsigned int)(k - k0) + 1u);
    };
    // the owner of row k+1 also publishes its source index and panel-start position
    auto publish_rowp = [&](int k) {
        if (own && i == k + 1) {
            ctrl->physp[k & 1][0] = phs;
            ctrl->physp[k & 1][1] = pho;
        }
    };

    // ---------------- step k0: v = the updated column k0
    double v = 0.0;
    {
        const int k = k0;
        Best best = no_candidate();
        bool nonfinite = false;
        if (own) {
            if (a.xprev) {
                v = __ldcg(a.xprev + i);
            } else {
                const int c0 = a.map_prev ? __ldg(a.map_prev + k0) : k0;
                v = skew_at(S, lds, phs, c0);
            }
            if (i == k + 1) ctrl->vtop[k & 1] = v;
            if (!finite_bits((unsigned long long)__double_as_longlong(v))) nonfinite = true;
            offer(best, v, i);
        }
        publish_rowp(k);
        publish(k, best, nonfinite);
    }

    for (int k = k0; k < kend; ++k) {
        // ---------------- gather the step-k candidates of all CTAs (the barrier)
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
            unsigned int bsrc = 0;
            if (!fail) {
#pragma unroll
                for (int j = 0; j < kPer; ++j) {
                    const int c = lane + 32 * j;
                    if (c >= G) continue;
                    const unsigned int pos = pi[j] & 0xffffu;
                    const int ipos = pos == kNoIdx ? INT_MAX : (int)pos;
                    if (better(pv[j], ipos, b.raw, b.i)) {
                        b.raw = pv[j];
                        b.i = ipos;
                        b.c = c;
                        bsrc = pi[j] >> 16;
                    }
                }
            }
            fail = __any_sync(0xffffffffu, fail);
            // the lane holding the winner hands over its source index
            b.c = (b.c << 16) | (int)bsrc;
            b = warp_best_all(b);
            if (lane == 0) {
                s_fail = fail;
                s_r = (b.i == INT_MAX) ? k + 1 : b.i;    // all NaN: keep the diagonal
                s_tau = as_double(b.raw);
                s_win = (b.i == INT_MAX) ? -1 : (b.c >> 16);
                s_psr = b.c & 0xffff;
            }
        }
        __syncthreads();
        if (s_fail) break;           // the map written below stays a valid permutation
        const int r = s_r, p = k + 1, nq = k - kb;
        const int win = s_win;
        // source index of the new column p (old row r); with no candidate (all NaN) the
        // pivot stays and row p's own index is used
        // ---------------- one round of loads: exchanged L rows, positions, v[k+1],
        // and this thread's entry of the new column p
        if (win >= 0) {
            for (int q = tid; q < nq; q += nthr) {
                s_w[q] = __ldcg(&slot(k, win)->row[q]);
                s_rp[q] = __ldcg(&ctrl->rowp[k & 1][q]);
            }
        }
        if (tid == 0) {
            const double vt = __ldcg(&ctrl->vtop[k & 1]);
            s_vtop = vt;
            if (win < 0) s_tau = vt;
            s_psp = __ldcg(&ctrl->physp[k & 1][0]);
            s_pop = __ldcg(&ctrl->physp[k & 1][1]);
            s_por = win >= 0 ? __ldcg(&slot(k, win)->aux[0]) : 0;
        }
        __syncthreads();
        const int psr = (win >= 0) ? s_psr : s_psp;   // source index of the new column p
        const double tau = s_tau, vtop = s_vtop;
        // the new row r (old row p) takes old row p's source index and position
        if (own && i == r && r != p) {
            phs = s_psp;
            pho = s_pop;
        } else if (own && i == p && r != p) {
            phs = psr;
            pho = s_por;
        }
        double x_new = 0.0;
        if (own && i > p) x_new = skew_at(S, lds, phs, psr);
        if (tid == 0) s_t[k - kb] = tau;
        if (blockIdx.x == 0 && tid == 0) {
            a.t[k] = tau;
            a.piv[p] = r;
        }
        // exchanged rows of the L columns kb+1 .. k: new row p = old row r (s_w) in the
        // CTA owning p, new row r = old row p (s_rp) in the CTA owning r; this panel's
        // own columns also in global memory
        if (r != p && win >= 0) {
            if (owner_cta(p) == (int)blockIdx.x) {
                const int ot = owner_tid(p);
                for (int q = tid; q < nq; q += nthr) {
                    s_L[q * nthr + ot] = s_w[q];
                    if (q >= nbj) Lcol(kb + 1 + q)[p] = s_w[q];
                }
            }
            if (owner_cta(r) == (int)blockIdx.x) {
                const int ot = owner_tid(r);
                for (int q = tid; q < nq; q += nthr) {
                    s_L[q * nthr + ot] = s_rp[q];
                    if (q >= nbj) Lcol(kb + 1 + q)[r] = s_rp[q];
                }
            }
        }
        const bool next = (k + 1 < kend);
        const bool form_x = (!next && a.with_x);
        if (next || form_x) {
            // h for step k+1 from the new row p: L[p, c] = s_w[c - kb - 1] for c <= k,
            // L[p, k+1] = 1; t[c] = s_t[c - kb] for c < k, t[k] = tau
            auto tq = [&](int q) -> double { return q == k ? tau : s_t[q - kb]; };
            for (int q = kb + 1 + tid; q <= k + 1; q += nthr) {
                double hq = 0.0;
                if (q - 1 >= kb + 1) hq = tq(q - 1) * s_w[q - 2 - kb];
                if (q + 1 <= k + 1) {
                    const double lq1 = (q + 1 == k + 1) ? 1.0 : s_w[q - kb];
                    hq -= tq(q) * lq1;
                }
                s_h[q - kb - 1] = hq;
            }
        }
        __syncthreads();

        Best best = no_candidate();
        bool nonfinite = false;
        if (own && i >= p) {
            // ---- finish step k for this row: L column k+1 (own column index k - k0)
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
            if (i > p && (next || form_x)) {
                // ---- step k+1 for this row (or the updated column kend)
                double acc0 = 0.0, acc1 = 0.0;
                int q = 0;
#pragma unroll 4
                for (; q + 1 <= nq; q += 2) {
                    acc0 += sL(q) * s_h[q];
                    acc1 += sL(q + 1) * s_h[q + 1];
                }
                if (q <= nq) acc0 += sL(q) * s_h[q];
                const double vn = x_new - (acc0 + acc1);
                if (!finite_bits((unsigned long long)__double_as_longlong(vn))) nonfinite = true;
                if (form_x) {
                    a.xout[i] = vn;
                } else {
                    v = vn;
                    if (i == p + 1) ctrl->vtop[(k + 1) & 1] = vn;
                    offer(best, vn, i);
                }
            }
        }
        if (next) {
            publish_rowp(k + 1);
            publish(k + 1, best, nonfinite);
        } else if (nonfinite) {
            raise_error(ctrl, SKEW_ERR_NONFINITE);
        }
    }
    if (own && a.map_out) a.map_out[i] = pho;
    // tags of this launch were base+1 .. base+(kend-k0); the next launch starts above
    if (blockIdx.x == 0 && tid == 0) st_release_u32(&ctrl->bar_gen, base + (unsigned int)(kend - k0) + 1u);
}

}  // namespace

// Rows per CTA of the look-ahead panel (one per thread): 128, so that a CTA's FP64
// gemv runs on all four schedulers of its multiprocessor.  Measured on GB300 (look-ahead
// factorization, ms): 32 rows per CTA up to 4096 rows and 64 up to 8192 gave 61.8 ms at
// n = 4096 and 257 ms at n = 8192, against 45.5 and 228 with 128: more CTAs in the
// grid-wide exchange cost more than the shorter gemv saves.  `force` (32 or 64)
// overrides, for such measurements.
int la_rows_per_cta(int64_t rows, int force) {
    if ((force == 32 || force == 64) && rows <= (int64_t)force * kMaxPanelGrid) return force;
    return 128;
}

int launch_panel_la(const PanelLAArgs &a, int sms, cudaStream_t stream) {
    const int64_t rows = (int64_t)a.n - a.k0 - 1;
    const int cols = (a.k0 - a.kb) + (a.kend - a.k0);
    if (rows < 1 || cols > kLaMaxCols || !panel_la_fits(a.n, a.k0, sms)) return SKEW_ERR_CUDA;
    const int nthr = la_rows_per_cta(rows, a.rows_per_cta);
    int64_t g = (rows + nthr - 1) / nthr;
    if (g < 1) g = 1;
    if (g > kMaxPanelGrid) return SKEW_ERR_CUDA;        // unreachable: rows <= 128 x sms
    const size_t smem = (size_t)(cols > 0 ? cols : 1) * nthr * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute((const void *)panel_la_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kLaMaxCols * kLaThreads * sizeof(double)));
    if (e != cudaSuccess) {
        set_last_error(e);
        return SKEW_ERR_CUDA;
    }
    PanelLAArgs args = a;
    void *params[] = {&args};
    e = cudaLaunchCooperativeKernel((const void *)panel_la_kernel, dim3((unsigned)g),
                                    dim3((unsigned)nthr), params, smem, stream);
    if (e != cudaSuccess) {
        set_last_error(e);
        return SKEW_ERR_CUDA;
    }
    note_launches(1);
    return SKEW_OK;
}

}  // namespace skew
