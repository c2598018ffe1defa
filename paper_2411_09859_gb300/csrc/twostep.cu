// twostep.cu -- Pfaffian-only factorization: the two-step elimination with pivoting
// at the even steps only (Wimmer's algorithm, as described in the notes to the
// two-step right-looking algorithm of Section 4.1: the second Gauss transform of
// each step, l_43, and tau_32 are skipped, since only every other sub-diagonal
// element of T enters the Pfaffian), blocked: left-looking inside a panel, one skew
// rank-2k trailing update per panel.
//
// Each pair of columns (k, k+1) is removed by the Schur complement of its 2 x 2 skew
// pivot block: X[k+2:, k+2:] += l y^T - y l^T with l = X[k+2:, k] / a,
// y = X[k+2:, k+1], a = X[k+1, k] after the exchange k+1 <-> r; Pf(X) =
// det(P) prod (-a).  Inside a panel starting at column k0 the current matrix is the
// stored X plus the panel's terms, X + sum_q (l_q y_q^T - y_q l_q^T), so pair j at
// column k = k0 + 2j reads
//   v   = X[:, k]   + sum_{q<j} (l_q y_q[k]   - y_q l_q[k])      (formed the step before)
//   y_j = X[:, k+1] + sum_{q<j} (l_q y_q[k+1] - y_q l_q[k+1])    (after the exchange)
// and forms the next pivot column k+2 with the terms of pairs 0..j.  After the panel
// the pairs (l_j, y_j) update the trailing block as one skew rank-2k operation.
//
// GPU organisation as in the shared-memory panel of panel.cu: row i has one owner
// thread for the whole panel, which keeps its stored entries l_q[i], y_q[i] in shared
// memory.  The single grid-wide exchange of a pair step carries, besides the argmax
// candidates (each with its stored row), the stored rows and v values of rows k+1 and
// k+2, so that after it every CTA can form -- redundantly -- what columns k+1 and k+2
// need: the new rows k+1 and k+2, l_j[k+2] and y_j[k+2].  An entry moved by the
// exchange is taken from its value before the exchange, so a pair step needs no
// second synchronisation: half the grid exchanges of the one-step panel.
#include <climits>

#include "argmax.cuh"
#include "common.cuh"

namespace skew {
namespace {

constexpr int kTsMaxNb = 96;     // panel width (columns), 48 pairs: 192 KB of rows

__global__ void __launch_bounds__(kPanelThreads)
twostep_panel_kernel(TwoStepArgs A) {
    extern __shared__ double s_S[];                 // [c][tid]: c = 2q: l_q, 2q+1: y_q
    __shared__ double s_W[kTsMaxNb], s_P1[kTsMaxNb], s_P2[kTsMaxNb];
    __shared__ double s_c1[kTsMaxNb], s_c2[kTsMaxNb + 2];
    __shared__ double s_a, s_vk1, s_vk2, s_xs1, s_xs2;
    __shared__ unsigned long long s_wraw[kPanelThreads / 32];   // per-warp candidates
    __shared__ int s_wi[kPanelThreads / 32];
    __shared__ int s_r, s_win, s_fail;
    __shared__ unsigned int s_base;

    Ctrl *ctrl = A.ctrl;
    const int n = A.n, k0 = A.k0, kend = A.kend;
    const int G = (int)gridDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double *X = A.X;
    const int64_t ldx = A.ldx, ldv = A.ldv;
    auto slot = [&](int j, int cta) -> ArgmaxPartial * {
        return A.part + (j & 1) * kMaxPanelGrid + cta;
    };
    auto S = [&](int c) -> double & { return s_S[c * kPanelThreads + tid]; };

    // this thread's row: chunk (tid / 32) * G + cta, lane tid % 32
    const int64_t i =
        (int64_t)k0 + 1 + ((int64_t)((tid >> 5) * G + (int)blockIdx.x) << 5) + (tid & 31);
    const bool own = i < n;
    if (tid == 0) {
        s_base = ld_acquire_u32(&ctrl->bar_gen);
        s_fail = ld_volatile_i32(&ctrl->err) != 0;
    }
    __syncthreads();
    if (s_fail) return;
    const unsigned int base = s_base;
    auto owner_cta = [&](int row) -> int { return ((row - k0 - 1) >> 5) % G; };
    auto owner_tid = [&](int row) -> int {
        const int j = row - k0 - 1;
        return (((j >> 5) / G) << 5) + (j & 31);
    };

    // Publish pair step j (column k = k0 + 2j): this CTA's best candidate row (> k)
    // with its nc = 2j stored entries, and -- from their owners -- the stored rows and
    // v of rows k+1 and k+2; then release the step tag.  One CTA barrier: every warp
    // leaves its best candidate in shared memory (and the owners of rows k+1, k+2
    // their v), then warp 0 alone finishes the reduction, copies the rows from shared
    // memory and releases, while the other warps go on to wait for the next gather.
    auto publish = [&](int j, Best best, bool nonfinite, double v) {
        const int k = k0 + 2 * j, nc = 2 * j;
        if (nonfinite) raise_error(ctrl, SKEW_ERR_NONFINITE);
        if (own && i == k + 1) ctrl->vtop[j & 1] = v;
        if (own && i == k + 2) ctrl->vnext[j & 1] = v;
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
        ArgmaxPartial *sp = slot(j, blockIdx.x);
        if (y.i != INT_MAX) {
            const int ot = owner_tid(y.i);
            for (int c = lane; c < nc; c += 32) sp->row[c] = s_S[c * kPanelThreads + ot];
        }
        if (k + 1 < n && owner_cta(k + 1) == (int)blockIdx.x) {
            const int ot = owner_tid(k + 1);
            for (int c = lane; c < nc; c += 32) ctrl->rowp[j & 1][c] = s_S[c * kPanelThreads + ot];
        }
        if (k + 2 < n && owner_cta(k + 2) == (int)blockIdx.x) {
            const int ot = owner_tid(k + 2);
            for (int c = lane; c < nc; c += 32) ctrl->rowq[j & 1][c] = s_S[c * kPanelThreads + ot];
        }
        // release: the CTA's writes before the barrier and warp 0's copies (ordered by
        // __syncwarp) become visible to any CTA that sees the tag
        __syncwarp();
        if (lane == 0) record_release(sp, y.raw, y.i, base + (unsigned int)j + 1u);
    };

    // ---------------- pair step 0: v = X[k0+1:, k0]
    double v = 0.0;
    {
        Best best = no_candidate();
        bool nonfinite = false;
        if (own) {
            v = __ldcg(X + (int64_t)k0 * ldx + i);
            if (!finite_bits((unsigned long long)__double_as_longlong(v))) nonfinite = true;
            offer(best, v, (int)i);
        }
        best.c = blockIdx.x;
        publish(0, best, nonfinite, v);
    }

    int npairs = 0;
    for (int j = 0;; ++j) {
        const int k = k0 + 2 * j;
        if (!(k < kend && k + 1 < n)) break;
        npairs = j + 1;
        // ---------------- gather the step-j candidates of all CTAs (the barrier)
        if (tid < 32) {
            constexpr int kPer = kMaxPanelGrid / 32;
            const unsigned int want = base + (unsigned int)j + 1u;
            unsigned int pending = 0;
#pragma unroll
            for (int q = 0; q < kPer; ++q)
                if (tid + 32 * q < G) pending |= 1u << q;
            int fail = 0;
            uint64_t t0 = 0;
            unsigned int polls = 0;
            unsigned long long pv[kPer];
            unsigned int pi[kPer];
            while (pending != 0u) {
#pragma unroll
                for (int q = 0; q < kPer; ++q)
                    if ((pending >> q) & 1u) {
                        unsigned long long rv;
                        unsigned int ri, rt;
                        record_poll(slot(j, tid + 32 * q), rv, ri, rt);
                        if (rt == want) {
                            pending &= ~(1u << q);
                            pv[q] = rv;
                            pi[q] = ri;
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
            if (!fail) {
#pragma unroll
                for (int q = 0; q < kPer; ++q) {
                    const int c = tid + 32 * q;
                    if (c < G && better(pv[q], (int)pi[q], b.raw, b.i)) {
                        b.raw = pv[q];
                        b.i = (int)pi[q];
                        b.c = c;
                    }
                }
            }
            fail = __any_sync(0xffffffffu, fail);
            b = warp_best_all(b);
            if (tid == 0) {
                s_fail = fail;
                s_r = (b.i == INT_MAX) ? k + 1 : b.i;     // all NaN: keep the diagonal
                s_a = as_double(b.raw);
                s_win = (b.i == INT_MAX) ? -1 : b.c;
            }
        }
        __syncthreads();
        if (s_fail) return;
        const int r = s_r, nc = 2 * j;
        const bool next = (k + 2 < kend) && (k + 3 < n);

        // ---------------- one round of loads
        if (s_win >= 0)
            for (int c = tid; c < nc; c += blockDim.x) s_W[c] = __ldcg(&slot(j, s_win)->row[c]);
        for (int c = tid; c < nc; c += blockDim.x) {
            s_P1[c] = __ldcg(&ctrl->rowp[j & 1][c]);
            s_P2[c] = (k + 2 < n) ? __ldcg(&ctrl->rowq[j & 1][c]) : 0.0;
        }
        if (tid == 0) {
            const double vk1 = __ldcg(&ctrl->vtop[j & 1]);
            s_vk1 = vk1;
            s_vk2 = (k + 2 < n) ? __ldcg(&ctrl->vnext[j & 1]) : 0.0;
            s_xs1 = (k + 2 < n) ? __ldcg(X + (int64_t)(k + 1) * ldx + (k + 2)) : 0.0;  // X[k+2,k+1]
            // X[r, k+2] before the exchange (only read when there is a next pair: then
            // no thread writes it in this step)
            s_xs2 = (next && r > k + 2) ? __ldcg(X + (int64_t)(k + 2) * ldx + r) : 0.0;
            if (s_win < 0) s_a = vk1;
        }
        double x_old = 0.0, xe = 0.0, x2 = 0.0;
        if (own && i >= k + 2) {
            x_old = __ldcg(X + (int64_t)(k + 1) * ldx + i);                   // X[i, k+1]
            if (r != k + 1) {
                if (i < r) xe = __ldcg(X + i * ldx + r);                      // X[r, i]
                else if (i > r) xe = __ldcg(X + (int64_t)r * ldx + i);        // X[i, r]
            }
            if (next && i >= k + 3 && r != k + 2)
                x2 = __ldcg(X + (int64_t)(k + 2) * ldx + i);                  // X[i, k+2]
        }
        __syncthreads();
        const double a = s_a;

        // ---------------- coefficients shared by all rows
        // y_j[i] = X_new[i, k+1] + sum_c S[c][i] c1[c] with the new row k+1 (R1):
        // c1[2q] = y_q[k+1] = R1[2q+1], c1[2q+1] = -l_q[k+1] = -R1[2q]
        for (int c = tid; c < nc; c += blockDim.x) {
            const int q2 = c & ~1;
            const double r1l = (r != k + 1) ? s_W[q2] : s_P1[q2];
            const double r1y = (r != k + 1) ? s_W[q2 + 1] : s_P1[q2 + 1];
            s_c1[c] = (c & 1) ? -r1l : r1y;
        }
        __syncthreads();
        if (next) {
            // v'[i] = X_new[i, k+2] + sum_c S[c][i] c2[c] over pairs 0..j, with the new row
            // k+2 (R2 for q < j; l_j[k+2], y_j[k+2] formed here for q = j)
            for (int c = tid; c < nc; c += blockDim.x) {
                const int q2 = c & ~1;
                const double r2l = (r == k + 2) ? s_P1[q2] : s_P2[q2];
                const double r2y = (r == k + 2) ? s_P1[q2 + 1] : s_P2[q2 + 1];
                s_c2[c] = (c & 1) ? -r2l : r2y;
            }
            if (tid < 32) {
                double dot = 0.0;
                for (int c = tid; c < nc; c += 32) {
                    const double r2 = (r == k + 2) ? s_P1[c] : s_P2[c];
                    dot = fma(r2, s_c1[c], dot);
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
                    dot += __shfl_down_sync(0xffffffffu, dot, off);
                if (tid == 0) {
                    const double vk2 = (r == k + 2) ? s_vk1 : s_vk2;                // v_new[k+2]
                    const double lk2 = (a != 0.0) ? vk2 / a : 0.0;                  // l_j[k+2]
                    const double xk = (r == k + 1) ? s_xs1 : ((r == k + 2) ? -s_xs1 : -s_xs2);
                    s_c2[nc] = xk + dot;                                           // y_j[k+2]
                    s_c2[nc + 1] = -lk2;
                }
            }
        }
        if (blockIdx.x == 0 && tid == 0) {
            A.a[k / 2] = a;
            A.piv[k + 1] = r;
        }
        __syncthreads();

        // ---------------- rows k+2 .. n-1
        Best best = no_candidate();
        bool nonfinite = false;
        if (own && i >= k + 2) {
            if (r != k + 1 && i == r) {             // row r takes the old row k+1
                for (int c = 0; c < nc; ++c) S(c) = s_P1[c];
                v = s_vk1;
            }
            const double l = (a != 0.0) ? v / a : 0.0;
            // the gemvs over the stored entries first: they need no global data, so the
            // loads of x_old, xe and x2 are still in flight while they run.  Both in one
            // loop, four independent accumulators: an FP64 FMA takes a few hundred cycles
            // on this part, and a warp is often alone on its scheduler here.
            const bool nxt = next && i >= k + 3;
            double acc0 = 0.0, acc1 = 0.0, b0 = 0.0, b1 = 0.0;
            {
                int c = 0;
#pragma unroll 4
                for (; c + 1 < nc; c += 2) {
                    acc0 = fma(S(c), s_c1[c], acc0);
                    acc1 = fma(S(c + 1), s_c1[c + 1], acc1);
                }
                if (nxt) {
#pragma unroll 4
                    for (c = 0; c + 1 < nc; c += 2) {
                        b0 = fma(S(c), s_c2[c], b0);
                        b1 = fma(S(c + 1), s_c2[c + 1], b1);
                    }
                }
            }
            double x1 = x_old;                      // X_new[i, k+1]
            if (r != k + 1) {
                if (i < r) {
                    x1 = -xe;
                    // X[r, i]; for i = k+2 inside the panel the entry lies in the next
                    // pivot column, which is formed in registers and never read again,
                    // while every CTA reads its old value (s_xs2) in this step: not
                    // written then, so that no CTA can read the new value early
                    if (i != k + 2 || !next) X[i * ldx + r] = -x_old;
                } else if (i == r) {
                    x1 = -x_old;
                } else {
                    x1 = xe;
                    X[(int64_t)r * ldx + i] = x_old; // X[i, r]
                }
            }
            const double y = x1 + (acc0 + acc1);
            S(nc) = l;
            S(nc + 1) = y;
            if (nxt) {
                double x2v = x2;                    // X_new[i, k+2]
                if (r == k + 2) x2v = x_old;
                else if (r > k + 2 && i == r) x2v = -s_xs1;
                b0 = fma(l, s_c2[nc], b0);          // the pair formed in this step
                b1 = fma(y, s_c2[nc + 1], b1);
                const double vn = x2v + (b0 + b1);
                if (!finite_bits((unsigned long long)__double_as_longlong(vn))) nonfinite = true;
                v = vn;
                offer(best, vn, (int)i);
            }
        }
        if (next) {
            best.c = blockIdx.x;
            publish(j + 1, best, nonfinite, v);
        } else if (nonfinite) {
            raise_error(ctrl, SKEW_ERR_NONFINITE);
        }
    }
    // the panel's pairs for the trailing update: rows kend .. n-1 of V
    if (own && i >= kend)
        for (int c = 0; c < 2 * npairs; ++c) A.V[i + (int64_t)c * ldv] = S(c);
    // tags of this launch were base+1 .. base+npairs; the next launch starts above
    if (blockIdx.x == 0 && tid == 0)
        st_release_u32(&ctrl->bar_gen, base + (unsigned int)npairs + 1u);
}

// log|Pf| = sum_j log|a_j|, sign = det(P) prod_j sign(-a_j): one CTA, each thread a
// fixed strided subset in index order, then a fixed-shape tree (timing independent).
constexpr int kFinThreads = 1024;

__global__ void __launch_bounds__(kFinThreads)
finish_twostep_kernel(int64_t n, const double *a, const int32_t *piv, const Ctrl *ctrl,
                      double *logabs, int32_t *sign, int32_t *info) {
    __shared__ double s_sum[kFinThreads];
    __shared__ int s_neg[kFinThreads];
    __shared__ int s_zero[kFinThreads];
    const int tid = threadIdx.x;
    const int64_t half = n / 2;
    double sum = 0.0;
    int neg = 0, first_zero = INT_MAX;
    for (int64_t j = tid; j < half; j += kFinThreads) {
        const double v = -a[j];
        if (v == 0.0) {
            if (j < first_zero) first_zero = (int)j;
        } else {
            if (v < 0.0) neg ^= 1;
            sum += log(fabs(v));
        }
    }
    for (int64_t q = tid; q < n; q += kFinThreads)
        if (piv[q] != (int32_t)q) neg ^= 1;
    s_sum[tid] = sum;
    s_neg[tid] = neg;
    s_zero[tid] = first_zero;
    __syncthreads();
    for (int w = kFinThreads / 2; w > 0; w >>= 1) {
        if (tid < w) {
            s_sum[tid] += s_sum[tid + w];
            s_neg[tid] ^= s_neg[tid + w];
            s_zero[tid] = min(s_zero[tid], s_zero[tid + w]);
        }
        __syncthreads();
    }
    if (tid == 0) {
        const bool zero = (n & 1) != 0 || s_zero[0] != INT_MAX;
        if (logabs) *logabs = zero ? -INFINITY : s_sum[0];
        if (sign) *sign = zero ? 0 : (s_neg[0] ? -1 : 1);
        if (info) {
            const int e = ctrl ? ctrl->err : 0;
            *info = e != 0 ? e : (s_zero[0] == INT_MAX ? 0 : 2 * s_zero[0] + 1);
        }
    }
}

}  // namespace

bool twostep_fits(int64_t n, int nb, int sms) {
    return nb >= 2 && nb <= kTsMaxNb && (nb & 1) == 0 && n - 1 <= (int64_t)sms * kPanelThreads;
}

int launch_twostep_panel(const TwoStepArgs &a, int sms, cudaStream_t stream) {
    const int64_t rows = (int64_t)a.n - a.k0 - 1;
    const int width = a.kend - a.k0;
    if (rows < 1 || width > kTsMaxNb || rows > (int64_t)sms * kPanelThreads) return SKEW_ERR_CUDA;
    // The attribute belongs to the current device's copy of the function: set it on
    // every launch (as the other panel launches do), which is cheap and keeps no
    // process-wide state shared between devices or threads.
    const size_t smem_max = (size_t)kTsMaxNb * kPanelThreads * sizeof(double);
    {
        cudaError_t e = cudaFuncSetAttribute((const void *)twostep_panel_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem_max);
        if (e != cudaSuccess) {
            set_last_error(e);
            return SKEW_ERR_CUDA;
        }
    }
    int64_t g = panel_grid(rows, sms);
    if (g > kMaxPanelGrid) g = kMaxPanelGrid;
    const int cols = width + (width & 1);
    const size_t smem = (size_t)cols * kPanelThreads * sizeof(double);
    TwoStepArgs args = a;
    void *params[] = {&args};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)twostep_panel_kernel,
                                                dim3((unsigned)g), dim3(kPanelThreads), params,
                                                smem, stream);
    if (e != cudaSuccess) {
        set_last_error(e);
        return SKEW_ERR_CUDA;
    }
    note_launches(1);
    return SKEW_OK;
}

int launch_finish_twostep(int64_t n, const double *a, const int32_t *piv, const Ctrl *ctrl,
                          double *logabs, int32_t *sign, int32_t *info, cudaStream_t stream) {
    finish_twostep_kernel<<<1, kFinThreads, 0, stream>>>(n, a, piv, ctrl, logabs, sign, info);
    note_launches(1);
    return check_launch();
}

}  // namespace skew
