// batched.cu -- many independent small/medium factorizations in one persistent launch.
//
// Each CTA factors whole matrices, one at a time, taken from a device work queue in
// descending order of size (largest first, so the launch ends evenly).  A matrix is
// factored in place in its own storage (at n <= 256 the whole lower triangle, at
// most 512 KB, stays in L2) by the pivoted right-looking algorithm of Section 4.1
// (Eq. (1)) with the pivoting of Section 5.2: per step k, the pivot of column k
// (largest magnitude, lowest index on ties), the symmetric exchange of k+1 and r in
// lower storage, the Gauss transform l = x_31 / chi_21, and the skew rank-2 update
// X33 += l x32^T - x32 l^T (two FMAs per stored entry).  Synchronisation is the CTA
// barrier only.  The Pfaffian and the info word of each matrix are written at the
// end, as in the single-matrix path.
#include <climits>

#include "common.cuh"

namespace skew {
namespace {

constexpr int kBatchThreads = 512;
constexpr unsigned long long kAbs = 0x7fffffffffffffffull;
constexpr unsigned long long kExp = 0x7ff0000000000000ull;

struct Cand {
    unsigned long long raw;  // bits of the signed value
    int i;
};

__device__ __forceinline__ bool cand_better(unsigned long long ra, int ia, unsigned long long rb,
                                            int ib) {
    const unsigned long long a = ra & kAbs, b = rb & kAbs;
    return (a > b) || (a == b && ia < ib);
}

__device__ __forceinline__ Cand warp_cand(Cand x) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long orw = __shfl_down_sync(0xffffffffu, x.raw, off);
        const int oi = __shfl_down_sync(0xffffffffu, x.i, off);
        if (cand_better(orw, oi, x.raw, x.i)) { x.raw = orw; x.i = oi; }
    }
    return x;
}

// The same reduction with warp reduce instructions, the result valid in every lane:
// the largest |v| bits (high word, then low word among the lanes that tie on it), then
// the lowest row among the lanes that tie on both.
__device__ __forceinline__ Cand warp_cand_all(Cand x) {
    const unsigned long long m = x.raw & kAbs;
    const unsigned int hi = (unsigned int)(m >> 32), lo = (unsigned int)m;
    const unsigned int mh = __reduce_max_sync(0xffffffffu, hi);
    const unsigned int ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
    const bool top = (hi == mh) && (lo == ml);
    const unsigned int mi = __reduce_min_sync(0xffffffffu, top ? (unsigned int)x.i : 0xffffffffu);
    const unsigned int win = __ballot_sync(0xffffffffu, top && (unsigned int)x.i == mi);
    Cand r;
    r.raw = __shfl_sync(0xffffffffu, x.raw, __ffs((int)win) - 1);
    r.i = (int)mi;
    return r;
}

struct BatchShared {
    unsigned long long w_raw[kBatchThreads / 32];
    int w_i[kBatchThreads / 32];
    int w_bad[kBatchThreads / 32];
    double w_sum[kBatchThreads / 32];
    int w_par[kBatchThreads / 32];
    int w_zero[kBatchThreads / 32];
    unsigned long long best_raw;
    int best_i;
    int bad;
    int item;
};

// argmax over the candidates of all threads; also ORs the non-finite flags
__device__ Cand block_cand(Cand x, bool bad, BatchShared &sh, bool &any_bad) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    x = warp_cand(x);
    const int wb = __any_sync(0xffffffffu, bad);
    if (lane == 0) { sh.w_raw[w] = x.raw; sh.w_i[w] = x.i; sh.w_bad[w] = wb; }
    __syncthreads();
    if (w == 0) {
        Cand y;
        y.raw = 0ull;
        y.i = INT_MAX;
        int b = 0;
        if (lane < kBatchThreads / 32) { y.raw = sh.w_raw[lane]; y.i = sh.w_i[lane]; b = sh.w_bad[lane]; }
        y = warp_cand(y);
        b = __any_sync(0xffffffffu, b);
        if (lane == 0) { sh.best_raw = y.raw; sh.best_i = y.i; sh.bad = b; }
    }
    __syncthreads();
    Cand r;
    r.raw = sh.best_raw;
    r.i = sh.best_i;
    any_bad = sh.bad != 0;
    return r;
}

__device__ void factor_one(const skew_problem &P, double *logabs, int32_t *sign, int32_t *info,
                           double *s_l, double *s_x, BatchShared &sh) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
    const int n = (int)P.n;
    double *X = P.A;
    const int64_t ldx = P.lda;
    double *L = P.L;
    const int64_t ldl = P.ldl;
    double *t = P.t;
    int32_t *piv = P.piv;

    for (int i = tid; i < n; i += nthr) piv[i] = i;
    if (L != nullptr)
        for (int j = warp; j < n; j += nwarps)
            for (int i = lane; i < n; i += 32) L[i + j * ldl] = (i == j) ? 1.0 : 0.0;
    bool nonfinite = false;
    __syncthreads();

    for (int k = 0; k + 1 < n; ++k) {
        const int p = k + 1;
        double *colk = X + (int64_t)k * ldx;
        // ---- pivot: largest |X[i, k]|, i > k (Definition of iamax, Section 5.1)
        Cand c;
        c.raw = 0ull;
        c.i = INT_MAX;
        bool bad = false;
        for (int i = p + tid; i < n; i += nthr) {
            const unsigned long long raw = (unsigned long long)__double_as_longlong(colk[i]);
            if ((raw & kExp) == kExp) { bad = true; continue; }
            if (cand_better(raw, i, c.raw, c.i)) { c.raw = raw; c.i = i; }
        }
        bool any_bad;
        const Cand best = block_cand(c, bad, sh, any_bad);
        nonfinite |= any_bad;
        const int r = (best.i == INT_MAX) ? p : best.i;
        // ---- exchange k+1 <-> r: pivot column, rows of L, trailing skew block
        if (r != p) {
            for (int i = p + 1 + tid; i < n; i += nthr) {
                double *colp = X + (int64_t)p * ldx;
                if (i < r) {
                    double *xri = X + (int64_t)i * ldx + r;
                    const double tmp = colp[i];
                    colp[i] = -*xri;
                    *xri = -tmp;
                } else if (i == r) {
                    colp[i] = -colp[i];
                } else {
                    double *colr = X + (int64_t)r * ldx;
                    const double tmp = colp[i];
                    colp[i] = colr[i];
                    colr[i] = tmp;
                }
            }
            if (L != nullptr)
                for (int c2 = 1 + tid; c2 <= k; c2 += nthr) {
                    double *lc = L + (int64_t)c2 * ldl;
                    const double tmp = lc[p];
                    lc[p] = lc[r];
                    lc[r] = tmp;
                }
            if (tid == 0) {
                const double tmp = colk[p];
                colk[p] = colk[r];
                colk[r] = tmp;
            }
        }
        __syncthreads();
        // ---- Gauss transform (Eq. (1)): tau = X[k+1, k], l = X[k+2:, k] / tau
        const double tau = colk[p];
        if (tid == 0) {
            t[k] = tau;
            piv[p] = r;
        }
        const double *colp = X + (int64_t)p * ldx;
        for (int i = p + 1 + tid; i < n; i += nthr) {
            const double l = (tau != 0.0) ? colk[i] / tau : 0.0;
            s_l[i] = l;
            s_x[i] = colp[i];
            if (L != nullptr) L[i + (int64_t)p * ldl] = l;
        }
        __syncthreads();
        // ---- X33 += l x32^T - x32 l^T on the strictly lower part (columns k+2..n-1)
        for (int j = k + 2 + warp; j < n; j += nwarps) {
            double *colj = X + (int64_t)j * ldx;
            const double xj = s_x[j], lj = s_l[j];
            for (int i = j + 1 + lane; i < n; i += 32)
                colj[i] = fma(-s_x[i], lj, fma(s_l[i], xj, colj[i]));
        }
        __syncthreads();
    }

    // ---- Pf = det(P) prod_i (-t[2i]) (Section 1), fixed reduction order
    double sum = 0.0;
    int par = 0, zero = 0;
    const int half = n / 2;
    if ((n & 1) == 0)
        for (int j = tid; j < half; j += nthr) {
            const double v = -t[2 * j];
            if (v == 0.0) zero = 1;
            else {
                if (v < 0.0) par ^= 1;
                sum += log(fabs(v));
            }
        }
    for (int i = tid; i < n; i += nthr)
        if (piv[i] != i) par ^= 1;
    int first_zero = INT_MAX;
    for (int j = tid; j + 1 < n; j += nthr)
        if (t[j] == 0.0 && j < first_zero) first_zero = j;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        sum += __shfl_down_sync(0xffffffffu, sum, off);
        par ^= __shfl_down_sync(0xffffffffu, par, off);
        zero |= __shfl_down_sync(0xffffffffu, zero, off);
        first_zero = min(first_zero, __shfl_down_sync(0xffffffffu, first_zero, off));
    }
    if (lane == 0) {
        sh.w_sum[warp] = sum;
        sh.w_par[warp] = par;
        sh.w_zero[warp] = zero;
        sh.w_i[warp] = first_zero;
    }
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        int pr = 0, z = 0, fz = INT_MAX;
        for (int w = 0; w < nwarps; ++w) {
            s += sh.w_sum[w];
            pr ^= sh.w_par[w];
            z |= sh.w_zero[w];
            fz = min(fz, sh.w_i[w]);
        }
        const bool pf_zero = (n & 1) || z;
        if (logabs) *logabs = pf_zero ? -INFINITY : s;
        if (sign) *sign = pf_zero ? 0 : (pr ? -1 : 1);
        if (info) *info = nonfinite ? SKEW_ERR_NONFINITE : (fz == INT_MAX ? 0 : fz + 1);
    }
    __syncthreads();
}

// ------------------------------------------------------------------------------------
// Blocked variant for n <= kBlkMaxN: the blocked right-looking algorithm of
// Section 4.2 (Variant 1) with the pivoted left-looking panel of Section 5.2, inside
// one CTA.  Panels of NB columns: each step forms v = X[k+1:, k] - Lp h from the
// panel's L columns kept in shared memory (h = T L[k, :]^T), takes the pivot, exchanges
// k+1 and r in place, and scales.  The trailing update is one skew rank-2k update
// with the pairs (a_j, w_j), W = A S (Section 2.2 theorem), plus the pair of the last
// Gauss transform, on FP64 DMMA (mma.sync.m8n8k4.f64): n^3/3 flops per matrix.
// ------------------------------------------------------------------------------------
constexpr int kBlkThreads = 256;
constexpr int kBlkNbMax = 32;     // panel widths 8, 16, 32 per size bucket (BatchedNb)
constexpr int kBlkMaxN = 512;

__device__ __forceinline__ void dmma884(double &c0, double &c1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(c0), "+d"(c1)
                 : "d"(a), "d"(b));
}

struct BlkShared {
    double h[kBlkNbMax + 1];
    double t[kBlkNbMax + 1];
    unsigned long long w_raw[kBlkThreads / 32];
    int w_i[kBlkThreads / 32];
    int w_bad[kBlkThreads / 32];
    unsigned long long best_raw;
    int best_i;
    int bad;
};

// argmax over the candidates of all threads (and the OR of their non-finite flags),
// valid in every thread on return.  One CTA barrier: each warp leaves its best in
// shared memory, then every warp reduces those itself.  The per-warp slots are next
// written by the following call, which comes after at least one more CTA barrier.
__device__ Cand blk_cand(Cand x, bool bad, BlkShared &sh, bool &any_bad) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    x = warp_cand_all(x);
    const int wb = __any_sync(0xffffffffu, bad);
    if (lane == 0) { sh.w_raw[w] = x.raw; sh.w_i[w] = x.i; sh.w_bad[w] = wb; }
    __syncthreads();
    Cand y;
    y.raw = 0ull;
    y.i = INT_MAX;
    int b = 0;
    if (lane < (int)(blockDim.x >> 5)) { y.raw = sh.w_raw[lane]; y.i = sh.w_i[lane]; b = sh.w_bad[lane]; }
    y = warp_cand_all(y);
    any_bad = __any_sync(0xffffffffu, b) != 0;
    return y;
}

// smem: Lp[NB][nmax] (panel L columns), Ws[NB/2+1][nmax] (odd W columns),
// sv[nmax] (v of the current step)
template <int NB, int WT>
__device__ void factor_one_blocked(const skew_problem &P, double *logabs, int32_t *sign,
                                   int32_t *info, double *smem, int nmax, BlkShared &sh,
                                   BatchShared &fin) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
    const int n = (int)P.n;
    double *X = P.A;
    const int64_t ldx = P.lda;
    double *L = P.L;
    const int64_t ldl = P.ldl;
    double *t = P.t;
    int32_t *piv = P.piv;
    double *Lp = smem;                                  // Lp[q * nmax + i]
    double *Ws = smem + (size_t)NB * nmax;              // Ws[pp * nmax + i]
    double *sv = Ws + (size_t)(NB / 2 + 1) * nmax;

    for (int i = tid; i < n; i += nthr) piv[i] = i;
    if (L != nullptr)
        for (int j = warp; j < n; j += nwarps)
            for (int i = lane; i < n; i += 32) L[i + j * ldl] = (i == j) ? 1.0 : 0.0;
    bool nonfinite = false;
    __syncthreads();

    // h for step k of the panel starting at k0 (L[k, k] = 1): into sh.h[q - k0 - 1]
    auto form_h = [&](int k, int k0) {
        for (int q = k0 + 1 + tid; q <= k; q += nthr) {
            double hq = 0.0;
            if (q - 1 >= k0 + 1) hq = sh.t[q - 1 - k0] * Lp[(q - 2 - k0) * nmax + k];
            if (q + 1 <= k) {
                const double lq1 = (q + 1 == k) ? 1.0 : Lp[(q - k0) * nmax + k];
                hq -= sh.t[q - k0] * lq1;
            }
            sh.h[q - k0 - 1] = hq;
        }
        __syncthreads();
    };

    for (int k0 = 0; k0 + 1 < n;) {
        const int kend = (k0 + NB < n - 1) ? k0 + NB : n - 1;
        const int b = kend - k0;
        // ---------------- the panel
        for (int k = k0; k < kend; ++k) {
            const int nq = k - k0, p = k + 1;
            form_h(k, k0);
            const double *colk = X + (int64_t)k * ldx;
            Cand c;
            c.raw = 0ull;
            c.i = INT_MAX;
            bool bad = false;
            for (int i = p + tid; i < n; i += nthr) {
                double v = colk[i];
                for (int q = 0; q < nq; ++q) v -= Lp[q * nmax + i] * sh.h[q];
                sv[i] = v;
                const unsigned long long raw = (unsigned long long)__double_as_longlong(v);
                if ((raw & kExp) == kExp) { bad = true; continue; }
                if (cand_better(raw, i, c.raw, c.i)) { c.raw = raw; c.i = i; }
            }
            bool any_bad;
            const Cand best = blk_cand(c, bad, sh, any_bad);
            nonfinite |= any_bad;
            const int r = (best.i == INT_MAX) ? p : best.i;
            // the exchange and the new L column in one phase: the column takes its
            // values from v before the exchange (row r gets old row p's v)
            const double tau = sv[r], vp = sv[p];
            if (r != p) {
                double *colp = X + (int64_t)p * ldx;
                for (int i = p + 1 + tid; i < n; i += nthr) {
                    if (i < r) {
                        double *xri = X + (int64_t)i * ldx + r;
                        const double tmp = colp[i];
                        colp[i] = -*xri;
                        *xri = -tmp;
                    } else if (i == r) {
                        colp[i] = -colp[i];
                    } else {
                        double *colr = X + (int64_t)r * ldx;
                        const double tmp = colp[i];
                        colp[i] = colr[i];
                        colr[i] = tmp;
                    }
                }
                for (int q = tid; q < nq; q += nthr) {
                    const double tmp = Lp[q * nmax + p];
                    Lp[q * nmax + p] = Lp[q * nmax + r];
                    Lp[q * nmax + r] = tmp;
                }
            }
            if (tid == 0) {
                sh.t[nq] = tau;
                t[k] = tau;
                piv[p] = r;
            }
            double *lnew = Lp + (size_t)nq * nmax;             // panel column k+1
            for (int i = p + tid; i < n; i += nthr) {
                const double val = (i == r) ? vp : sv[i];
                lnew[i] = (i == p) ? 1.0 : ((tau != 0.0) ? val / tau : 0.0);
            }
            __syncthreads();
        }
        const int s = kend;
        if (s < n - 1) {
            // ---------------- the updated column x = X[s+1:, s] (left-looking, k = s)
            form_h(s, k0);
            double *cols = X + (int64_t)s * ldx;
            for (int i = s + 1 + tid; i < n; i += nthr) {
                double v = cols[i];
                for (int q = 0; q < b; ++q) v -= Lp[q * nmax + i] * sh.h[q];
                cols[i] = v;
            }
            __syncthreads();
            // ---------------- odd W columns (W = A S), the last pair merged with x
            const int npairs = b / 2 + (b & 1);
            for (int i = s + 1 + tid; i < n; i += nthr) {
                for (int pp = 0; pp < npairs; ++pp) {
                    const int j = 2 * pp + 1;
                    double w;
                    if (j < b) {
                        w = -sh.t[j] * Lp[(j - 1) * nmax + i];             // t_p[j-1] = t[k0+j]
                        if (j + 1 < b) w += sh.t[j + 1] * Lp[(j + 1) * nmax + i];
                        if (j == b - 1) w += cols[i];
                    } else {
                        w = cols[i];                                      // b odd: (a_{b-1}, x)
                    }
                    Ws[(size_t)pp * nmax + i] = w;
                }
            }
            __syncthreads();
            // ---------------- C = X[s+1:, s+1:] += sum_p (a_p w_p^T - w_p a_p^T), DMMA
            const int m = n - s - 1;
            const int K = 2 * npairs;                  // U = [a | -w], V = [w | a]
            const int K4 = (K + 3) / 4 * 4;
            const int nt = (m + WT - 1) / WT;
            const int ntiles = nt * (nt + 1) / 2;
            const int g = lane >> 2, tg = lane & 3;
            auto acol = [&](int pp) { return (2 * pp + 1 < b) ? 2 * pp + 1 : b - 1; };
            for (int tile = warp; tile < ntiles; tile += nwarps) {
                int bi = 0;
                while ((bi + 1) * (bi + 2) / 2 <= tile) ++bi;
                const int bj = tile - bi * (bi + 1) / 2;
                const bool diag = bi == bj;   // a diagonal tile: its sub-tiles on or below the diagonal
                constexpr int FR = WT / 8;    // 8 x 8 DMMA sub-tiles per warp-tile side
                double acc[FR][FR][2];
#pragma unroll
                for (int mi = 0; mi < FR; ++mi)
#pragma unroll
                    for (int ni = 0; ni < FR; ++ni) acc[mi][ni][0] = acc[mi][ni][1] = 0.0;
                for (int kb = 0; kb < K4; kb += 4) {
                    const int kc = kb + tg;
                    double af[FR], bf[FR];
#pragma unroll
                    for (int mi = 0; mi < FR; ++mi) {
                        const int li = bi * WT + mi * 8 + g;          // local row in C
                        const int i = s + 1 + li;
                        double u = 0.0;
                        if (li < m && kc < K)
                            u = kc < npairs ? Lp[acol(kc) * nmax + i] : -Ws[(size_t)(kc - npairs) * nmax + i];
                        af[mi] = u;
                    }
#pragma unroll
                    for (int ni = 0; ni < FR; ++ni) {
                        const int lj = bj * WT + ni * 8 + g;
                        const int j = s + 1 + lj;
                        double v = 0.0;
                        if (lj < m && kc < K)
                            v = kc < npairs ? Ws[(size_t)kc * nmax + j] : Lp[acol(kc - npairs) * nmax + j];
                        bf[ni] = v;
                    }
#pragma unroll
                    for (int mi = 0; mi < FR; ++mi)
#pragma unroll
                        for (int ni = 0; ni < FR; ++ni)
                            if (!diag || mi >= ni)   // above the diagonal: nothing stored
                                dmma884(acc[mi][ni][0], acc[mi][ni][1], af[mi], bf[ni]);
                }
#pragma unroll
                for (int mi = 0; mi < FR; ++mi) {
                    const int li = bi * WT + mi * 8 + g;
#pragma unroll
                    for (int ni = 0; ni < FR; ++ni)
#pragma unroll
                        for (int cc = 0; cc < 2; ++cc) {
                            const int lj = bj * WT + ni * 8 + 2 * tg + cc;
                            if (li < m && lj < m && li > lj) {
                                double *dst = X + (int64_t)(s + 1 + lj) * ldx + (s + 1 + li);
                                *dst = *dst + acc[mi][ni][cc];
                            }
                        }
                }
            }
        }
        // ---------------- L: the panel's columns, and its exchanges on earlier columns
        if (L != nullptr) {
            for (int q = warp; q < b; q += nwarps) {
                const int col = k0 + 1 + q;
                for (int i = col + lane; i < n; i += 32) L[i + (int64_t)col * ldl] = Lp[(size_t)q * nmax + i];
            }
            for (int c2 = 1 + tid; c2 <= k0; c2 += nthr) {
                double *lc = L + (int64_t)c2 * ldl;
                for (int k = k0; k < kend; ++k) {
                    const int r = piv[k + 1], p = k + 1;
                    if (r != p) {
                        const double tmp = lc[p];
                        lc[p] = lc[r];
                        lc[r] = tmp;
                    }
                }
            }
        }
        __syncthreads();
        k0 = kend;
    }

    // ---- Pf = det(P) prod_i (-t[2i]) (Section 1), fixed reduction order
    double sum = 0.0;
    int par = 0, zero = 0;
    const int half = n / 2;
    if ((n & 1) == 0)
        for (int j = tid; j < half; j += nthr) {
            const double v = -t[2 * j];
            if (v == 0.0) zero = 1;
            else {
                if (v < 0.0) par ^= 1;
                sum += log(fabs(v));
            }
        }
    for (int i = tid; i < n; i += nthr)
        if (piv[i] != i) par ^= 1;
    int first_zero = INT_MAX;
    for (int j = tid; j + 1 < n; j += nthr)
        if (t[j] == 0.0 && j < first_zero) first_zero = j;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        sum += __shfl_down_sync(0xffffffffu, sum, off);
        par ^= __shfl_down_sync(0xffffffffu, par, off);
        zero |= __shfl_down_sync(0xffffffffu, zero, off);
        first_zero = min(first_zero, __shfl_down_sync(0xffffffffu, first_zero, off));
    }
    if (lane == 0) {
        fin.w_sum[warp] = sum;
        fin.w_par[warp] = par;
        fin.w_zero[warp] = zero;
        fin.w_i[warp] = first_zero;
    }
    __syncthreads();
    if (tid == 0) {
        double sm = 0.0;
        int pr = 0, z = 0, fz = INT_MAX;
        for (int w = 0; w < nwarps; ++w) {
            sm += fin.w_sum[w];
            pr ^= fin.w_par[w];
            z |= fin.w_zero[w];
            fz = min(fz, fin.w_i[w]);
        }
        const bool pf_zero = (n & 1) || z;
        if (logabs) *logabs = pf_zero ? -INFINITY : sm;
        if (sign) *sign = pf_zero ? 0 : (pr ? -1 : 1);
        if (info) *info = nonfinite ? SKEW_ERR_NONFINITE : (fz == INT_MAX ? 0 : fz + 1);
    }
    __syncthreads();
}

// ------------------------------------------------------------------------------------
// Pfaffian-only batched variant: the two-step elimination (only the even-step Gauss
// transforms; each pair of columns removed by the Schur complement of its 2 x 2 skew
// pivot block; notes to the two-step right-looking algorithm, Section 4.1), blocked
// inside one CTA: panels of NB columns (NB/2 pairs) formed left-looking from
// the panel's vectors kept in shared memory, then one skew rank-2k update
// X[k1:, k1:] += sum_j (l_j y_j^T - y_j l_j^T) on FP64 DMMA.  Half the pivot searches
// (and CTA barriers) of factor_one_blocked and no W.  P.t receives the n/2 pivot-block
// entries a_j, P.piv the even-step exchanges (identity elsewhere); P.L is not used.
// smem: Vp[NB][nmax] (c = 2q: l_q, 2q+1: y_q), sv[nmax].
// ------------------------------------------------------------------------------------
template <int NB, int WT>
__device__ void pfaff_one_twostep(const skew_problem &P, double *logabs, int32_t *sign,
                                  int32_t *info, double *smem, int nmax, BlkShared &sh,
                                  BatchShared &fin) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
    const int n = (int)P.n;
    double *X = P.A;
    const int64_t ldx = P.lda;
    double *aout = P.t;
    int32_t *piv = P.piv;
    double *Vp = smem;                                  // Vp[c * nmax + i]
    double *sv = smem + (size_t)NB * nmax;

    for (int i = tid; i < n; i += nthr) piv[i] = i;
    bool nonfinite = false;
    __syncthreads();

    for (int k0 = 0; k0 + 1 < n;) {
        int np = 0;
        for (int k = k0; k < k0 + NB && k + 1 < n; k += 2) ++np;
        for (int j = 0; j < np; ++j) {
            const int k = k0 + 2 * j, nc = 2 * j, p = k + 1;
            // v = X[:, k] + sum_c Vp[c][i] h[c]:  h[2q] = y_q[k], h[2q+1] = -l_q[k]
            for (int c = tid; c < nc; c += nthr)
                sh.h[c] = (c & 1) ? -Vp[(size_t)(c - 1) * nmax + k] : Vp[(size_t)(c + 1) * nmax + k];
            __syncthreads();
            const double *colk = X + (int64_t)k * ldx;
            Cand cd;
            cd.raw = 0ull;
            cd.i = INT_MAX;
            bool bad = false;
            for (int i = p + tid; i < n; i += nthr) {
                double v = colk[i];
                for (int c = 0; c < nc; ++c) v += Vp[(size_t)c * nmax + i] * sh.h[c];
                sv[i] = v;
                const unsigned long long raw = (unsigned long long)__double_as_longlong(v);
                if ((raw & kExp) == kExp) { bad = true; continue; }
                if (cand_better(raw, i, cd.raw, cd.i)) { cd.raw = raw; cd.i = i; }
            }
            bool any_bad;
            const Cand best = blk_cand(cd, bad, sh, any_bad);
            nonfinite |= any_bad;
            const int r = (best.i == INT_MAX) ? p : best.i;
            // the exchange and the coefficients of the new row p in one phase: each
            // thread handling a panel vector c swaps its rows p and r and writes the
            // coefficient that vector's old row r gives (h[2q] = y_q[p], h[2q+1] =
            // -l_q[p] of the new row p); v is taken before the exchange below
            const double a = sv[r], vp = sv[p];
            for (int c = tid; c < nc; c += nthr) {
                const double vr = Vp[(size_t)c * nmax + r];
                if (r != p) {
                    Vp[(size_t)c * nmax + r] = Vp[(size_t)c * nmax + p];
                    Vp[(size_t)c * nmax + p] = vr;
                }
                if (c & 1) sh.t[c - 1] = vr;
                else sh.t[c + 1] = -vr;
            }
            if (r != p) {
                // exchange of indices p and r in X[p:, p:] (lower storage)
                double *colp = X + (int64_t)p * ldx;
                for (int i = p + 1 + tid; i < n; i += nthr) {
                    if (i < r) {
                        double *xri = X + (int64_t)i * ldx + r;
                        const double tmp = colp[i];
                        colp[i] = -*xri;
                        *xri = -tmp;
                    } else if (i == r) {
                        colp[i] = -colp[i];
                    } else {
                        double *colr = X + (int64_t)r * ldx;
                        const double tmp = colp[i];
                        colp[i] = colr[i];
                        colr[i] = tmp;
                    }
                }
            }
            if (tid == 0) {
                aout[k / 2] = a;
                piv[p] = r;
            }
            __syncthreads();
            // y = X[:, k+1] + sum_c Vp[c][i] h[c] with h from the new row k+1;  l = v / a
            const double *colp = X + (int64_t)p * ldx;
            for (int i = p + 1 + tid; i < n; i += nthr) {
                double y = colp[i];
                for (int c = 0; c < nc; ++c) y += Vp[(size_t)c * nmax + i] * sh.t[c];
                const double val = (i == r) ? vp : sv[i];
                Vp[(size_t)nc * nmax + i] = (a != 0.0) ? val / a : 0.0;
                Vp[(size_t)(nc + 1) * nmax + i] = y;
            }
            __syncthreads();
        }
        const int k1 = k0 + 2 * np;
        const int m = n - k1;
        if (m >= 2) {
            // C = X[k1:, k1:] += sum_q (l_q y_q^T - y_q l_q^T): U = [l | -y], V = [y | l]
            const int K = 2 * np;
            const int K4 = (K + 3) / 4 * 4;
            const int nt = (m + WT - 1) / WT;
            const int ntiles = nt * (nt + 1) / 2;
            const int g = lane >> 2, tg = lane & 3;
            for (int tile = warp; tile < ntiles; tile += nwarps) {
                int bi = 0;
                while ((bi + 1) * (bi + 2) / 2 <= tile) ++bi;
                const int bj = tile - bi * (bi + 1) / 2;
                const bool diag = bi == bj;   // a diagonal tile: its sub-tiles on or below the diagonal
                constexpr int FR = WT / 8;    // 8 x 8 DMMA sub-tiles per warp-tile side
                double acc[FR][FR][2];
#pragma unroll
                for (int mi = 0; mi < FR; ++mi)
#pragma unroll
                    for (int ni = 0; ni < FR; ++ni) acc[mi][ni][0] = acc[mi][ni][1] = 0.0;
                for (int kb = 0; kb < K4; kb += 4) {
                    const int kc = kb + tg;
                    double af[FR], bf[FR];
#pragma unroll
                    for (int mi = 0; mi < FR; ++mi) {
                        const int li = bi * WT + mi * 8 + g;
                        const int i = k1 + li;
                        double u = 0.0;
                        if (li < m && kc < K)
                            u = kc < np ? Vp[(size_t)(2 * kc) * nmax + i]
                                        : -Vp[(size_t)(2 * (kc - np) + 1) * nmax + i];
                        af[mi] = u;
                    }
#pragma unroll
                    for (int ni = 0; ni < FR; ++ni) {
                        const int lj = bj * WT + ni * 8 + g;
                        const int j = k1 + lj;
                        double v = 0.0;
                        if (lj < m && kc < K)
                            v = kc < np ? Vp[(size_t)(2 * kc + 1) * nmax + j]
                                        : Vp[(size_t)(2 * (kc - np)) * nmax + j];
                        bf[ni] = v;
                    }
#pragma unroll
                    for (int mi = 0; mi < FR; ++mi)
#pragma unroll
                        for (int ni = 0; ni < FR; ++ni)
                            if (!diag || mi >= ni)   // above the diagonal: nothing stored
                                dmma884(acc[mi][ni][0], acc[mi][ni][1], af[mi], bf[ni]);
                }
#pragma unroll
                for (int mi = 0; mi < FR; ++mi) {
                    const int li = bi * WT + mi * 8 + g;
#pragma unroll
                    for (int ni = 0; ni < FR; ++ni)
#pragma unroll
                        for (int cc = 0; cc < 2; ++cc) {
                            const int lj = bj * WT + ni * 8 + 2 * tg + cc;
                            if (li < m && lj < m && li > lj) {
                                double *dst = X + (int64_t)(k1 + lj) * ldx + (k1 + li);
                                *dst = *dst + acc[mi][ni][cc];
                            }
                        }
                }
            }
        }
        __syncthreads();
        k0 = k1;
    }

    // ---- Pf = det(P) prod_j (-a_j), fixed reduction order
    double sum = 0.0;
    int par = 0, first_zero = INT_MAX;
    const int half = n / 2;
    for (int j = tid; j < half; j += nthr) {
        const double v = -aout[j];
        if (v == 0.0) {
            if (j < first_zero) first_zero = j;
        } else {
            if (v < 0.0) par ^= 1;
            sum += log(fabs(v));
        }
    }
    for (int i = tid; i < n; i += nthr)
        if (piv[i] != i) par ^= 1;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        sum += __shfl_down_sync(0xffffffffu, sum, off);
        par ^= __shfl_down_sync(0xffffffffu, par, off);
        first_zero = min(first_zero, __shfl_down_sync(0xffffffffu, first_zero, off));
    }
    if (lane == 0) {
        fin.w_sum[warp] = sum;
        fin.w_par[warp] = par;
        fin.w_i[warp] = first_zero;
    }
    __syncthreads();
    if (tid == 0) {
        double sm = 0.0;
        int pr = 0, fz = INT_MAX;
        for (int w = 0; w < nwarps; ++w) {
            sm += fin.w_sum[w];
            pr ^= fin.w_par[w];
            fz = min(fz, fin.w_i[w]);
        }
        const bool pf_zero = (n & 1) || fz != INT_MAX;
        if (logabs) *logabs = pf_zero ? -INFINITY : sm;
        if (sign) *sign = pf_zero ? 0 : (pr ? -1 : 1);
        if (info) *info = nonfinite ? SKEW_ERR_NONFINITE : (fz == INT_MAX ? 0 : 2 * fz + 1);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kBlkThreads, 2)
batched_twostep_kernel(int count, const skew_problem *problems, const int32_t *order,
                       unsigned int *counter, double *logabs, int32_t *sign, int32_t *info,
                       int max_n, BatchedNb tab) {
    extern __shared__ double s_blk[];
    __shared__ BlkShared sh;
    __shared__ BatchShared fin;
    for (;;) {
        if (threadIdx.x == 0) fin.item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int item = fin.item;
        __syncthreads();
        if (item >= count) return;
        const int b = order[item];
        const skew_problem P = problems[b];
        const int n = (int)P.n;
        if (n < 0 || n > max_n || (n > 0 && P.A == nullptr) || P.lda < (n > 1 ? n : 1) ||
            (n > 1 && P.t == nullptr) || (n > 0 && P.piv == nullptr)) {
            if (threadIdx.x == 0 && info) info[b] = -2;
            continue;
        }
        double *la = logabs ? logabs + b : nullptr;
        int32_t *sg = sign ? sign + b : nullptr, *inf = info ? info + b : nullptr;
        const int nm = max_n > 1 ? max_n : 1;
        const bool wt16 = batched_wt_for(tab, n) == 16;
        switch (batched_nb_for(tab, n)) {
            case 8:
                if (wt16) pfaff_one_twostep<8, 16>(P, la, sg, inf, s_blk, nm, sh, fin);
                else pfaff_one_twostep<8, 32>(P, la, sg, inf, s_blk, nm, sh, fin);
                break;
            case 32:
                if (wt16) pfaff_one_twostep<32, 16>(P, la, sg, inf, s_blk, nm, sh, fin);
                else pfaff_one_twostep<32, 32>(P, la, sg, inf, s_blk, nm, sh, fin);
                break;
            default:
                if (wt16) pfaff_one_twostep<16, 16>(P, la, sg, inf, s_blk, nm, sh, fin);
                else pfaff_one_twostep<16, 32>(P, la, sg, inf, s_blk, nm, sh, fin);
                break;
        }
    }
}

__global__ void __launch_bounds__(kBlkThreads, 2)
batched_blocked_kernel(int count, const skew_problem *problems, const int32_t *order,
                       unsigned int *counter, double *logabs, int32_t *sign, int32_t *info,
                       int max_n, BatchedNb tab) {
    extern __shared__ double s_blk[];
    __shared__ BlkShared sh;
    __shared__ BatchShared fin;
    for (;;) {
        if (threadIdx.x == 0) fin.item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int item = fin.item;
        __syncthreads();
        if (item >= count) return;
        const int b = order[item];
        const skew_problem P = problems[b];
        const int n = (int)P.n;
        if (n < 0 || n > max_n || (n > 0 && P.A == nullptr) || P.lda < (n > 1 ? n : 1) ||
            (P.L != nullptr && P.ldl < (n > 1 ? n : 1)) || (n > 1 && P.t == nullptr) ||
            (n > 0 && P.piv == nullptr)) {
            if (threadIdx.x == 0 && info) info[b] = -2;
            continue;
        }
        double *la = logabs ? logabs + b : nullptr;
        int32_t *sg = sign ? sign + b : nullptr, *inf = info ? info + b : nullptr;
        const int nm = max_n > 1 ? max_n : 1;
        const bool wt16 = batched_wt_for(tab, n) == 16;
        switch (batched_nb_for(tab, n)) {
            case 8:
                if (wt16) factor_one_blocked<8, 16>(P, la, sg, inf, s_blk, nm, sh, fin);
                else factor_one_blocked<8, 32>(P, la, sg, inf, s_blk, nm, sh, fin);
                break;
            case 32:
                if (wt16) factor_one_blocked<32, 16>(P, la, sg, inf, s_blk, nm, sh, fin);
                else factor_one_blocked<32, 32>(P, la, sg, inf, s_blk, nm, sh, fin);
                break;
            default:
                if (wt16) factor_one_blocked<16, 16>(P, la, sg, inf, s_blk, nm, sh, fin);
                else factor_one_blocked<16, 32>(P, la, sg, inf, s_blk, nm, sh, fin);
                break;
        }
    }
}

// Persistent: each CTA takes the next matrix of the size-ordered queue.
__global__ void __launch_bounds__(kBatchThreads)
batched_kernel(int count, const skew_problem *problems, const int32_t *order,
               unsigned int *counter, double *logabs, int32_t *sign, int32_t *info, int max_n) {
    extern __shared__ double s_vec[];
    __shared__ BatchShared sh;
    for (;;) {
        if (threadIdx.x == 0) sh.item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int item = sh.item;
        __syncthreads();
        if (item >= count) return;
        const int b = order[item];
        const skew_problem P = problems[b];
        const int n = (int)P.n;
        if (n < 0 || n > max_n || (n > 0 && P.A == nullptr) || P.lda < (n > 1 ? n : 1) ||
            (P.L != nullptr && P.ldl < (n > 1 ? n : 1)) || (n > 1 && P.t == nullptr) ||
            (n > 0 && P.piv == nullptr)) {
            if (threadIdx.x == 0 && info) info[b] = -2;   // a bad problem descriptor
            continue;
        }
        factor_one(P, logabs ? logabs + b : nullptr, sign ? sign + b : nullptr,
                   info ? info + b : nullptr, s_vec, s_vec + (n > 0 ? n : 1), sh);
    }
}

// Counting sort of the problems by order, largest first (one CTA).
__global__ void __launch_bounds__(1024)
order_kernel(int count, const skew_problem *problems, int max_n, int32_t *order,
             unsigned int *counter, unsigned int *hist) {
    for (int v = threadIdx.x; v <= max_n + 1; v += blockDim.x) hist[v] = 0u;
    if (threadIdx.x == 0) *counter = 0u;
    __syncthreads();
    for (int b = threadIdx.x; b < count; b += blockDim.x) {
        int64_t n = problems[b].n;
        int key = (n < 0 || n > max_n) ? 0 : (int)(max_n - n);   // descending size
        atomicAdd(&hist[key], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int run = 0;
        for (int v = 0; v <= max_n; ++v) {
            const unsigned int h = hist[v];
            hist[v] = run;
            run += h;
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < count; b += blockDim.x) {
        int64_t n = problems[b].n;
        int key = (n < 0 || n > max_n) ? 0 : (int)(max_n - n);
        const unsigned int pos = atomicAdd(&hist[key], 1u);
        order[pos] = b;
    }
}

// the widest panel any order <= max_n takes (shared memory is sized for it)
int widest_nb(const BatchedNb &t, int max_n) {
    if (t.count == 0) return 16;
    int w = 0;
    for (int i = 0; i < t.count; ++i) {
        w = t.nb[i] > w ? t.nb[i] : w;
        if (t.n_upper[i] >= max_n) break;
    }
    return w;
}

}  // namespace

int launch_batched_twostep(int count, const skew_problem *problems, double *logabs,
                           int32_t *sign, int32_t *info, int max_n, void *ws,
                           cudaStream_t stream, int sms) {
    if (max_n > kBlkMaxN) return SKEW_ERR_CUDA;            // callers check
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    char *base = static_cast<char *>(ws);
    unsigned int *counter = reinterpret_cast<unsigned int *>(base);
    int32_t *order = reinterpret_cast<int32_t *>(base + al(sizeof(unsigned int)));
    unsigned int *hist = reinterpret_cast<unsigned int *>(
        base + al(sizeof(unsigned int)) + al(sizeof(int32_t) * (size_t)(count > 0 ? count : 1)));
    order_kernel<<<1, 1024, 0, stream>>>(count, problems, max_n, order, counter, hist);
    note_launches(1);
    SKEW_TRY_STATUS(check_launch());
    const size_t nm = (size_t)(max_n > 1 ? max_n : 1);
    const BatchedNb tab = batched_nb_table();
    const size_t smem = sizeof(double) * nm * (widest_nb(tab, max_n) + 1);
    cudaError_t e = cudaFuncSetAttribute((const void *)batched_twostep_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
        set_last_error(e);
        return SKEW_ERR_CUDA;
    }
    const int thr = tab.threads == 128 ? 128 : kBlkThreads;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_twostep_kernel,
                                                      thr, smem);
    if (e != cudaSuccess || per_sm < 1) {
        if (e != cudaSuccess) set_last_error(e);
        return SKEW_ERR_CUDA;
    }
    int grid = sms * per_sm;
    if (grid > count) grid = count;
    batched_twostep_kernel<<<grid, thr, smem, stream>>>(count, problems, order, counter,
                                                                logabs, sign, info, max_n, tab);
    note_launches(1);
    return check_launch();
}

size_t batched_workspace_bytes(int count, int max_n) {
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    return al(sizeof(unsigned int)) + al(sizeof(int32_t) * (size_t)(count > 0 ? count : 1)) +
           al(sizeof(unsigned int) * (size_t)(max_n + 2));
}

int launch_batched(int count, const skew_problem *problems, double *logabs, int32_t *sign,
                   int32_t *info, int max_n, void *ws, cudaStream_t stream, int sms) {
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    char *base = static_cast<char *>(ws);
    unsigned int *counter = reinterpret_cast<unsigned int *>(base);
    int32_t *order = reinterpret_cast<int32_t *>(base + al(sizeof(unsigned int)));
    unsigned int *hist = reinterpret_cast<unsigned int *>(
        base + al(sizeof(unsigned int)) + al(sizeof(int32_t) * (size_t)(count > 0 ? count : 1)));
    order_kernel<<<1, 1024, 0, stream>>>(count, problems, max_n, order, counter, hist);
    note_launches(1);
    SKEW_TRY_STATUS(check_launch());
    if (max_n <= kBlkMaxN) {
        // blocked variant: Lp, Ws and sv in shared memory
        const size_t nm = (size_t)(max_n > 1 ? max_n : 1);
        const BatchedNb tab = batched_nb_table();
        const int wnb = widest_nb(tab, max_n);
        const size_t bsmem = sizeof(double) * nm * (wnb + (wnb / 2 + 1) + 1);
        cudaError_t e = cudaFuncSetAttribute((const void *)batched_blocked_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)bsmem);
        if (e != cudaSuccess) {
            set_last_error(e);
            return SKEW_ERR_CUDA;
        }
        const int thr = tab.threads == 128 ? 128 : kBlkThreads;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_blocked_kernel,
                                                          thr, bsmem);
        if (e != cudaSuccess || per_sm < 1) {
            if (e != cudaSuccess) set_last_error(e);
            return SKEW_ERR_CUDA;
        }
        int grid = sms * per_sm;
        if (grid > count) grid = count;
        batched_blocked_kernel<<<grid, thr, bsmem, stream>>>(
            count, problems, order, counter, logabs, sign, info, max_n, tab);
        note_launches(1);
        return check_launch();
    }
    const size_t smem = 2 * sizeof(double) * (size_t)(max_n > 1 ? max_n : 1);
    static_assert(kBatchThreads == 512, "launch shape");
    cudaError_t e = cudaFuncSetAttribute((const void *)batched_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) {
        set_last_error(e);
        return SKEW_ERR_CUDA;
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel, kBatchThreads, smem);
    if (e != cudaSuccess || per_sm < 1) {
        if (e != cudaSuccess) set_last_error(e);
        return SKEW_ERR_CUDA;
    }
    int grid = sms * per_sm;
    if (grid > count) grid = count;
    batched_kernel<<<grid, kBatchThreads, smem, stream>>>(count, problems, order, counter,
                                                          logabs, sign, info, max_n);
    note_launches(1);
    return check_launch();
}

}  // namespace skew
