// panel_la_cluster.cu -- the look-ahead panel (panel_la.cu) run by one thread-block
// cluster, beside the previous panel's trailing update.
//
// The column steps are those of panel_la.cu: the left-looking column over the previous
// panel's and this panel's L columns (Section 4.2, skew_tridiag_gemv, with kb = the
// previous panel's k0), read from the state S before the previous trailing update
// through a position map, with this panel's exchanges deferred into the map (Section
// 5.2 pivoting).  The per-step exchange is that of panel_cluster.cu: each warp leaves
// its best candidate (with the candidate row's source index and panel-start position)
// and its L row in its CTA's shared memory, one cluster barrier, then warp 0 of every
// CTA gathers all candidates through distributed shared memory, fetches the winner's
// row and forms h; one CTA barrier hands the step to the row warps.
//
// The cluster (at most 16 CTAs of 256 rows: trailing blocks up to 4096 rows, at most
// 96 L columns) takes at least 200 KB of shared memory per CTA, so that no CTA of the
// concurrent update is placed beside it: the update's FP64 work would otherwise share
// the multiprocessors of this latency-bound kernel.  No spin waits; every exit is
// uniform and follows a last cluster barrier.
#include <climits>

#include <cooperative_groups.h>

#include "argmax.cuh"
#include "common.cuh"

namespace cg = cooperative_groups;

namespace skew {
namespace {

constexpr int kLcMaxCols = 96;
constexpr int kLcThreads = 256;               // rows per CTA, one per thread
constexpr int kLcWarps = kLcThreads / 32;
constexpr int kLcLds = kLcThreads + 1;        // s_L column stride (distinct banks per row)
constexpr size_t kLcClaim = 200 * 1024;       // dynamic shared memory taken per CTA
constexpr unsigned int kLcNoPos = 0xffffu;

// One warp's best candidate: v bits and (position | source << 16 | panel-start position
// << 32 | bad << 48), 16 bytes read remotely in one load.
struct __align__(16) LcSlot {
    unsigned long long raw;
    unsigned long long meta;
};

struct LcPub {
    LcSlot slot[kLcWarps];
    double vtop;                      // v[k+1] (the CTA that owns row k+1)
    int psp, pop;                     // row k+1's source index and panel-start position
    double row[kLcWarps][kLcMaxCols];  // L[candidate, kb+1 .. k] of each warp's candidate
    double rowp[kLcMaxCols];          // L[k+1, kb+1 .. k]
};

// X[a, c] of the skew matrix held in the strictly lower triangle of S (a != c)
__device__ __forceinline__ double skew_at_lc(const double *S, int64_t lds, int a, int c) {
    return a > c ? __ldg(S + a + (int64_t)c * lds) : -__ldg(S + c + (int64_t)a * lds);
}

__global__ void __launch_bounds__(kLcThreads)
panel_la_cluster_kernel(PanelLAArgs a) {
    extern __shared__ double s_L[];          // [c * kLcLds + tid]: L column kb+1+c of the row
    __shared__ LcPub s_pub[2];
    __shared__ double s_t[kLcMaxCols + 1];   // t[c], index c - kb
    __shared__ double s_h[kLcMaxCols + 1];
    __shared__ double s_w[kLcMaxCols];       // the winner's L row (new row p)
    __shared__ double s_rp[kLcMaxCols];      // row p's L row (new row r)
    __shared__ double s_tau, s_vtop;
    __shared__ int s_r, s_win, s_fail, s_psr, s_por, s_psp, s_pop;

    cg::cluster_group cluster = cg::this_cluster();
    Ctrl *ctrl = a.ctrl;
    const int n = a.n, kb = a.kb, k0 = a.k0, kend = a.kend;
    const int nbj = k0 - kb;                 // L columns of the previous panel
    const int G = (int)gridDim.x;            // the cluster size, a power of two
    const int lg = __ffs(G) - 1;
    const int me = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double *S = a.S;
    const int64_t lds = a.lds, ldl = a.ldl;
    auto Lcol = [&](int q) -> double * { return a.Lp + (int64_t)(q - k0 - 1) * ldl; };
    auto sL = [&](int c) -> double & { return s_L[c * kLcLds + tid]; };

    // this thread's row: 32-row chunk (warp G + cta), lane
    const int i = k0 + 1 + (((warp << lg) + me) << 5) + lane;
    const bool own = i < n;
    auto owner_cta = [&](int row) -> int { return ((row - k0 - 1) >> 5) & (G - 1); };
    auto owner_warp = [&](int row) -> int { return ((row - k0 - 1) >> 5) >> lg; };
    auto owner_tid = [&](int row) -> int {
        return (owner_warp(row) << 5) | ((row - k0 - 1) & 31);
    };
    const bool fail0 = ld_volatile_i32(&ctrl->err) != 0;

    // source index (phs) and panel-start position (pho) of this thread's row; the
    // previous panel's L columns of the row and its t
    int phs = 0, pho = i;
    if (own) phs = a.map_prev ? __ldg(a.map_prev + i) : i;
    for (int c = 0; c < nbj; ++c) sL(c) = own ? __ldg(a.Lprev + i + (int64_t)c * a.ldlp) : 0.0;
    for (int c = tid; c < nbj; c += kLcThreads) s_t[c] = __ldcg(a.t + kb + c);

    // Show this warp's step-k candidate (with its row's source index and panel-start
    // position) and its L row over columns kb+1 .. k; the owner of row k+1 its row,
    // v, source index and position; then the cluster barrier.
    auto publish = [&](int k, Best best, bool bad, double vtop_mine) {
        __syncwarp();
        best.c = (int)(((unsigned int)phs << 16) | ((unsigned int)pho & 0xffffu));
        best = warp_best_all(best);
        const unsigned long long wbad = __any_sync(0xffffffffu, bad) ? 1ull : 0ull;
        LcPub &pb = s_pub[k & 1];
        const int nq = k - kb;
        if (lane == 0) {
            LcSlot sl;
            sl.raw = best.raw;
            const unsigned long long pos =
                best.i == INT_MAX ? (unsigned long long)kLcNoPos : (unsigned long long)best.i;
            const unsigned long long src = ((unsigned int)best.c >> 16) & 0xffffu;
            const unsigned long long p0 = (unsigned int)best.c & 0xffffu;
            sl.meta = pos | (src << 16) | (p0 << 32) | (wbad << 48);
            pb.slot[warp] = sl;
        }
        if (best.i != INT_MAX) {
            const int ot = owner_tid(best.i);
            for (int q = lane; q < nq; q += 32) pb.row[warp][q] = s_L[q * kLcLds + ot];
        }
        if (k + 1 < n && owner_cta(k + 1) == me && owner_warp(k + 1) == warp) {
            const int ot = owner_tid(k + 1);
            for (int q = lane; q < nq; q += 32) pb.rowp[q] = s_L[q * kLcLds + ot];
        }
        if (own && i == k + 1) {
            pb.vtop = vtop_mine;
            pb.psp = phs;
            pb.pop = pho;
        }
        cluster.sync();
    };

    // ---------------- step k0: v = the updated column k0
    double v = 0.0;
    {
        const int k = k0;
        Best best = no_candidate();
        bool bad = fail0;
        if (own) {
            if (a.xprev) {
                v = __ldcg(a.xprev + i);
            } else {
                const int c0 = a.map_prev ? __ldg(a.map_prev + k0) : k0;
                v = skew_at_lc(S, lds, phs, c0);
            }
            if (!finite_bits((unsigned long long)__double_as_longlong(v))) bad = true;
            offer(best, v, i);
        }
        publish(k, best, bad, v);
    }

    bool failed = false;
    for (int k = k0; k < kend; ++k) {
        const int p = k + 1, nq = k - kb;
        const bool next = (k + 1 < kend);
        const bool form_x = (!next && a.with_x);
        if (warp == 0) {
            // ---------------- every warp's candidate of every CTA (up to four per lane)
            const LcPub *pp = cluster.map_shared_rank(&s_pub[k & 1], (unsigned)owner_cta(p));
            for (int q = lane; q < nq; q += 32) s_rp[q] = pp->rowp[q];   // row p: known already
            const double vt = pp->vtop;
            const int psp = pp->psp, pop = pp->pop;
            LcSlot sl[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {      // all remote loads first, then compare
                const int sidx = lane + 32 * u;
                if (sidx < (G << 3)) {
                    const LcPub *rp = cluster.map_shared_rank(&s_pub[k & 1], (unsigned)(sidx >> 3));
                    sl[u] = rp->slot[sidx & 7];
                } else {
                    sl[u].raw = 0ull;
                    sl[u].meta = kLcNoPos;
                }
            }
            Best b = no_candidate();
            int anybad = 0;
            unsigned long long bmeta = kLcNoPos;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                anybad |= (int)((sl[u].meta >> 48) & 1ull);
                const unsigned int pos = (unsigned int)(sl[u].meta & 0xffffull);
                const int ipos = pos == kLcNoPos ? INT_MAX : (int)pos;
                if (better(sl[u].raw, ipos, b.raw, b.i)) {
                    b.raw = sl[u].raw;
                    b.i = ipos;
                    b.c = lane + 32 * u;
                    bmeta = sl[u].meta;
                }
            }
            anybad = __any_sync(0xffffffffu, anybad);
            b = warp_best_all(b);
            // the winning lane (the one whose slot index won) hands over the meta
            const int wl = (b.i == INT_MAX) ? 0 : (b.c & 31);
            const unsigned long long wmeta = __shfl_sync(0xffffffffu, bmeta, wl);
            const int r = (b.i == INT_MAX) ? p : b.i;       // all NaN: keep the diagonal
            const int win = (b.i == INT_MAX) ? -1 : b.c;
            const double tau = (win < 0) ? vt : as_double(b.raw);
            if (!anybad) {
                if (win >= 0) {
                    const LcPub *wp = cluster.map_shared_rank(&s_pub[k & 1], (unsigned)(win >> 3));
                    for (int q = lane; q < nq; q += 32) s_w[q] = wp->row[win & 7][q];
                }
                __syncwarp();
                if (next || form_x) {
                    // h over columns kb+1 .. k+1 from the new row p: L[p, c] = s_w[c - kb - 1]
                    // for c <= k, L[p, k+1] = 1; t[c] = s_t[c - kb] for c < k, t[k] = tau
                    auto tq = [&](int q) -> double { return q == k ? tau : s_t[q - kb]; };
                    for (int q = kb + 1 + lane; q <= k + 1; q += 32) {
                        double hq = 0.0;
                        if (q - 1 >= kb + 1) hq = tq(q - 1) * s_w[q - 2 - kb];
                        if (q + 1 <= k + 1) {
                            const double lq1 = (q + 1 == k + 1) ? 1.0 : s_w[q - kb];
                            hq -= tq(q) * lq1;
                        }
                        s_h[q - kb - 1] = hq;
                    }
                }
            }
            if (lane == 0) {
                s_fail = anybad;
                s_r = r;
                s_tau = tau;
                s_vtop = vt;
                s_win = win;
                s_psr = (int)((wmeta >> 16) & 0xffffull);
                s_por = (int)((wmeta >> 32) & 0xffffull);
                s_psp = psp;
                s_pop = pop;
                s_t[nq] = tau;
                if (me == 0 && !anybad) {
                    a.t[k] = tau;
                    a.piv[p] = r;
                }
            }
        }
        __syncthreads();
        if (s_fail) {              // the same decision in every CTA: leave together
            failed = true;
            break;
        }
        const int r = s_r, win = s_win;
        const double tau = s_tau, vtop = s_vtop;
        const int psr = (win >= 0) ? s_psr : s_psp;     // source index of the new column p
        // the new row r (old row p) takes old row p's source index and position; the new
        // row p those of the winner
        if (own && i == r && r != p) {
            phs = s_psp;
            pho = s_pop;
        } else if (own && i == p && r != p) {
            phs = psr;
            pho = s_por;
        }
        double x_new = 0.0;
        if (own && i > p) x_new = skew_at_lc(S, lds, phs, psr);
        // exchanged rows of the L columns kb+1 .. k, by the warps that own them; this
        // panel's own columns also in global memory
        if (r != p && win >= 0) {
            if (owner_cta(p) == me && owner_warp(p) == warp) {
                const int ot = owner_tid(p);
                for (int q = lane; q < nq; q += 32) {
                    s_L[q * kLcLds + ot] = s_w[q];
                    if (q >= nbj) Lcol(kb + 1 + q)[p] = s_w[q];
                }
            }
            if (owner_cta(r) == me && owner_warp(r) == warp) {
                const int ot = owner_tid(r);
                for (int q = lane; q < nq; q += 32) {
                    s_L[q * kLcLds + ot] = s_rp[q];
                    if (q >= nbj) Lcol(kb + 1 + q)[r] = s_rp[q];
                }
            }
            __syncwarp();
        }

        Best best = no_candidate();
        bool bad = false;
        double vnext_top = 0.0;
        if (own && i >= p) {
            // ---- finish step k for this row: L column k+1
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
                if (!finite_bits((unsigned long long)__double_as_longlong(vn))) bad = true;
                if (form_x) {
                    a.xout[i] = vn;
                } else {
                    v = vn;
                    vnext_top = vn;
                    offer(best, vn, i);
                }
            }
        }
        if (next) {
            publish(k + 1, best, bad, vnext_top);
        } else if (bad) {
            raise_error(ctrl, SKEW_ERR_NONFINITE);
        }
    }
    if (failed && me == 0 && tid == 0 && !fail0) raise_error(ctrl, SKEW_ERR_NONFINITE);
    // the map stays a valid permutation on every exit (the update that follows reads it)
    if (own && a.map_out) a.map_out[i] = pho;
    // no CTA leaves while another may still read its shared memory
    cluster.sync();
}

}  // namespace

// Whether a look-ahead panel of `rows` trailing rows and `cols` L columns can run as
// one cluster (and clusters of 16 such CTAs can be resident: `cluster_ok`).
bool panel_la_cluster_fits(int64_t rows, int cols) {
    return rows >= 1 && rows <= 16LL * kLcThreads && cols <= kLcMaxCols;
}

int launch_panel_la_cluster(const PanelLAArgs &a, cudaStream_t stream) {
    const int64_t rows = (int64_t)a.n - a.k0 - 1;
    const int cols = (a.k0 - a.kb) + (a.kend - a.k0);
    if (!panel_la_cluster_fits(rows, cols)) return SKEW_ERR_CUDA;
    int g = 1;
    while (g < 16 && (int64_t)g * 128 < rows) g <<= 1;
    cudaError_t e = cudaFuncSetAttribute((const void *)panel_la_cluster_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kLcClaim);
    if (e == cudaSuccess && g > 8)
        e = cudaFuncSetAttribute((const void *)panel_la_cluster_kernel,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) {
        set_last_error(e);
        return SKEW_ERR_CUDA;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)g);
    cfg.blockDim = dim3(kLcThreads);
    cfg.dynamicSmemBytes = kLcClaim;     // >= cols * kLcLds doubles
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)g;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    PanelLAArgs args = a;
    e = cudaLaunchKernelEx(&cfg, panel_la_cluster_kernel, args);
    if (e != cudaSuccess) {
        set_last_error(e);
        return SKEW_ERR_CUDA;
    }
    note_launches(1);
    return SKEW_OK;
}

// Whether clusters of 16 look-ahead panel CTAs (256 threads, the claimed shared memory)
// can be resident on this device.
int panel_la_cluster_supported(int *ok) {
    *ok = 0;
    cudaError_t e = cudaFuncSetAttribute((const void *)panel_la_cluster_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kLcClaim);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void *)panel_la_cluster_kernel,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SKEW_OK;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(kLcThreads);
    cfg.dynamicSmemBytes = kLcClaim;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&clusters, (const void *)panel_la_cluster_kernel, &cfg);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SKEW_OK;
    }
    *ok = clusters >= 1 ? 1 : 0;
    return SKEW_OK;
}

}  // namespace skew
