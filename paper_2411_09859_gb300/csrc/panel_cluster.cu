// panel_cluster.cu -- the pivoted left-looking panel for narrow trailing blocks, run by
// one thread-block cluster that exchanges each step's pivot candidates through
// distributed shared memory.
//
// The column steps are those of the shared-memory panel in panel.cu (Section 5.2:
// left-looking column v = X[k+1:, k] - L[k+1:, k0+1 .. k] h with h = T L[k, :]^T,
// Section 4.2; r = argmax |v| with the lowest index on ties; exchange of k+1 and r in
// the unfactored matrix and in the panel's L rows; t[k] = v[k+1] and L[k+2:, k+1] =
// v[k+2:] / t[k], Eq. (1)).  What differs is the per-step exchange.  There every CTA
// publishes its best candidate in global memory with a release-stored step tag and
// polls all the others' tags.  Here the whole grid is ONE cluster of at most 16 CTAs:
// each WARP leaves its best candidate and that row's L values (and the warp that owns
// row k+1 that row's L values and v[k+1]) in its CTA's shared memory, one cluster
// barrier makes them visible, and warp 0 of every CTA reads all the warps' candidates
// from the other CTAs' shared memory, then the winner's L row, and forms h; one CTA
// barrier hands the step to the other warps.  A step thus has one cluster barrier and
// one CTA barrier, and no CTA-wide candidate reduction.  The cluster barrier also
// orders the step's global writes (the exchanged entries of X) for the next step's
// readers.
//
// Used for trailing blocks of at most 16 x 256 rows (every row of the panel has its own
// thread), where a grid-wide exchange through L2 dominates a column step.  The
// cluster's CTAs are co-scheduled by the hardware, so there is no spin wait at all: no
// step can stall on a CTA that is not running.  Every exit is taken by all CTAs at the
// same point (the error flags travel with the candidates), after a last cluster
// barrier, so that no CTA leaves while another still reads its shared memory.
#include <climits>

#include <cooperative_groups.h>

#include "argmax.cuh"
#include "common.cuh"

namespace cg = cooperative_groups;

namespace skew {
namespace {

constexpr int kClMaxNb = 96;
constexpr int kClThreads = 256;     // up to 256 rows per CTA, one per thread
constexpr int kClWarps = kClThreads / 32;
constexpr int kClLds = kClThreads + 1;  // s_L column stride: a row's entries in distinct banks

// One warp's best candidate of a step (16 bytes: read remotely in one load).
struct __align__(16) ClusterSlot {
    unsigned long long raw;          // bits of the signed v
    int idx;                         // its row (INT_MAX: none)
    int bad;                         // a non-finite v or a recorded error in this warp
};

// What a CTA shows the cluster for one step (double-buffered by step parity).
struct ClusterPub {
    ClusterSlot slot[kClWarps];
    double vtop;                     // v[k+1] (written by the CTA that owns row k+1)
    double row[kClWarps][kClMaxNb];  // L[slot idx, k0+1 .. k] of each warp's candidate
    double rowp[kClMaxNb];           // L[k+1, k0+1 .. k] (the CTA that owns row k+1)
};

__global__ void __launch_bounds__(kClThreads)
panel_cluster_kernel(PanelArgs a) {
    extern __shared__ double s_L[];          // [q * kClLds + threadIdx.x], q < kend - k0
    __shared__ ClusterPub s_pub[2];
    __shared__ double s_t[kClMaxNb + 1];     // t of the panel's steps so far
    __shared__ double s_h[kClMaxNb + 1];     // h of the current step
    __shared__ double s_w[kClMaxNb];         // the winner's L row (the new row p)
    __shared__ double s_rp[kClMaxNb];        // row p's L row (the new row r)
    __shared__ double s_tau, s_vtop;
    __shared__ int s_r, s_win, s_fail;

    cg::cluster_group cluster = cg::this_cluster();
    Ctrl *ctrl = a.ctrl;
    const int n = a.n, k0 = a.k0, kend = a.kend;
    const int G = (int)gridDim.x;                   // = the cluster size, a power of two
    const int lg = __ffs(G) - 1;
    const int me = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double *X = a.X;
    const int64_t ldx = a.ldx, ldl = a.ldl;
    auto Lcol = [&](int q) -> double * { return a.Lp + (int64_t)(q - k0 - 1) * ldl; };
    auto sL = [&](int q) -> double & { return s_L[q * kClLds + tid]; };

    // this thread's row: 32-row chunk (warp G + cta), lane tid % 32
    const int64_t i = (int64_t)k0 + 1 + ((int64_t)((warp << lg) + me) << 5) + lane;
    const bool own = i < n;
    auto owner_cta = [&](int row) -> int { return ((row - k0 - 1) >> 5) & (G - 1); };
    auto owner_warp = [&](int row) -> int { return ((row - k0 - 1) >> 5) >> lg; };
    auto owner_tid = [&](int row) -> int {
        return (owner_warp(row) << 5) | ((row - k0 - 1) & 31);
    };
    // an error recorded before this launch (read by every CTA; the first exchange
    // makes the decision uniform)
    const bool fail0 = ld_volatile_i32(&ctrl->err) != 0;

    // Show this warp's step-k candidate to the cluster: its slot and its L row in
    // s_pub[k & 1] (and row k+1's L row, if this warp owns row k+1), then the cluster
    // barrier.  No CTA-wide reduction: the gather reads every warp's slot.
    auto publish = [&](int k, Best best, bool bad, double vtop_mine) {
        __syncwarp();                        // this warp's s_L writes of the step
        best = warp_best_all(best);
        const int wbad = __any_sync(0xffffffffu, bad);
        ClusterPub &pb = s_pub[k & 1];
        const int nq = k - k0;
        if (lane == 0) {
            ClusterSlot sl;
            sl.raw = best.raw;
            sl.idx = best.i;
            sl.bad = wbad;
            pb.slot[warp] = sl;
        }
        if (best.i != INT_MAX) {
            const int ot = owner_tid(best.i);
            for (int q = lane; q < nq; q += 32) pb.row[warp][q] = s_L[q * kClLds + ot];
        }
        if (k + 1 < n && owner_cta(k + 1) == me && owner_warp(k + 1) == warp) {
            const int ot = owner_tid(k + 1);
            for (int q = lane; q < nq; q += 32) pb.rowp[q] = s_L[q * kClLds + ot];
        }
        if (own && i == k + 1) pb.vtop = vtop_mine;
        cluster.sync();
    };

    // ---------------- step k0: v = X[k0+1:, k0]
    double v = 0.0;
    {
        const int k = k0;
        Best best = no_candidate();
        bool bad = fail0;
        if (own) {
            v = __ldcg(X + (int64_t)k * ldx + i);
            if (!finite_bits((unsigned long long)__double_as_longlong(v))) bad = true;
            offer(best, v, (int)i);
        }
        publish(k, best, bad, v);
    }

    bool failed = false;
    for (int k = k0; k < kend; ++k) {
        const int p = k + 1, nq = k - k0;
        const bool next = (k + 1 < kend);
        const bool form_x = (!next && a.with_x);
        double *colp = X + (int64_t)p * ldx;
        // column p of this row does not depend on the pivot: its load goes first
        double x_old = 0.0, xe = 0.0;
        if (own && i > p) x_old = __ldcg(colp + i);
        if (warp == 0) {
            // ---------------- the cluster's step-k candidates (the barrier was the last
            // one of publish): every warp's slot of every CTA, up to four per lane
            const ClusterPub *pp = cluster.map_shared_rank(&s_pub[k & 1], (unsigned)owner_cta(p));
            for (int q = lane; q < nq; q += 32) s_rp[q] = pp->rowp[q];   // row p: known already
            const double vt = pp->vtop;
            // all remote loads first (G <= 16: at most four slots per lane), then compare
            ClusterSlot sl[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int sidx = lane + 32 * u;
                if (sidx < (G << 3)) {
                    const ClusterPub *rp =
                        cluster.map_shared_rank(&s_pub[k & 1], (unsigned)(sidx >> 3));
                    sl[u] = rp->slot[sidx & 7];
                } else {
                    sl[u].raw = 0ull;
                    sl[u].idx = INT_MAX;
                    sl[u].bad = 0;
                }
            }
            Best b = no_candidate();
            int anybad = 0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                anybad |= sl[u].bad;
                if (better(sl[u].raw, sl[u].idx, b.raw, b.i)) {
                    b.raw = sl[u].raw;
                    b.i = sl[u].idx;
                    b.c = lane + 32 * u;
                }
            }
            anybad = __any_sync(0xffffffffu, anybad);
            b = warp_best_all(b);
            const int r = (b.i == INT_MAX) ? p : b.i;       // all NaN: keep the diagonal
            const int win = (b.i == INT_MAX) ? -1 : b.c;
            const double tau = (win < 0) ? vt : as_double(b.raw);
            if (!anybad) {
                // the winner's L row, then h = T L[p, :]^T over columns k0+1 .. k+1
                if (win >= 0) {
                    const ClusterPub *wp =
                        cluster.map_shared_rank(&s_pub[k & 1], (unsigned)(win >> 3));
                    for (int q = lane; q < nq; q += 32) s_w[q] = wp->row[win & 7][q];
                }
                __syncwarp();
                if (next || form_x) {
                    auto tq = [&](int q) -> double { return q == k ? tau : s_t[q - k0]; };
                    for (int q = k0 + 1 + lane; q <= k + 1; q += 32) {
                        double hq = 0.0;
                        if (q - 1 >= k0 + 1) hq = tq(q - 1) * s_w[q - 2 - k0];
                        if (q + 1 <= k + 1) {
                            const double lq1 = (q + 1 == k + 1) ? 1.0 : s_w[q - k0];
                            hq -= tq(q) * lq1;
                        }
                        s_h[q - k0 - 1] = hq;
                    }
                }
            }
            if (lane == 0) {
                s_fail = anybad;
                s_r = r;
                s_tau = tau;
                s_vtop = vt;
                s_win = win;
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
        if (own && i > p && r != p) {
            if (i < r) xe = __ldcg(X + i * ldx + r);                 // X[r, i]
            else if (i > r) xe = __ldcg(X + (int64_t)r * ldx + i);   // X[i, r]
        }
        // exchanged rows of the panel's L columns k0+1..k, by the warps that own them
        if (r != p && win >= 0) {
            if (owner_cta(p) == me && owner_warp(p) == warp) {
                const int ot = owner_tid(p);
                for (int q = lane; q < nq; q += 32) {
                    s_L[q * kClLds + ot] = s_w[q];
                    Lcol(k0 + 1 + q)[p] = s_w[q];
                }
            }
            if (owner_cta(r) == me && owner_warp(r) == warp) {
                const int ot = owner_tid(r);
                for (int q = lane; q < nq; q += 32) {
                    s_L[q * kClLds + ot] = s_rp[q];
                    Lcol(k0 + 1 + q)[r] = s_rp[q];
                }
            }
            __syncwarp();
        }

        Best best = no_candidate();
        bool bad = false;
        double vnext_top = 0.0;
        if (own && i >= p) {
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
                // symmetric exchange of p and r in the strictly lower storage
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
                if (next || form_x) {
                    const double vn = xn - (acc0 + acc1);
                    if (!finite_bits((unsigned long long)__double_as_longlong(vn))) bad = true;
                    if (form_x) {
                        colp[i] = vn;
                    } else {
                        v = vn;
                        vnext_top = vn;
                        offer(best, vn, (int)i);
                    }
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
    // no CTA leaves while another may still read its shared memory
    cluster.sync();
}

}  // namespace

bool panel_cluster_fits(int64_t rows, int width) {
    return rows >= 1 && rows <= 16LL * kClThreads && width <= kClMaxNb;
}

// CTAs of a cluster panel: the power of two that gives at most 128 rows each, at most
// 16 (then up to 256 rows each).
int cluster_grid(int64_t rows) {
    int g = 1;
    while (g < 16 && (int64_t)g * 128 < rows) g <<= 1;
    return g;
}

int launch_panel_cluster(const PanelArgs &a, cudaStream_t stream) {
    const int64_t rows = (int64_t)a.n - a.k0 - 1;
    const int width = a.kend - a.k0;
    if (!panel_cluster_fits(rows, width)) return SKEW_ERR_CUDA;
    const int g = cluster_grid(rows);
    const size_t smem = (size_t)(width > 0 ? width : 1) * kClLds * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute((const void *)panel_cluster_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kClMaxNb * kClLds * sizeof(double)));
    if (e == cudaSuccess && g > 8)
        e = cudaFuncSetAttribute((const void *)panel_cluster_kernel,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) {
        set_last_error(e);
        return SKEW_ERR_CUDA;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)g);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)g;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    PanelArgs args = a;
    e = cudaLaunchKernelEx(&cfg, panel_cluster_kernel, args);
    if (e != cudaSuccess) {
        set_last_error(e);
        return SKEW_ERR_CUDA;
    }
    note_launches(1);
    return SKEW_OK;
}

// Whether clusters of every size the cluster panel launches (1 .. 16 CTAs of 256
// threads with the largest shared memory) can be resident on this device.
int panel_cluster_supported(int *ok) {
    *ok = 0;
    cudaError_t e = cudaFuncSetAttribute((const void *)panel_cluster_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kClMaxNb * kClLds * sizeof(double)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void *)panel_cluster_kernel,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SKEW_OK;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = (size_t)kClMaxNb * kClLds * sizeof(double);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&clusters, (const void *)panel_cluster_kernel, &cfg);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SKEW_OK;
    }
    *ok = clusters >= 1 ? 1 : 0;
    return SKEW_OK;
}

}  // namespace skew
