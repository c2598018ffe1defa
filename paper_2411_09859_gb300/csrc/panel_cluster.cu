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
// each CTA leaves its candidate (and its L row, and row k+1's row and v if it owns row
// k+1) in its own shared memory, one cluster barrier makes them visible, and every CTA
// reads them from the other CTAs' shared memory.  The cluster barrier also orders the
// step's global writes (the exchanged entries of X) for the next step's readers.
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

// What a CTA shows the cluster for one step (double-buffered by step parity).
struct ClusterPub {
    unsigned long long raw;          // the CTA's best candidate: bits of the signed v
    int idx;                         // its row (INT_MAX: none)
    int bad;                         // a non-finite v or a recorded error in this CTA
    double vtop;                     // v[k+1] (written by the CTA that owns row k+1)
    double row[kClMaxNb];            // L[idx, k0+1 .. k]
    double rowp[kClMaxNb];           // L[k+1, k0+1 .. k] (the CTA that owns row k+1)
};

__global__ void __launch_bounds__(kClThreads)
panel_cluster_kernel(PanelArgs a) {
    extern __shared__ double s_L[];          // [q][threadIdx.x], q < kend - k0
    __shared__ ClusterPub s_pub[2];
    __shared__ double s_h[kClMaxNb + 1];
    __shared__ double s_t[kClMaxNb + 1];
    __shared__ double s_w[kClMaxNb + 1];
    __shared__ double s_rp[kClMaxNb + 1];
    __shared__ unsigned long long s_wraw[kClThreads / 32];
    __shared__ int s_wi[kClThreads / 32];
    __shared__ int s_wbad[kClThreads / 32];
    __shared__ double s_tau, s_vtop;
    __shared__ int s_r, s_win, s_fail;

    cg::cluster_group cluster = cg::this_cluster();
    Ctrl *ctrl = a.ctrl;
    const int n = a.n, k0 = a.k0, kend = a.kend;
    const int G = (int)gridDim.x;                   // = the cluster size
    const int me = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double *X = a.X;
    const int64_t ldx = a.ldx, ldl = a.ldl;
    auto Lcol = [&](int q) -> double * { return a.Lp + (int64_t)(q - k0 - 1) * ldl; };
    auto sL = [&](int q) -> double & { return s_L[q * kClThreads + tid]; };

    // this thread's row: chunk warp * G + cta, lane tid % 32
    const int64_t i = (int64_t)k0 + 1 + ((int64_t)(warp * G + me) << 5) + lane;
    const bool own = i < n;
    auto owner_cta = [&](int row) -> int { return ((row - k0 - 1) >> 5) % G; };
    auto owner_tid = [&](int row) -> int {
        const int j = row - k0 - 1;
        return (((j >> 5) / G) << 5) + (j & 31);
    };
    // an error recorded before this launch (read by every CTA; the first exchange
    // makes the decision uniform)
    const bool fail0 = ld_volatile_i32(&ctrl->err) != 0;

    // Show this CTA's step-k candidate to the cluster: reduce over the CTA, copy the
    // candidate's L row (and row k+1's, with v[k+1], if this CTA owns row k+1) into
    // s_pub[k & 1], then the cluster barrier.
    auto publish = [&](int k, Best best, bool bad, double vtop_mine) {
        best = warp_best_all(best);
        const int wbad = __any_sync(0xffffffffu, bad);
        if (lane == 0) {
            s_wraw[warp] = best.raw;
            s_wi[warp] = best.i;
            s_wbad[warp] = wbad;
        }
        ClusterPub &pb = s_pub[k & 1];
        if (own && i == k + 1) pb.vtop = vtop_mine;
        __syncthreads();
        if (warp == 0) {
            Best y = no_candidate();
            int yb = 0;
            if (lane < kClThreads / 32) {
                y.raw = s_wraw[lane];
                y.i = s_wi[lane];
                yb = s_wbad[lane];
            }
            y = warp_best_all(y);
            yb = __any_sync(0xffffffffu, yb);
            if (lane == 0) {
                pb.raw = y.raw;
                pb.idx = y.i;
                pb.bad = yb;
            }
            const int nq = k - k0;
            if (y.i != INT_MAX) {
                const int ot = owner_tid(y.i);
                for (int q = lane; q < nq; q += 32) pb.row[q] = s_L[q * kClThreads + ot];
            }
            if (k + 1 < n && owner_cta(k + 1) == me) {
                const int ot = owner_tid(k + 1);
                for (int q = lane; q < nq; q += 32) pb.rowp[q] = s_L[q * kClThreads + ot];
            }
        }
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
        // ---------------- the step-k candidates of the cluster (the barrier was the
        // last one of publish); warp 0 reads them from every CTA's shared memory
        if (warp == 0) {
            Best b = no_candidate();
            int anybad = 0;
            for (int c = lane; c < G; c += 32) {
                const ClusterPub *rp = cluster.map_shared_rank(&s_pub[k & 1], (unsigned)c);
                const unsigned long long pr = rp->raw;
                const int pi = rp->idx;
                anybad |= rp->bad;
                if (better(pr, pi, b.raw, b.i)) { b.raw = pr; b.i = pi; b.c = c; }
            }
            anybad = __any_sync(0xffffffffu, anybad);
            b = warp_best_all(b);
            if (lane == 0) {
                s_fail = anybad;
                s_r = (b.i == INT_MAX) ? k + 1 : b.i;    // all NaN: keep the diagonal
                s_tau = as_double(b.raw);
                s_win = (b.i == INT_MAX) ? -1 : b.c;
            }
        }
        __syncthreads();
        if (s_fail) {              // the same decision in every CTA: leave together
            failed = true;
            break;
        }
        const int r = s_r, p = k + 1, nq = k - k0;
        // ---------------- the winner's row, row k+1's row and v[k+1], from the CTAs
        // that hold them; and this thread's entries of X for the exchange
        const int op = owner_cta(p);
        if (s_win >= 0) {
            const ClusterPub *wp = cluster.map_shared_rank(&s_pub[k & 1], (unsigned)s_win);
            const ClusterPub *pp = cluster.map_shared_rank(&s_pub[k & 1], (unsigned)op);
            for (int q = tid; q < nq; q += kClThreads) {
                s_w[q] = wp->row[q];
                s_rp[q] = pp->rowp[q];
            }
        }
        if (tid == 0) {
            const ClusterPub *pp = cluster.map_shared_rank(&s_pub[k & 1], (unsigned)op);
            const double vt = pp->vtop;
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
        if (tid == 0) s_t[k - k0] = tau;
        if (me == 0 && tid == 0) {
            a.t[k] = tau;
            a.piv[p] = r;
        }
        // exchanged rows of the panel's L columns k0+1..k
        if (r != p && s_win >= 0) {
            if (owner_cta(p) == me) {
                const int ot = owner_tid(p);
                for (int q = tid; q < nq; q += kClThreads) {
                    s_L[q * kClThreads + ot] = s_w[q];
                    Lcol(k0 + 1 + q)[p] = s_w[q];
                }
            }
            if (owner_cta(r) == me) {
                const int ot = owner_tid(r);
                for (int q = tid; q < nq; q += kClThreads) {
                    s_L[q * kClThreads + ot] = s_rp[q];
                    Lcol(k0 + 1 + q)[r] = s_rp[q];
                }
            }
        }
        const bool next = (k + 1 < kend);
        const bool form_x = (!next && a.with_x);
        if (next || form_x) {
            auto tq = [&](int q) -> double { return q == k ? tau : s_t[q - k0]; };
            for (int q = k0 + 1 + tid; q <= k + 1; q += kClThreads) {
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

// CTAs of a cluster panel: one per 128 rows, at most 16 (then up to 256 rows each).
int cluster_grid(int64_t rows) {
    int64_t g = (rows + 127) / 128;
    if (g > 16) g = 16;
    if (g < 1) g = 1;
    return (int)g;
}

int launch_panel_cluster(const PanelArgs &a, cudaStream_t stream) {
    const int64_t rows = (int64_t)a.n - a.k0 - 1;
    const int width = a.kend - a.k0;
    if (!panel_cluster_fits(rows, width)) return SKEW_ERR_CUDA;
    const int g = cluster_grid(rows);
    const size_t smem = (size_t)(width > 0 ? width : 1) * kClThreads * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute((const void *)panel_cluster_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kClMaxNb * kClThreads * sizeof(double)));
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
                                         (int)(kClMaxNb * kClThreads * sizeof(double)));
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
    cfg.dynamicSmemBytes = (size_t)kClMaxNb * kClThreads * sizeof(double);
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
