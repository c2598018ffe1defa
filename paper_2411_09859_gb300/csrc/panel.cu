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
// GPU organisation: one CTA per SM (cooperative launch), rows of each column step
// spread over all threads (consecutive threads -> consecutive rows, so column reads
// of X and L are coalesced).  Each step has two grid barriers: after the gemv and the
// per-CTA argmax, and after the exchange and the scaling.  The unscaled v lives in L's
// column k+1 between the two phases; data written by other CTAs inside this launch
// is read with ld.global.cg (L2, never a stale L1 line).
#include <cfloat>
#include <climits>

#include "common.cuh"

namespace skew {
namespace {

__device__ __forceinline__ bool better(double va, int ia, double vb, int ib) {
    // (|va|, ia) beats (|vb|, ib): larger magnitude, then lower index.  A NaN
    // magnitude never wins (its comparisons are false).
    double a = fabs(va), b = fabs(vb);
    return (a > b) || (a == b && ia < ib);
}

struct Best {
    double v;
    int i;
};

__device__ __forceinline__ Best warp_best(Best x) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        double ov = __shfl_down_sync(0xffffffffu, x.v, off);
        int oi = __shfl_down_sync(0xffffffffu, x.i, off);
        if (better(ov, oi, x.v, x.i)) { x.v = ov; x.i = oi; }
    }
    return x;
}

// Reduce one Best per thread to thread 0 of the CTA.
__device__ Best block_best(Best x) {
    __shared__ double s_v[kPanelThreads / 32];
    __shared__ int s_i[kPanelThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    x = warp_best(x);
    if (lane == 0) { s_v[w] = x.v; s_i[w] = x.i; }
    __syncthreads();
    if (w == 0) {
        Best y;
        // (0, INT_MAX) is the "no candidate" value: any real entry beats it, because a
        // finite |v| > 0 is larger and |v| == 0 wins on the index
        y.v = (lane < kPanelThreads / 32) ? s_v[lane] : 0.0;
        y.i = (lane < kPanelThreads / 32) ? s_i[lane] : INT_MAX;
        x = warp_best(y);
    }
    __syncthreads();
    return x;
}

__global__ void __launch_bounds__(kPanelThreads)
panel_kernel(PanelArgs a) {
    __shared__ double s_h[kMaxNb + 1];
    __shared__ double s_tau, s_vtop;
    __shared__ int s_r;

    Ctrl *ctrl = a.ctrl;
    const int n = a.n, k0 = a.k0, kend = a.kend;
    const unsigned int G = gridDim.x;
    const int64_t nthreads = (int64_t)G * blockDim.x;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned int gen = 0;
    if (threadIdx.x == 0) gen = ld_acquire_u32(&ctrl->bar_gen);
    if (ld_volatile_i32(&ctrl->err) != 0) return;

    // L(i, q) for panel columns q in [k0+1, kend]
    auto Lcol = [&](int q) -> double * { return a.Lp + (int64_t)(q - k0 - 1) * a.ldl; };
    double *X = a.X;
    const int64_t ldx = a.ldx;

    // h = T L[k, :]^T restricted to the panel, into s_h[q - k0 - 1]
    auto form_h = [&](int k) {
        for (int q = k0 + 1 + threadIdx.x; q <= k; q += blockDim.x) {
            double hq = 0.0;
            if (q - 1 >= k0 + 1) hq = __ldcg(a.t + (q - 1)) * __ldcg(Lcol(q - 1) + k);
            if (q + 1 <= k) hq -= __ldcg(a.t + q) * __ldcg(Lcol(q + 1) + k);
            s_h[q - k0 - 1] = hq;
        }
        __syncthreads();
    };

    for (int k = k0; k < kend; ++k) {
        // ---------------- phase A: v = X[k+1:, k] - L[k+1:, k0+1..k] h; local argmax
        form_h(k);
        const int nq = k - k0;                   // panel columns already formed
        double *vcol = Lcol(k + 1);              // v is parked in L's column k+1
        const double *xk = X + (int64_t)k * ldx;
        Best best;
        best.v = 0.0;
        best.i = INT_MAX;
        bool nonfinite = false;
        for (int64_t i = k + 1 + gtid; i < n; i += nthreads) {
            double v = __ldcg(xk + i);
            for (int q = 0; q < nq; ++q) v -= __ldcg(a.Lp + (int64_t)q * a.ldl + i) * s_h[q];
            vcol[i] = v;
            if (i == k + 1) ctrl->vtop = v;
            if (!isfinite(v)) nonfinite = true;
            if (better(v, (int)i, best.v, best.i)) { best.v = v; best.i = (int)i; }
        }
        if (nonfinite) raise_error(ctrl, SKEW_ERR_NONFINITE);
        best = block_best(best);
        if (threadIdx.x == 0) {
            a.part[blockIdx.x].val = best.v;
            a.part[blockIdx.x].idx = best.i;
        }
        if (!grid_barrier(ctrl, G, gen)) return;

        // ---------------- phase B: global argmax, exchange k+1 <-> r, scale
        if (threadIdx.x < 32) {
            Best b;
            b.v = 0.0;
            b.i = INT_MAX;
            for (unsigned int c = threadIdx.x; c < G; c += 32) {
                double pv = __ldcg(&a.part[c].val);
                int pi = __ldcg(&a.part[c].idx);
                if (better(pv, pi, b.v, b.i)) { b.v = pv; b.i = pi; }
            }
            b = warp_best(b);
            if (threadIdx.x == 0) {
                int r = (b.i == INT_MAX) ? k + 1 : b.i;   // all NaN: keep the diagonal
                s_r = r;
                s_vtop = __ldcg(&ctrl->vtop);
                s_tau = (b.i == INT_MAX) ? s_vtop : b.v;
            }
        }
        __syncthreads();
        const int r = s_r, p = k + 1;
        const double tau = s_tau, vtop = s_vtop;
        if (gtid == 0) {
            a.t[k] = tau;
            a.piv[p] = r;
        }
        for (int64_t i = p + gtid; i < n; i += nthreads) {
            // L column k+1: 1 on the diagonal, v / tau below it (v[p] and v[r] exchanged)
            if (i == p) {
                vcol[i] = 1.0;
            } else {
                double v = (i == r) ? vtop : vcol[i];
                vcol[i] = (tau != 0.0) ? v / tau : 0.0;
            }
            if (r != p && i > p) {
                // symmetric exchange of indices p and r in the strictly lower storage
                double *colp = X + (int64_t)p * ldx;
                if (i < r) {
                    double *xri = X + (int64_t)i * ldx + r;    // X[r, i]
                    double tmp = __ldcg(colp + i);
                    colp[i] = -__ldcg(xri);
                    *xri = -tmp;
                } else if (i == r) {
                    colp[i] = -__ldcg(colp + i);
                } else {
                    double *colr = X + (int64_t)r * ldx;
                    double tmp = __ldcg(colp + i);
                    colp[i] = __ldcg(colr + i);
                    colr[i] = tmp;
                }
            }
        }
        // rows p and r of the panel's L columns k0+1 .. k
        if (r != p && blockIdx.x == 0) {
            for (int q = threadIdx.x; q < nq; q += blockDim.x) {
                double *col = a.Lp + (int64_t)q * a.ldl;
                double tmp = __ldcg(col + p);
                col[p] = __ldcg(col + r);
                col[r] = tmp;
            }
        }
        const bool last = (k + 1 == kend);
        if (!last || a.with_x) {
            if (!grid_barrier(ctrl, G, gen)) return;
        }
    }

    // ---------------- the updated column s = kend (for the fused trailing update)
    if (a.with_x) {
        const int s = kend;
        form_h(s);
        const int nq = s - k0;
        double *xs = X + (int64_t)s * ldx;
        bool nonfinite = false;
        for (int64_t i = s + 1 + gtid; i < n; i += nthreads) {
            double v = __ldcg(xs + i);
            for (int q = 0; q < nq; ++q) v -= __ldcg(a.Lp + (int64_t)q * a.ldl + i) * s_h[q];
            xs[i] = v;
            if (!isfinite(v)) nonfinite = true;
        }
        if (nonfinite) raise_error(ctrl, SKEW_ERR_NONFINITE);
    }
}

}  // namespace

int launch_panel(const PanelArgs &a, int grid, cudaStream_t stream) {
    PanelArgs args = a;
    void *params[] = {&args};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)panel_kernel, dim3(grid),
                                                dim3(kPanelThreads), params, 0, stream);
    if (e != cudaSuccess) {
        set_last_error(e);
        return SKEW_ERR_CUDA;
    }
    note_launches(1);
    return SKEW_OK;
}

int panel_max_blocks_per_sm(int *out) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, panel_kernel,
                                                                  kPanelThreads, 0);
    if (e != cudaSuccess) {
        set_last_error(e);
        return SKEW_ERR_CUDA;
    }
    return SKEW_OK;
}

}  // namespace skew
