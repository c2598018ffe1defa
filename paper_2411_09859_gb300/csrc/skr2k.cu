// skr2k.cu -- skew-symmetric rank-2k update of a strictly lower triangle on FP64
// tensor cores (DMMA, mma.sync.m8n8k4.f64).
//
//     C := beta C + alpha * sum_p (a_p w_p^T - w_p a_p^T),   strictly lower part only
//
// evaluated as the GEMM  C += U V^T  with U = [a_1 .. a_K, -w_1 .. -w_K] and
// V = [w_1 .. w_K, a_1 .. a_K] restricted to lower tiles (skew_rank2k, table of
// BLAS-like operations, Section 4.2).  The pairs (a_p, w_p) come from:
//
//   Rank2k  : a_p = X[:, p], w_p = Y[:, p].
//   Tridiag : A T A^T with T = S - S^T (Section 2.2 theorem): W = A S has only odd
//             columns, w_j = t[j] a_{j+1} - t[j-1] a_{j-1} (j odd, a_b := 0), and
//             A T A^T = W A^T - A W^T = -sum_{j odd} (a_j w_j^T - w_j a_j^T); so the
//             pairs are (a_j, w_j) with the sign folded into alpha.  This is the
//             "form W after the panel" two-step route of Section 4.2.
//   Fused   : the trailing update of one panel of the blocked right-looking
//             algorithm (Section 4.2 Variant 1): X44 -= A T_p A^T followed by the
//             last Gauss transform X44 += l x^T - x l^T, where l is A's last column
//             and x the already updated column.  Both are one update: the pairs of
//             Tridiag with x added to w_{b-1} when b is even (l = a_{b-1} is then
//             already a pair), or the extra pair (a_{b-1}, x) when b is odd.
//
// Out of place (Cin != nullptr, the look-ahead factorization): the old C is read from
// another buffer through a map of rows/columns (the panel's deferred exchanges) and C
// is only written; the update is otherwise the same.
//
// W is never stored: each CTA forms the pair columns of its row block while it
// stages them into shared memory (the GPU counterpart of forming T A^T while
// packing, Section 4.3).  FP64 throughput on this part is what bounds the kernel
// (about 1 TFLOP/s for the whole GPU), so the tile loop is kept simple: 64 x 64
// CTA tiles, four warps of 32 x 32, 16 pairs (32 K-columns) staged per round.
#include <atomic>
#include <climits>
#include <cmath>

#include "common.cuh"
#include "pairs.cuh"

namespace skew {
namespace {

constexpr int BM = 64;            // CTA tile (rows and columns)
constexpr int PC = 16;            // pairs per staging round
constexpr int KC = 2 * PC;        // K columns per staging round
constexpr int LDS = KC + 4;       // padded smem row (doubles): conflict-free fragments
constexpr int kThreads = 128;     // four warps
constexpr int64_t kSplitWaves = 8;  // updates of at most this many waves cut their tail

__device__ __forceinline__ void dmma_8x8x4(double &c0, double &c1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(c0), "+d"(c1)
                 : "d"(a), "d"(b));
}

// Lower-triangular tile index -> (bi, bj), bi >= bj, idx = bi (bi + 1) / 2 + bj.
__device__ __forceinline__ void tri_tile(int64_t idx, int64_t &bi, int64_t &bj) {
    int64_t r = (int64_t)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
    while (r * (r + 1) / 2 > idx) --r;
    while ((r + 1) * (r + 2) / 2 <= idx) ++r;
    bi = r;
    bj = idx - r * (r + 1) / 2;
}

// One TS x TS tile of C with rows I0.. and columns J0..: four warps of TS/2 x TS/2,
// each F x F DMMA fragments of 8 x 8 (F = TS / 16).
template <PairKind KIND, bool MAPPED, int TS>
__device__ __forceinline__ void skr2k_tile(int64_t I0, int64_t J0, int64_t m, double *C,
                                           int64_t ldc, double alpha, double beta,
                                           const PairSource<KIND> &src, const double *Cin,
                                           int64_t ldcin, const int32_t *map, int64_t nin,
                                           double (&Us)[BM][LDS], double (&Vs)[BM][LDS]) {
    constexpr int F = TS / 16;                     // fragments per warp and dimension
    constexpr int WT = TS / 2;                     // warp tile
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;       // warp quadrant
    const int g = lane >> 2, tg = lane & 3;        // fragment coordinates

    double acc[F][F][2];
#pragma unroll
    for (int mi = 0; mi < F; ++mi)
#pragma unroll
        for (int ni = 0; ni < F; ++ni) acc[mi][ni][0] = acc[mi][ni][1] = 0.0;

    const int64_t np = src.npairs();
    for (int64_t p0 = 0; p0 < np; p0 += PC) {
        const int nv = (int)((np - p0) < PC ? (np - p0) : PC);
        // ---- stage U rows I0.. and V rows J0.. for pairs p0 .. p0+PC-1
        for (int it = tid; it < TS * PC; it += kThreads) {
            const int r = it % TS, pp = it / TS;
            double ai = 0.0, wi = 0.0, aj = 0.0, wj = 0.0;
            if (pp < nv) {
                if (I0 + r < m) src.get(p0 + pp, I0 + r, ai, wi);
                if (J0 + r < m) src.get(p0 + pp, J0 + r, aj, wj);
            }
            Us[r][pp] = ai;
            Us[r][PC + pp] = -wi;
            Vs[r][pp] = wj;
            Vs[r][PC + pp] = aj;
        }
        __syncthreads();
        // ---- DMMA over the valid K columns of this round: [a | -w] x [w | a]^T
        const int ksteps = (nv + 3) / 4;
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
#pragma unroll 1
            for (int ks = 0; ks < ksteps; ++ks) {
                const int kc = half * PC + ks * 4 + tg;
                double af[F], bf[F];
#pragma unroll
                for (int mi = 0; mi < F; ++mi) af[mi] = Us[wm * WT + mi * 8 + g][kc];
#pragma unroll
                for (int ni = 0; ni < F; ++ni) bf[ni] = Vs[wn * WT + ni * 8 + g][kc];
#pragma unroll
                for (int mi = 0; mi < F; ++mi)
#pragma unroll
                    for (int ni = 0; ni < F; ++ni)
                        dmma_8x8x4(acc[mi][ni][0], acc[mi][ni][1], af[mi], bf[ni]);
            }
        }
        __syncthreads();
    }

    // ---- epilogue: strictly lower entries inside the block.  All C loads of a row
    // block are issued before its stores, so their latencies overlap.  Out of place,
    // the old entry (gi, gj) is entry (map[gi], map[gj]) of the skew matrix Cin.
    int cmap[F][2];
    if (MAPPED) {
#pragma unroll
        for (int ni = 0; ni < F; ++ni)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int64_t gj = J0 + wn * WT + ni * 8 + 2 * tg + c;
                cmap[ni][c] = gj < m ? __ldg(map + gj) : 0;
            }
    }
#pragma unroll
    for (int mi = 0; mi < F; ++mi) {
        const int64_t gi = I0 + wm * WT + mi * 8 + g;
        double cv[F][2];
        const int rmap = (MAPPED && gi < m) ? __ldg(map + gi) : 0;
#pragma unroll
        for (int ni = 0; ni < F; ++ni)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int64_t gj = J0 + wn * WT + ni * 8 + 2 * tg + c;
                const bool in = gi < m && gj < m && gi > gj && beta != 0.0;
                if (!in) {
                    cv[ni][c] = 0.0;
                } else if (!MAPPED) {
                    cv[ni][c] = C[gi + gj * ldc];
                } else {
                    // a map left by a failed panel is still read inside Cin
                    const int a = rmap, b = cmap[ni][c];
                    if ((uint64_t)a >= (uint64_t)nin || (uint64_t)b >= (uint64_t)nin || a == b)
                        cv[ni][c] = 0.0;
                    else
                        cv[ni][c] = a > b ? __ldg(Cin + a + (int64_t)b * ldcin)
                                          : -__ldg(Cin + b + (int64_t)a * ldcin);
                }
            }
#pragma unroll
        for (int ni = 0; ni < F; ++ni) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int64_t gj = J0 + wn * WT + ni * 8 + 2 * tg + c;
                if (gi < m && gj < m && gi > gj) {
                    double *dst = C + gi + gj * ldc;
                    const double upd = alpha * acc[mi][ni][c];
                    *dst = (beta == 0.0) ? upd : ((beta == 1.0) ? cv[ni][c] + upd : beta * cv[ni][c] + upd);
                }
            }
        }
    }
}


// Whole 64 x 64 lower tiles, one per block.
template <PairKind KIND, bool MAPPED>
__global__ void __launch_bounds__(kThreads, 2)
skr2k_kernel(int64_t m, double *C, int64_t ldc, double alpha, double beta,
             PairSource<KIND> src, const double *Cin, int64_t ldcin, const int32_t *map,
             int64_t nin) {
    __shared__ double Us[BM][LDS];
    __shared__ double Vs[BM][LDS];
    int64_t bi, bj;
    tri_tile(blockIdx.x, bi, bj);
    skr2k_tile<KIND, MAPPED, BM>(bi * BM, bj * BM, m, C, ldc, alpha, beta, src, Cin, ldcin,
                                 map, nin, Us, Vs);
}

// The lower tiles from `tile0` on, cut into four 32 x 32 quarters, one per block (a
// quarter entirely above the diagonal does nothing): the partial last wave of an
// update, a quarter as long as whole tiles would make it.
template <PairKind KIND, bool MAPPED>
__global__ void __launch_bounds__(kThreads, 2)
skr2k_quarter_kernel(int64_t m, double *C, int64_t ldc, double alpha, double beta,
                     PairSource<KIND> src, const double *Cin, int64_t ldcin,
                     const int32_t *map, int64_t nin, int64_t tile0) {
    __shared__ double Us[BM][LDS];
    __shared__ double Vs[BM][LDS];
    const int64_t q = blockIdx.x;
    int64_t bi, bj;
    tri_tile(tile0 + (q >> 2), bi, bj);
    const int si = (int)((q >> 1) & 1), sj = (int)(q & 1);
    if (bi == bj && si < sj) return;               // above the diagonal
    skr2k_tile<KIND, MAPPED, BM / 2>(bi * BM + si * (BM / 2), bj * BM + sj * (BM / 2), m, C,
                                     ldc, alpha, beta, src, Cin, ldcin, map, nin, Us, Vs);
}

// Both in one launch: blocks below `nfull` take whole tiles 0 .. nfull-1, the rest the
// quarters of the tiles from nfull on.  Used by the look-ahead's out-of-place update,
// which shares the device with a panel: its quarters then fill the slots as they free
// up, where a second launch would wait for the whole tiles to drain.  (Holding both tile
// sizes makes the whole-tile path of this kernel slower than skr2k_kernel's, so the
// in-place update keeps two launches.)
template <PairKind KIND, bool MAPPED>
__global__ void __launch_bounds__(kThreads, 2)
skr2k_mixed_kernel(int64_t m, double *C, int64_t ldc, double alpha, double beta,
                   PairSource<KIND> src, const double *Cin, int64_t ldcin, const int32_t *map,
                   int64_t nin, int64_t nfull) {
    __shared__ double Us[BM][LDS];
    __shared__ double Vs[BM][LDS];
    const int64_t b = blockIdx.x;
    int64_t bi, bj;
    if (b < nfull) {
        tri_tile(b, bi, bj);
        skr2k_tile<KIND, MAPPED, BM>(bi * BM, bj * BM, m, C, ldc, alpha, beta, src, Cin,
                                     ldcin, map, nin, Us, Vs);
    } else {
        const int64_t q = b - nfull;
        tri_tile(nfull + (q >> 2), bi, bj);
        const int si = (int)((q >> 1) & 1), sj = (int)(q & 1);
        if (bi == bj && si < sj) return;           // above the diagonal
        skr2k_tile<KIND, MAPPED, BM / 2>(bi * BM + si * (BM / 2), bj * BM + sj * (BM / 2), m,
                                         C, ldc, alpha, beta, src, Cin, ldcin, map, nin, Us,
                                         Vs);
    }
}

// Blocks of the update kernel resident on the current device at once (one wave), per
// device and instantiation, looked up once; 0 if the query fails (then every tile
// stays whole).
template <PairKind KIND>
int64_t skr2k_wave(bool mapped) {
    constexpr int kDevices = 64;
    static std::atomic<long long> cached[kDevices][2];         // 0: not looked up yet
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevices) {
        cudaGetLastError();
        return 0;
    }
    std::atomic<long long> &slot = cached[dev][mapped ? 1 : 0];
    long long w = slot.load();
    if (w > 0) return w;
    int sms = 0, per = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = mapped ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                         &per, skr2k_kernel<KIND, true>, kThreads, 0)
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                         &per, skr2k_kernel<KIND, false>, kThreads, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    w = (long long)per * sms;
    slot.store(w);
    return w;
}

template <PairKind KIND>
int launch_kind(const Skr2kArgs &a, cudaStream_t stream) {
    if (a.m <= 1) return SKEW_OK;
    const int64_t nt = (a.m + BM - 1) / BM;
    const int64_t tiles = nt * (nt + 1) / 2;
    if (tiles > INT_MAX) return SKEW_ERR_CUDA;      // unreachable: orders are capped
    PairSource<KIND> src{a.P, a.ldp, a.Q, a.ldq, a.tt, a.x, a.b};
    // whole waves of 64 x 64 tiles, then the rest as quarters in a second launch -- for
    // updates of at most kSplitWaves waves, where the partial last wave is a large share
    // of the time
    const bool mapped = a.Cin != nullptr;
    const int64_t wave = skr2k_wave<KIND>(mapped);
    const int64_t nfull =
        (wave > 0 && tiles <= kSplitWaves * wave) ? (tiles / wave) * wave : tiles;
    if (mapped && nfull < tiles) {
        const int64_t blocks = nfull + 4 * (tiles - nfull);
        skr2k_mixed_kernel<KIND, true><<<(unsigned)blocks, kThreads, 0, stream>>>(
            a.m, a.C, a.ldc, a.alpha, a.beta, src, a.Cin, a.ldcin, a.map, a.nin, nfull);
        note_launches(1);
        return check_launch();
    }
    if (nfull > 0) {
        if (mapped)
            skr2k_kernel<KIND, true><<<(unsigned)nfull, kThreads, 0, stream>>>(
                a.m, a.C, a.ldc, a.alpha, a.beta, src, a.Cin, a.ldcin, a.map, a.nin);
        else
            skr2k_kernel<KIND, false><<<(unsigned)nfull, kThreads, 0, stream>>>(
                a.m, a.C, a.ldc, a.alpha, a.beta, src, nullptr, 0, nullptr, 0);
        note_launches(1);
    }
    if (nfull < tiles) {
        const unsigned nq = (unsigned)(4 * (tiles - nfull));
        skr2k_quarter_kernel<KIND, false><<<nq, kThreads, 0, stream>>>(
            a.m, a.C, a.ldc, a.alpha, a.beta, src, nullptr, 0, nullptr, 0, nfull);
        note_launches(1);
    }
    return check_launch();
}

}  // namespace

int launch_skr2k(PairKind kind, const Skr2kArgs &a, cudaStream_t stream) {
    switch (kind) {
        case PairKind::Rank2k: return launch_kind<PairKind::Rank2k>(a, stream);
        case PairKind::Tridiag: return launch_kind<PairKind::Tridiag>(a, stream);
        default: return launch_kind<PairKind::Fused>(a, stream);
    }
}

}  // namespace skew
