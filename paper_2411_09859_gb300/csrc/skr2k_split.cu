// skr2k_split.cu -- the skew rank-2k update C += U V^T (strictly lower part) with the
// FP64 operands split into 8-bit digit slices multiplied on the fifth-generation tensor
// cores (tcgen05.mma kind::f16, bf16 inputs, FP32 accumulators in tensor memory), the
// slices loaded by TMA, and the products recombined exactly in 64-bit integers.
//
// This is the error-free splitting of Ozaki, Ogita, Oishi and Rump (2012), "Error-
// free transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", in fixed-point form with balanced digits:
//
//   - every row i of the pair columns (a_p, w_p) gets the exponent E_i of its
//     largest entry; each entry x becomes the signed integer X = trunc(x 2^(54-E_i)),
//     |X| < 2^55 (exact for entries within a factor 4 of the row maximum), written
//     with seven base-256 digits X = sum_{s=1..7} d_s 2^(8(7-s)): d_7 .. d_2 balanced
//     in [-128, 127], d_1 what remains (|d_1| <= 128); every digit is exact in bf16;
//   - U = [a | -w] and V = [w | a] (64 columns, zero padded past the pairs);
//   - (U V^T)[i,j] ~ 2^(E_i+E_j-54) acc with acc = sum_{d=2..9} P_d 2^(58-8d) and
//     P_d = sum_{s+t=d} U_s V_t^T.  |P_d| <= 7 * 64 * 2^14 < 2^24, so each P_d is an
//     exact FP32 tensor-core sum and its conversion to an integer is exact; acc is
//     exact up to the truncation of the lowest bits of P_8 and P_9 (|acc| < 2^62).
//
// The products with s + t > 9 and the bits below 2^(E_i-54) are dropped: the result
// differs from the exact update by at most about 1.1 * 2^-53 * K * (max row entry of
// U) * (max row entry of V) -- the size of FP64 rounding in an ordinary dot product,
// but measured against row maxima rather than entry by entry.  K = 2 * pairs <= 64.
// So that a large sub-diagonal entry of T (w_j carries t_j), or a large trailing column
// in the two-step update, does not raise the row maxima, each pair of a factorization's
// trailing update is first balanced by exact powers of two, (a_p, w_p) -> (2^e_p a_p,
// 2^-e_p w_p), with e_p from the pair's column maxima; this leaves its term
// a_p w_p^T - w_p a_p^T unchanged (split_colexp_kernel, balance_exp).
//
// Update kernel: persistent, one CTA per SM, tiles of 128 rows x 32 columns of the
// lower triangle of C, each CTA taking a contiguous run of tiles (consecutive tiles
// share their 128-row block, so the U slices are loaded once per run).  For one digit
// s of U, the products with every digit t of V are a single MMA: the V slices t = 1..T
// lie one after another in shared memory, so together they form one B operand of
// 32 T rows, and the result columns (t, j) are exactly the accumulator columns of the
// groups d = s + t, 32 columns per group.  Seven MMAs per K-step (N = 256, 224, 192,
// ..., 64; the first one reads one extra all-zero slice so that it initialises all
// eight groups) cover the 34 slice products.  Warp roles:
//   warp 0   TMA producer: U slices of the row block (7 x 128 x 64 bf16, 112 KB, one
//            3-D box) and V slices of the column block (7 x 32 x 64, 28 KB) into three
//            V buffers;
//   warp 1   allocates 512 tensor-memory columns (two accumulators of 8 groups x 32
//            columns, so the MMAs of the next tile overlap the epilogue of this one);
//            one thread issues the 28 MMAs of a tile and commits them to an mbarrier;
//   warps 2-17 epilogue: warp w reads lanes 32 (w mod 4) .. +31 (its 32 rows) and one
//            8-column quarter of the tile for all eight groups, combines them in 64-bit
//            integers, and updates C in FP64.
// Every wait is bounded (kSplitTimeoutNs); on a timeout the kernel records
// SKEW_ERR_TIMEOUT, every role leaves its loop, the issued copies and MMAs are waited
// for (bounded again), the tensor memory is freed and the kernel returns.
#include <climits>
#include <mutex>

#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "pairs.cuh"
#include "tc.cuh"

namespace skew {
namespace {

constexpr int kSlices = 7;
constexpr int kGroups = 8;                  // d = s + t = 2 .. 9
constexpr int kK = 64;                      // columns of U and V (bf16): one 128-byte row
constexpr int kTM = 128;                    // tile rows (MMA M)
constexpr int kTN = 32;                     // tile columns = accumulator columns per group
constexpr int kEpiWarps = 16;
constexpr int kEpiCols = 8;                 // tile columns per epilogue warp
constexpr int kThreads = 32 * (2 + kEpiWarps);   // producer, MMA, epilogue
constexpr int kVBufs = 3;
constexpr uint32_t kAccCols = kGroups * kTN;            // 256 per accumulator
constexpr uint32_t kTmemCols = 2 * kAccCols;            // two accumulators
constexpr uint32_t kUSlice = kTM * kK * 2;              // 16384
constexpr uint32_t kVSlice = kTN * kK * 2;              // 4096
constexpr uint32_t kUBytes = kSlices * kUSlice;         // 114688
constexpr uint32_t kVLoad = kSlices * kVSlice;          // 28672: slices 1..7
constexpr uint32_t kVBuf = (kSlices + 1) * kVSlice;     // 32768: + one zero slice
constexpr size_t kSmemBytes = 1024 + kUBytes + kVBufs * kVBuf + 256;
static_assert(kSmemBytes <= 227 * 1024, "shared memory");
static_assert(kTmemCols <= 512, "tensor memory");
constexpr uint64_t kSplitTimeoutNs = 2000000000ull;    // 2 s

// unbiased exponent and 53-bit significand of |x| (subnormals: exponent -1022)
__device__ __forceinline__ void decompose(double x, int &ex, unsigned long long &mant) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ef = (int)((b >> 52) & 0x7ff);
    mant = b & 0x000fffffffffffffull;
    if (ef == 0) {
        ex = -1022;
    } else {
        ex = ef - 1023;
        mant |= 0x0010000000000000ull;
    }
}

__device__ __forceinline__ int exponent_of(double x) {
    int ex;
    unsigned long long m;
    decompose(x, ex, m);
    return m == 0 ? INT_MIN / 2 : ex;
}

// X = trunc(x 2^(54-E)) with the sign of x (|x| < 2^(E+1), so |X| < 2^55)
__device__ __forceinline__ long long fixed55(double x, int E) {
    int ex;
    unsigned long long m;
    decompose(x, ex, m);
    const int sh = ex - E + 2;             // |x| = m 2^(ex-52); X = m 2^(ex+2-E)
    unsigned long long X;
    if (sh >= 0) X = m << sh;              // sh <= 2
    else if (sh <= -64) X = 0ull;
    else X = m >> (-sh);
    return x < 0.0 ? -(long long)X : (long long)X;
}

__device__ __forceinline__ unsigned int bf16_bits(int d) {
    const __nv_bfloat16 h = __int2bfloat16_rn(d);   // |d| <= 128: exact
    return (unsigned int)*reinterpret_cast<const unsigned short *>(&h);
}

__device__ __forceinline__ unsigned int pack2(int lo, int hi) {
    return bf16_bits(lo) | (bf16_bits(hi) << 16);
}

// 2^e as a double (|e| <= 1000: a normal number)
__device__ __forceinline__ double pow2(int e) {
    return __longlong_as_double((long long)(1023 + e) << 52);
}

// Balancing of the pairs (trailing updates of the factorizations): the term
// a_p w_p^T - w_p a_p^T is unchanged when a_p is scaled by 2^e_p and w_p by 2^-e_p
// (exactly, both being powers of two).  With Ea_p and Ew_p the largest exponents in
// the columns a_p and w_p, e_p = ceil((Ew_p - Ea_p) / 2) brings both columns to the
// same size, so that no column of a row lies far below the row's largest entry only
// because the pairs differ in scale (a large T entry in w_j = t_j a_{j+1} - ..., or a
// large trailing column y in the two-step update); the digits then keep the precision
// of every column (the bound below is measured against row maxima).
constexpr int kNoExp = (int)0x80808080;      // the byte pattern the column maxima start from

__device__ __forceinline__ int balance_exp(int ea, int ew) {
    if (ea < -1100 || ew < -1100) return 0;  // an all-zero column
    const int e = (ew - ea + 1) >> 1;
    return e > 400 ? 400 : (e < -400 ? -400 : e);
}

// Column maxima of the exponents of the pairs: colexp[p] for a_p, colexp[32 + p] for
// w_p (four threads per row as in the pre-pass; reduced per CTA, then atomicMax).
template <PairKind KIND>
__global__ void __launch_bounds__(256)
split_colexp_kernel(int64_t m, PairSource<KIND> src, int P, int *colexp) {
    __shared__ int s_max[64];
    const int64_t i = (int64_t)blockIdx.x * 64 + (threadIdx.x >> 2);
    const int g = threadIdx.x & 3;
    if (threadIdx.x < 64) s_max[threadIdx.x] = kNoExp;
    __syncthreads();
    int ea[8], ew[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int p = 8 * g + q;
        ea[q] = ew[q] = kNoExp;
        if (i < m && p < P) {
            double av, wv;
            src.get(p, i, av, wv);
            ea[q] = exponent_of(av) < -1100 ? kNoExp : exponent_of(av);
            ew[q] = exponent_of(wv) < -1100 ? kNoExp : exponent_of(wv);
        }
        // the lanes holding the same pairs differ in lane bits 2, 3, 4
#pragma unroll
        for (int off = 4; off < 32; off <<= 1) {
            ea[q] = max(ea[q], __shfl_xor_sync(0xffffffffu, ea[q], off));
            ew[q] = max(ew[q], __shfl_xor_sync(0xffffffffu, ew[q], off));
        }
    }
    if ((threadIdx.x & 31) < 4) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            atomicMax(&s_max[8 * g + q], ea[q]);
            atomicMax(&s_max[32 + 8 * g + q], ew[q]);
        }
    }
    __syncthreads();
    if (threadIdx.x < 64 && s_max[threadIdx.x] != kNoExp) atomicMax(&colexp[threadIdx.x], s_max[threadIdx.x]);
}

// Pre-pass, four threads per row i (thread g of the row takes pairs 8g .. 8g+7): the
// pairs balanced by 2^(+-e_p) (balance_exp, when colexp is given), the exponent E_i of the row's
// largest balanced entry, and the digit slices Zu[s][i][0..63] = digits of [a | -w],
// Zv[s][i][0..63] = digits of [w | a] (pair p in column p of each half, zero past P).
template <PairKind KIND>
__global__ void __launch_bounds__(256)
split_prepare_kernel(int64_t m, PairSource<KIND> src, int P, unsigned short *Zu,
                     unsigned short *Zv, int *rowexp, const int *colexp) {
    const int64_t i = (int64_t)blockIdx.x * 64 + (threadIdx.x >> 2);
    const int g = threadIdx.x & 3;
    double av[8], wv[8];
    int E = INT_MIN / 2;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int p = 8 * g + q;
        av[q] = 0.0;
        wv[q] = 0.0;
        if (i < m && p < P) {
            src.get(p, i, av[q], wv[q]);
            const int e = colexp ? balance_exp(__ldg(colexp + p), __ldg(colexp + 32 + p)) : 0;
            if (e != 0) {
                av[q] *= pow2(e);
                wv[q] *= pow2(-e);
            }
            E = max(E, max(exponent_of(av[q]), exponent_of(wv[q])));
        }
    }
    E = max(E, __shfl_xor_sync(0xffffffffu, E, 1));
    E = max(E, __shfl_xor_sync(0xffffffffu, E, 2));
    if (i >= m) return;
    if (E < -1022) E = -1022;                  // an all-zero row
    if (g == 0) rowexp[i] = E;
    long long Xa[8], Xw[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        Xa[q] = fixed55(av[q], E);
        Xw[q] = fixed55(wv[q], E);
    }
    const size_t slice = (size_t)m * kK;
    // digits from the least significant (slice 7) up; slice 1 takes what remains
#pragma unroll
    for (int s = kSlices - 1; s >= 0; --s) {
        int da[8], dw[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (s > 0) {
                da[q] = (int)((Xa[q] + 128) & 255) - 128;
                dw[q] = (int)((Xw[q] + 128) & 255) - 128;
                Xa[q] = (Xa[q] - da[q]) >> 8;
                Xw[q] = (Xw[q] - dw[q]) >> 8;
            } else {
                da[q] = (int)Xa[q];
                dw[q] = (int)Xw[q];
            }
        }
        unsigned short *zu = Zu + s * slice + (size_t)i * kK + 8 * g;
        unsigned short *zv = Zv + s * slice + (size_t)i * kK + 8 * g;
        const uint4 ua = make_uint4(pack2(da[0], da[1]), pack2(da[2], da[3]), pack2(da[4], da[5]),
                                    pack2(da[6], da[7]));
        const uint4 uw = make_uint4(pack2(dw[0], dw[1]), pack2(dw[2], dw[3]), pack2(dw[4], dw[5]),
                                    pack2(dw[6], dw[7]));
        const uint4 nw = make_uint4(pack2(-dw[0], -dw[1]), pack2(-dw[2], -dw[3]),
                                    pack2(-dw[4], -dw[5]), pack2(-dw[6], -dw[7]));
        *reinterpret_cast<uint4 *>(zu) = ua;
        *reinterpret_cast<uint4 *>(zu + 32) = nw;
        *reinterpret_cast<uint4 *>(zv) = uw;
        *reinterpret_cast<uint4 *>(zv + 32) = ua;
    }
}

// An integer-valued FP32 |f| <= 2^22 as an int32 without a conversion instruction:
// f + 1.5 2^23 is exact and lies in [2^23, 2^24], and its bit pattern minus that of
// 1.5 2^23 is f.  The group sums P_2 .. P_5 (at most four slice products over 64
// columns of digits |d| <= 128: |P_d| <= 4 * 64 * 2^14 = 2^22) take this path; it
// relieves the conversion unit, which the other groups still use.
__device__ __forceinline__ int small_int_of(float f) {
    return __float_as_int(__fadd_rn(f, 12582912.0f)) - 0x4B400000;
}

// v * 2^e2 outside the normal range of the result (rare; kept out of line so that its
// FP64 operations are not executed speculatively for every entry)
__device__ __noinline__ double scaled_to_double_slow(long long v, int e2) {
    return ldexp((double)v, e2);
}

// v * 2^e2 rounded to nearest (ties to even), two equivalent ways: HW converts v to FP64
// (one rounding to 53 bits) and scales it exactly through the exponent field; otherwise
// the same rounding is built with integer operations.  The epilogue uses both, on
// alternate columns, so that the FP64 pipe (which also does the final add) and the
// integer pipe share the work.  Results outside the normal range take the out-of-line
// path.
template <bool HW>
__device__ __forceinline__ double scaled_to_double(long long v, int e2) {
    if (HW) {
        const long long bits = __double_as_longlong(__ll2double_rn(v));
        const int be = (int)((bits >> 52) & 0x7ff);
        if (be == 0) return 0.0;                      // v == 0
        const int E = be + e2;
        if (E <= 0 || E >= 2047) return scaled_to_double_slow(v, e2);
        return __longlong_as_double(bits + ((long long)e2 << 52));
    }
    if (v == 0) return 0.0;
    const bool neg = v < 0;
    unsigned long long u = neg ? (unsigned long long)(-v) : (unsigned long long)v;
    const int lz = __clzll((long long)u);
    u <<= lz;                                         // leading one at bit 63
    int E = 63 - lz + e2 + 1023;
    unsigned long long mant = (u >> 11) & 0x000fffffffffffffull;
    const unsigned long long rem = u & 0x7ffull;
    if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) {
        ++mant;
        if (mant == 0x0010000000000000ull) {
            mant = 0;
            ++E;
        }
    }
    if (E <= 0 || E >= 2047) return scaled_to_double_slow(v, e2);
    const unsigned long long bits =
        ((unsigned long long)neg << 63) | ((unsigned long long)E << 52) | mant;
    return __longlong_as_double((long long)bits);
}

// Lower tiles of the (128-row x 32-column) grid in row-block order: row block bi holds
// column blocks 0 .. 4 bi + 3 (the last row block is cut at the last column block), so
// tile idx belongs to the largest bi with 2 bi (bi + 1) <= idx.
__device__ __forceinline__ void tile_of(int64_t idx, int &bi, int &bj) {
    int64_t r = (int64_t)((sqrt(2.0 * (double)idx + 1.0) - 1.0) * 0.5);
    while (r > 0 && 2 * r * (r + 1) > idx) --r;
    while (2 * (r + 1) * (r + 2) <= idx) ++r;
    bi = (int)r;
    bj = (int)(idx - 2 * r * (r + 1));
}

// Walks the tiles lo, lo+1, ... of the same order in O(1) per step.
struct TileWalk {
    int bi, bj;
    int64_t nbj;
    __device__ __forceinline__ TileWalk(int64_t idx, int64_t nbj_) : nbj(nbj_) { tile_of(idx, bi, bj); }
    __device__ __forceinline__ void next() {
        const int64_t cols = 4 * (int64_t)bi + 4 < nbj ? 4 * (int64_t)bi + 4 : nbj;
        if (++bj >= cols) {
            ++bi;
            bj = 0;
        }
    }
};

struct SplitShared {
    uint64_t u_full, u_empty, v_full[kVBufs], v_empty[kVBufs], acc_full[2], acc_empty[2], drain;
    uint32_t tmem;
    int abort;
};
static_assert(sizeof(SplitShared) <= 256, "barrier block");

// Bounded wait for the phase of the given parity; false on a timeout (recorded in
// *err when err is given) or when another role has given up.
__device__ __forceinline__ bool wait_phase(uint64_t *bar, uint32_t parity, SplitShared *sh,
                                           int *err) {
    return tc::mbar_wait_bounded(bar, parity, &sh->abort, err, SKEW_ERR_TIMEOUT, kSplitTimeoutNs);
}

// The 8 entries C[i, j0 .. j0+7] of the strictly lower part that a thread updates
// (0 elsewhere, and not read when beta = 0); issued before the accumulator is ready.
__device__ __forceinline__ void load_row(const double *crow, int64_t ldc, int64_t i, int64_t j0,
                                         int64_t m, bool interior, bool read,
                                         double (&cv)[kEpiCols]) {
#pragma unroll
    for (int k = 0; k < kEpiCols; ++k) {
        const int64_t j = j0 + k;
        const bool in = interior || (i < m && j < m && i > j);
        cv[k] = (in && read) ? crow[k * ldc] : 0.0;
    }
}

// C[i,j] = beta C[i,j] + alpha 2^(E_i+E_j-54) acc[k] for the 8 columns j0 .. j0+7 of
// row i, strictly lower part only.  PLAIN: alpha = beta = 1 (one FP64 add per entry).
template <bool PLAIN>
__device__ __forceinline__ void store_row(double *crow, int64_t ldc, int64_t i, int64_t j0,
                                          int64_t m, bool interior, int Ei, int Ej_lane,
                                          const long long (&acc)[kEpiCols],
                                          const double (&cv)[kEpiCols], double alpha,
                                          double beta) {
#pragma unroll
    for (int k = 0; k < kEpiCols; ++k) {
        const int Ej = __shfl_sync(0xffffffffu, Ej_lane, k);
        const int64_t j = j0 + k;
        if (!(interior || (i < m && j < m && i > j))) continue;
        const double upd = (k & 1) ? scaled_to_double<true>(acc[k], Ei + Ej - 54)
                                   : scaled_to_double<false>(acc[k], Ei + Ej - 54);
        if (PLAIN) crow[k * ldc] = cv[k] + upd;
        else crow[k * ldc] = fma(beta, cv[k], alpha * upd);
    }
}

__global__ void __launch_bounds__(kThreads, 1)
split_tc_kernel(int64_t m, double *C, int64_t ldc, double alpha, double beta,
                const __grid_constant__ CUtensorMap mapU, const __grid_constant__ CUtensorMap mapV,
                const int *rowexp, int64_t ntiles, int64_t nbj, int *err) {
    extern __shared__ unsigned char split_raw[];
    unsigned char *base =
        split_raw + ((1024u - (tc::smem_u32(split_raw) & 1023u)) & 1023u);   // 1024-aligned
    unsigned char *sU = base;
    unsigned char *sV = base + kUBytes;                                        // kVBufs buffers
    SplitShared *sh = reinterpret_cast<SplitShared *>(base + kUBytes + kVBufs * kVBuf);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t lo = (int64_t)blockIdx.x * ntiles / gridDim.x;
    const int64_t hi = (int64_t)(blockIdx.x + 1) * ntiles / gridDim.x;

    // the zero slice after the seven V slices of every buffer (read by the N = 256 MMA)
    for (int b = 0; b < kVBufs; ++b)
        for (int o = threadIdx.x * 16; o < (int)kVSlice; o += kThreads * 16)
            *reinterpret_cast<uint4 *>(sV + b * kVBuf + kVLoad + o) = make_uint4(0, 0, 0, 0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        tc::mbar_init(&sh->u_full, 1);
        tc::mbar_init(&sh->u_empty, 1);
        for (int b = 0; b < kVBufs; ++b) {
            tc::mbar_init(&sh->v_full[b], 1);
            tc::mbar_init(&sh->v_empty[b], 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(&sh->acc_full[a], 1);
            tc::mbar_init(&sh->acc_empty[a], kEpiWarps / 2);   // one warp group per accumulator
        }
        tc::mbar_init(&sh->drain, 1);
        sh->abort = 0;
        tc::fence_barrier_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(&sh->tmem, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = sh->tmem;

    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------------------- producer
        tc::tma_prefetch_map(&mapU);
        tc::tma_prefetch_map(&mapV);
        uint32_t u_loads = 0, v_loads[kVBufs] = {0, 0, 0};
        int prev_bi = -1;
        TileWalk tw(lo, nbj);
        for (int64_t idx = lo; idx < hi; ++idx, tw.next()) {
            const int bi = tw.bi, bj = tw.bj;
            if (bi != prev_bi) {
                if (u_loads > 0 && !wait_phase(&sh->u_empty, (u_loads - 1) & 1, sh, err)) break;
                tc::mbar_arrive_expect_tx(&sh->u_full, kUBytes);
                tc::tma_load_3d(sU, &mapU, 0, bi * kTM, 0, &sh->u_full);
                ++u_loads;
                prev_bi = bi;
            }
            const int b = (int)((idx - lo) % kVBufs);
            if (!wait_phase(&sh->v_empty[b], (v_loads[b] & 1) ^ 1, sh, err)) break;
            tc::mbar_arrive_expect_tx(&sh->v_full[b], kVLoad);
            tc::tma_load_3d(sV + b * kVBuf, &mapV, 0, bj * kTN, 0, &sh->v_full[b]);
            ++v_loads[b];
        }
        // every issued copy has landed before the shared memory is released
        if (u_loads > 0) wait_phase(&sh->u_full, (u_loads - 1) & 1, sh, nullptr);
        for (int b = 0; b < kVBufs; ++b)
            if (v_loads[b] > 0) wait_phase(&sh->v_full[b], (v_loads[b] - 1) & 1, sh, nullptr);
    } else if (warp == 1 && lane == 0) {
        // ---------------------------------------------------------------- MMA issue
        const uint32_t u_addr = tc::smem_u32(sU), v_addr = tc::smem_u32(sV);
        uint32_t u_uses = 0;
        int prev_bi = -1;
        TileWalk tw(lo, nbj);
        for (int64_t idx = lo; idx < hi; ++idx) {
            const int bi = tw.bi;
            tw.next();                               // tw is now the next tile
            if (bi != prev_bi) {
                if (!wait_phase(&sh->u_full, u_uses & 1, sh, err)) break;
                ++u_uses;
                prev_bi = bi;
            }
            const int64_t tau = idx - lo;
            const int b = (int)(tau % kVBufs);
            const int ab = (int)(tau & 1);
            if (!wait_phase(&sh->v_full[b], (uint32_t)((tau / kVBufs) & 1), sh, err)) break;
            if (!wait_phase(&sh->acc_empty[ab], (uint32_t)(((tau >> 1) & 1) ^ 1), sh, err)) break;
            tc::fence_after_sync();
            const uint32_t vb = v_addr + (uint32_t)b * kVBuf;
            const uint32_t acc_base = tmem + (uint32_t)ab * kAccCols;
#pragma unroll 1
            for (int s = 1; s <= kSlices; ++s) {
                // digit s of U times V slices 1..T into groups s+1 .. s+T
                const int T = s == 1 ? kSlices + 1 : (kSlices < 9 - s ? kSlices : 9 - s);
                const uint32_t idesc = tc::idesc_bf16_f32(kTM, kTN * T);
                const uint32_t dt = acc_base + (uint32_t)(s - 1) * kTN;
#pragma unroll
                for (int ks = 0; ks < kK / 16; ++ks) {
                    const uint64_t ad = tc::sdesc_kmajor_sw128(u_addr + (s - 1) * kUSlice + ks * 32);
                    const uint64_t bd = tc::sdesc_kmajor_sw128(vb + ks * 32);
                    tc::mma_bf16(dt, ad, bd, idesc, (s > 1 || ks > 0) ? 1u : 0u);
                }
            }
            tc::mma_commit(&sh->acc_full[ab]);
            tc::mma_commit(&sh->v_empty[b]);
            if (idx + 1 >= hi || tw.bi != bi) tc::mma_commit(&sh->u_empty);
        }
        // every issued MMA has completed before the tensor memory is released
        tc::mma_commit(&sh->drain);
        wait_phase(&sh->drain, 0, sh, nullptr);
    } else if (warp >= 2) {
        // ---------------------------------------------------------------- epilogue
        // Two groups of 8 warps take alternate tiles (group g: accumulator g), so the
        // FP64 adds of one group overlap the integer work of the other.  In a group,
        // warp w reads lanes 32 (w mod 4) .. +31 and one 16-column half of the tile, as
        // two passes of 8 columns.
        const int e = warp - 2;
        const int grp = e >> 3;
        const int q = warp & 3;                      // lane quarter of the tensor memory
        const int ch = (e >> 2) & 1;                 // 16-column half of the tile
        const bool plain = alpha == 1.0 && beta == 1.0;
        const bool read = beta != 0.0;
        TileWalk tw(lo, nbj);
        if (grp == 1) tw.next();
        for (int64_t idx = lo + grp; idx < hi; idx += 2, tw.next(), tw.next()) {
            const int64_t tau = idx - lo;
            const int64_t r0 = (int64_t)tw.bi * kTM + q * 32;
            const int64_t i = r0 + lane;
            const int Ei = i < m ? __ldg(rowexp + i) : 0;
            const uint32_t ta = tmem + (uint32_t)grp * kAccCols + ((uint32_t)(q * 32) << 16);
            bool ok = true;
#pragma unroll 1
            for (int ps = 0; ps < 2; ++ps) {
                const int cofs = ch * 16 + ps * kEpiCols;      // column offset in the tile
                const int64_t j0 = (int64_t)tw.bj * kTN + cofs;
                // everything that does not depend on the accumulator is loaded first
                const bool interior =
                    r0 + 31 < m && j0 + kEpiCols - 1 < m && r0 > j0 + kEpiCols - 1;
                double *crow = C + i + j0 * ldc;
                const int Ej_lane =
                    (lane < kEpiCols && j0 + lane < m) ? __ldg(rowexp + j0 + lane) : 0;
                double cv[kEpiCols];
                load_row(crow, ldc, i, j0, m, interior, read, cv);
                if (ps == 0) {
                    int got = 1;
                    if (lane == 0)
                        got = wait_phase(&sh->acc_full[grp], (uint32_t)((tau >> 1) & 1), sh, err);
                    if (!__shfl_sync(0xffffffffu, got, 0)) {   // warp-uniform (tcgen05.ld)
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                }
                // acc = Q23 2^34 + Q45 2^18 + Q67 2^2 + Q89 2^-14 with Q = 256 P_d + P_(d+1)
                // (|Q| < 2^31: exact in 32 bits).  Q89 only reaches acc shifted right by
                // 14, so it is formed in FP32: its rounding (< 2^7) stays below one unit.
                long long acc[kEpiCols];
#pragma unroll
                for (int h = 0; h < 2; ++h) {        // groups 2..5, then 6..9
                    uint32_t r[4][kEpiCols];
#pragma unroll
                    for (int g = 0; g < 4; ++g)
                        tc::tmem_ld8(ta + (uint32_t)(4 * h + g) * kTN + cofs, r[g]);
                    tc::tmem_ld_wait();
                    if (h == 1 && ps == 1) {         // the accumulator can take a new tile
                        tc::fence_before_sync();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&sh->acc_empty[grp]);
                    }
#pragma unroll
                    for (int k = 0; k < kEpiCols; ++k) {
                        const float f0 = __uint_as_float(r[0][k]), f1 = __uint_as_float(r[1][k]);
                        const float f2 = __uint_as_float(r[2][k]), f3 = __uint_as_float(r[3][k]);
                        if (h == 0) {                // P_2 .. P_5: |P_d| <= 2^22
                            const long long Qa =
                                (long long)(small_int_of(f0) * 256 + small_int_of(f1));
                            const long long Qb =
                                (long long)(small_int_of(f2) * 256 + small_int_of(f3));
                            acc[k] = (Qa << 34) + (Qb << 18);
                        } else {
                            const long long Qa =
                                (long long)(__float2int_rn(f0) * 256 + __float2int_rn(f1));
                            acc[k] += (Qa << 2) +
                                      (long long)__float2int_rd(fmaf(f2, 256.0f, f3) * 0x1p-14f);
                        }
                    }
                }
                if (plain)
                    store_row<true>(crow, ldc, i, j0, m, interior, Ei, Ej_lane, acc, cv, alpha, beta);
                else
                    store_row<false>(crow, ldc, i, j0, m, interior, Ei, Ej_lane, acc, cv, alpha, beta);
            }
            if (!ok) break;
            if (lane < 16) {   // bring this group's next block of C (32 x 16) towards L2
                TileWalk nx = tw;
                nx.next();
                nx.next();
                const int64_t nr0 = (int64_t)nx.bi * kTM + q * 32;
                const int64_t j = (int64_t)nx.bj * kTN + ch * 16 + lane;
                if (idx + 2 < hi && nr0 < m && j < m && nr0 + 31 > j) {
                    const int64_t rl = (nr0 + 31 < m ? nr0 + 31 : m - 1);
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(C + nr0 + j * ldc));
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(C + (nr0 + rl) / 2 + j * ldc));
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(C + rl + j * ldc));
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

// ---------------------------------------------------------------- tensor maps (host)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// [7][m][64] bf16 slices; box of 64 x rows x 7, 128-byte swizzle, rows past m read as 0
int make_slice_map(CUtensorMap *map, const unsigned short *Z, int64_t m, int rows) {
    EncodeTiledFn enc = encode_fn();
    if (enc == nullptr) return SKEW_ERR_CUDA;
    const cuuint64_t dims[3] = {(cuuint64_t)kK, (cuuint64_t)m, (cuuint64_t)kSlices};
    const cuuint64_t strides[2] = {(cuuint64_t)kK * 2, (cuuint64_t)m * kK * 2};
    const cuuint32_t box[3] = {(cuuint32_t)kK, (cuuint32_t)rows, (cuuint32_t)kSlices};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                           const_cast<unsigned short *>(Z), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? SKEW_OK : SKEW_ERR_CUDA;
}

size_t rowexp_bytes(int64_t m) {
    return ((size_t)(m > 0 ? m : 1) * sizeof(int) + 255) & ~size_t(255);
}

size_t slice_bytes(int64_t m) {
    const size_t z = (size_t)kSlices * (size_t)(m > 0 ? m : 1) * kK * sizeof(unsigned short);
    return (z + 1023) & ~size_t(1023);
}

template <PairKind KIND>
int launch_split_kind(const Skr2kArgs &a, void *scratch, int *err, int sms,
                      cudaStream_t stream) {
    if (a.m <= 1) return SKEW_OK;
    if (a.m > INT_MAX / 2) return SKEW_ERR_CUDA;
    PairSource<KIND> src{a.P, a.ldp, a.Q, a.ldq, a.tt, a.x, a.b};
    int P;
    if (KIND == PairKind::Rank2k) P = (int)a.b;
    else if (KIND == PairKind::Tridiag) P = (int)(a.b / 2);
    else P = (int)(a.b / 2 + (a.b & 1));
    if (P > 32) return SKEW_ERR_CUDA;             // guarded by the callers (<= 32 pairs)
    if (P < 0) P = 0;
    char *base = static_cast<char *>(scratch);
    unsigned short *Zu = reinterpret_cast<unsigned short *>(base);
    unsigned short *Zv = reinterpret_cast<unsigned short *>(base + slice_bytes(a.m));
    int *rowexp = reinterpret_cast<int *>(base + 2 * slice_bytes(a.m));
    int *colexp = reinterpret_cast<int *>(base + 2 * slice_bytes(a.m) + rowexp_bytes(a.m));
    const int pgrid = (int)((a.m + 63) / 64);            // 64 rows per 256-thread CTA
    if (a.balance) {
        SKEW_TRY(cudaMemsetAsync(colexp, 0x80, 64 * sizeof(int), stream));
        split_colexp_kernel<KIND><<<pgrid, 256, 0, stream>>>(a.m, src, P, colexp);
        note_launches(1);
        SKEW_TRY_STATUS(check_launch());
    }
    split_prepare_kernel<KIND><<<pgrid, 256, 0, stream>>>(a.m, src, P, Zu, Zv, rowexp,
                                                         a.balance ? colexp : nullptr);
    note_launches(1);
    SKEW_TRY_STATUS(check_launch());

    CUtensorMap mapU, mapV;
    SKEW_TRY_STATUS(make_slice_map(&mapU, Zu, a.m, kTM));
    SKEW_TRY_STATUS(make_slice_map(&mapV, Zv, a.m, kTN));
    const int64_t nbi = (a.m + kTM - 1) / kTM, nbj = (a.m + kTN - 1) / kTN;
    const int64_t ntiles = 2 * (nbi - 1) * nbi + nbj;
    const int grid = (int)(ntiles < sms ? ntiles : sms);
    cudaError_t e = cudaFuncSetAttribute((const void *)split_tc_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemBytes);
    if (e != cudaSuccess) {
        set_last_error(e);
        return SKEW_ERR_CUDA;
    }
    split_tc_kernel<<<grid, kThreads, kSmemBytes, stream>>>(a.m, a.C, a.ldc, a.alpha, a.beta,
                                                           mapU, mapV, rowexp, ntiles, nbj, err);
    note_launches(1);
    return check_launch();
}

}  // namespace

size_t split_scratch_bytes(int64_t m) {
    return 2 * slice_bytes(m) + rowexp_bytes(m) + 256;      // + the 64 column exponents
}

int launch_skr2k_split(PairKind kind, const Skr2kArgs &a, void *scratch, int *err, int sms,
                       cudaStream_t stream) {
    switch (kind) {
        case PairKind::Rank2k:
            return launch_split_kind<PairKind::Rank2k>(a, scratch, err, sms, stream);
        case PairKind::Tridiag:
            return launch_split_kind<PairKind::Tridiag>(a, scratch, err, sms, stream);
        default: return launch_split_kind<PairKind::Fused>(a, scratch, err, sms, stream);
    }
}

}  // namespace skew
