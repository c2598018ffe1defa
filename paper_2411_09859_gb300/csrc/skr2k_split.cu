// skr2k_split.cu -- the skew rank-2k update C += U V^T (strictly lower part) with
// FP64 operands split into 8-bit digit slices multiplied on bf16 tensor cores
// (mma.sync.m16n8k16, FP32 accumulation), recombined exactly in 64-bit integers.
//
// This is the error-free splitting of Ozaki, Ogita, Oishi and Rump (2012), "Error-
// free transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", in fixed-point form:
//
//   - every row i of the pair columns (a_p, w_p) gets the exponent E_i of its
//     largest entry; each entry x becomes the 56-bit integer X = trunc(|x| 2^(55-E_i))
//     (|x| < 2^(E_i+1)) with the sign of x, cut into seven 8-bit digits
//     x ~ sign * sum_{s=1..7} d_s 2^(E_i+1-8s), 0 <= d_s <= 255 (exact in bf16);
//   - U = [a | -w] and V = [w | a] share the digits of the row (negation flips a
//     sign bit, V swaps the halves);
//   - (U V^T)[i,j] ~ 2^(E_i+E_j+2) sum_{d=2..8} 2^(-8d) P_d[i,j] with
//     P_d = sum_{s+t=d} U_s V_t^T.  Over a K-chunk of 32 columns every P_d is an
//     integer below 7 * 32 * 255^2 < 2^24, so its FP32 tensor-core sum is exact;
//     chunk results are added as integers into a 64-bit fixed-point accumulator
//     (weight 2^(56-8d)), and one conversion to FP64 plus one FP64 add per entry
//     finishes the update.
//
// The products with s + t > 8 and the digits beyond the seventh are dropped: the
// result differs from the exact update by about 2^-53 * K * (max row entry of U) *
// (max row entry of V), the size of FP64 rounding in an ordinary dot product, but
// measured against row maxima rather than entry by entry.  K (2 * pairs) is limited
// to 64 so that the accumulator cannot overflow.
#include <climits>
#include <cuda_bf16.h>

#include "common.cuh"
#include "pairs.cuh"

namespace skew {
namespace {

constexpr int kSlices = 7;
constexpr int kTile = 64;
constexpr int kChunk = 32;               // K columns per staging round
constexpr int kRowPad = kChunk + 8;      // bf16 per smem row (conflict-free fragments)
constexpr int kThreads = 128;

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

// 56-bit fixed point of |x| relative to 2^(E+1): X = trunc(|x| 2^(55-E))
__device__ __forceinline__ unsigned long long fixed56(double x, int E) {
    int ex;
    unsigned long long m;
    decompose(x, ex, m);
    const int sh = ex - E + 3;              // |x| = m 2^(ex-52); X = m 2^(ex-52+55-E)
    if (sh >= 0) return m << sh;             // sh <= 3: at most 56 bits
    if (sh <= -64) return 0ull;
    return m >> (-sh);
}

__device__ __forceinline__ unsigned short bf16_bits_of_digit(unsigned int d, bool neg) {
    // d in [0, 255] is exact in bf16
    const __nv_bfloat16 h = __uint2bfloat16_rn(d);
    unsigned short u = *reinterpret_cast<const unsigned short *>(&h);
    if (neg && d != 0) u ^= 0x8000u;
    return u;
}

// Pre-pass: for each row i, the exponent E_i of its largest pair entry and the seven
// digit slices of its a-part (columns [0, P)) and w-part (columns [P32, P32+P)) into
// Z[s][i][kk] (bf16, row length 2*P32, zero padded).
template <PairKind KIND>
__global__ void __launch_bounds__(256)
split_prepare_kernel(int64_t m, PairSource<KIND> src, int P, int P32, unsigned short *Z,
                     int *rowexp) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int E = INT_MIN / 2;
    for (int p = 0; p < P; ++p) {
        double av, wv;
        src.get(p, i, av, wv);
        E = max(E, max(exponent_of(av), exponent_of(wv)));
    }
    if (E < -1022) E = -1022;                  // an all-zero row
    rowexp[i] = E;
    const int KP = 2 * P32;
    const size_t slice_stride = (size_t)m * KP;
    unsigned short *zrow = Z + (size_t)i * KP;
    for (int half = 0; half < 2; ++half) {
        for (int p0 = 0; p0 < P32; p0 += 8) {
            unsigned long long X[8];
            bool neg[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int p = p0 + q;
                X[q] = 0ull;
                neg[q] = false;
                if (p < P) {
                    double av, wv;
                    src.get(p, i, av, wv);
                    const double v = half == 0 ? av : wv;
                    X[q] = fixed56(v, E);
                    neg[q] = v < 0.0;
                }
            }
#pragma unroll
            for (int s = 0; s < kSlices; ++s) {
                unsigned int w[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const unsigned int d0 = (unsigned int)(X[2 * q] >> (48 - 8 * s)) & 0xffu;
                    const unsigned int d1 = (unsigned int)(X[2 * q + 1] >> (48 - 8 * s)) & 0xffu;
                    w[q] = (unsigned int)bf16_bits_of_digit(d0, neg[2 * q]) |
                           ((unsigned int)bf16_bits_of_digit(d1, neg[2 * q + 1]) << 16);
                }
                uint4 *dst = reinterpret_cast<uint4 *>(zrow + s * slice_stride + half * P32 + p0);
                *dst = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    }
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned int (&a)[4],
                                         const unsigned int (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
        "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// v * 2^e2 rounded to nearest (ties to even), built with integer operations
__device__ __forceinline__ double scaled_to_double(long long v, int e2) {
    if (v == 0) return 0.0;
    const bool neg = v < 0;
    unsigned long long u = neg ? (unsigned long long)(-v) : (unsigned long long)v;
    const int lz = __clzll((long long)u);
    u <<= lz;                                  // leading one at bit 63
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
    if (E <= 0 || E >= 2047) return ldexp((double)v, e2);   // outside the normal range
    const unsigned long long bits =
        ((unsigned long long)neg << 63) | ((unsigned long long)E << 52) | mant;
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ void tri_tile(int64_t idx, int64_t &bi, int64_t &bj) {
    int64_t r = (int64_t)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
    while (r * (r + 1) / 2 > idx) --r;
    while ((r + 1) * (r + 2) / 2 <= idx) ++r;
    bi = r;
    bj = idx - r * (r + 1) / 2;
}

__global__ void __launch_bounds__(kThreads, 3)
split_update_kernel(int64_t m, double *C, int64_t ldc, double alpha, double beta,
                    const unsigned short *Z, const int *rowexp, int P32) {
    // U slices of the tile's rows I and V slices of its rows J (bf16 bit patterns),
    // in dynamic shared memory: [kSlices][kTile][kRowPad] each
    extern __shared__ __align__(16) unsigned char split_smem[];
    typedef unsigned short SliceTile[kTile][kRowPad];
    SliceTile *Us = reinterpret_cast<SliceTile *>(split_smem);
    SliceTile *Vs = reinterpret_cast<SliceTile *>(split_smem + sizeof(SliceTile) * kSlices);

    int64_t bi, bj;
    tri_tile(blockIdx.x, bi, bj);
    const int64_t I0 = bi * kTile, J0 = bj * kTile;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;
    const int g = lane >> 2, tg = lane & 3;
    const int KP = 2 * P32;
    const size_t slice_stride = (size_t)m * KP;

    long long acc[2][4][4];                    // [mi][ni][c] fixed point, weight 2^-56
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[mi][ni][c] = 0;

    const int nchunks = KP / kChunk;
    for (int ch = 0; ch < nchunks; ++ch) {
        // U columns [ch*32, ch*32+32) of [a | -w] and the same columns of V = [w | a].
        // The digits are copied as stored (+a, +w) with cp.async, all copies of a
        // thread in flight at once (rows past m are zero-filled); a chunk of the w-part
        // of U enters the accumulator with a minus sign instead.
        const int ucol = ch * kChunk;
        const bool uneg = ucol >= P32;                        // U holds -w here
        const int vcol = uneg ? ucol - P32 : ucol + P32;      // the other half
        for (int it = tid; it < kSlices * kTile * (kChunk / 8); it += kThreads) {
            const int seg = it % (kChunk / 8);
            const int r = (it / (kChunk / 8)) % kTile;
            const int s = it / ((kChunk / 8) * kTile);
            const bool iu = I0 + r < m, jv = J0 + r < m;
            const unsigned short *su =
                iu ? Z + s * slice_stride + (size_t)(I0 + r) * KP + ucol + seg * 8 : Z;
            const unsigned short *sv =
                jv ? Z + s * slice_stride + (size_t)(J0 + r) * KP + vcol + seg * 8 : Z;
            const unsigned int du = (unsigned int)__cvta_generic_to_shared(&Us[s][r][seg * 8]);
            const unsigned int dv = (unsigned int)__cvta_generic_to_shared(&Vs[s][r][seg * 8]);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(du), "l"(su),
                         "r"(iu ? 16 : 0)
                         : "memory");
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dv), "l"(sv),
                         "r"(jv ? 16 : 0)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
#pragma unroll 1
        for (int d = 2; d <= kSlices + 1; ++d) {
            float f[2][4][4];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni)
#pragma unroll
                    for (int c = 0; c < 4; ++c) f[mi][ni][c] = 0.0f;
            const int s_lo = d - kSlices > 1 ? d - kSlices : 1;
            const int s_hi = d - 1 < kSlices ? d - 1 : kSlices;
#pragma unroll 1
            for (int s = s_lo; s <= s_hi; ++s) {
                const int t = d - s;
#pragma unroll
                for (int ks = 0; ks < kChunk / 16; ++ks) {
                    const int kb = ks * 16 + 2 * tg;
                    unsigned int a[2][4], b[4][2];
#pragma unroll
                    for (int mi = 0; mi < 2; ++mi) {
                        const int r0 = wm * 32 + mi * 16 + g;
                        a[mi][0] = *reinterpret_cast<const unsigned int *>(&Us[s - 1][r0][kb]);
                        a[mi][1] = *reinterpret_cast<const unsigned int *>(&Us[s - 1][r0 + 8][kb]);
                        a[mi][2] = *reinterpret_cast<const unsigned int *>(&Us[s - 1][r0][kb + 8]);
                        a[mi][3] = *reinterpret_cast<const unsigned int *>(&Us[s - 1][r0 + 8][kb + 8]);
                    }
#pragma unroll
                    for (int ni = 0; ni < 4; ++ni) {
                        const int c0 = wn * 32 + ni * 8 + g;
                        b[ni][0] = *reinterpret_cast<const unsigned int *>(&Vs[t - 1][c0][kb]);
                        b[ni][1] = *reinterpret_cast<const unsigned int *>(&Vs[t - 1][c0][kb + 8]);
                    }
#pragma unroll
                    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                        for (int ni = 0; ni < 4; ++ni) mma_bf16(f[mi][ni], a[mi], b[ni]);
                }
            }
            // exact integers below 2^24: add with weight 2^(56-8d) (d = 8: 2^-8, truncated)
            const int shl = 56 - 8 * d;
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        long long q = (long long)__float2int_rn(f[mi][ni][c]);
                        q = shl >= 0 ? (q << shl) : (q >> (-shl));
                        acc[mi][ni][c] += uneg ? -q : q;
                    }
        }
        __syncthreads();
    }

    // epilogue: C[i,j] = beta C[i,j] + alpha 2^(E_i+E_j+2-56) acc, strictly lower part.
    // All loads of a row block (row exponents, C entries) are issued before any
    // store, so their latencies overlap instead of adding up.
    int Ej[4][2];
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int64_t gj = J0 + wn * 32 + ni * 8 + 2 * tg + c;
            Ej[ni][c] = gj < m ? __ldg(rowexp + gj) : 0;
        }
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
        int Ei[2];
        double cv[2][4][2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t gi = I0 + wm * 32 + mi * 16 + g + 8 * h;
            Ei[h] = gi < m ? __ldg(rowexp + gi) : 0;
#pragma unroll
            for (int ni = 0; ni < 4; ++ni)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int64_t gj = J0 + wn * 32 + ni * 8 + 2 * tg + c;
                    const bool in = gi < m && gj < m && gi > gj && beta != 0.0;
                    cv[h][ni][c] = in ? C[gi + gj * ldc] : 0.0;
                }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t gi = I0 + wm * 32 + mi * 16 + g + 8 * h;
#pragma unroll
            for (int ni = 0; ni < 4; ++ni)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int64_t gj = J0 + wn * 32 + ni * 8 + 2 * tg + c;
                    if (gi >= m || gj >= m || gi <= gj) continue;
                    const double upd =
                        scaled_to_double(acc[mi][ni][2 * h + c], Ei[h] + Ej[ni][c] + 2 - 56);
                    double *dst = C + gi + gj * ldc;
                    if (beta == 1.0 && alpha == 1.0) *dst = cv[h][ni][c] + upd;
                    else if (beta == 0.0) *dst = alpha * upd;
                    else *dst = beta * cv[h][ni][c] + alpha * upd;
                }
        }
    }
}

template <PairKind KIND>
int launch_split_kind(const Skr2kArgs &a, void *scratch, cudaStream_t stream) {
    if (a.m <= 1) return SKEW_OK;
    PairSource<KIND> src{a.P, a.ldp, a.Q, a.ldq, a.tt, a.x, a.b};
    int P;
    if (KIND == PairKind::Rank2k) P = (int)a.b;
    else if (KIND == PairKind::Tridiag) P = (int)(a.b / 2);
    else P = (int)(a.b / 2 + (a.b & 1));
    const int P32 = P <= 0 ? 32 : ((P + 31) / 32) * 32;
    if (P32 > 32) return SKEW_ERR_CUDA;           // guarded by the callers (<= 32 pairs)
    char *base = static_cast<char *>(scratch);
    unsigned short *Z = reinterpret_cast<unsigned short *>(base);
    int *rowexp = reinterpret_cast<int *>(base + split_z_bytes(a.m));
    const int pgrid = (int)((a.m + 255) / 256);
    split_prepare_kernel<KIND><<<pgrid, 256, 0, stream>>>(a.m, src, P, P32, Z, rowexp);
    note_launches(1);
    SKEW_TRY_STATUS(check_launch());
    const int64_t nt = (a.m + kTile - 1) / kTile;
    const int64_t tiles = nt * (nt + 1) / 2;
    if (tiles > INT_MAX) return SKEW_ERR_CUDA;
    const size_t smem = 2 * sizeof(unsigned short) * kSlices * kTile * kRowPad;
    static_assert(2 * sizeof(unsigned short) * kSlices * kTile * kRowPad <= 227 * 1024, "smem");
    cudaError_t e = cudaFuncSetAttribute((const void *)split_update_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
        set_last_error(e);
        return SKEW_ERR_CUDA;
    }
    split_update_kernel<<<(unsigned)tiles, kThreads, smem, stream>>>(a.m, a.C, a.ldc, a.alpha,
                                                                     a.beta, Z, rowexp, P32);
    note_launches(1);
    return check_launch();
}

}  // namespace

size_t split_z_bytes(int64_t m) {
    // seven slices of m rows of 64 bf16 (the largest K), 256-byte aligned
    const size_t z = (size_t)kSlices * (size_t)(m > 0 ? m : 1) * 64 * sizeof(unsigned short);
    return (z + 255) & ~size_t(255);
}

size_t split_scratch_bytes(int64_t m) {
    return split_z_bytes(m) + (((size_t)(m > 0 ? m : 1) * sizeof(int) + 255) & ~size_t(255));
}

int launch_skr2k_split(PairKind kind, const Skr2kArgs &a, void *scratch, cudaStream_t stream) {
    switch (kind) {
        case PairKind::Rank2k: return launch_split_kind<PairKind::Rank2k>(a, scratch, stream);
        case PairKind::Tridiag: return launch_split_kind<PairKind::Tridiag>(a, scratch, stream);
        default: return launch_split_kind<PairKind::Fused>(a, scratch, stream);
    }
}

}  // namespace skew
