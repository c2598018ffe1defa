// pairs.cuh -- the (a_p, w_p) column pairs of a skew rank-2k update
//     C := beta C + alpha * sum_p (a_p w_p^T - w_p a_p^T)
// as formed by the update kernels (see skr2k.cu for the three kinds).
#pragma once

#include "common.cuh"

namespace skew {

template <PairKind KIND>
struct PairSource {
    const double *P;
    int64_t ldp;
    const double *Q;
    int64_t ldq;
    const double *tt;
    const double *x;
    int64_t b;

    __device__ __forceinline__ int64_t npairs() const {
        if (KIND == PairKind::Rank2k) return b;
        if (KIND == PairKind::Tridiag) return b / 2;
        return b / 2 + (b & 1);
    }
    // (a_p, w_p) at row i (0 <= i < m)
    __device__ __forceinline__ void get(int64_t p, int64_t i, double &av, double &wv) const {
        if (KIND == PairKind::Rank2k) {
            av = P[i + p * ldp];
            wv = Q[i + p * ldq];
            return;
        }
        const int64_t j = 2 * p + 1;
        if (j < b) {
            av = P[i + j * ldp];
            double w = -tt[j - 1] * P[i + (j - 1) * ldp];
            if (j + 1 < b) w += tt[j] * P[i + (j + 1) * ldp];
            if (KIND == PairKind::Fused && j == b - 1) w += x[i];
            wv = w;
        } else {                                    // Fused, b odd: (a_{b-1}, x)
            av = P[i + (b - 1) * ldp];
            wv = x[i];
        }
    }
};


}  // namespace skew
