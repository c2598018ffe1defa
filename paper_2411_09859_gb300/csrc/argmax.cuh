// argmax.cuh -- the pivot search of the panel kernels: candidates (|v|, row) compared
// as integers, reduced within a warp and within a CTA.
#pragma once

#include <climits>

#include "common.cuh"

namespace skew {
namespace {

// Pivot candidates are compared on the bits of |v| as unsigned integers (for
// non-negative IEEE doubles the order of the bit patterns is the order of the
// values), then on the row index: larger magnitude wins, the lower index wins a tie.
// FP64 instructions are avoided because they are slow on this part.  A NaN is never
// a candidate.  (0, INT_MAX) is the "no candidate" value: any real entry beats it,
// since |v| > 0 is larger and |v| == 0 wins on the index.
constexpr unsigned long long kAbsMask = 0x7fffffffffffffffull;
constexpr unsigned long long kExpMask = 0x7ff0000000000000ull;

__device__ __forceinline__ bool finite_bits(unsigned long long raw) {
    return (raw & kExpMask) != kExpMask;
}

struct Best {
    unsigned long long raw;   // bits of the signed v
    int i;                    // row
    int c;                    // CTA that published it
};

__device__ __forceinline__ bool better(unsigned long long ra, int ia, unsigned long long rb,
                                       int ib) {
    const unsigned long long a = ra & kAbsMask, b = rb & kAbsMask;
    return (a > b) || (a == b && ia < ib);
}

__device__ __forceinline__ Best no_candidate() {
    Best b;
    b.raw = 0ull;
    b.i = INT_MAX;
    b.c = 0;
    return b;
}

// Offer row i with value v; NaN is skipped.
__device__ __forceinline__ void offer(Best &b, double v, int i) {
    const unsigned long long raw = (unsigned long long)__double_as_longlong(v);
    if ((raw & kAbsMask) > kExpMask) return;          // NaN
    if (better(raw, i, b.raw, b.i)) { b.raw = raw; b.i = i; }
}

__device__ __forceinline__ Best warp_best(Best x) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long orw = __shfl_down_sync(0xffffffffu, x.raw, off);
        const int oi = __shfl_down_sync(0xffffffffu, x.i, off);
        const int oc = __shfl_down_sync(0xffffffffu, x.c, off);
        if (better(orw, oi, x.raw, x.i)) { x.raw = orw; x.i = oi; x.c = oc; }
    }
    return x;
}

// The same reduction with warp reduce instructions, the result valid in every lane:
// the largest |v| bits (high word, then low word among the lanes that tie on it), the
// lowest row among the lanes that tie on both, and the CTA field of that lane.  Fewer
// dependent steps than the five-level shuffle tree above.
__device__ __forceinline__ Best warp_best_all(Best x) {
    const unsigned long long m = x.raw & kAbsMask;
    const unsigned int hi = (unsigned int)(m >> 32), lo = (unsigned int)m;
    const unsigned int mh = __reduce_max_sync(0xffffffffu, hi);
    const unsigned int ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
    const bool top = (hi == mh) && (lo == ml);
    const unsigned int mi = __reduce_min_sync(0xffffffffu, top ? (unsigned int)x.i : 0xffffffffu);
    const unsigned int win = __ballot_sync(0xffffffffu, top && (unsigned int)x.i == mi);
    const int src = __ffs((int)win) - 1;
    Best r;
    r.raw = __shfl_sync(0xffffffffu, x.raw, src);
    r.i = (int)mi;
    r.c = __shfl_sync(0xffffffffu, x.c, src);
    return r;
}

// Reduce one Best per thread; the result is valid in every thread on return.
__device__ Best block_best(Best x) {
    __shared__ unsigned long long s_raw[kPanelThreads / 32];
    __shared__ int s_i[kPanelThreads / 32];
    __shared__ Best s_res;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    x = warp_best(x);
    if (lane == 0) { s_raw[w] = x.raw; s_i[w] = x.i; }
    __syncthreads();
    if (w == 0) {
        Best y = no_candidate();
        if (lane < kPanelThreads / 32) { y.raw = s_raw[lane]; y.i = s_i[lane]; }
        y = warp_best(y);
        if (lane == 0) s_res = y;
    }
    __syncthreads();
    return s_res;
}

// A panel CTA's step record {val, idx, tag} (the first 16 bytes of its ArgmaxPartial)
// is written and read as ONE 128-bit access, so a reader that sees the step's tag has
// that step's candidate in the same load (no second round trip).
__device__ __forceinline__ void record_poll(const ArgmaxPartial *p, unsigned long long &val,
                                            unsigned int &idx, unsigned int &tag) {
    unsigned long long lo, hi;
    asm volatile(
        "{\n\t.reg .b128 t;\n\tld.relaxed.gpu.global.b128 t, [%2];\n\t"
        "mov.b128 {%0, %1}, t;\n\t}"
        : "=l"(lo), "=l"(hi)
        : "l"(p)
        : "memory");
    val = lo;
    idx = (unsigned int)(hi & 0xffffffffull);
    tag = (unsigned int)(hi >> 32);
}
__device__ __forceinline__ void record_release(ArgmaxPartial *p, unsigned long long val, int idx,
                                               unsigned int tag) {
    const unsigned long long hi =
        ((unsigned long long)tag << 32) | (unsigned long long)(unsigned int)idx;
    asm volatile(
        "{\n\t.reg .b128 t;\n\tmov.b128 t, {%1, %2};\n\t"
        "st.release.gpu.global.b128 [%0], t;\n\t}" ::"l"(p),
        "l"(val), "l"(hi)
        : "memory");
}

__device__ __forceinline__ double as_double(unsigned long long raw) {
    return __longlong_as_double((long long)raw);
}

}  // namespace
}  // namespace skew
