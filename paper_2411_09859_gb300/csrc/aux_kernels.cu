// aux_kernels.cu -- prologue, deferred row exchanges of L, and the Pfaffian read-off.
#include <climits>

#include "common.cuh"
#include "tc.cuh"

namespace skew {
namespace {

constexpr int kAuxThreads = 256;

// One CTA per column j (grid-stride over columns): L[:, j] := e_j when L is given,
// and a scan of the strictly lower part of A's column j for NaN / infinity.
__global__ void __launch_bounds__(kAuxThreads)
prologue_kernel(int64_t n, const double *A, int64_t lda, double *L, int64_t ldl,
                int32_t *piv, Ctrl *ctrl) {
    bool bad = false;
    for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
        const double *a = A + j * lda;
        for (int64_t i = j + 1 + threadIdx.x; i < n; i += blockDim.x)
            if (!isfinite(a[i])) bad = true;
        if (L != nullptr) {
            double *l = L + j * ldl;
            for (int64_t i = threadIdx.x; i < n; i += blockDim.x) l[i] = (i == j) ? 1.0 : 0.0;
        }
        if (threadIdx.x == 0) piv[j] = (int32_t)j;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) raise_error(ctrl, SKEW_ERR_NONFINITE);
}

// pivot_rows (Section 5.2): the panel's exchanges k+1 <-> piv[k+1], k = k0..kend-1,
// applied in order to rows of the L columns left of the panel (1 .. k0).  One thread
// per column; the exchanges of a column are sequential, as their order matters.
__global__ void __launch_bounds__(kAuxThreads)
pivot_rows_kernel(double *L, int64_t ldl, const int32_t *piv, int k0, int kend) {
    __shared__ int s_piv[kMaxNb];
    for (int k = k0 + threadIdx.x; k < kend; k += blockDim.x) s_piv[k - k0] = piv[k + 1];
    __syncthreads();
    const int64_t c = 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c > k0) return;
    double *col = L + c * ldl;
    for (int k = k0; k < kend; ++k) {
        const int r = s_piv[k - k0], p = k + 1;
        if (r != p) {
            double tmp = col[p];
            col[p] = col[r];
            col[r] = tmp;
        }
    }
}

// Pf(X) = det(P) Pf(T), Pf(T) = prod_i T[2i, 2i+1] = prod_i (-t[2i]) (Section 1,
// Eq. (T)), det(P) = (-1)^(#{i : piv[i] != i}).  One CTA; each thread accumulates a
// fixed strided subset in index order, then a fixed-shape tree: the result does not
// depend on timing.  Also resolves the info word: a device error recorded in ctrl,
// else 1 + the first j with t[j] == 0, else 0.
constexpr int kFinishThreads = 1024;

__global__ void __launch_bounds__(kFinishThreads)
finish_kernel(int64_t n, const double *t, const int32_t *piv, const Ctrl *ctrl,
              double *logabs, int32_t *sign, int32_t *info) {
    __shared__ double s_sum[kFinishThreads];
    __shared__ int s_neg[kFinishThreads];
    __shared__ int s_zero[kFinishThreads];
    const int tid = threadIdx.x;
    const int64_t half = n / 2;
    double sum = 0.0;
    int neg = 0, zero_even = 0;
    int first_zero = INT_MAX;
    for (int64_t j = tid; j < n - 1; j += kFinishThreads) {
        const double tj = t[j];
        if (tj == 0.0 && j < first_zero) first_zero = (int)j;
        if ((j & 1) == 0 && j / 2 < half) {
            const double v = -tj;              // T[j, j+1]
            if (v == 0.0) zero_even = 1;
            else {
                if (v < 0.0) neg ^= 1;
                sum += log(fabs(v));
            }
        }
    }
    for (int64_t i = tid; i < n; i += kFinishThreads)
        if (piv[i] != (int32_t)i) neg ^= 1;
    s_sum[tid] = sum;
    s_neg[tid] = neg | (zero_even << 1);
    s_zero[tid] = first_zero;
    __syncthreads();
    for (int w = kFinishThreads / 2; w > 0; w >>= 1) {
        if (tid < w) {
            s_sum[tid] += s_sum[tid + w];
            s_neg[tid] = (s_neg[tid] ^ (s_neg[tid + w] & 1)) | (s_neg[tid] & 2) |
                         (s_neg[tid + w] & 2);
            s_zero[tid] = min(s_zero[tid], s_zero[tid + w]);
        }
        __syncthreads();
    }
    if (tid == 0) {
        const bool odd = (n & 1) != 0;
        const bool zero = odd || (s_neg[0] & 2);
        if (logabs) *logabs = zero ? -INFINITY : s_sum[0];
        if (sign) *sign = zero ? 0 : ((s_neg[0] & 1) ? -1 : 1);
        if (info) {
            int e = ctrl ? ctrl->err : 0;
            *info = e != 0 ? e : (s_zero[0] == INT_MAX ? 0 : s_zero[0] + 1);
        }
    }
}

__global__ void selftest_wait_kernel(Ctrl *ctrl, unsigned int expected, uint64_t timeout_ns) {
    unsigned int gen = 0;
    if (threadIdx.x == 0) gen = ld_acquire_u32(&ctrl->bar_gen);
    grid_barrier(ctrl, expected, gen, timeout_ns);
}

// An mbarrier that no thread ever arrives on, waited for with the bounded wait of the
// tensor-core kernels: the wait gives up after timeout_ns and records the timeout.
__global__ void selftest_mbar_kernel(int *err, uint64_t timeout_ns) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        abort_flag = 0;
        tc::fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) tc::mbar_wait_bounded(&bar, 0, &abort_flag, err, SKEW_ERR_TIMEOUT, timeout_ns);
    __syncthreads();
}

}  // namespace

int launch_selftest_mbar(int *err, uint64_t timeout_ns, cudaStream_t stream) {
    selftest_mbar_kernel<<<1, 32, 0, stream>>>(err, timeout_ns);
    note_launches(1);
    return check_launch();
}

int launch_selftest_wait(Ctrl *ctrl, int blocks, uint64_t timeout_ns, cudaStream_t stream) {
    selftest_wait_kernel<<<blocks, 32, 0, stream>>>(ctrl, (unsigned int)blocks + 1u, timeout_ns);
    note_launches(1);
    return check_launch();
}

int launch_prologue(int64_t n, const double *A, int64_t lda, double *L, int64_t ldl,
                    int32_t *piv, Ctrl *ctrl, cudaStream_t stream) {
    if (n <= 0) return SKEW_OK;
    int grid = (int)(n < 4096 ? n : 4096);
    prologue_kernel<<<grid, kAuxThreads, 0, stream>>>(n, A, lda, L, ldl, piv, ctrl);
    note_launches(1);
    return check_launch();
}

int launch_pivot_rows(int64_t n, double *L, int64_t ldl, const int32_t *piv, int k0,
                      int kend, cudaStream_t stream) {
    (void)n;
    if (k0 < 1 || kend <= k0) return SKEW_OK;
    int grid = (k0 + kAuxThreads - 1) / kAuxThreads;
    pivot_rows_kernel<<<grid, kAuxThreads, 0, stream>>>(L, ldl, piv, k0, kend);
    note_launches(1);
    return check_launch();
}

int launch_finish(int64_t n, const double *t, const int32_t *piv, const Ctrl *ctrl,
                  double *logabs, int32_t *sign, int32_t *info, cudaStream_t stream) {
    finish_kernel<<<1, kFinishThreads, 0, stream>>>(n, t, piv, ctrl, logabs, sign, info);
    note_launches(1);
    return check_launch();
}

}  // namespace skew
