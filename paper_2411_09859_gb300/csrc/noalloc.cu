// noalloc.cu -- skew_pfaffian_noalloc: the Pfaffian entry point for callers that
// must not have the library allocate device memory.
//
// Who needs it: programs whose device memory is owned by another allocator (a
// framework that reserves nearly all of HBM for its own caching pool, where a
// library-side allocation fails or fragments that pool), and latency-bound loops
// that cannot afford an allocation call or a pool growing on their critical path.
// skew_pfaffian already accepts a caller-provided workspace; this entry point is for
// callers that cannot provide one either.
//
// The workspace lives in one file-scope device array of fixed size, created when
// the library is loaded on a device and held there until the process exits.  Its
// device address is looked up once per device, with that device current, on the
// first call made on it.
#include <mutex>

#include "common.cuh"

// Fixed scratch of the allocation-free entry point: 16 MiB on every device that
// loads the library.
constexpr size_t kNoallocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[kMaxDevices];   // device address of g_noalloc_scratch, per device
}  // namespace

using namespace skew;

extern "C" int skew_pfaffian_noalloc(int64_t n, double *A, int64_t lda, double *logabs,
                                     int32_t *sign, int32_t *info, int nb, void *stream) {
    if (n < 0 || n > kMaxOrder) return -1;
    const int64_t ld_min = n > 1 ? n : 1;
    if (A == nullptr && n > 0) return -2;
    if (lda < ld_min) return -3;
    if (logabs == nullptr) return -4;
    if (sign == nullptr) return -5;
    if (nb < 0 || nb > kMaxNb) return -7;
    const int nb_eff = nb == 0 ? skew_default_nb(n) : nb;
    if (skew_workspace_bytes(n, nb_eff, 0) > kNoallocScratchBytes) return SKEW_ERR_SCRATCH_LIMIT;

    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return SKEW_ERR_NODEVICE;
    }
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (g_noalloc_ptr[dev] == nullptr) {
            // host code sees only a stand-in for the array: ask the runtime for its
            // address on this (current) device
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || p == nullptr) {
                set_last_error(e);
                cudaGetLastError();
                return SKEW_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = p;
        }
        scratch = g_noalloc_ptr[dev];
    }
    // skew_pfaffian clears the part of the workspace that must start at zero (its
    // control block) in stream order, and allocates nothing when given a workspace.
    return skew_pfaffian(n, A, lda, logabs, sign, nullptr, nullptr, info, nb_eff, scratch,
                         kNoallocScratchBytes, stream);
}
