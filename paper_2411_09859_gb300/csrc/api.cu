// api.cu -- the C ABI (include/skewltlt.h): argument checks, workspace, and the
// panel loop of the pivoted blocked right-looking factorization.
//
// Per panel k0 .. kend-1 (Section 4.2 Variant 1 with the pivoted panel of
// Section 5.2), all enqueued on the caller's stream with no host synchronisation:
//   1. panel kernel (cooperative): the nb pivoted left-looking steps, then the
//      updated column x = X[kend+1:, kend] for the fused trailing update;
//   2. pivot_rows on the L columns left of the panel (skipped when L is not kept);
//   3. skew rank-2k trailing update of X[kend+1:, kend+1:] (Fused pairs).
// Then one kernel reads off log|Pf|, its sign and the info word.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace skew {

static std::atomic<uint64_t> g_launches{0};
static thread_local char g_last_error[256] = "";

void note_launches(uint64_t count) { g_launches.fetch_add(count); }

void set_last_error(cudaError_t e) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", cudaGetErrorName(e),
             cudaGetErrorString(e));
}

int check_launch() {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(e);
        return SKEW_ERR_CUDA;
    }
    return SKEW_OK;
}

// ------------------------------------------------------------------ per-kernel timing
namespace {
enum ProfKind { kProfPrologue = 0, kProfPanel = 1, kProfPivotRows = 2, kProfSkr2k = 3,
                kProfFinish = 4, kProfBatched = 5 };
struct ProfRec {
    int kind;
    cudaEvent_t a, b;
    double flops, bytes;
};
std::mutex g_prof_mutex;
std::atomic<bool> g_prof_on{false};
std::vector<ProfRec> g_prof;
std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t take_event() {
    std::lock_guard<std::mutex> lock(g_prof_mutex);
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Brackets one launch with events on `st` while profiling is enabled.
// Each stage of a call is an NVTX range named for its kind (a host-side range around
// the launch: it marks when the work was enqueued, which is what a profiler needs to
// select the stage's kernels, e.g. ncu --nvtx --nvtx-include "skr2k/").  With no tool
// attached an NVTX call returns at once.  With profiling on, the stage is also
// bracketed by two CUDA events on its stream.
const char *const kProfNames[] = {"prologue", "panel", "pivot_rows", "skr2k", "finish", "batched"};

struct ProfScope {
    bool on;
    ProfRec r;
    cudaStream_t st;
    ProfScope(int kind, cudaStream_t stream, double flops, double bytes)
        : on(g_prof_on.load()), st(stream) {
        nvtxRangePushA(kProfNames[kind]);
        if (!on) return;
        r.kind = kind;
        r.flops = flops;
        r.bytes = bytes;
        r.a = take_event();
        r.b = take_event();
        if (!r.a || !r.b || cudaEventRecord(r.a, st) != cudaSuccess) {
            cudaGetLastError();
            on = false;
        }
    }
    ~ProfScope() {
        nvtxRangePop();
        if (!on) return;
        if (cudaEventRecord(r.b, st) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        std::lock_guard<std::mutex> lock(g_prof_mutex);
        g_prof.push_back(r);
    }
};

double skr2k_flops(int64_t m, int64_t npairs) { return 2.0 * (double)npairs * (double)m * (double)(m - 1); }
double skr2k_bytes(int64_t m) { return 2.0 * 8.0 * (double)m * (double)(m - 1) / 2.0; }
}  // namespace

// ------------------------------------------------------------------ per-device state
namespace {
constexpr int kMaxDevices = 64;
std::mutex g_dev_mutex;
DeviceInfo g_dev[kMaxDevices];
bool g_dev_ready[kMaxDevices];
cudaMemPool_t g_pool[kMaxDevices];
bool g_pool_ready[kMaxDevices];

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// A side stream with fork/join events: pivot_rows runs on it, overlapping the next
// trailing update (it touches only L columns left of the current panel).  Pooled
// per device; a pooled stream may still hold earlier work, which only orders it.
struct SideStream {
    cudaStream_t stream;
    cudaEvent_t fork, join;
};
std::vector<SideStream> g_side_pool[kMaxDevices];

int side_acquire(int dev, SideStream *out) {
    {
        std::lock_guard<std::mutex> lock(g_dev_mutex);
        if (!g_side_pool[dev].empty()) {
            *out = g_side_pool[dev].back();
            g_side_pool[dev].pop_back();
            return SKEW_OK;
        }
    }
    SKEW_TRY(cudaStreamCreateWithFlags(&out->stream, cudaStreamNonBlocking));
    SKEW_TRY(cudaEventCreateWithFlags(&out->fork, cudaEventDisableTiming));
    SKEW_TRY(cudaEventCreateWithFlags(&out->join, cudaEventDisableTiming));
    return SKEW_OK;
}

void side_release(int dev, const SideStream &s) {
    std::lock_guard<std::mutex> lock(g_dev_mutex);
    g_side_pool[dev].push_back(s);
}

// Streams of the look-ahead factorization: the panels on a stream of the highest
// priority (so that their CTAs are placed as soon as the running trailing update leaves
// room on a multiprocessor) and pivot_rows on another, with the events that order
// them.  Pooled per device like the side streams.
struct LaStreams {
    cudaStream_t panel, rows;
    cudaEvent_t fork, panel_done, upd_done[2], pjoin, rjoin;
};
std::vector<LaStreams> g_la_pool[kMaxDevices];

int la_acquire(int dev, LaStreams *out) {
    {
        std::lock_guard<std::mutex> lock(g_dev_mutex);
        if (!g_la_pool[dev].empty()) {
            *out = g_la_pool[dev].back();
            g_la_pool[dev].pop_back();
            return SKEW_OK;
        }
    }
    int lo = 0, hi = 0;
    SKEW_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    SKEW_TRY(cudaStreamCreateWithPriority(&out->panel, cudaStreamNonBlocking, hi));
    SKEW_TRY(cudaStreamCreateWithFlags(&out->rows, cudaStreamNonBlocking));
    cudaEvent_t *evs[] = {&out->fork, &out->panel_done, &out->upd_done[0], &out->upd_done[1],
                          &out->pjoin, &out->rjoin};
    for (cudaEvent_t *e : evs) SKEW_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    return SKEW_OK;
}

void la_release(int dev, const LaStreams &s) {
    std::lock_guard<std::mutex> lock(g_dev_mutex);
    g_la_pool[dev].push_back(s);
}

std::atomic<int> g_lookahead{1};
// Trailing order below which a look-ahead factorization goes on without it (-1: the
// default, kLaSwitchRows)
std::atomic<long long> g_la_switch{-1};
// Where an update of m trailing rows (about m^2 nb flops at 1 TFLOP/s) stops hiding a
// look-ahead panel (nb column steps of 7-10 us): m^2 ~ 7e6 to 1e7, whatever the width.
// Measured best: 2560 at n = 4096, width 32; 2048-3072 at n = 8192, width 64.
constexpr long long kLaSwitchRows = 2560;
std::atomic<int> g_cluster_panel{1};

// Library-private stream-ordered pool: freed blocks stay reserved for reuse (release
// threshold = max), so repeated calls do not map and unmap device memory.
int device_pool(int dev, cudaMemPool_t *out) {
    std::lock_guard<std::mutex> lock(g_dev_mutex);
    if (!g_pool_ready[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        SKEW_TRY(cudaMemPoolCreate(&g_pool[dev], &props));
        uint64_t thr = UINT64_MAX;
        SKEW_TRY(cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &thr));
        g_pool_ready[dev] = true;
    }
    *out = g_pool[dev];
    return SKEW_OK;
}

}  // namespace

int pool_alloc(void **p, size_t bytes, cudaStream_t st) {
    int dev;
    SKEW_TRY(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    SKEW_TRY_STATUS(device_pool(dev, &pool));
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes ? bytes : 256, pool, st);
    if (e != cudaSuccess) {
        set_last_error(e);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? SKEW_ERR_NOMEM : SKEW_ERR_CUDA;
    }
    return SKEW_OK;
}

int current_device_info(DeviceInfo *out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return SKEW_ERR_NODEVICE;
    }
    {
        std::lock_guard<std::mutex> lock(g_dev_mutex);
        if (g_dev_ready[dev]) {
            *out = g_dev[dev];
            return SKEW_OK;
        }
    }
    int major = 0, minor = 0, sms = 0;
    SKEW_TRY(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
    SKEW_TRY(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
    SKEW_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (major != 10 || minor != 3) return SKEW_ERR_NODEVICE;
    int bps = 0;
    SKEW_TRY_STATUS(panel_max_blocks_per_sm(&bps));
    if (bps < 1) return SKEW_ERR_CUDA;
    DeviceInfo di;
    di.device = dev;
    di.sms = sms;
    di.panel_grid_max = sms;                       // one panel CTA per SM
    if (di.panel_grid_max > kMaxPanelGrid) di.panel_grid_max = kMaxPanelGrid;
    SKEW_TRY_STATUS(panel_cluster_supported(&di.cluster_ok));
    SKEW_TRY_STATUS(panel_la_cluster_supported(&di.cluster_la_ok));
    std::lock_guard<std::mutex> lock(g_dev_mutex);
    g_dev[dev] = di;
    g_dev_ready[dev] = true;
    *out = di;
    return SKEW_OK;
}

WsLayout workspace_layout(int64_t n, int nb, bool with_L, int precision) {
    WsLayout w;
    size_t off = 0;
    w.ctrl = off;
    off += align256(sizeof(Ctrl));
    w.partials = off;
    off += align256(sizeof(ArgmaxPartial) * 2 * kMaxPanelGrid);
    w.tbuf = off;
    off += align256(sizeof(double) * (size_t)(n > 1 ? n : 1));
    w.pivbuf = off;
    off += align256(sizeof(int32_t) * (size_t)(n > 1 ? n : 1));
    w.lbuf = off;
    if (!with_L) off += align256(sizeof(double) * (size_t)(n > 1 ? n : 1) * (size_t)nb);
    w.split = off;
    if (precision == SKEW_PRECISION_SPLIT_BF16) off += split_scratch_bytes(n);
    w.total = off;
    return w;
}

LaLayout workspace_layout_la(int64_t n, int nb, bool with_L) {
    LaLayout l;
    l.base = workspace_layout(n, nb, with_L, SKEW_PRECISION_FP64);
    const size_t nn = (size_t)(n > 1 ? n : 1);
    size_t off = l.base.total;
    l.mat2 = off;
    off += align256(nn * nn * sizeof(double));
    l.maps = off;
    off += 2 * align256(nn * sizeof(int32_t));
    l.xs = off;
    off += 2 * align256(nn * sizeof(double));
    l.lbuf2 = off;
    if (!with_L) off += align256(nn * (size_t)nb * sizeof(double));
    l.total = off;
    return l;
}

bool cluster_panel_enabled() { return g_cluster_panel.load() != 0; }

bool lookahead_applies(int64_t n, int nb, int precision, const DeviceInfo &di) {
    const int mode = g_lookahead.load();          // 0 off, 1 by order, 2 always, 32..128
    if (mode == 0 || precision != SKEW_PRECISION_FP64 || nb < 2 || nb > kLaMaxCols / 2 ||
        n - 1 <= nb || !panel_la_fits(n, 0, di.sms))
        return false;
    return mode != 1 || lookahead_wanted(n, di.cluster_ok && cluster_panel_enabled());
}

// ------------------------------------------------------------------ the factorization
namespace {

// Rows of L sent to host memory while the factorization runs (skew_ltlt_host with a
// page-locked L): a row of L is final once the panel of its step and that panel's
// pivot_rows are done (later exchanges only touch rows below the panel), so each
// panel's strip of rows, over all n columns, is copied on `copy` after them.
struct HostRows {
    double *L_host = nullptr;
    int64_t ldl_host = 0;
    cudaStream_t copy = nullptr;
    cudaEvent_t ev = nullptr;      // reused: each wait captures the last record
    bool used = false;
};

// Copy rows [r0, r1) of the device L (all n columns) to the host after the work
// already submitted on `after`.
int host_rows_strip(HostRows *hr, const double *L, int64_t ldl, int64_t n, int64_t r0,
                    int64_t r1, cudaStream_t after) {
    if (hr == nullptr || hr->L_host == nullptr || r1 <= r0) return SKEW_OK;
    cudaError_t e = cudaEventRecord(hr->ev, after);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hr->copy, hr->ev, 0);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(hr->L_host + r0, hr->ldl_host * sizeof(double), L + r0,
                              ldl * sizeof(double), (size_t)(r1 - r0) * sizeof(double),
                              (size_t)n, cudaMemcpyDeviceToHost, hr->copy);
    if (e != cudaSuccess) {
        set_last_error(e);
        return SKEW_ERR_CUDA;
    }
    hr->used = true;
    return SKEW_OK;
}

// The blocks from s on, factored like the plain path (panel, pivot_rows beside the
// next update, in-place fused update) on the state X = S_j left by the last look-ahead
// update.  Column s of X is the last look-ahead panel's updated column (kept by
// position in xlast), which that update does not write.
int factor_rest_plain(int64_t n, double *X, int64_t ldx, int64_t s, const double *xlast,
                      int64_t jnext, double *L, int64_t ldl, double *const *lbuf, bool with_L,
                      double *t, int32_t *piv, Ctrl *ctrl, ArgmaxPartial *part, int nb,
                      cudaStream_t st, LaStreams &ls, const DeviceInfo &di,
                      HostRows *host_rows) {
    cudaError_t e = cudaMemcpyAsync(X + (s + 1) + s * ldx, xlast + (s + 1),
                                    sizeof(double) * (size_t)(n - s - 1),
                                    cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) { set_last_error(e); return SKEW_ERR_CUDA; }
    int status = SKEW_OK;
    int64_t jj = jnext;
    for (int64_t k0 = s; k0 < n - 1 && status == SKEW_OK; ++jj) {
        const int64_t kend = (k0 + nb < n - 1) ? k0 + nb : n - 1;
        const bool with_x = kend < n - 1;
        PanelArgs pa;
        pa.X = X;
        pa.ldx = ldx;
        pa.Lp = with_L ? L + (k0 + 1) * ldl : lbuf[jj & 1];
        pa.ldl = with_L ? ldl : n;
        pa.t = t;
        pa.piv = piv;
        pa.ctrl = ctrl;
        pa.part = part;
        pa.n = (int)n;
        pa.k0 = (int)k0;
        pa.kend = (int)kend;
        pa.with_x = with_x ? 1 : 0;
        {
            double pf = 0.0;
            for (int64_t k = k0; k < kend; ++k) pf += 2.0 * (double)(n - k - 1) * (double)(k - k0);
            ProfScope ps(kProfPanel, st, pf, 8.0 * 6.0 * (double)(n - k0) * (double)(kend - k0));
            if (di.cluster_ok && cluster_panel_enabled() &&
                panel_cluster_fits(n - k0 - 1, (int)(kend - k0)))
                status = launch_panel_cluster(pa, st);
            else
                status = launch_panel(pa, di.panel_grid_max, st);
        }
        if (status != SKEW_OK) break;
        if (with_L && k0 >= 1) {
            e = cudaEventRecord(ls.fork, st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(ls.rows, ls.fork, 0);
            if (e != cudaSuccess) { set_last_error(e); status = SKEW_ERR_CUDA; break; }
            {
                ProfScope ps(kProfPivotRows, ls.rows, 0.0,
                             4.0 * 8.0 * (double)k0 * (double)(kend - k0));
                status = launch_pivot_rows(n, L, ldl, piv, (int)k0, (int)kend, ls.rows);
            }
            if (status != SKEW_OK) break;
            status = host_rows_strip(host_rows, L, ldl, n, k0 + 1, kend + 1, ls.rows);
            if (status != SKEW_OK) break;
        }
        if (with_x) {
            Skr2kArgs sa;
            sa.m = n - kend - 1;
            sa.C = X + (kend + 1) + (kend + 1) * ldx;
            sa.ldc = ldx;
            sa.alpha = 1.0;
            sa.beta = 1.0;
            sa.P = pa.Lp + (kend + 1);
            sa.ldp = pa.ldl;
            sa.Q = nullptr;
            sa.ldq = 0;
            sa.tt = t + k0 + 1;
            sa.x = X + (kend + 1) + kend * ldx;
            sa.b = kend - k0;
            ProfScope ps(kProfSkr2k, st, skr2k_flops(sa.m, sa.b / 2 + (sa.b & 1)),
                         skr2k_bytes(sa.m));
            status = launch_skr2k(PairKind::Fused, sa, st);
        }
        k0 = kend;
    }
    return status;
}

// The blocked factorization with look-ahead: the panel of block j+1 runs on its own
// stream beside the trailing update of block j.  It reads the state S_{j-1} before
// that update (left-looking over blocks j and j+1, exchanges deferred, see
// panel_la.cu); the update of block j reads S_{j-1} through block j's exchanges and
// writes S_j into the other of two buffers (A and a workspace copy), so neither
// writes what the other reads.  Order:
//   panel j+1  after panel j (its stream) and update j-1 (S_{j-1} complete);
//   update j   after update j-1 (the caller's stream) and panel j;
//   pivot_rows of panel j (on L columns 1 .. k0_j)  after panel j and update j-1,
//              which reads the L columns of block j-1.
int factor_la(int64_t n, double *A, int64_t lda, double *L, int64_t ldl, double *t,
              int32_t *piv, int32_t *info, double *logabs, int32_t *sign, int nb, char *base,
              const LaLayout &lay, cudaStream_t st, bool with_L, const DeviceInfo &di,
              HostRows *host_rows) {
    Ctrl *ctrl = reinterpret_cast<Ctrl *>(base + lay.base.ctrl);
    ArgmaxPartial *part = reinterpret_cast<ArgmaxPartial *>(base + lay.base.partials);
    if (t == nullptr) t = reinterpret_cast<double *>(base + lay.base.tbuf);
    if (piv == nullptr) piv = reinterpret_cast<int32_t *>(base + lay.base.pivbuf);
    double *B = reinterpret_cast<double *>(base + lay.mat2);
    const size_t nn = (size_t)n;
    int32_t *maps[2] = {reinterpret_cast<int32_t *>(base + lay.maps),
                        reinterpret_cast<int32_t *>(base + lay.maps + align256(nn * sizeof(int32_t)))};
    double *xs[2] = {reinterpret_cast<double *>(base + lay.xs),
                     reinterpret_cast<double *>(base + lay.xs + align256(nn * sizeof(double)))};
    double *lbuf[2] = {reinterpret_cast<double *>(base + lay.base.lbuf),
                       reinterpret_cast<double *>(base + lay.lbuf2)};
    // S_j lives in B for even j and in A for odd j; S_{-1} is A
    auto sbuf = [&](int64_t j) -> double * { return (j >= 0 && (j & 1) == 0) ? B : A; };
    auto sld = [&](int64_t j) -> int64_t { return (j >= 0 && (j & 1) == 0) ? (int64_t)n : lda; };
    // L columns of the block starting at k0 (block index j)
    auto lblock = [&](int64_t k0, int64_t j) -> double * {
        return with_L ? L + (k0 + 1) * ldl : lbuf[j & 1];
    };
    const int64_t lld = with_L ? ldl : (int64_t)n;

    LaStreams ls{};
    SKEW_TRY_STATUS(la_acquire(di.device, &ls));
    int status = SKEW_OK;
    bool p_used = false, r_used = false;
    do {
        cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(part, 0, sizeof(ArgmaxPartial) * 2 * kMaxPanelGrid, st);
        if (e != cudaSuccess) { set_last_error(e); status = SKEW_ERR_CUDA; break; }
        {
            ProfScope ps(kProfPrologue, st, 0.0,
                         8.0 * (double)n * (double)(n - 1) / 2.0 +
                             (with_L ? 8.0 * (double)n * (double)n : 0.0));
            status = launch_prologue(n, A, lda, with_L ? L : nullptr, ldl, piv, ctrl, st);
        }
        if (status != SKEW_OK) break;
        e = cudaEventRecord(ls.fork, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ls.panel, ls.fork, 0);
        if (e == cudaSuccess && with_L) e = cudaStreamWaitEvent(ls.rows, ls.fork, 0);
        if (e != cudaSuccess) { set_last_error(e); status = SKEW_ERR_CUDA; break; }
        p_used = true;
        r_used = with_L;

        auto panel_prof = [&](int64_t kb, int64_t k0, int64_t kend, bool with_x, double &pf,
                              double &pb) {
            pf = 0.0;
            pb = 0.0;
            for (int64_t k = k0; k <= kend; ++k) {
                if (k == kend && !with_x) break;
                const double rows = (double)(n - k - 1);
                pf += 2.0 * rows * (double)(k - kb);
                pb += 8.0 * rows * 2.0;
            }
        };
        // a look-ahead panel as one cluster where it fits, else grid-wide
        auto launch_la_panel = [&](const PanelLAArgs &pa) -> int {
            const int64_t rows = n - (int64_t)pa.k0 - 1;
            const int cols = (pa.k0 - pa.kb) + (pa.kend - pa.k0);
            if (di.cluster_la_ok && cluster_panel_enabled() && pa.rows_per_cta == 0 &&
                panel_la_cluster_fits(rows, cols))
                return launch_panel_la_cluster(pa, ls.panel);
            return launch_panel_la(pa, di.sms, ls.panel);
        };
        // panel 0: the first block, from A itself
        int64_t k0 = 0, kend = (nb < n - 1) ? nb : n - 1;
        {
            PanelLAArgs pa;
            pa.S = A;
            pa.lds = lda;
            pa.map_prev = nullptr;
            pa.xprev = nullptr;
            pa.Lprev = nullptr;
            pa.ldlp = lld;
            pa.Lp = lblock(0, 0);
            pa.ldl = lld;
            pa.t = t;
            pa.piv = piv;
            pa.map_out = maps[0];
            pa.xout = xs[0];
            pa.ctrl = ctrl;
            pa.part = part;
            pa.n = (int)n;
            pa.kb = 0;
            pa.k0 = 0;
            pa.kend = (int)kend;
            pa.with_x = kend < n - 1 ? 1 : 0;
            pa.rows_per_cta = g_lookahead.load() > 2 ? g_lookahead.load() : 0;
            double pf, pb;
            panel_prof(0, 0, kend, pa.with_x != 0, pf, pb);
            ProfScope ps(kProfPanel, ls.panel, pf, pb);
            status = launch_la_panel(pa);
        }
        if (status != SKEW_OK) break;
        // rows 0 .. kend of L are final after the first panel
        if (with_L) status = host_rows_strip(host_rows, L, ldl, n, 0, kend + 1, ls.panel);
        if (status != SKEW_OK) break;
        e = cudaEventRecord(ls.panel_done, ls.panel);
        if (e != cudaSuccess) { set_last_error(e); status = SKEW_ERR_CUDA; break; }

        for (int64_t j = 0;; ++j) {
            const int64_t s = kend;                  // this block: k0 .. kend-1
            const bool has_update = s < n - 1;
            // The waits on panel j come first (they capture its event before panel j+1
            // records it again); panel j+1 is submitted before update j, so that the
            // panel (a high-priority stream, possibly one thread-block cluster) is
            // placed before the update's CTAs fill the multiprocessors.
            if (has_update) {
                e = cudaStreamWaitEvent(st, ls.panel_done, 0);
                if (e != cudaSuccess) { set_last_error(e); status = SKEW_ERR_CUDA; break; }
            }
            // ---- pivot_rows of panel j on L columns 1 .. k0
            if (with_L && k0 >= 1) {
                e = cudaStreamWaitEvent(ls.rows, ls.panel_done, 0);
                if (e == cudaSuccess && j >= 1)
                    e = cudaStreamWaitEvent(ls.rows, ls.upd_done[(j - 1) & 1], 0);
                if (e != cudaSuccess) { set_last_error(e); status = SKEW_ERR_CUDA; break; }
                {
                    ProfScope ps(kProfPivotRows, ls.rows, 0.0,
                                 4.0 * 8.0 * (double)k0 * (double)(kend - k0));
                    status = launch_pivot_rows(n, L, ldl, piv, (int)k0, (int)kend, ls.rows);
                }
                if (status != SKEW_OK) break;
                status = host_rows_strip(host_rows, L, ldl, n, k0 + 1, kend + 1, ls.rows);
                if (status != SKEW_OK) break;
            }
            if (!has_update) break;
            // Below the switch order the panel of a block costs more than the update it
            // would hide: update j is the last look-ahead update, and the remaining blocks
            // are factored like the plain path, in place on S_j.
            const long long sw = g_la_switch.load();
            const bool la_next = (n - s - 1) > (sw < 0 ? kLaSwitchRows : sw);
            // ---- panel j+1, beside update j: reads S_{j-1}
            const int64_t k0n = kend, kendn = (kend + nb < n - 1) ? kend + nb : n - 1;
            if (la_next && j >= 1) {
                e = cudaStreamWaitEvent(ls.panel, ls.upd_done[(j - 1) & 1], 0);
                if (e != cudaSuccess) { set_last_error(e); status = SKEW_ERR_CUDA; break; }
            }
            if (la_next) {
                PanelLAArgs pa;
                pa.S = sbuf(j - 1);
                pa.lds = sld(j - 1);
                pa.map_prev = maps[j & 1];
                pa.xprev = xs[j & 1];
                pa.Lprev = lblock(k0, j);
                pa.ldlp = lld;
                pa.Lp = lblock(k0n, j + 1);
                pa.ldl = lld;
                pa.t = t;
                pa.piv = piv;
                pa.map_out = maps[(j + 1) & 1];
                pa.xout = xs[(j + 1) & 1];
                pa.ctrl = ctrl;
                pa.part = part;
                pa.n = (int)n;
                pa.kb = (int)k0;
                pa.k0 = (int)k0n;
                pa.kend = (int)kendn;
                pa.with_x = kendn < n - 1 ? 1 : 0;
                pa.rows_per_cta = g_lookahead.load() > 2 ? g_lookahead.load() : 0;
                {
                    double pf, pb;
                    panel_prof(k0, k0n, kendn, pa.with_x != 0, pf, pb);
                    ProfScope ps(kProfPanel, ls.panel, pf, pb);
                    status = launch_la_panel(pa);
                }
                if (status != SKEW_OK) break;
                e = cudaEventRecord(ls.panel_done, ls.panel);
                if (e != cudaSuccess) { set_last_error(e); status = SKEW_ERR_CUDA; break; }
            }
            if (has_update) {
                // ---- update j: S_j = (S_{j-1} through block j's exchanges) + pairs
                Skr2kArgs sa;
                sa.m = n - s - 1;
                double *dst = sbuf(j);
                const int64_t ldd = sld(j);
                sa.C = dst + (s + 1) + (s + 1) * ldd;
                sa.ldc = ldd;
                sa.Cin = sbuf(j - 1);
                sa.ldcin = sld(j - 1);
                sa.map = maps[j & 1] + (s + 1);
                sa.nin = n;
                sa.alpha = 1.0;
                sa.beta = 1.0;
                sa.P = lblock(k0, j) + (s + 1);
                sa.ldp = lld;
                sa.Q = nullptr;
                sa.ldq = 0;
                sa.tt = t + k0 + 1;
                sa.x = xs[j & 1] + (s + 1);
                sa.b = kend - k0;
                {
                    ProfScope ps(kProfSkr2k, st, skr2k_flops(sa.m, sa.b / 2 + (sa.b & 1)),
                                 skr2k_bytes(sa.m));
                    status = launch_skr2k(PairKind::Fused, sa, st);
                }
                if (status != SKEW_OK) break;
                e = cudaEventRecord(ls.upd_done[j & 1], st);
                if (e != cudaSuccess) { set_last_error(e); status = SKEW_ERR_CUDA; break; }
            }
            if (!la_next) {
                status = factor_rest_plain(n, sbuf(j), sld(j), s, xs[j & 1], j + 1, L, ldl,
                                           lbuf, with_L, t, piv, ctrl, part, nb, st, ls, di,
                                           host_rows);
                break;
            }
            k0 = k0n;
            kend = kendn;
        }
        if (status != SKEW_OK) break;
    } while (0);

    // join: the caller's stream waits for the last panel and the last pivot_rows
    if (p_used) {
        cudaError_t e = cudaEventRecord(ls.pjoin, ls.panel);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ls.pjoin, 0);
        if (e != cudaSuccess && status == SKEW_OK) { set_last_error(e); status = SKEW_ERR_CUDA; }
    }
    if (r_used) {
        cudaError_t e = cudaEventRecord(ls.rjoin, ls.rows);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ls.rjoin, 0);
        if (e != cudaSuccess && status == SKEW_OK) { set_last_error(e); status = SKEW_ERR_CUDA; }
    }
    if (status == SKEW_OK) {
        ProfScope ps(kProfFinish, st, 0.0, 12.0 * (double)n);
        status = launch_finish(n, t, piv, ctrl, logabs, sign, info, st);
    }
    la_release(di.device, ls);
    return status;
}

int factor(int64_t n, double *A, int64_t lda, double *L, int64_t ldl, double *t,
           int32_t *piv, int32_t *info, double *logabs, int32_t *sign, int nb,
           void *workspace, size_t workspace_bytes, cudaStream_t st, bool with_L,
           int precision, HostRows *host_rows = nullptr) {
    DeviceInfo di;
    SKEW_TRY_STATUS(current_device_info(&di));
    if (nb == 0) nb = skew_default_nb(n);
    if (lookahead_applies(n, nb, precision, di)) {
        const LaLayout llay = workspace_layout_la(n, nb, with_L);
        char *lb = static_cast<char *>(workspace);
        if (lb == nullptr || workspace_bytes >= llay.total) {
            bool lown = false;
            if (lb == nullptr) {
                SKEW_TRY_STATUS(pool_alloc(reinterpret_cast<void **>(&lb), llay.total, st));
                lown = true;
            }
            int rc = factor_la(n, A, lda, L, ldl, t, piv, info, logabs, sign, nb, lb, llay, st,
                               with_L, di, host_rows);
            if (lown) {
                cudaError_t e = cudaFreeAsync(lb, st);
                if (e != cudaSuccess && rc == SKEW_OK) {
                    set_last_error(e);
                    rc = SKEW_ERR_CUDA;
                }
            }
            return rc;
        }
        // a caller's workspace sized for the plain path: factor without look-ahead
    }
    const WsLayout lay = workspace_layout(n, nb, with_L, precision);
    char *base = static_cast<char *>(workspace);
    bool own = false;
    if (base == nullptr) {
        SKEW_TRY_STATUS(pool_alloc(reinterpret_cast<void **>(&base), lay.total, st));
        own = true;
    } else if (workspace_bytes < lay.total) {
        return -11;
    }
    int status = SKEW_OK;
    Ctrl *ctrl = reinterpret_cast<Ctrl *>(base + lay.ctrl);
    ArgmaxPartial *part = reinterpret_cast<ArgmaxPartial *>(base + lay.partials);
    if (t == nullptr) t = reinterpret_cast<double *>(base + lay.tbuf);
    if (piv == nullptr) piv = reinterpret_cast<int32_t *>(base + lay.pivbuf);
    double *Lbuf = with_L ? nullptr : reinterpret_cast<double *>(base + lay.lbuf);

    SideStream side{};
    bool have_side = false;
    if (with_L && n > nb + 1) {
        status = side_acquire(di.device, &side);
        if (status != SKEW_OK) {
            if (own) cudaFreeAsync(base, st);
            return status;
        }
        have_side = true;
    }
    bool side_used = false;

    do {
        // control block and the step tags of the argmax partials start at zero
        cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(part, 0, sizeof(ArgmaxPartial) * 2 * kMaxPanelGrid, st);
        if (e != cudaSuccess) { set_last_error(e); status = SKEW_ERR_CUDA; break; }
        {
            ProfScope ps(kProfPrologue, st, 0.0,
                         8.0 * (double)n * (double)(n - 1) / 2.0 +
                             (with_L ? 8.0 * (double)n * (double)n : 0.0));
            status = launch_prologue(n, A, lda, with_L ? L : nullptr, ldl, piv, ctrl, st);
        }
        if (status != SKEW_OK) break;
        for (int64_t k0 = 0; k0 < n - 1 && status == SKEW_OK;) {
            const int64_t kend = (k0 + nb < n - 1) ? k0 + nb : n - 1;
            const int64_t s = kend;
            const bool with_x = s < n - 1;
            PanelArgs pa;
            pa.X = A;
            pa.ldx = lda;
            if (with_L) {
                pa.Lp = L + (k0 + 1) * ldl;
                pa.ldl = ldl;
            } else {
                pa.Lp = Lbuf;
                pa.ldl = n;
            }
            pa.t = t;
            pa.piv = piv;
            pa.ctrl = ctrl;
            pa.part = part;
            pa.n = (int)n;
            pa.k0 = (int)k0;
            pa.kend = (int)kend;
            pa.with_x = with_x ? 1 : 0;
            {
                double pf = 0.0, pb = 0.0;
                for (int64_t k = k0; k < kend; ++k) {
                    const double rows = (double)(n - k - 1);
                    pf += 2.0 * rows * (double)(k - k0);
                    pb += 8.0 * rows * 6.0;
                }
                if (with_x) {
                    pf += 2.0 * (double)(n - s - 1) * (double)(s - k0);
                    pb += 8.0 * (double)(n - s - 1) * 2.0;
                }
                ProfScope ps(kProfPanel, st, pf, pb);
                if (di.cluster_ok && cluster_panel_enabled() &&
                    panel_cluster_fits(n - k0 - 1, (int)(kend - k0)))
                    status = launch_panel_cluster(pa, st);
                else
                    status = launch_panel(pa, di.panel_grid_max, st);
            }
            if (status != SKEW_OK) break;
            if (with_L && k0 >= 1) {
                // fork: pivot_rows after this panel, beside the next trailing update
                cudaStream_t ps_stream = st;
                if (have_side) {
                    e = cudaEventRecord(side.fork, st);
                    if (e == cudaSuccess) e = cudaStreamWaitEvent(side.stream, side.fork, 0);
                    if (e != cudaSuccess) { set_last_error(e); status = SKEW_ERR_CUDA; break; }
                    ps_stream = side.stream;
                    side_used = true;
                }
                {
                    ProfScope ps(kProfPivotRows, ps_stream, 0.0,
                                 4.0 * 8.0 * (double)k0 * (double)(kend - k0));
                    status = launch_pivot_rows(n, L, ldl, piv, (int)k0, (int)kend, ps_stream);
                }
                if (status != SKEW_OK) break;
                // rows k0+1 .. kend of L are final
                status = host_rows_strip(host_rows, L, ldl, n, k0 + 1, kend + 1, ps_stream);
                if (status != SKEW_OK) break;
            } else if (with_L && k0 == 0) {
                // rows 0 .. kend of L are final after the first panel
                status = host_rows_strip(host_rows, L, ldl, n, 0, kend + 1, st);
                if (status != SKEW_OK) break;
            }
            if (with_x) {
                Skr2kArgs sa;
                sa.m = n - s - 1;
                sa.C = A + (s + 1) + (s + 1) * lda;
                sa.ldc = lda;
                sa.alpha = 1.0;
                sa.beta = 1.0;
                sa.P = pa.Lp + (s + 1);
                sa.ldp = pa.ldl;
                sa.Q = nullptr;
                sa.ldq = 0;
                sa.tt = t + k0 + 1;
                sa.x = A + (s + 1) + s * lda;
                sa.b = kend - k0;
                ProfScope ps(kProfSkr2k, st, skr2k_flops(sa.m, sa.b / 2 + (sa.b & 1)),
                             skr2k_bytes(sa.m));
                sa.balance = 1;
                if (precision == SKEW_PRECISION_SPLIT_BF16)
                    status = launch_skr2k_split(PairKind::Fused, sa, base + lay.split, &ctrl->err, di.sms, st);
                else
                    status = launch_skr2k(PairKind::Fused, sa, st);
            }
            k0 = kend;
        }
        if (status != SKEW_OK) break;
        ProfScope ps(kProfFinish, st, 0.0, 12.0 * (double)n);
        status = launch_finish(n, t, piv, ctrl, logabs, sign, info, st);
    } while (0);

    if (side_used) {
        // join: the caller's stream waits for the last pivot_rows
        cudaError_t e = cudaEventRecord(side.join, side.stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, side.join, 0);
        if (e != cudaSuccess && status == SKEW_OK) {
            set_last_error(e);
            status = SKEW_ERR_CUDA;
        }
    }
    if (have_side) side_release(di.device, side);

    if (own) {
        cudaError_t e = cudaFreeAsync(base, st);
        if (e != cudaSuccess && status == SKEW_OK) {
            set_last_error(e);
            status = SKEW_ERR_CUDA;
        }
    }
    return status;
}

// The two-step (Pfaffian-only) elimination: per panel of nb columns (nb/2 pairs), the
// two-step panel kernel, then one skew rank-2k update of the trailing block with the
// panel's pairs (l_j, y_j): X[k1:, k1:] += sum_j (l_j y_j^T - y_j l_j^T).
int factor_twostep(int64_t n, double *A, int64_t lda, double *a, int32_t *piv, int32_t *info,
                   double *logabs, int32_t *sign, int nb, void *workspace,
                   size_t workspace_bytes, cudaStream_t st, int precision) {
    DeviceInfo di;
    SKEW_TRY_STATUS(current_device_info(&di));
    if (!twostep_fits(n, nb, di.panel_grid_max)) return -1;
    const WsLayout lay = workspace_layout(n, nb, false, precision);
    char *base = static_cast<char *>(workspace);
    bool own = false;
    if (base == nullptr) {
        SKEW_TRY_STATUS(pool_alloc(reinterpret_cast<void **>(&base), lay.total, st));
        own = true;
    } else if (workspace_bytes < lay.total) {
        return -12;
    }
    int status = SKEW_OK;
    Ctrl *ctrl = reinterpret_cast<Ctrl *>(base + lay.ctrl);
    ArgmaxPartial *part = reinterpret_cast<ArgmaxPartial *>(base + lay.partials);
    if (a == nullptr) a = reinterpret_cast<double *>(base + lay.tbuf);
    if (piv == nullptr) piv = reinterpret_cast<int32_t *>(base + lay.pivbuf);
    double *V = reinterpret_cast<double *>(base + lay.lbuf);     // n x nb
    do {
        cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(part, 0, sizeof(ArgmaxPartial) * 2 * kMaxPanelGrid, st);
        if (e == cudaSuccess && n >= 2) e = cudaMemsetAsync(a, 0, sizeof(double) * (size_t)(n / 2), st);
        if (e != cudaSuccess) { set_last_error(e); status = SKEW_ERR_CUDA; break; }
        {
            ProfScope ps(kProfPrologue, st, 0.0, 8.0 * (double)n * (double)(n - 1) / 2.0);
            status = launch_prologue(n, A, lda, nullptr, 0, piv, ctrl, st);
        }
        if (status != SKEW_OK) break;
        for (int64_t k0 = 0; k0 + 1 < n && status == SKEW_OK;) {
            int64_t np = 0;
            for (int64_t k = k0; k < k0 + nb && k + 1 < n; k += 2) ++np;
            const int64_t k1 = k0 + 2 * np;                      // first column left
            TwoStepArgs ta;
            ta.X = A;
            ta.ldx = lda;
            ta.V = V;
            ta.ldv = n;
            ta.a = a;
            ta.piv = piv;
            ta.ctrl = ctrl;
            ta.part = part;
            ta.n = (int)n;
            ta.k0 = (int)k0;
            ta.kend = (int)k1;
            {
                double pf = 0.0, pb = 0.0;
                for (int64_t j = 0; j < np; ++j) {
                    const double rows = (double)(n - k0 - 2 * j - 2);
                    pf += 2.0 * rows * (double)(4 * j + 2);
                    pb += 8.0 * rows * 6.0;
                }
                ProfScope ps(kProfPanel, st, pf, pb);
                status = launch_twostep_panel(ta, di.panel_grid_max, st);
            }
            if (status != SKEW_OK) break;
            const int64_t m = n - k1;
            if (m >= 2) {
                Skr2kArgs sa;
                sa.m = m;
                sa.C = A + k1 + k1 * lda;
                sa.ldc = lda;
                sa.alpha = 1.0;
                sa.beta = 1.0;
                sa.P = V + k1;                  // l_j: column 2j
                sa.ldp = 2 * n;
                sa.Q = V + n + k1;              // y_j: column 2j+1
                sa.ldq = 2 * n;
                sa.tt = nullptr;
                sa.x = nullptr;
                sa.b = np;
                ProfScope ps(kProfSkr2k, st, skr2k_flops(m, np), skr2k_bytes(m));
                sa.balance = 1;
                if (precision == SKEW_PRECISION_SPLIT_BF16)
                    status = launch_skr2k_split(PairKind::Rank2k, sa, base + lay.split, &ctrl->err,
                                                di.sms, st);
                else
                    status = launch_skr2k(PairKind::Rank2k, sa, st);
            }
            k0 = k1;
        }
        if (status != SKEW_OK) break;
        ProfScope ps(kProfFinish, st, 0.0, 12.0 * (double)n);
        status = launch_finish_twostep(n, a, piv, ctrl, logabs, sign, info, st);
    } while (0);
    if (own) {
        cudaError_t e = cudaFreeAsync(base, st);
        if (e != cudaSuccess && status == SKEW_OK) {
            set_last_error(e);
            status = SKEW_ERR_CUDA;
        }
    }
    return status;
}

}  // namespace
}  // namespace skew

namespace skew {
namespace {
std::mutex g_bnb_mutex;
BatchedNb g_bnb = {0, {0}, {0}, {0}, 256};
}  // namespace

BatchedNb batched_nb_table() {
    std::lock_guard<std::mutex> lock(g_bnb_mutex);
    return g_bnb;
}
}  // namespace skew

using namespace skew;

namespace {
// Context of the host-buffer call, one per device, created on first use and kept
// until skew_trim_memory: the stream, the phase events, and the device buffers (grown
// when a larger order arrives).  Calls on one device are serialised by its mutex.
struct HostCall {
    std::mutex mu;
    bool ready = false;
    cudaStream_t st = nullptr;
    cudaStream_t copy = nullptr;   // rows of L to host memory during the factorization
    cudaEvent_t ev_rows = nullptr, ev_join = nullptr;
    cudaEvent_t ev[4] = {};
    void *buf = nullptr;          // dA | dL | dt | dpiv | dlog | dsign | dinfo
    size_t buf_bytes = 0;
    float ms[3] = {0.f, 0.f, 0.f};
    bool have_ms = false;
};
HostCall g_host[kMaxDevices];

int host_ready(HostCall &h) {
    if (h.ready) return SKEW_OK;
    SKEW_TRY(cudaStreamCreateWithFlags(&h.st, cudaStreamNonBlocking));
    SKEW_TRY(cudaStreamCreateWithFlags(&h.copy, cudaStreamNonBlocking));
    SKEW_TRY(cudaEventCreateWithFlags(&h.ev_rows, cudaEventDisableTiming));
    SKEW_TRY(cudaEventCreateWithFlags(&h.ev_join, cudaEventDisableTiming));
    for (cudaEvent_t &e : h.ev) SKEW_TRY(cudaEventCreate(&e));
    h.ready = true;
    return SKEW_OK;
}

int host_release_buffers(HostCall &h) {
    if (h.buf == nullptr) return SKEW_OK;
    cudaError_t e = cudaFreeAsync(h.buf, h.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h.st);
    h.buf = nullptr;
    h.buf_bytes = 0;
    if (e != cudaSuccess) {
        set_last_error(e);
        return SKEW_ERR_CUDA;
    }
    return SKEW_OK;
}
}  // namespace

extern "C" {

int skew_version(void) { return 100; }   // 0.1.0

const char *skew_last_error(void) { return g_last_error; }

uint64_t skew_kernel_launches(void) { return g_launches.load(); }

// Panel-width table installed by skew_set_nb_table (an autotuner's result), else the
// built-in rule; each entry also says whether that order range takes the look-ahead
// (-1: the built-in rule).  Guarded by a mutex: installs are rare, reads take a
// snapshot.
namespace {
struct NbEntry {
    int64_t n_upper;
    int nb;
    int lookahead;
};
std::mutex g_nb_mutex;
std::vector<NbEntry> g_nb_table;
}  // namespace

}  // extern "C"

namespace skew {
// Whether order n takes the look-ahead: the table's choice, else on for
// 3072 <= n <= 10240 (measured on GB300: at n = 4096 / 8192 the look-ahead saves 10 % /
// 5 %; at 2048 and from 12288 up the panel's extra FP64 work and its share of the
// multiprocessors cost as much as the overlap saves).
bool lookahead_wanted(int64_t n, bool cluster_panel) {
    {
        std::lock_guard<std::mutex> lock(g_nb_mutex);
        if (!g_nb_table.empty()) {
            int la = g_nb_table.back().lookahead;
            for (const auto &e : g_nb_table)
                if (n <= e.n_upper) { la = e.lookahead; break; }
            if (la >= 0) return la != 0;
        }
    }
    // Built-in rule (measured on GB300): with cluster panels the look-ahead (its panels
    // also clusters, up to the switch order) wins around n = 4096 and loses at 2048 and
    // 8192; with grid-wide panels it wins from about 3072 to 10240.
    return cluster_panel ? (n >= 3072 && n <= 5120) : (n >= 3072 && n <= 10240);
}
}  // namespace skew

extern "C" {

int skew_set_nb_table_ex(int count, const int64_t *n_upper, const int32_t *nb,
                         const int32_t *lookahead) {
    if (count < 0) return -1;
    if (count > 0 && (n_upper == nullptr)) return -2;
    if (count > 0 && (nb == nullptr)) return -3;
    std::vector<NbEntry> t;
    for (int i = 0; i < count; ++i) {
        if (nb[i] < 1 || nb[i] > kMaxNb) return -3;
        if (i > 0 && n_upper[i] <= n_upper[i - 1]) return -2;
        const int la = lookahead ? lookahead[i] : -1;
        if (la < -1 || la > 1) return -4;
        t.push_back({n_upper[i], nb[i], la});
    }
    std::lock_guard<std::mutex> lock(g_nb_mutex);
    g_nb_table.swap(t);
    return SKEW_OK;
}

int skew_set_nb_table(int count, const int64_t *n_upper, const int32_t *nb) {
    return skew_set_nb_table_ex(count, n_upper, nb, nullptr);
}

int skew_set_batched_tiles(int count, const int32_t *n_upper, const int32_t *nb,
                           const int32_t *warp_tile) {
    if (count < 0 || count > 8) return -1;
    if (count > 0 && n_upper == nullptr) return -2;
    if (count > 0 && nb == nullptr) return -3;
    BatchedNb t = {count, {0}, {0}, {0}, 256};
    for (int i = 0; i < count; ++i) {
        if (nb[i] != 8 && nb[i] != 16 && nb[i] != 32) return -3;
        if (n_upper[i] < 1 || (i > 0 && n_upper[i] <= n_upper[i - 1])) return -2;
        const int wt = warp_tile ? warp_tile[i] : 32;
        if (wt != 16 && wt != 32) return -4;
        t.n_upper[i] = n_upper[i];
        t.nb[i] = nb[i];
        t.wt[i] = wt;
    }
    std::lock_guard<std::mutex> lock(g_bnb_mutex);
    t.threads = g_bnb.threads;
    g_bnb = t;
    return SKEW_OK;
}

int skew_set_batched_threads(int threads) {
    if (threads != 128 && threads != 256) return -1;
    std::lock_guard<std::mutex> lock(g_bnb_mutex);
    const int old = g_bnb.threads;
    g_bnb.threads = threads;
    return old;
}

int skew_set_batched_nb_table(int count, const int32_t *n_upper, const int32_t *nb) {
    return skew_set_batched_tiles(count, n_upper, nb, nullptr);
}

int skew_get_batched_nb(int n) {
    return batched_nb_for(batched_nb_table(), n);
}

int skew_get_batched_warp_tile(int n) {
    return batched_wt_for(batched_nb_table(), n);
}

int skew_default_nb(int64_t n) {
    {
        std::lock_guard<std::mutex> lock(g_nb_mutex);
        if (!g_nb_table.empty()) {
            for (const auto &e : g_nb_table)
                if (n <= e.n_upper) return e.nb;
            return g_nb_table.back().nb;
        }
    }
    if (n <= 256) return 16;
    if (n <= 2048) return 32;
    return 64;
}

size_t skew_workspace_bytes(int64_t n, int nb, int with_L) {
    if (n < 0) return 0;
    if (nb <= 0) nb = skew_default_nb(n);
    if (nb > kMaxNb) nb = kMaxNb;
    return workspace_layout(n, nb, with_L != 0).total;
}

size_t skew_workspace_bytes_lookahead(int64_t n, int nb, int with_L) {
    if (n < 0) return 0;
    if (nb <= 0) nb = skew_default_nb(n);
    if (nb > kMaxNb) nb = kMaxNb;
    if (nb > kLaMaxCols / 2 || n >= 65535) return workspace_layout(n, nb, with_L != 0).total;
    return workspace_layout_la(n, nb, with_L != 0).total;
}

int skew_lookahead_used(int64_t n, int nb, int precision) {
    DeviceInfo di;
    if (current_device_info(&di) != SKEW_OK) return 0;
    if (nb <= 0) nb = skew_default_nb(n);
    return lookahead_applies(n, nb, precision, di) ? 1 : 0;
}

int skew_set_cluster_panel(int on) {
    return g_cluster_panel.exchange(on != 0 ? 1 : 0);
}

long long skew_set_lookahead_switch(long long rows) {
    return g_la_switch.exchange(rows < 0 ? -1 : rows);
}

int skew_set_lookahead(int mode) {
    const int old = g_lookahead.load();
    g_lookahead.store((mode == 2 || mode == 32 || mode == 64 || mode == 128) ? mode
                                                                            : (mode != 0 ? 1 : 0));
    return old;
}

int skew_profile_enable(int on) {
    g_prof_on.store(on != 0);
    return SKEW_OK;
}

int skew_profile_read(skew_kernel_stat *stats) {
    if (stats == nullptr) return -1;
    for (int k = 0; k < SKEW_KIND_COUNT; ++k) stats[k] = skew_kernel_stat{0.0, 0.0, 0.0, 0};
    std::vector<ProfRec> recs;
    {
        std::lock_guard<std::mutex> lock(g_prof_mutex);
        recs.swap(g_prof);
    }
    int status = SKEW_OK;
    for (const ProfRec &r : recs) {
        float ms = 0.0f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) {
            set_last_error(e);
            status = SKEW_ERR_CUDA;
        } else if (r.kind >= 0 && r.kind < SKEW_KIND_COUNT) {
            stats[r.kind].ms += ms;
            stats[r.kind].flops += r.flops;
            stats[r.kind].bytes += r.bytes;
            stats[r.kind].launches += 1;
        }
    }
    std::lock_guard<std::mutex> lock(g_prof_mutex);
    for (const ProfRec &r : recs) {
        g_event_pool.push_back(r.a);
        g_event_pool.push_back(r.b);
    }
    return status;
}

int skew_selftest_bounded_wait(double timeout_s, int32_t *status) {
    if (!(timeout_s > 0.0 && timeout_s <= 10.0)) return -1;
    if (status == nullptr) return -2;
    DeviceInfo di;
    SKEW_TRY_STATUS(current_device_info(&di));
    cudaStream_t st;
    SKEW_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    void *p = nullptr;
    int rc = pool_alloc(&p, sizeof(Ctrl), st);
    if (rc == SKEW_OK) {
        Ctrl *ctrl = static_cast<Ctrl *>(p);
        cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st);
        if (e != cudaSuccess) { set_last_error(e); rc = SKEW_ERR_CUDA; }
        if (rc == SKEW_OK)
            rc = launch_selftest_wait(ctrl, 2, (uint64_t)(timeout_s * 1e9), st);
        if (rc == SKEW_OK) {
            e = cudaMemcpyAsync(status, &ctrl->err, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) { set_last_error(e); rc = SKEW_ERR_CUDA; }
        }
        cudaFreeAsync(p, st);
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess && rc == SKEW_OK) { set_last_error(e); rc = SKEW_ERR_CUDA; }
    cudaStreamDestroy(st);
    return rc;
}

int skew_selftest_mbarrier_wait(double timeout_s, int32_t *status) {
    if (!(timeout_s > 0.0 && timeout_s <= 10.0)) return -1;
    if (status == nullptr) return -2;
    DeviceInfo di;
    SKEW_TRY_STATUS(current_device_info(&di));
    cudaStream_t st;
    SKEW_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    void *p = nullptr;
    int rc = pool_alloc(&p, sizeof(int), st);
    if (rc == SKEW_OK) {
        int *err = static_cast<int *>(p);
        cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
        if (e != cudaSuccess) { set_last_error(e); rc = SKEW_ERR_CUDA; }
        if (rc == SKEW_OK) rc = launch_selftest_mbar(err, (uint64_t)(timeout_s * 1e9), st);
        if (rc == SKEW_OK) {
            e = cudaMemcpyAsync(status, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) { set_last_error(e); rc = SKEW_ERR_CUDA; }
        }
        cudaFreeAsync(p, st);
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess && rc == SKEW_OK) { set_last_error(e); rc = SKEW_ERR_CUDA; }
    cudaStreamDestroy(st);
    return rc;
}

int skew_pool_usage(size_t *used_now, size_t *used_high, int reset_high) {
    int dev;
    SKEW_TRY(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    SKEW_TRY_STATUS(device_pool(dev, &pool));
    unsigned long long now = 0, high = 0;   // the attributes are 64-bit values
    SKEW_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &now));
    SKEW_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &high));
    if (used_now) *used_now = (size_t)now;
    if (used_high) *used_high = (size_t)high;
    if (reset_high) {
        unsigned long long zero = 0;
        SKEW_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
    }
    return SKEW_OK;
}

int skew_trim_memory(void) {
    int dev;
    SKEW_TRY(cudaGetDevice(&dev));
    if (dev >= 0 && dev < kMaxDevices) {
        std::lock_guard<std::mutex> lock(g_host[dev].mu);
        SKEW_TRY_STATUS(host_release_buffers(g_host[dev]));
    }
    cudaMemPool_t pool;
    SKEW_TRY_STATUS(device_pool(dev, &pool));
    SKEW_TRY(cudaMemPoolTrimTo(pool, 0));
    return SKEW_OK;
}

int skew_ltlt(int64_t n, double *A, int64_t lda, double *L, int64_t ldl, double *t,
              int32_t *piv, int32_t *info, int nb, void *workspace,
              size_t workspace_bytes, void *stream) {
    if (n < 0 || n > kMaxOrder) return -1;
    const int64_t ld_min = n > 1 ? n : 1;
    if (A == nullptr && n > 0) return -2;
    if (lda < ld_min) return -3;
    if (L == nullptr && n > 0) return -4;
    if (ldl < ld_min) return -5;
    if (t == nullptr && n >= 2) return -6;
    if (piv == nullptr && n >= 1) return -7;
    if (nb < 0 || nb > kMaxNb) return -9;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n == 0) {
        if (info) SKEW_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t), st));
        return SKEW_OK;
    }
    return factor(n, A, lda, L, ldl, t, piv, info, nullptr, nullptr, nb, workspace,
                  workspace_bytes, st, true, SKEW_PRECISION_FP64);
}

int skew_pfaffian(int64_t n, double *A, int64_t lda, double *logabs, int32_t *sign,
                  double *t, int32_t *piv, int32_t *info, int nb, void *workspace,
                  size_t workspace_bytes, void *stream) {
    if (n < 0 || n > kMaxOrder) return -1;
    const int64_t ld_min = n > 1 ? n : 1;
    if (A == nullptr && n > 0) return -2;
    if (lda < ld_min) return -3;
    if (logabs == nullptr) return -4;
    if (sign == nullptr) return -5;
    if (nb < 0 || nb > kMaxNb) return -9;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n == 0) {
        // Pf of the empty matrix is 1
        DeviceInfo di;
        SKEW_TRY_STATUS(current_device_info(&di));
        SKEW_TRY_STATUS(launch_finish(0, nullptr, nullptr, nullptr, logabs, sign, info, st));
        return SKEW_OK;
    }
    return factor(n, A, lda, nullptr, 0, t, piv, info, logabs, sign, nb, workspace,
                  workspace_bytes, st, false, SKEW_PRECISION_FP64);
}

size_t skew_workspace_bytes_ex(int64_t n, int nb, int with_L, int precision) {
    if (n < 0 || (precision != SKEW_PRECISION_FP64 && precision != SKEW_PRECISION_SPLIT_BF16))
        return 0;
    if (nb <= 0) nb = skew_default_nb(n);
    if (nb > kMaxNb) nb = kMaxNb;
    return workspace_layout(n, nb, with_L != 0, precision).total;
}

int skew_ltlt_ex(int64_t n, double *A, int64_t lda, double *L, int64_t ldl, double *t,
                 int32_t *piv, int32_t *info, int nb, int precision, void *workspace,
                 size_t workspace_bytes, void *stream) {
    if (precision != SKEW_PRECISION_FP64 && precision != SKEW_PRECISION_SPLIT_BF16) return -10;
    if (precision == SKEW_PRECISION_FP64)
        return skew_ltlt(n, A, lda, L, ldl, t, piv, info, nb, workspace, workspace_bytes, stream);
    if (n < 0 || n > kMaxOrder) return -1;
    const int64_t ld_min = n > 1 ? n : 1;
    if (A == nullptr && n > 0) return -2;
    if (lda < ld_min) return -3;
    if (L == nullptr && n > 0) return -4;
    if (ldl < ld_min) return -5;
    if (t == nullptr && n >= 2) return -6;
    if (piv == nullptr && n >= 1) return -7;
    if (nb < 0 || nb > 64) return -9;                  // split update: at most 32 pairs
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n == 0) {
        if (info) SKEW_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t), st));
        return SKEW_OK;
    }
    if (nb == 0 && skew_default_nb(n) > 64) nb = 64;
    if (workspace != nullptr &&
        workspace_bytes < workspace_layout(n, nb == 0 ? skew_default_nb(n) : nb, true, precision).total)
        return -12;
    return factor(n, A, lda, L, ldl, t, piv, info, nullptr, nullptr, nb, workspace,
                  workspace_bytes, st, true, precision);
}

int skew_pfaffian_ex(int64_t n, double *A, int64_t lda, double *logabs, int32_t *sign,
                     double *t, int32_t *piv, int32_t *info, int nb, int precision,
                     void *workspace, size_t workspace_bytes, void *stream) {
    if (precision != SKEW_PRECISION_FP64 && precision != SKEW_PRECISION_SPLIT_BF16) return -10;
    if (precision == SKEW_PRECISION_FP64)
        return skew_pfaffian(n, A, lda, logabs, sign, t, piv, info, nb, workspace,
                             workspace_bytes, stream);
    if (n < 0 || n > kMaxOrder) return -1;
    const int64_t ld_min = n > 1 ? n : 1;
    if (A == nullptr && n > 0) return -2;
    if (lda < ld_min) return -3;
    if (logabs == nullptr) return -4;
    if (sign == nullptr) return -5;
    if (nb < 0 || nb > 64) return -9;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n == 0) return skew_pfaffian(n, A, lda, logabs, sign, t, piv, info, nb, nullptr, 0, stream);
    if (nb == 0 && skew_default_nb(n) > 64) nb = 64;
    if (workspace != nullptr &&
        workspace_bytes < workspace_layout(n, nb == 0 ? skew_default_nb(n) : nb, false, precision).total)
        return -12;
    return factor(n, A, lda, nullptr, 0, t, piv, info, logabs, sign, nb, workspace,
                  workspace_bytes, st, false, precision);
}

int skew_rank2k_ex(int64_t m, int64_t k, double alpha, const double *X, int64_t ldx,
                   const double *Y, int64_t ldy, double beta, double *C, int64_t ldc,
                   int precision, void *stream) {
    if (precision != SKEW_PRECISION_FP64 && precision != SKEW_PRECISION_SPLIT_BF16) return -11;
    if (precision == SKEW_PRECISION_FP64)
        return skew_rank2k(m, k, alpha, X, ldx, Y, ldy, beta, C, ldc, stream);
    if (m < 0 || m > kMaxOrder) return -1;
    if (k < 0 || k > 32) return -2;                    // split update: at most 32 pairs
    const int64_t ld_min = m > 1 ? m : 1;
    const bool need_ops = m > 1 && k > 0;
    if (X == nullptr && need_ops) return -4;
    if (ldx < ld_min) return -5;
    if (Y == nullptr && need_ops) return -6;
    if (ldy < ld_min) return -7;
    if (C == nullptr && m > 1) return -9;
    if (ldc < ld_min) return -10;
    if (m <= 1) return SKEW_OK;
    DeviceInfo di;
    SKEW_TRY_STATUS(current_device_info(&di));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void *scratch = nullptr;
    SKEW_TRY_STATUS(pool_alloc(&scratch, split_scratch_bytes(m), st));
    Skr2kArgs sa;
    sa.m = m;
    sa.C = C;
    sa.ldc = ldc;
    sa.alpha = alpha;
    sa.beta = beta;
    sa.P = X;
    sa.ldp = ldx;
    sa.Q = Y;
    sa.ldq = ldy;
    sa.tt = nullptr;
    sa.x = nullptr;
    sa.b = k;
    int status;
    {
        ProfScope ps(kProfSkr2k, st, skr2k_flops(m, k), skr2k_bytes(m));
        status = launch_skr2k_split(PairKind::Rank2k, sa, scratch, nullptr, di.sms, st);
    }
    cudaError_t e = cudaFreeAsync(scratch, st);
    if (e != cudaSuccess && status == SKEW_OK) {
        set_last_error(e);
        status = SKEW_ERR_CUDA;
    }
    return status;
}

int skew_pfaffian_from_factors(int64_t n, const double *t, const int32_t *piv,
                               double *logabs, int32_t *sign, void *stream) {
    if (n < 0 || n > kMaxOrder) return -1;
    if (t == nullptr && n >= 2) return -2;
    if (piv == nullptr && n >= 1) return -3;
    if (logabs == nullptr) return -4;
    if (sign == nullptr) return -5;
    DeviceInfo di;
    SKEW_TRY_STATUS(current_device_info(&di));
    return launch_finish(n, t, piv, nullptr, logabs, sign, nullptr,
                         static_cast<cudaStream_t>(stream));
}

int skew_rank2k(int64_t m, int64_t k, double alpha, const double *X, int64_t ldx,
                const double *Y, int64_t ldy, double beta, double *C, int64_t ldc,
                void *stream) {
    if (m < 0 || m > kMaxOrder) return -1;
    if (k < 0) return -2;
    const int64_t ld_min = m > 1 ? m : 1;
    const bool need_ops = m > 1 && k > 0;
    if (X == nullptr && need_ops) return -4;
    if (ldx < ld_min) return -5;
    if (Y == nullptr && need_ops) return -6;
    if (ldy < ld_min) return -7;
    if (C == nullptr && m > 1) return -9;
    if (ldc < ld_min) return -10;
    if (m <= 1) return SKEW_OK;
    DeviceInfo di;
    SKEW_TRY_STATUS(current_device_info(&di));
    Skr2kArgs sa;
    sa.m = m;
    sa.C = C;
    sa.ldc = ldc;
    sa.alpha = alpha;
    sa.beta = beta;
    sa.P = X;
    sa.ldp = ldx;
    sa.Q = Y;
    sa.ldq = ldy;
    sa.tt = nullptr;
    sa.x = nullptr;
    sa.b = k;
    ProfScope ps(kProfSkr2k, static_cast<cudaStream_t>(stream), skr2k_flops(m, k), skr2k_bytes(m));
    return launch_skr2k(PairKind::Rank2k, sa, static_cast<cudaStream_t>(stream));
}

int skew_tridiag_rankk(int64_t m, int64_t b, double alpha, const double *A,
                       int64_t lda, const double *t, double beta, double *C,
                       int64_t ldc, void *stream) {
    if (m < 0 || m > kMaxOrder) return -1;
    if (b < 0) return -2;
    const int64_t ld_min = m > 1 ? m : 1;
    const bool need_ops = m > 1 && b > 1;
    if (A == nullptr && need_ops) return -4;
    if (lda < ld_min) return -5;
    if (t == nullptr && need_ops) return -6;
    if (C == nullptr && m > 1) return -8;
    if (ldc < ld_min) return -9;
    if (m <= 1) return SKEW_OK;
    DeviceInfo di;
    SKEW_TRY_STATUS(current_device_info(&di));
    Skr2kArgs sa;
    sa.m = m;
    sa.C = C;
    sa.ldc = ldc;
    sa.alpha = -alpha;            // A T A^T = -sum_j (a_j w_j^T - w_j a_j^T)
    sa.beta = beta;
    sa.P = A;
    sa.ldp = lda;
    sa.Q = nullptr;
    sa.ldq = 0;
    sa.tt = t;
    sa.x = nullptr;
    sa.b = b;
    ProfScope ps(kProfSkr2k, static_cast<cudaStream_t>(stream), skr2k_flops(m, b / 2), skr2k_bytes(m));
    return launch_skr2k(PairKind::Tridiag, sa, static_cast<cudaStream_t>(stream));
}

size_t skew_batched_workspace_bytes(int count, int max_n) {
    if (count < 0 || max_n < 0 || max_n > SKEW_BATCH_MAX_N) return 0;
    return batched_workspace_bytes(count, max_n);
}

int skew_ltlt_batched(int count, const skew_problem *problems, double *logabs,
                      int32_t *sign, int32_t *info, int max_n, void *workspace,
                      size_t workspace_bytes, void *stream) {
    if (count < 0) return -1;
    if (problems == nullptr && count > 0) return -2;
    if (max_n < 0 || max_n > SKEW_BATCH_MAX_N) return -6;
    const size_t need = batched_workspace_bytes(count, max_n);
    if (workspace != nullptr && workspace_bytes < need) return -8;
    if (count == 0) return SKEW_OK;
    DeviceInfo di;
    SKEW_TRY_STATUS(current_device_info(&di));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void *ws = workspace;
    bool own = false;
    if (ws == nullptr) {
        SKEW_TRY_STATUS(pool_alloc(&ws, need, st));
        own = true;
    }
    int status;
    {
        ProfScope ps(kProfBatched, st, 0.0, 0.0);
        status = launch_batched(count, problems, logabs, sign, info, max_n, ws, st, di.sms);
    }
    if (own) {
        cudaError_t e = cudaFreeAsync(ws, st);
        if (e != cudaSuccess && status == SKEW_OK) {
            set_last_error(e);
            status = SKEW_ERR_CUDA;
        }
    }
    return status;
}

size_t skew_workspace_bytes_twostep(int64_t n, int nb, int precision) {
    if (n < 0) return 0;
    if (nb <= 0) nb = 64;
    if (nb > kMaxNb) nb = kMaxNb;
    return workspace_layout(n, nb, false, precision).total;
}

int skew_pfaffian_twostep(int64_t n, double *A, int64_t lda, double *logabs, int32_t *sign,
                          double *a, int32_t *piv, int32_t *info, int nb, int precision,
                          void *workspace, size_t workspace_bytes, void *stream) {
    if (n < 0 || n > kMaxOrder) return -1;
    const int64_t ld_min = n > 1 ? n : 1;
    if (A == nullptr && n > 0) return -2;
    if (lda < ld_min) return -3;
    if (nb == 0) nb = 64;
    if (nb < 2 || nb > 96 || (nb & 1)) return -9;
    if (precision != SKEW_PRECISION_FP64 && precision != SKEW_PRECISION_SPLIT_BF16) return -10;
    if (precision == SKEW_PRECISION_SPLIT_BF16 && nb > 64) return -9;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return factor_twostep(n, A, lda, a, piv, info, logabs, sign, nb, workspace, workspace_bytes,
                          st, precision);
}

int skew_pfaffian_batched(int count, const skew_problem *problems, double *logabs,
                          int32_t *sign, int32_t *info, int max_n, void *workspace,
                          size_t workspace_bytes, void *stream) {
    if (count < 0) return -1;
    if (problems == nullptr && count > 0) return -2;
    if (max_n < 0 || max_n > 512) return -6;
    const size_t need = batched_workspace_bytes(count, max_n);
    if (workspace != nullptr && workspace_bytes < need) return -8;
    if (count == 0) return SKEW_OK;
    DeviceInfo di;
    SKEW_TRY_STATUS(current_device_info(&di));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void *ws = workspace;
    bool own = false;
    if (ws == nullptr) {
        SKEW_TRY_STATUS(pool_alloc(&ws, need, st));
        own = true;
    }
    int status;
    {
        ProfScope ps(kProfBatched, st, 0.0, 0.0);
        status = launch_batched_twostep(count, problems, logabs, sign, info, max_n, ws, st, di.sms);
    }
    if (own) {
        cudaError_t e = cudaFreeAsync(ws, st);
        if (e != cudaSuccess && status == SKEW_OK) {
            set_last_error(e);
            status = SKEW_ERR_CUDA;
        }
    }
    return status;
}

// Columns per host-link copy of A's lower triangle (skew_ltlt_host).
constexpr int64_t kHostCopyCols = 256;

int skew_ltlt_host(int64_t n, const double *A_host, int64_t lda, double *L_host,
                   int64_t ldl, double *t_host, int32_t *piv_host, double *logabs,
                   int32_t *sign, int32_t *info, int nb) {
    if (n < 0 || n > kMaxOrder) return -1;
    const int64_t ld_min = n > 1 ? n : 1;
    if (A_host == nullptr && n > 0) return -2;
    if (lda < ld_min) return -3;
    if (L_host != nullptr && ldl < ld_min) return -5;
    if (nb < 0 || nb > kMaxNb) return -11;
    DeviceInfo di;
    SKEW_TRY_STATUS(current_device_info(&di));
    int dev;
    SKEW_TRY(cudaGetDevice(&dev));
    HostCall &h = g_host[dev];
    std::lock_guard<std::mutex> lock(h.mu);
    SKEW_TRY_STATUS(host_ready(h));
    cudaStream_t st = h.st;
    const size_t nn = (size_t)(n > 0 ? n : 1);
    const size_t mat = align256(nn * nn * sizeof(double));
    const size_t vec = align256(nn * sizeof(double));
    const size_t need = mat + (L_host ? mat : 0) + 2 * vec + 3 * 256;
    if (need > h.buf_bytes) {
        SKEW_TRY_STATUS(host_release_buffers(h));
        SKEW_TRY_STATUS(pool_alloc(&h.buf, need, st));
        h.buf_bytes = need;
    }
    char *b = static_cast<char *>(h.buf);
    double *dA = reinterpret_cast<double *>(b);
    b += mat;
    double *dL = nullptr;
    if (L_host) {
        dL = reinterpret_cast<double *>(b);
        b += mat;
    }
    double *dt = reinterpret_cast<double *>(b);
    b += vec;
    int32_t *dpiv = reinterpret_cast<int32_t *>(b);
    b += vec;
    double *dlog = reinterpret_cast<double *>(b);
    int32_t *dsign = reinterpret_cast<int32_t *>(b + 256);
    int32_t *dinfo = reinterpret_cast<int32_t *>(b + 512);
    int status = SKEW_OK;
    double h_log = 0.0;
    int32_t h_sign = 0, h_info = 0;
    h.have_ms = false;
    do {
        // Only the lower triangle of A is read, so only it crosses the host link: in
        // blocks of kHostCopyCols columns, rows from the block's first column down (half
        // the bytes of the whole matrix; the device's upper triangle is never read).
        cudaError_t e = cudaEventRecord(h.ev[0], st);
        for (int64_t c0 = 0; e == cudaSuccess && c0 < n; c0 += kHostCopyCols) {
            const int64_t w = (n - c0 < kHostCopyCols) ? n - c0 : kHostCopyCols;
            e = cudaMemcpy2DAsync(dA + c0 + c0 * n, n * sizeof(double), A_host + c0 + c0 * lda,
                                  lda * sizeof(double), (size_t)(n - c0) * sizeof(double),
                                  (size_t)w, cudaMemcpyHostToDevice, st);
        }
        if (e == cudaSuccess) e = cudaEventRecord(h.ev[1], st);
        if (e != cudaSuccess) { set_last_error(e); status = SKEW_ERR_CUDA; break; }
        // a page-locked L receives its final rows while the factorization runs (plain
        // path); otherwise, and on the look-ahead path, L is copied after it
        HostRows hr;
        if (L_host && n > 0) {
            cudaPointerAttributes pa;
            if (cudaPointerGetAttributes(&pa, L_host) == cudaSuccess &&
                pa.type == cudaMemoryTypeHost) {
                hr.L_host = L_host;
                hr.ldl_host = ldl;
                hr.copy = h.copy;
                hr.ev = h.ev_rows;
            } else {
                cudaGetLastError();
            }
        }
        if (L_host && hr.L_host) {
            status = factor(n, dA, ld_min, dL, ld_min, dt, dpiv, dinfo, nullptr, nullptr,
                            nb == 0 ? skew_default_nb(n) : nb, nullptr, 0, st, true,
                            SKEW_PRECISION_FP64, &hr);
            if (status == SKEW_OK) status = skew_pfaffian_from_factors(n, dt, dpiv, dlog, dsign, st);
        } else if (L_host) {
            status = skew_ltlt(n, dA, ld_min, dL, ld_min, dt, dpiv, dinfo, nb, nullptr, 0, st);
            if (status == SKEW_OK) status = skew_pfaffian_from_factors(n, dt, dpiv, dlog, dsign, st);
        } else {
            status = skew_pfaffian(n, dA, ld_min, dlog, dsign, dt, dpiv, dinfo, nb, nullptr, 0, st);
        }
        if (status != SKEW_OK) break;
        e = cudaEventRecord(h.ev[2], st);
        if (e == cudaSuccess && hr.used) {      // the last rows' copies, then the rest
            e = cudaEventRecord(h.ev_join, h.copy);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h.ev_join, 0);
        }
        if (e == cudaSuccess && L_host && n > 0 && !hr.used)
            e = (ldl == n) ? cudaMemcpyAsync(L_host, dL, (size_t)n * n * sizeof(double),
                                             cudaMemcpyDeviceToHost, st)
                           : cudaMemcpy2DAsync(L_host, ldl * sizeof(double), dL,
                                               n * sizeof(double), n * sizeof(double), n,
                                               cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && t_host && n > 1)
            e = cudaMemcpyAsync(t_host, dt, (n - 1) * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && piv_host && n > 0)
            e = cudaMemcpyAsync(piv_host, dpiv, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&h_log, dlog, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&h_sign, dsign, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&h_info, dinfo, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaEventRecord(h.ev[3], st);
        if (e != cudaSuccess) { set_last_error(e); status = SKEW_ERR_CUDA; break; }
    } while (0);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess && status == SKEW_OK) {
        set_last_error(e);
        status = SKEW_ERR_CUDA;
    }
    // on every exit no copy into the caller's L is left in flight
    cudaError_t ec = cudaStreamSynchronize(h.copy);
    if (ec != cudaSuccess && status == SKEW_OK) {
        set_last_error(ec);
        status = SKEW_ERR_CUDA;
    }
    if (status == SKEW_OK) {
        bool ok = true;
        for (int i = 0; i < 3 && ok; ++i)
            ok = cudaEventElapsedTime(&h.ms[i], h.ev[i], h.ev[i + 1]) == cudaSuccess;
        if (!ok) cudaGetLastError();
        h.have_ms = ok;
        if (n == 0) {   // empty factorization: Pf = 1
            h_info = 0;
        }
        if (logabs) *logabs = h_log;
        if (sign) *sign = h_sign;
        if (info) *info = h_info;
    }
    return status;
}

int skew_ltlt_host_timing(float *h2d_ms, float *device_ms, float *d2h_ms) {
    int dev;
    SKEW_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return SKEW_ERR_NODEVICE;
    HostCall &h = g_host[dev];
    std::lock_guard<std::mutex> lock(h.mu);
    if (!h.have_ms) return -1;             // no completed call on this device
    if (h2d_ms) *h2d_ms = h.ms[0];
    if (device_ms) *device_ms = h.ms[1];
    if (d2h_ms) *d2h_ms = h.ms[2];
    return SKEW_OK;
}

}  // extern "C"
