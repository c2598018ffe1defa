// server.cu -- a continuous-batching Pfaffian/factorization server (host runtime).
//
// Requests (a device matrix each) are queued by skew_server_submit.  A worker thread
//   - admits queued requests in arrival order while their device memory fits in the
//     budget: the resident buffers (the matrix copy, t, piv, optionally L), held until
//     the request is released, and the workspace its launch allocates (its own call's,
//     or its share of a batched launch), held until its work has finished; admission
//     happens as soon as memory frees up, also while other work is running;
//   - launches admitted work on the first free stream: all admitted small requests of
//     one kind together in one batched launch (skew_ltlt_batched for requests that keep
//     their factors, skew_pfaffian_batched for Pfaffian-only ones), or one large
//     request as a skew_ltlt / skew_pfaffian / skew_pfaffian_twostep call -- so work
//     submitted while other work is on the GPU is batched and overlaps it on other
//     streams;
//   - detects completions through events and wakes waiters.
// Factors stay resident in device memory until skew_server_release.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct HostResult {   // page-locked, written by the device through async copies
    double logabs;
    int32_t sign;
    int32_t info;
};

enum class ReqState { Queued, Admitted, Running, Done, Failed };

struct Request {
    uint64_t ticket = 0;
    int64_t n = 0;
    int mode = SKEW_SERVE_FACTORS;  // SKEW_SERVE_*
    const double *src = nullptr;   // caller's matrix (read before completion)
    int64_t src_ld = 0;
    double *A = nullptr, *L = nullptr, *t = nullptr;
    int32_t *piv = nullptr;
    double *d_logabs = nullptr;
    int32_t *d_sign = nullptr, *d_info = nullptr;
    HostResult *host = nullptr;
    size_t bytes = 0;              // resident buffers (matrix, factors, result words)
    size_t ws_bytes = 0;           // transient workspace of its launch, held until done
    bool ws_held = false;          // ws_bytes counted in `used`
    int lane = -1;                 // stream its work was enqueued on
    ReqState state = ReqState::Queued;
    int status = SKEW_OK;
    Clock::time_point t_submit, t_admit, t_launch, t_done;
};

struct Lane {                      // one stream and what runs on it
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<uint64_t> tickets;
    skew_problem *h_table = nullptr;   // page-locked descriptor staging
    skew_problem *d_table = nullptr;
    int table_cap = 0;
};

}  // namespace

struct skew_server {
    int device = 0;
    size_t budget = 0, used = 0;
    int small_n_max = 512;
    std::vector<Lane> lanes;
    std::mutex mu;
    std::condition_variable cv_done, cv_work;
    std::deque<uint64_t> queue;      // queued, not admitted
    std::deque<uint64_t> admitted;   // admitted, not launched
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    std::vector<HostResult *> host_free;   // page-locked result slots
    std::vector<HostResult *> host_chunks;
    int worker_status = SKEW_OK;
};

namespace {

// Largest order a request of this kind may have to join a batched launch (the
// Pfaffian-only batched kernel takes orders up to 512).
int64_t batch_limit(const skew_server *s, const Request &r) {
    const int64_t lim = s->small_n_max;
    return (r.mode == SKEW_SERVE_PFAFFIAN && lim > 512) ? 512 : lim;
}

size_t request_bytes(int64_t n, bool want_L) {
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t nn = (size_t)(n > 0 ? n : 1);
    size_t b = al(nn * nn * sizeof(double)) + al(nn * sizeof(double)) + al(nn * sizeof(int32_t)) +
               al(sizeof(double)) + 2 * al(sizeof(int32_t));
    if (want_L) b += al(nn * nn * sizeof(double));
    return b;
}

// Device memory a request's launch allocates for the duration of its work: the
// workspace of its own call, or its share of a batched launch (a descriptor, the
// batch's result words and the batched kernel's counters).
size_t request_ws_bytes(const skew_server *s, const Request &r) {
    // (the look-ahead figures cover both paths of skew_ltlt / skew_pfaffian)
    if (r.n <= batch_limit(s, r)) return 1024 + skew::batched_workspace_bytes(1, (int)r.n);
    if (r.mode == SKEW_SERVE_FACTORS_L) return skew_workspace_bytes_lookahead(r.n, 0, 1);
    if (r.mode == SKEW_SERVE_PFAFFIAN) {
        const size_t a = skew_workspace_bytes_twostep(r.n, 0, SKEW_PRECISION_FP64);
        const size_t b = skew_workspace_bytes_lookahead(r.n, 0, 0);   // fallback of large orders
        return a > b ? a : b;
    }
    return skew_workspace_bytes_lookahead(r.n, 0, 0);
}

// The launch of the request has ended (completed or failed): its workspace is back.
void drop_ws(skew_server *s, Request &r) {
    if (!r.ws_held) return;
    s->used -= r.ws_bytes;
    r.ws_held = false;
}

HostResult *take_host_slot(skew_server *s) {
    if (s->host_free.empty()) {
        HostResult *chunk = nullptr;
        if (cudaHostAlloc(&chunk, 256 * sizeof(HostResult), cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        s->host_chunks.push_back(chunk);
        for (int i = 0; i < 256; ++i) s->host_free.push_back(chunk + i);
    }
    HostResult *h = s->host_free.back();
    s->host_free.pop_back();
    return h;
}

// Allocate a request's device buffers on `st` and copy its matrix in.
int materialise(Request &r, cudaStream_t st) {
    const size_t nn = (size_t)(r.n > 0 ? r.n : 1);
    void *p;
    auto alloc = [&](size_t bytes) -> int { return skew::pool_alloc(&p, bytes, st); };
    SKEW_TRY_STATUS(alloc(nn * nn * sizeof(double)));
    r.A = static_cast<double *>(p);
    SKEW_TRY_STATUS(alloc(nn * sizeof(double)));
    r.t = static_cast<double *>(p);
    SKEW_TRY_STATUS(alloc(nn * sizeof(int32_t)));
    r.piv = static_cast<int32_t *>(p);
    SKEW_TRY_STATUS(alloc(sizeof(double)));
    r.d_logabs = static_cast<double *>(p);
    SKEW_TRY_STATUS(alloc(sizeof(int32_t)));
    r.d_sign = static_cast<int32_t *>(p);
    SKEW_TRY_STATUS(alloc(sizeof(int32_t)));
    r.d_info = static_cast<int32_t *>(p);
    if (r.mode == SKEW_SERVE_FACTORS_L) {
        SKEW_TRY_STATUS(alloc(nn * nn * sizeof(double)));
        r.L = static_cast<double *>(p);
    }
    if (r.n > 0)
        SKEW_TRY(cudaMemcpy2DAsync(r.A, r.n * sizeof(double), r.src, r.src_ld * sizeof(double),
                                   r.n * sizeof(double), r.n, cudaMemcpyDeviceToDevice, st));
    return SKEW_OK;
}

void free_request(Request &r, cudaStream_t st) {
    void *bufs[] = {r.A, r.L, r.t, r.piv, r.d_logabs, r.d_sign, r.d_info};
    for (void *b : bufs)
        if (b) cudaFreeAsync(b, st);
    r.A = r.L = r.t = nullptr;
    r.piv = nullptr;
    r.d_logabs = nullptr;
    r.d_sign = r.d_info = nullptr;
}

int copy_results_back(Request &r, cudaStream_t st) {
    SKEW_TRY(cudaMemcpyAsync(&r.host->logabs, r.d_logabs, sizeof(double), cudaMemcpyDeviceToHost, st));
    SKEW_TRY(cudaMemcpyAsync(&r.host->sign, r.d_sign, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SKEW_TRY(cudaMemcpyAsync(&r.host->info, r.d_info, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    return SKEW_OK;
}

// Launch the next unit of admitted work on lane `ln` (lock held).  Returns false when
// nothing was launched.
bool launch_next(skew_server *s, int lane_index) {
    Lane &ln = s->lanes[lane_index];
    if (s->admitted.empty()) return false;
    Request &first = s->reqs[s->admitted.front()];
    ln.tickets.clear();
    int status = SKEW_OK;
    const bool pf_only = first.mode == SKEW_SERVE_PFAFFIAN;
    if (first.n <= batch_limit(s, first)) {
        // every admitted small request of the first one's kind goes into one batched
        // launch
        std::deque<uint64_t> rest;
        int max_n = 0;
        for (uint64_t tk : s->admitted) {
            Request &r = s->reqs[tk];
            if (r.n <= batch_limit(s, r) && (r.mode == SKEW_SERVE_PFAFFIAN) == pf_only) {
                ln.tickets.push_back(tk);
                if (r.n > max_n) max_n = (int)r.n;
            } else {
                rest.push_back(tk);
            }
        }
        s->admitted.swap(rest);
        const int count = (int)ln.tickets.size();
        if (count > ln.table_cap) {
            if (ln.h_table) cudaFreeHost(ln.h_table);
            if (ln.d_table) cudaFree(ln.d_table);
            int cap = count < 64 ? 64 : count * 2;
            if (cudaHostAlloc(&ln.h_table, cap * sizeof(skew_problem), cudaHostAllocDefault) != cudaSuccess ||
                cudaMalloc(&ln.d_table, cap * sizeof(skew_problem)) != cudaSuccess) {
                cudaGetLastError();
                status = SKEW_ERR_NOMEM;
            } else {
                ln.table_cap = cap;
            }
        }
        for (int i = 0; i < count && status == SKEW_OK; ++i) {
            Request &r = s->reqs[ln.tickets[i]];
            status = materialise(r, ln.stream);
            skew_problem &pr = ln.h_table[i];
            pr.n = r.n;
            pr.A = r.A;
            pr.lda = r.n > 1 ? r.n : 1;
            pr.L = r.L;
            pr.ldl = r.n > 1 ? r.n : 1;
            pr.t = r.t;
            pr.piv = r.piv;
        }
        // results of a batch land in per-request device words, gathered afterwards
        if (status == SKEW_OK) {
            cudaError_t e = cudaMemcpyAsync(ln.d_table, ln.h_table, count * sizeof(skew_problem),
                                            cudaMemcpyHostToDevice, ln.stream);
            if (e != cudaSuccess) { skew::set_last_error(e); status = SKEW_ERR_CUDA; }
        }
        if (status == SKEW_OK) {
            // the batch's logabs/sign/info arrays, then scattered to each request
            double *la = nullptr;
            int32_t *sg = nullptr, *inf = nullptr;
            cudaError_t e = cudaSuccess;
            status = skew::pool_alloc((void **)&la, count * sizeof(double), ln.stream);
            if (status == SKEW_OK) status = skew::pool_alloc((void **)&sg, count * sizeof(int32_t), ln.stream);
            if (status == SKEW_OK) status = skew::pool_alloc((void **)&inf, count * sizeof(int32_t), ln.stream);
            if (status == SKEW_OK)
                status = pf_only
                             ? skew_pfaffian_batched(count, ln.d_table, la, sg, inf, max_n, nullptr, 0,
                                                     ln.stream)
                             : skew_ltlt_batched(count, ln.d_table, la, sg, inf, max_n, nullptr, 0,
                                                 ln.stream);
            for (int i = 0; i < count && status == SKEW_OK; ++i) {
                Request &r = s->reqs[ln.tickets[i]];
                e = cudaMemcpyAsync(&r.host->logabs, la + i, sizeof(double), cudaMemcpyDeviceToHost, ln.stream);
                if (e == cudaSuccess) e = cudaMemcpyAsync(&r.host->sign, sg + i, sizeof(int32_t), cudaMemcpyDeviceToHost, ln.stream);
                if (e == cudaSuccess) e = cudaMemcpyAsync(&r.host->info, inf + i, sizeof(int32_t), cudaMemcpyDeviceToHost, ln.stream);
                if (e == cudaSuccess) e = cudaMemcpyAsync(r.d_logabs, la + i, sizeof(double), cudaMemcpyDeviceToDevice, ln.stream);
                if (e == cudaSuccess) e = cudaMemcpyAsync(r.d_sign, sg + i, sizeof(int32_t), cudaMemcpyDeviceToDevice, ln.stream);
                if (e == cudaSuccess) e = cudaMemcpyAsync(r.d_info, inf + i, sizeof(int32_t), cudaMemcpyDeviceToDevice, ln.stream);
                if (e != cudaSuccess) { skew::set_last_error(e); status = SKEW_ERR_CUDA; }
            }
            if (la) cudaFreeAsync(la, ln.stream);
            if (sg) cudaFreeAsync(sg, ln.stream);
            if (inf) cudaFreeAsync(inf, ln.stream);
        }
    } else {
        ln.tickets.push_back(s->admitted.front());
        s->admitted.pop_front();
        Request &r = s->reqs[ln.tickets[0]];
        status = materialise(r, ln.stream);
        const int64_t ld = r.n > 1 ? r.n : 1;
        if (status == SKEW_OK) {
            if (r.mode == SKEW_SERVE_FACTORS_L) {
                status = skew_ltlt(r.n, r.A, ld, r.L, ld, r.t, r.piv, r.d_info, 0, nullptr, 0, ln.stream);
                if (status == SKEW_OK)
                    status = skew_pfaffian_from_factors(r.n, r.t, r.piv, r.d_logabs, r.d_sign, ln.stream);
            } else if (r.mode == SKEW_SERVE_PFAFFIAN) {
                // the two-step elimination; an order too large for its panel (-1) takes
                // the factorization's Pfaffian instead
                status = skew_pfaffian_twostep(r.n, r.A, ld, r.d_logabs, r.d_sign, r.t, r.piv,
                                               r.d_info, 0, SKEW_PRECISION_FP64, nullptr, 0,
                                               ln.stream);
                if (status == -1)
                    status = skew_pfaffian(r.n, r.A, ld, r.d_logabs, r.d_sign, r.t, r.piv, r.d_info,
                                           0, nullptr, 0, ln.stream);
            } else {
                status = skew_pfaffian(r.n, r.A, ld, r.d_logabs, r.d_sign, r.t, r.piv, r.d_info, 0,
                                       nullptr, 0, ln.stream);
            }
        }
        if (status == SKEW_OK) status = copy_results_back(r, ln.stream);
    }
    // The tickets stay Running, also when the launch failed part way, until the lane's
    // event shows that everything enqueued so far (copies from the caller's matrix,
    // kernels, copies into the result slots) has finished; the completion pass then
    // marks them Done, or Failed with the status kept here.
    const auto launched = Clock::now();
    for (uint64_t tk : ln.tickets) {
        Request &r = s->reqs[tk];
        r.state = ReqState::Running;
        r.status = status;
        r.lane = lane_index;
        r.t_launch = launched;
    }
    cudaError_t e = cudaEventRecord(ln.done, ln.stream);
    if (e != cudaSuccess) {
        // no event: wait for the lane's stream here instead
        skew::set_last_error(e);
        cudaGetLastError();
        cudaStreamSynchronize(ln.stream);
        cudaGetLastError();
        const auto now = Clock::now();
        for (uint64_t tk : ln.tickets) {
            Request &r = s->reqs[tk];
            r.state = ReqState::Failed;
            if (r.status == SKEW_OK) r.status = SKEW_ERR_CUDA;
            r.t_done = now;
            drop_ws(s, r);
        }
        ln.tickets.clear();
        s->cv_done.notify_all();
        return true;
    }
    ln.busy = true;
    return true;
}

void worker_main(skew_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        bool progressed = false;
        // 1. completions
        for (Lane &ln : s->lanes) {
            if (!ln.busy) continue;
            cudaError_t q = cudaEventQuery(ln.done);
            if (q == cudaErrorNotReady) continue;
            const auto now = Clock::now();
            for (uint64_t tk : ln.tickets) {
                Request &r = s->reqs[tk];
                r.t_done = now;
                if (q == cudaSuccess && r.status == SKEW_OK) {
                    r.state = ReqState::Done;
                } else {
                    if (q != cudaSuccess) {
                        skew::set_last_error(q);
                        r.status = SKEW_ERR_CUDA;
                    }
                    r.state = ReqState::Failed;
                }
                drop_ws(s, r);
            }
            if (q != cudaSuccess) cudaGetLastError();
            ln.tickets.clear();
            ln.busy = false;
            progressed = true;
            s->cv_done.notify_all();
        }
        // 2. admission, in arrival order, while memory fits the budget
        while (!s->queue.empty()) {
            Request &r = s->reqs[s->queue.front()];
            if (s->used + r.bytes + r.ws_bytes > s->budget) break;
            s->used += r.bytes + r.ws_bytes;
            r.ws_held = true;
            r.t_admit = Clock::now();
            r.state = ReqState::Admitted;
            s->admitted.push_back(r.ticket);
            s->queue.pop_front();
            progressed = true;
        }
        // 3. launches on free lanes
        for (int li = 0; li < (int)s->lanes.size(); ++li)
            if (!s->lanes[li].busy && !s->admitted.empty()) progressed |= launch_next(s, li);
        bool any_busy = false;
        for (Lane &ln : s->lanes) any_busy |= ln.busy;
        if (s->stop && !any_busy && s->admitted.empty()) break;
        if (!progressed) {
            // in-flight work: poll events again soon; idle: sleep until submitted
            if (any_busy)
                s->cv_work.wait_for(lock, std::chrono::microseconds(20));
            else
                s->cv_work.wait_for(lock, std::chrono::milliseconds(50));
        }
    }
}

}  // namespace

using namespace skew;

extern "C" {

int skew_server_create(size_t device_budget_bytes, int n_streams, int small_n_max,
                       skew_server **out) {
    if (device_budget_bytes == 0) return -1;
    if (n_streams < 1 || n_streams > 64) return -2;
    if (small_n_max < 0 || small_n_max > SKEW_BATCH_MAX_N) return -3;
    if (out == nullptr) return -4;
    DeviceInfo di;
    SKEW_TRY_STATUS(current_device_info(&di));
    skew_server *s = new skew_server();
    s->device = di.device;
    s->budget = device_budget_bytes;
    s->small_n_max = small_n_max;
    s->lanes.resize(n_streams);
    for (Lane &ln : s->lanes) {
        if (cudaStreamCreateWithFlags(&ln.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ln.done, cudaEventDisableTiming) != cudaSuccess) {
            cudaError_t e = cudaGetLastError();
            set_last_error(e);
            for (Lane &l2 : s->lanes) {
                if (l2.stream) cudaStreamDestroy(l2.stream);
                if (l2.done) cudaEventDestroy(l2.done);
            }
            delete s;
            return SKEW_ERR_CUDA;
        }
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return SKEW_OK;
}

int skew_server_submit(skew_server *s, int64_t n, const double *A, int64_t lda, int mode,
                       uint64_t *ticket) {
    if (s == nullptr) return -1;
    if (n < 0 || n > kMaxOrder) return -2;
    if (A == nullptr && n > 0) return -3;
    if (lda < (n > 1 ? n : 1)) return -4;
    if (mode != SKEW_SERVE_FACTORS && mode != SKEW_SERVE_FACTORS_L && mode != SKEW_SERVE_PFAFFIAN)
        return -5;
    if (ticket == nullptr) return -6;
    const size_t bytes = request_bytes(n, mode == SKEW_SERVE_FACTORS_L);
    std::lock_guard<std::mutex> lock(s->mu);
    Request r;
    r.n = n;
    r.mode = mode;
    r.bytes = bytes;
    r.ws_bytes = request_ws_bytes(s, r);
    if (bytes + r.ws_bytes > s->budget) return SKEW_ERR_NOMEM;
    r.ticket = s->next_ticket++;
    r.src = A;
    r.src_ld = lda;
    r.t_submit = Clock::now();
    r.host = take_host_slot(s);
    if (r.host == nullptr) return SKEW_ERR_NOMEM;
    *ticket = r.ticket;
    s->queue.push_back(r.ticket);
    s->reqs.emplace(r.ticket, r);
    s->cv_work.notify_one();
    return SKEW_OK;
}

int skew_server_poll(skew_server *s, uint64_t ticket, int *done) {
    if (s == nullptr) return -1;
    if (done == nullptr) return -3;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return -2;
    const ReqState st = it->second.state;
    *done = (st == ReqState::Done || st == ReqState::Failed) ? 1 : 0;
    return SKEW_OK;
}

int skew_server_wait(skew_server *s, uint64_t ticket, double timeout_s, double *logabs,
                     int32_t *sign, int32_t *info, const double **t, const int32_t **piv,
                     const double **L, double *latency_s) {
    if (s == nullptr) return -1;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return -2;
    auto finished = [&] {
        const ReqState st = s->reqs[ticket].state;
        return st == ReqState::Done || st == ReqState::Failed;
    };
    if (timeout_s < 0) {
        s->cv_done.wait(lock, finished);
    } else if (!s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), finished)) {
        return SKEW_ERR_TIMEOUT;
    }
    Request &r = s->reqs[ticket];
    if (r.state == ReqState::Failed) return r.status;
    if (logabs) *logabs = r.host->logabs;
    if (sign) *sign = r.host->sign;
    if (info) *info = r.host->info;
    const bool factors = r.mode != SKEW_SERVE_PFAFFIAN;   // Pfaffian-only: none kept
    if (t) *t = factors ? r.t : nullptr;
    if (piv) *piv = factors ? r.piv : nullptr;
    if (L) *L = r.L;
    if (latency_s) *latency_s = std::chrono::duration<double>(r.t_done - r.t_submit).count();
    return SKEW_OK;
}

int skew_server_timing(skew_server *s, uint64_t ticket, double *queued_s, double *waiting_s,
                       double *running_s) {
    if (s == nullptr) return -1;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return -2;
    const Request &r = it->second;
    if (r.state != ReqState::Done && r.state != ReqState::Failed) return SKEW_ERR_BUSY;
    if (r.lane < 0) return SKEW_ERR_BUSY;            // failed before it was launched
    auto sec = [](Clock::time_point a, Clock::time_point b) {
        return std::chrono::duration<double>(b - a).count();
    };
    if (queued_s) *queued_s = sec(r.t_submit, r.t_admit);
    if (waiting_s) *waiting_s = sec(r.t_admit, r.t_launch);
    if (running_s) *running_s = sec(r.t_launch, r.t_done);
    return SKEW_OK;
}

int skew_server_release(skew_server *s, uint64_t ticket) {
    if (s == nullptr) return -1;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return -2;
    Request &r = it->second;
    if (r.state != ReqState::Done && r.state != ReqState::Failed && r.state != ReqState::Queued)
        return SKEW_ERR_BUSY;      // admitted or running: not released
    if (r.state == ReqState::Queued) {
        for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
            if (*q == ticket) { s->queue.erase(q); break; }
    } else {
        // freed in the order of the stream its work ran on
        free_request(r, s->lanes[r.lane >= 0 ? r.lane : 0].stream);
        s->used -= r.bytes;
    }
    s->host_free.push_back(r.host);
    s->reqs.erase(it);
    s->cv_work.notify_one();
    return SKEW_OK;
}

int skew_server_copy_factors(skew_server *s, uint64_t ticket, double *t_host, int32_t *piv_host,
                             double *L_host, int64_t ldl) {
    if (s == nullptr) return -1;
    double *t;
    int32_t *piv;
    double *L;
    int64_t n;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return -2;
        Request &r = it->second;
        if (r.state != ReqState::Done) return r.state == ReqState::Failed ? r.status : SKEW_ERR_BUSY;
        if (r.mode == SKEW_SERVE_PFAFFIAN) return -3;   // no factors kept
        if (L_host != nullptr && (r.L == nullptr || ldl < (r.n > 1 ? r.n : 1))) return -5;
        t = r.t;
        piv = r.piv;
        L = r.L;
        n = r.n;
    }
    // the buffers stay valid: only the caller releases its ticket
    cudaSetDevice(s->device);
    if (t_host && n > 1) SKEW_TRY(cudaMemcpy(t_host, t, (n - 1) * sizeof(double), cudaMemcpyDeviceToHost));
    if (piv_host && n > 0) SKEW_TRY(cudaMemcpy(piv_host, piv, n * sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (L_host && n > 0)
        SKEW_TRY(cudaMemcpy2D(L_host, ldl * sizeof(double), L, n * sizeof(double), n * sizeof(double),
                              n, cudaMemcpyDeviceToHost));
    return SKEW_OK;
}

int skew_server_stats(skew_server *s, size_t *used_bytes, int *queued, int *in_flight) {
    if (s == nullptr) return -1;
    std::lock_guard<std::mutex> lock(s->mu);
    if (used_bytes) *used_bytes = s->used;
    if (queued) *queued = (int)s->queue.size();
    if (in_flight) {
        int k = (int)s->admitted.size();
        for (Lane &ln : s->lanes) k += (int)ln.tickets.size();
        *in_flight = k;
    }
    return SKEW_OK;
}

int skew_server_destroy(skew_server *s) {
    if (s == nullptr) return -1;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        s->queue.clear();   // not yet admitted: dropped
        s->cv_work.notify_one();
    }
    s->worker.join();
    cudaSetDevice(s->device);
    for (auto &kv : s->reqs)
        free_request(kv.second, s->lanes[kv.second.lane >= 0 ? kv.second.lane : 0].stream);
    for (Lane &ln : s->lanes) {
        cudaStreamSynchronize(ln.stream);
        if (ln.h_table) cudaFreeHost(ln.h_table);
        if (ln.d_table) cudaFree(ln.d_table);
        cudaEventDestroy(ln.done);
        cudaStreamDestroy(ln.stream);
    }
    for (HostResult *c : s->host_chunks) cudaFreeHost(c);
    delete s;
    return SKEW_OK;
}

}  // extern "C"
