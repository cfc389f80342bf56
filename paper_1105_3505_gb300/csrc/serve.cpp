// Request loop with continuous admission (lfmm_server_* in include/lfmm.h).
//
// A server owns n_slots worker threads, each with its own non-blocking CUDA streams.
// Submitted requests wait in arrival order; a free worker admits the oldest one as
// soon as its estimated device footprint fits the memory budget next to the requests
// already running (and the device's free memory, counting what the stream-ordered
// pool holds unused).  Every admitted request builds its plan and evaluates on its
// worker's stream, so requests that arrive while others run overlap with them on the
// device.  The model-box operators and the phi tables are cached process-wide and
// stay resident; plan workspaces come from the stream-ordered pool, which keeps freed
// memory for reuse.  A request's result does not depend on what runs beside it: each
// request owns its plan, stream and buffers.
//
// Overload policy (lfmm_server_set_limits): a bounded queue, a refusal at submit when the
// predicted wait (the smoothed run times of the requests queued ahead, by class and size,
// over the slots) exceeds the latency budget, and shedding of requests that waited past
// it anyway; cancellation removes a queued request.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <algorithm>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "lfmm_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

// leaf size of the float-float path in the server (its M2L costs ~15 binary32 operations
// per multiply-add, so larger leaves that trade M2L boxes for near-field pairs pay off)
constexpr int kServeLeafDF = 192;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Job {
    lfmm_request req{};
    lfmm_opts opts{};
    int cls = 0;  // 0: mixed path, 1: binary64 path
    int64_t est = 0;
    double est_ms = 0.0;  // predicted run time (overload policy)
    Clock::time_point t_submit, t_admit, t_done;
    lfmm_request_stats stats{};
    bool done = false;
};

// Conservative device footprint of a request before its plan exists (coordinates,
// buckets, staging, expansions and the tree temporaries), corrected once the plan
// reports its own size.
int64_t estimate_bytes(const lfmm_request& r, const lfmm_opts& o) {
    const int64_t n = r.n_src + r.n_tgt;
    const int64_t esz = o.precision == LFMM_MIXED ? 4 : 8;
    const int64_t np = o.p <= 9 ? 32 : 64;
    return 160 * n + 4 * np * esz * (n / 8 + 1) + ((int64_t)64 << 20);
}

}  // namespace

struct lfmm_server {
    int device = 0;
    int n_slots = 0;
    int64_t budget = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<int64_t> pending;
    std::unordered_map<int64_t, Job> jobs;
    int64_t next_ticket = 1;
    int64_t in_flight = 0;
    int running = 0;
    int running_cls[2] = {0, 0};
    int max_cls[2] = {0, 0};  // binary64 requests leave slots to the mixed ones
    int max_pending = 0;      // overload policy (lfmm_server_set_limits); 0: no limit
    double max_queue_ms = 0.0;
    // measured run times per class and size bucket (log2 of the point count), smoothed;
    // the predicted work queued ahead of a new request is their sum over `pending`
    double run_ms_fit[2][40] = {};
    double pending_ms = 0.0;
    bool stopping = false;

    static int size_bucket(const Job& j) {
        int b = 0;
        while (b < 39 && ((int64_t)2 << b) <= j.req.n_src + j.req.n_tgt) ++b;
        return b;
    }
    // predicted run time of a request from the nearest measured bucket of its class,
    // scaled by the point count; 0 while nothing is measured
    double predict_ms(const Job& j) const {
        const int b = size_bucket(j);
        for (int d = 0; d < 40; ++d)
            for (int bb : {b - d, b + d})
                if (bb >= 0 && bb < 40 && run_ms_fit[j.cls][bb] > 0.0)
                    return run_ms_fit[j.cls][bb] * std::max(0.25, std::min(4.0, std::ldexp(1.0, b - bb)));
        return 0.0;
    }
    void learn(const Job& j, double run_ms) {
        double& m = run_ms_fit[j.cls][size_bucket(j)];
        m = m > 0.0 ? 0.8 * m + 0.2 * run_ms : run_ms;
    }
    std::vector<std::thread> workers;

    // free device memory plus what the default pool holds but does not use
    int64_t available() {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            return INT64_MAX;
        }
        int64_t pooled = 0;
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
            uint64_t reserved = 0, used = 0;
            if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
                cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess &&
                reserved > used)
                pooled = (int64_t)(reserved - used);
        }
        cudaGetLastError();
        return (int64_t)fr + pooled;
    }

    // The budget was sized from the device's available memory at creation; the device is
    // asked again (a driver call, kept out of the common path since every waiting worker
    // evaluates this under the lock) only once the budget is more than half committed.
    bool fits(const Job& j) {
        if (running == 0) return true;  // progress: a lone request always runs
        if (in_flight + j.est > budget) return false;
        if (2 * (in_flight + j.est) <= budget) return true;
        return j.est + ((int64_t)256 << 20) <= available();
    }

    // Completes a waiting request without running it (status EBUSY or ECANCELED).
    // Caller holds mu and removes the ticket from `pending`.
    void finish_unrun(Job& j, int status, Clock::time_point now) {
        j.t_admit = j.t_done = now;
        j.stats.status = status;
        j.stats.precision = j.opts.precision;
        j.stats.queue_ms = ms_between(j.t_submit, now);
        j.stats.run_ms = 0.0;
        j.stats.total_ms = j.stats.queue_ms;
        j.done = true;
    }

    // Overload policy: sheds every waiting request whose wait exceeds the latency budget.
    // Caller holds mu; returns whether any was shed (waiters must then be woken).
    bool shed_expired() {
        if (max_queue_ms <= 0.0 || pending.empty()) return false;
        const Clock::time_point now = Clock::now();
        bool any = false;
        for (size_t i = 0; i < pending.size();) {
            Job& j = jobs[pending[i]];
            if (ms_between(j.t_submit, now) > max_queue_ms) {
                finish_unrun(j, LFMM_EBUSY, now);
                pending_ms -= j.est_ms;
                pending.erase(pending.begin() + (std::ptrdiff_t)i);
                any = true;
            } else {
                ++i;
            }
        }
        return any;
    }

    // Position in `pending` of the request to start next, or -1.  Requests start in
    // arrival order; a later one may pass the oldest only when the oldest waits for a
    // slot of its class (binary64 requests may not take every slot), never when it
    // waits for memory, so large requests are not starved.
    int64_t pick() {
        for (size_t i = 0; i < pending.size(); ++i) {
            const Job& j = jobs[pending[i]];
            if (running_cls[j.cls] >= max_cls[j.cls]) continue;  // class full: look further
            return fits(j) ? (int64_t)i : -1;
        }
        return -1;
    }

    void worker_main() {
        cudaSetDevice(device);
        // two streams per worker: mixed-path requests (short, latency-bound) run at the
        // highest priority so that their blocks are scheduled ahead of the long M2L
        // kernels of binary64-level requests sharing the device
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) cudaGetLastError();
        cudaStream_t sp[2] = {nullptr, nullptr};
        for (int c = 0; c < 2; ++c)
            if (cudaStreamCreateWithPriority(&sp[c], cudaStreamNonBlocking, c == 0 ? greatest : least) != cudaSuccess) {
                cudaGetLastError();
                sp[c] = nullptr;
            }
        for (;;) {
            int64_t ticket;
            Job* job;
            {
                std::unique_lock<std::mutex> lk(mu);
                int64_t at = -1;
                cv_work.wait(lk, [&] {
                    if (shed_expired()) cv_done.notify_all();
                    return (stopping && pending.empty()) || (at = pick()) >= 0;
                });
                if (pending.empty()) break;  // stopping and drained
                ticket = pending[at];
                pending.erase(pending.begin() + at);
                job = &jobs[ticket];
                pending_ms -= job->est_ms;
                job->t_admit = Clock::now();
                in_flight += job->est;
                ++running;
                ++running_cls[job->cls];
            }
            int st = run(*job, sp[job->cls]);
            {
                std::lock_guard<std::mutex> lk(mu);
                job->t_done = Clock::now();
                in_flight -= job->est;
                --running;
                --running_cls[job->cls];
                if (st == LFMM_OK) learn(*job, ms_between(job->t_admit, job->t_done));
                job->stats.status = st;
                job->stats.precision = job->opts.precision;
                job->stats.queue_ms = ms_between(job->t_submit, job->t_admit);
                job->stats.run_ms = ms_between(job->t_admit, job->t_done);
                job->stats.total_ms = ms_between(job->t_submit, job->t_done);
                job->done = true;
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
        for (cudaStream_t s : sp)
            if (s) {
                cudaStreamSynchronize(s);
                cudaStreamDestroy(s);
            }
    }

    int run(Job& j, cudaStream_t s) {
        lfmm_plan* plan = nullptr;
        int st = lfmm_plan_create(&plan, j.req.src_xy, j.req.n_src, j.req.tgt_xy, j.req.n_tgt, &j.opts, s);
        if (st) return st;
        lfmm_plan_info info;
        if (lfmm_plan_get_info(plan, &info) == LFMM_OK) {
            j.stats.device_bytes = info.device_bytes;
            std::lock_guard<std::mutex> lk(mu);
            const int64_t actual = std::max<int64_t>(info.device_bytes, 1);
            in_flight += actual - j.est;  // replace the estimate by the plan's own size
            j.est = actual;
        }
        st = lfmm_eval(plan, j.req.f, j.req.u, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (!st && e != cudaSuccess) st = LFMM_ECUDA;
        const int st2 = lfmm_plan_destroy(plan);
        return st ? st : st2;
    }
};

extern "C" {

int lfmm_server_create(lfmm_server** out, int32_t n_slots, int64_t hbm_budget_bytes) {
    if (!out) return lfmm::fail(LFMM_EINVAL, "NULL server out-pointer");
    *out = nullptr;
    if (n_slots < 1 || n_slots > 64) return lfmm::fail(LFMM_EINVAL, "n_slots must be in [1, 64]");
    if (hbm_budget_bytes < 0) return lfmm::fail(LFMM_EINVAL, "hbm_budget_bytes must be >= 0");
    lfmm_server* sv = new (std::nothrow) lfmm_server();
    if (!sv) return lfmm::fail(LFMM_ENOMEM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&sv->device);
    if (e != cudaSuccess) {
        delete sv;
        return lfmm::fail(LFMM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    }
    sv->n_slots = n_slots;
    sv->max_cls[0] = n_slots;
    sv->max_cls[1] = n_slots > 1 ? n_slots - std::max(1, n_slots / 4) : 1;
    sv->budget = hbm_budget_bytes;
    if (sv->budget == 0) sv->budget = (int64_t)(0.8 * (double)sv->available());
    for (int i = 0; i < n_slots; ++i) sv->workers.emplace_back([sv] { sv->worker_main(); });
    *out = sv;
    return LFMM_OK;
}

int lfmm_server_submit(lfmm_server* sv, const lfmm_request* req, int64_t* ticket) {
    if (!sv || !req || !ticket) return lfmm::fail(LFMM_EINVAL, "NULL argument");
    if (!req->src_xy || !req->tgt_xy || !req->f || !req->u) return lfmm::fail(LFMM_EINVAL, "NULL request buffer");
    if (req->n_src < 1 || req->n_tgt < 1) return lfmm::fail(LFMM_EINVAL, "empty request");
    if (!(req->tol > 0.0)) return lfmm::fail(LFMM_EINVAL, "request tol must be > 0");
    Job j;
    j.req = *req;
    lfmm_opts_default(&j.opts);
    // tolerance -> path: the mixed path reaches ~2e-7; the float-float path at p = 16
    // reaches binary64-level accuracy (~1e-14) on the FP32 pipes
    if (req->tol >= 1e-6) {
        j.opts.precision = LFMM_MIXED;
        j.opts.p = 8;
        j.cls = 0;
    } else {
        j.opts.precision = LFMM_DF;
        j.opts.p = 16;
        j.opts.leaf_size = kServeLeafDF;
        j.cls = 1;
    }
    j.est = estimate_bytes(*req, j.opts);
    j.t_submit = Clock::now();
    bool shed = false;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stopping) return lfmm::fail(LFMM_EINVAL, "server is shutting down");
        shed = sv->shed_expired();
        if (sv->max_pending > 0 && (int64_t)sv->pending.size() >= sv->max_pending) {
            if (shed) sv->cv_done.notify_all();
            return lfmm::fail(LFMM_EBUSY, "server queue full (" + std::to_string(sv->pending.size()) +
                                              " requests waiting for admission)");
        }
        j.est_ms = sv->predict_ms(j);
        const double wait_ms = sv->pending_ms / sv->n_slots;
        if (sv->max_queue_ms > 0.0 && wait_ms > sv->max_queue_ms) {
            if (shed) sv->cv_done.notify_all();
            return lfmm::fail(LFMM_EBUSY, "predicted wait " + std::to_string(wait_ms) +
                                              " ms exceeds the server's latency budget");
        }
        *ticket = sv->next_ticket++;
        sv->jobs.emplace(*ticket, j);
        sv->pending.push_back(*ticket);
        sv->pending_ms += j.est_ms;
    }
    if (shed) sv->cv_done.notify_all();
    sv->cv_work.notify_all();
    return LFMM_OK;
}

int lfmm_server_set_limits(lfmm_server* sv, int32_t max_pending, double max_queue_ms) {
    if (!sv) return lfmm::fail(LFMM_EINVAL, "NULL server");
    if (max_pending < 0 || !(max_queue_ms >= 0.0)) return lfmm::fail(LFMM_EINVAL, "limits must be >= 0");
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->max_pending = max_pending;
        sv->max_queue_ms = max_queue_ms;
    }
    sv->cv_work.notify_all();
    return LFMM_OK;
}

int lfmm_server_cancel(lfmm_server* sv, int64_t ticket) {
    if (!sv) return lfmm::fail(LFMM_EINVAL, "NULL server");
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = std::find(sv->pending.begin(), sv->pending.end(), ticket);
        if (it == sv->pending.end())
            return lfmm::fail(LFMM_EINVAL, sv->jobs.count(ticket) ? "request already admitted or finished"
                                                                   : "unknown ticket");
        sv->finish_unrun(sv->jobs[ticket], LFMM_ECANCELED, Clock::now());
        sv->pending_ms -= sv->jobs[ticket].est_ms;
        sv->pending.erase(it);
    }
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
    return LFMM_OK;
}

int lfmm_server_wait(lfmm_server* sv, int64_t ticket, lfmm_request_stats* stats) {
    if (!sv) return lfmm::fail(LFMM_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(ticket);
    if (it == sv->jobs.end()) return lfmm::fail(LFMM_EINVAL, "unknown ticket");
    sv->cv_done.wait(lk, [&] { return it->second.done; });
    const lfmm_request_stats st = it->second.stats;
    sv->jobs.erase(it);
    lk.unlock();
    if (stats) *stats = st;
    if (st.status) return lfmm::fail(st.status, "request failed: " + std::string(lfmm_status_string(st.status)));
    return LFMM_OK;
}

int lfmm_server_destroy(lfmm_server* sv) {
    if (!sv) return LFMM_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stopping = true;
    }
    sv->cv_work.notify_all();
    for (auto& t : sv->workers) t.join();
    delete sv;
    return LFMM_OK;
}

}  // extern "C"
