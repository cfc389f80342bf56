// Launch counting and per-phase CUDA-event timing (see lfmm_profile_* in include/lfmm.h).
#include <atomic>
#include <map>
#include <mutex>
#include <utility>

#include "lfmm_internal.h"

namespace lfmm {

namespace {
std::atomic<int64_t> g_launches{0};
std::atomic<bool> g_enabled{false};
std::mutex g_mu;
double g_ms[LFMM_NUM_PHASES] = {0};
int64_t g_cnt[LFMM_NUM_PHASES] = {0};
struct Pending {
    int phase;
    cudaEvent_t a, b;
    int launches;
};
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free_events;

cudaEvent_t get_event() {
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_free_events.empty()) {
        cudaEvent_t e = g_free_events.back();
        g_free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}
}  // namespace

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
bool profiling_enabled() { return g_enabled.load(std::memory_order_relaxed); }

PhaseTimer::PhaseTimer(int phase, cudaStream_t s) : phase_(phase), s_(s) {
    if (!profiling_enabled()) return;
    a_ = get_event();
    b_ = get_event();
    if (a_) cudaEventRecord(a_, s_);
}

PhaseTimer::~PhaseTimer() {
    if (!a_ || !b_) return;
    cudaEventRecord(b_, s_);
    std::lock_guard<std::mutex> g(g_mu);
    g_pending.push_back({phase_, a_, b_, launches_});
}

void profile_flush() {
    std::vector<Pending> pend;
    {
        std::lock_guard<std::mutex> g(g_mu);
        pend.swap(g_pending);
    }
    for (auto& p : pend) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            std::lock_guard<std::mutex> g(g_mu);
            g_ms[p.phase] += ms;
            g_cnt[p.phase] += p.launches;
        }
        cudaGetLastError();
        std::lock_guard<std::mutex> g(g_mu);
        g_free_events.push_back(p.a);
        g_free_events.push_back(p.b);
    }
}

}  // namespace lfmm

extern "C" {

int lfmm_profile_enable(int enable) {
    if (!enable) lfmm::profile_flush();
    lfmm::g_enabled.store(enable != 0);
    return LFMM_OK;
}

int lfmm_profile_read(double* ms, int64_t* launches, int reset) {
    lfmm::profile_flush();
    std::lock_guard<std::mutex> g(lfmm::g_mu);
    for (int i = 0; i < LFMM_NUM_PHASES; ++i) {
        if (ms) ms[i] = lfmm::g_ms[i];
        if (launches) launches[i] = lfmm::g_cnt[i];
        if (reset) {
            lfmm::g_ms[i] = 0;
            lfmm::g_cnt[i] = 0;
        }
    }
    return LFMM_OK;
}

int64_t lfmm_launch_count(void) { return lfmm::g_launches.load(); }

}  // extern "C"

namespace lfmm {

namespace {
std::mutex g_attr_mu;
std::map<const void*, size_t> g_smem_limit;
std::map<std::pair<const void*, std::pair<int, size_t>>, int> g_occ;
}  // namespace

cudaError_t ensure_dynamic_smem(const void* func, size_t bytes) {
    std::lock_guard<std::mutex> g(g_attr_mu);
    size_t& cur = g_smem_limit[func];
    if (bytes <= cur) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return clear_and_return(e);
    cur = bytes;
    return cudaSuccess;
}

int blocks_per_sm(const void* func, int threads, size_t smem) {
    std::lock_guard<std::mutex> g(g_attr_mu);
    auto key = std::make_pair(func, std::make_pair(threads, smem));
    auto it = g_occ.find(key);
    if (it != g_occ.end()) return it->second;
    int n = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, func, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        n = 1;
    }
    n = n < 1 ? 1 : n;
    g_occ[key] = n;
    return n;
}

}  // namespace lfmm
