// Autotuner (lfmm_autotune in include/lfmm.h): expansion order, leaf size and the
// tensor-core levels chosen by measurement, cached process-wide.
//
// The error of every candidate is measured against a reference evaluation of the same
// points by the float-float path at p = 16 (relative error ~1e-13, far below every
// tolerance the tuner accepts), with one fixed pseudo-random zero-sum charge vector;
// times are CUDA-event medians of plan creation + evaluation on the caller's stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "lfmm_internal.h"

namespace {

using lfmm::fail;

struct Key {
    int precision, tol_dec, ls, lt, lp, tree;
    bool operator<(const Key& o) const {
        return std::tie(precision, tol_dec, ls, lt, lp, tree) < std::tie(o.precision, o.tol_dec, o.ls, o.lt, o.lp, o.tree);
    }
};
struct Entry {
    int p, leaf_size, tc_min_level;
    double rel_err, ms;
    int m2l_tile = 0, m2l_stages = 0, m2l_split = 0;
};

std::mutex g_mu;
std::map<Key, Entry> g_cache;

int ceil_log2(int64_t v) {
    int k = 0;
    while (((int64_t)1 << k) < v) ++k;
    return k;
}

// splitmix64: the charge vector of the measurements (any fixed values would do)
uint64_t splitmix64(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct Problem {
    const int32_t* src;
    int64_t ns;
    const int64_t* soff;
    const int32_t* tgt;
    int64_t nt;
    const int64_t* toff;
    int64_t np;
};

int create(const Problem& pr, const lfmm_opts& o, lfmm_plan** plan, cudaStream_t s) {
    if (pr.soff) return lfmm_forest_create(plan, pr.src, pr.soff, pr.tgt, pr.toff, pr.np, &o, s);
    return lfmm_plan_create(plan, pr.src, pr.ns, pr.tgt, pr.nt, &o, s);
}

struct Bufs {
    double* f = nullptr;
    double* u = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t s = nullptr;
    ~Bufs() {
        if (f) cudaFreeAsync(f, s);
        if (u) cudaFreeAsync(u, s);
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        cudaStreamSynchronize(s);
        cudaGetLastError();
    }
};

// One measured configuration: `timed` steps of create + eval (after one untimed),
// median time in *ms (when timed > 0) and u of the last step in `u_host`.
int measure(const Problem& pr, const lfmm_opts& o, Bufs& b, int timed, std::vector<double>& u_host, double* ms) {
    std::vector<float> t;
    for (int k = 0; k <= timed; ++k) {
        lfmm_plan* plan = nullptr;
        if (k > 0) LFMM_CUDA_TRY(cudaEventRecord(b.a, b.s));
        int st = create(pr, o, &plan, b.s);
        if (st) return st;
        st = lfmm_eval(plan, b.f, b.u, b.s);
        if (k > 0) cudaEventRecord(b.b, b.s);
        const int st2 = lfmm_plan_destroy(plan);
        if (st) return st;
        if (st2) return st2;
        LFMM_CUDA_TRY(cudaStreamSynchronize(b.s));
        if (k > 0) {
            float e = 0.f;
            LFMM_CUDA_TRY(cudaEventElapsedTime(&e, b.a, b.b));
            t.push_back(e);
        }
    }
    u_host.resize((size_t)pr.nt);
    LFMM_CUDA_TRY(cudaMemcpyAsync(u_host.data(), b.u, (size_t)pr.nt * sizeof(double), cudaMemcpyDeviceToHost, b.s));
    LFMM_CUDA_TRY(cudaStreamSynchronize(b.s));
    if (ms) {
        std::sort(t.begin(), t.end());
        *ms = t.empty() ? 0.0 : (double)t[t.size() / 2];
    }
    return LFMM_OK;
}

double rel_err(const std::vector<double>& u, const std::vector<double>& ref) {
    double num = 0.0, den = 0.0;
    for (size_t i = 0; i < ref.size(); ++i) {
        num = std::max(num, std::fabs(u[i] - ref[i]));
        den = std::max(den, std::fabs(ref[i]));
    }
    if (!(num == num)) return INFINITY;  // NaN
    return den > 0.0 ? num / den : num;
}

}  // namespace

extern "C" {

int lfmm_autotune(const int32_t* src_xy, int64_t n_src, const int64_t* src_offsets, const int32_t* tgt_xy,
                  int64_t n_tgt, const int64_t* tgt_offsets, int64_t n_problems, double tol, const lfmm_opts* base,
                  lfmm_tune_result* result, void* stream) {
    if (!src_xy || !tgt_xy || !result) return fail(LFMM_EINVAL, "NULL argument");
    if (n_src < 1 || n_tgt < 1) return fail(LFMM_EINVAL, "empty problem");
    if ((src_offsets == nullptr) != (tgt_offsets == nullptr)) return fail(LFMM_EINVAL, "give both offset arrays or none");
    if (!src_offsets && n_problems != 1) return fail(LFMM_EINVAL, "n_problems must be 1 without offsets");
    if (n_problems < 1) return fail(LFMM_EINVAL, "n_problems must be >= 1");
    if (!(tol >= 1e-13 && tol <= 1e-2)) return fail(LFMM_EINVAL, "tol must be in [1e-13, 1e-2]");
    lfmm_opts o0;
    if (base) o0 = *base;
    else lfmm_opts_default(&o0);
    std::memset(result, 0, sizeof(*result));
    const bool mixed = tol >= 1e-6;
    o0.precision = mixed ? LFMM_MIXED : LFMM_DF;
    o0.tc_min_level = 0;
    const Problem pr{src_xy, n_src, src_offsets, tgt_xy, n_tgt, tgt_offsets, n_problems};
    const Key key{o0.precision, (int)std::floor(std::log10(tol) + 1e-9), ceil_log2(n_src), ceil_log2(n_tgt),
                  ceil_log2(n_problems), src_offsets ? LFMM_TREE_PRUNED : o0.tree};
    {
        std::lock_guard<std::mutex> g(g_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            result->opts = o0;
            result->opts.p = it->second.p;
            result->opts.leaf_size = it->second.leaf_size;
            result->opts.tc_min_level = it->second.tc_min_level;
            result->opts.m2l_tile = it->second.m2l_tile;
            result->opts.m2l_stages = it->second.m2l_stages;
            result->opts.m2l_split = it->second.m2l_split;
            result->rel_err = it->second.rel_err;
            result->ms = it->second.ms;
            result->from_cache = 1;
            return LFMM_OK;
        }
    }

    Bufs b;
    b.s = (cudaStream_t)stream;
    LFMM_CUDA_TRY(cudaEventCreate(&b.a));
    LFMM_CUDA_TRY(cudaEventCreate(&b.b));
    LFMM_CUDA_TRY(lfmm::dev_malloc((void**)&b.f, (size_t)n_src * sizeof(double), b.s));
    LFMM_CUDA_TRY(lfmm::dev_malloc((void**)&b.u, (size_t)n_tgt * sizeof(double), b.s));
    {
        // uniform in (-1, 1), each problem shifted to zero sum
        std::vector<double> f((size_t)n_src);
        uint64_t seed = 0x6C666D6D74756E65ull;
        for (auto& v : f) v = (double)(splitmix64(seed) >> 11) * 0x1.0p-52 - 1.0;
        for (int64_t i = 0; i < n_problems; ++i) {
            const int64_t a = src_offsets ? src_offsets[i] : 0, e = src_offsets ? src_offsets[i + 1] : n_src;
            double m = 0.0;
            for (int64_t j = a; j < e; ++j) m += f[(size_t)j];
            m /= (double)std::max<int64_t>(1, e - a);
            for (int64_t j = a; j < e; ++j) f[(size_t)j] -= m;
        }
        LFMM_CUDA_TRY(cudaMemcpyAsync(b.f, f.data(), f.size() * sizeof(double), cudaMemcpyHostToDevice, b.s));
        LFMM_CUDA_TRY(cudaStreamSynchronize(b.s));
    }
    std::vector<double> ref, u;
    {
        lfmm_opts r = o0;
        r.precision = LFMM_DF;
        r.p = 16;
        r.leaf_size = 128;
        r.tc_min_level = 0;
        r.flags = 0;
        const int st = measure(pr, r, b, 0, ref, nullptr);
        if (st) return st;
    }
    const double goal = 0.5 * tol;
    int candidates = 0;
    // 3. p at leaf size 64
    const std::vector<int> ps = mixed ? std::vector<int>{4, 5, 6, 7, 8, 9} : std::vector<int>{10, 12, 14, 16, 17};
    lfmm_opts best = o0;
    best.leaf_size = 64;
    double best_err = INFINITY;
    bool met = false;
    for (int p : ps) {
        lfmm_opts c = best;
        c.p = p;
        if (measure(pr, c, b, 0, u, nullptr) != LFMM_OK) continue;
        ++candidates;
        const double e = rel_err(u, ref);
        best.p = p;
        best_err = e;
        if (e <= goal) {
            met = true;
            break;
        }
    }
    if (!met)
        return fail(LFMM_EUNSUPPORTED, "autotune: no expansion order reaches tol / 2 (best " + std::to_string(best_err) + ")");
    // 4. leaf size, then (mixed, single problem) the first tensor-core level
    double best_ms = INFINITY;
    const std::vector<int> leaves = mixed ? std::vector<int>{32, 64, 128} : std::vector<int>{64, 128, 192};
    lfmm_opts pick = best;
    for (int leaf : leaves) {
        lfmm_opts c = best;
        c.leaf_size = leaf;
        double ms = 0.0;
        if (measure(pr, c, b, 3, u, &ms) != LFMM_OK) continue;
        ++candidates;
        const double e = rel_err(u, ref);
        if (e > goal) continue;
        if (ms < best_ms) {
            best_ms = ms;
            best_err = e;
            pick = c;
        }
    }
    if (!(best_ms < INFINITY)) return fail(LFMM_EUNSUPPORTED, "autotune: no leaf size met the tolerance");
    if (mixed && !src_offsets) {
        lfmm_plan* plan = nullptr;
        int L = 0;
        if (create(pr, pick, &plan, b.s) == LFMM_OK) {
            lfmm_plan_info info;
            if (lfmm_plan_get_info(plan, &info) == LFMM_OK) L = info.L;
            lfmm_plan_destroy(plan);
        }
        for (int tc : {L, L - 1, 99}) {
            if (tc < 2 || tc == (pick.tc_min_level == 0 ? lfmm::kDefaultTcMinLevel : pick.tc_min_level)) continue;
            lfmm_opts c = pick;
            c.tc_min_level = tc;
            double ms = 0.0;
            if (measure(pr, c, b, 3, u, &ms) != LFMM_OK) continue;
            ++candidates;
            const double e = rel_err(u, ref);
            if (e > goal) continue;
            if (ms < best_ms) {
                best_ms = ms;
                best_err = e;
                pick = c;
            }
        }
    }
    // 5. M2L tiling: the tensor-core tile width and TMA ring depth (mixed, single problem,
    // when tensor-core levels are in use), then the K-split of the coarse-level / list
    // M2L kernels; each candidate must still meet the tolerance
    auto try_opts = [&](const lfmm_opts& c) {
        double ms = 0.0;
        if (measure(pr, c, b, 3, u, &ms) != LFMM_OK) return;
        ++candidates;
        const double e = rel_err(u, ref);
        if (e > goal) return;
        if (ms < best_ms) {
            best_ms = ms;
            best_err = e;
            pick = c;
        }
    };
    if (mixed && !src_offsets && pick.tc_min_level != 99) {
        for (int tile : {64, 32, 16}) {
            lfmm_opts c = pick;
            c.m2l_tile = tile;
            try_opts(c);
        }
        for (int stages : {2, 4}) {
            lfmm_opts c = pick;
            c.m2l_stages = stages;
            try_opts(c);
        }
    }
    {
        const lfmm_opts base_pick = pick;
        for (int split : {1, 2, 4, 8}) {
            lfmm_opts c = base_pick;
            c.m2l_split = split;
            try_opts(c);
        }
    }
    if (base) pick.flags = base->flags;
    result->opts = pick;
    result->rel_err = best_err;
    result->ms = best_ms;
    result->candidates = candidates;
    result->from_cache = 0;
    std::lock_guard<std::mutex> g(g_mu);
    g_cache[key] = Entry{pick.p, pick.leaf_size, pick.tc_min_level, best_err, best_ms, pick.m2l_tile, pick.m2l_stages,
                         pick.m2l_split};
    return LFMM_OK;
}

int lfmm_tune_cache_clear(void) {
    std::lock_guard<std::mutex> g(g_mu);
    g_cache.clear();
    return LFMM_OK;
}

int lfmm_tune_cache_save(const char* path) {
    if (!path) return fail(LFMM_EINVAL, "NULL path");
    FILE* fp = std::fopen(path, "w");
    if (!fp) return fail(LFMM_EINVAL, std::string("cannot open ") + path);
    std::lock_guard<std::mutex> g(g_mu);
    for (const auto& kv : g_cache) {
        const Key& k = kv.first;
        const Entry& e = kv.second;
        std::fprintf(fp, "lfmm-tune-2 %d %d %d %d %d %d %d %d %d %.6e %.6e %d %d %d\n", k.precision, k.tol_dec, k.ls,
                     k.lt, k.lp, k.tree, e.p, e.leaf_size, e.tc_min_level, e.rel_err, e.ms, e.m2l_tile, e.m2l_stages,
                     e.m2l_split);
    }
    const bool ok = std::fclose(fp) == 0;
    return ok ? LFMM_OK : fail(LFMM_EINVAL, std::string("write failed: ") + path);
}

int lfmm_tune_cache_load(const char* path) {
    if (!path) return fail(LFMM_EINVAL, "NULL path");
    FILE* fp = std::fopen(path, "r");
    if (!fp) return fail(LFMM_EINVAL, std::string("cannot open ") + path);
    char line[512];
    int st = LFMM_OK;
    int n = 0;
    while (std::fgets(line, sizeof line, fp)) {
        ++n;
        Key k;
        Entry e;
        char tag[32];
        // version 1 lines carry no M2L tiling (the library's rules)
        const int got = std::sscanf(line, "%31s %d %d %d %d %d %d %d %d %d %lf %lf %d %d %d", tag, &k.precision,
                                    &k.tol_dec, &k.ls, &k.lt, &k.lp, &k.tree, &e.p, &e.leaf_size, &e.tc_min_level,
                                    &e.rel_err, &e.ms, &e.m2l_tile, &e.m2l_stages, &e.m2l_split);
        const bool v1 = got == 12 && std::strcmp(tag, "lfmm-tune-1") == 0;
        const bool v2 = got == 15 && std::strcmp(tag, "lfmm-tune-2") == 0;
        if (v1) e.m2l_tile = e.m2l_stages = e.m2l_split = 0;
        if ((!v1 && !v2) || (k.precision != LFMM_MIXED && k.precision != LFMM_DF && k.precision != LFMM_FP64) ||
            e.p < 2 || e.p > 17 || e.leaf_size < 1 || e.tc_min_level < 0 ||
            (e.m2l_tile != 0 && e.m2l_tile != 16 && e.m2l_tile != 32 && e.m2l_tile != 64 && e.m2l_tile != 128) ||
            (e.m2l_stages != 0 && (e.m2l_stages < 2 || e.m2l_stages > 4)) || e.m2l_split < 0 || e.m2l_split > 9) {
            st = fail(LFMM_EINVAL, std::string("malformed tuning line ") + std::to_string(n) + " in " + path);
            break;
        }
        std::lock_guard<std::mutex> g(g_mu);
        g_cache[k] = e;
    }
    std::fclose(fp);
    return st;
}

}  // extern "C"
