// C ABI of liblfmm.so: plans, evaluation, diagnostics (declared in include/lfmm.h).
#include <algorithm>
#include <atomic>
#include <climits>
#include <cstring>
#include <mutex>
#include <new>

#include "lfmm_internal.h"

namespace lfmm {

namespace {
thread_local std::string t_last_error;
}

void set_error(const std::string& msg) { t_last_error = msg; }

int fail(int status, const std::string& msg) {
    t_last_error = msg;
    return status;
}

const char* last_error_cstr() { return t_last_error.c_str(); }

// lfmm_fault_inject_alloc: allocations left until the failing one (0: disarmed)
std::atomic<int64_t> g_alloc_fail_in{0};

cudaError_t dev_malloc(void** ptr, size_t bytes, cudaStream_t s) {
    int64_t n = g_alloc_fail_in.load(std::memory_order_relaxed);
    while (n > 0) {
        if (g_alloc_fail_in.compare_exchange_weak(n, n - 1)) {
            if (n == 1) {
                *ptr = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    return cudaMallocAsync(ptr, bytes, s);
}

}  // namespace lfmm

using namespace lfmm;

struct lfmm_plan {
    int device = 0;
    int num_sms = 0;
    lfmm_opts opts{};
    int64_t ns = 0, nt = 0;
    int64_t x0 = 0, y0 = 0;
    int K = 0, L = 0, side = 1;
    int P = 0, NP = 32;
    int max_src = 0, max_tgt = 0;
    const DeviceOps* ops = nullptr;
    cudaStream_t last_stream = nullptr;
    // device buffers (plan-owned, stream-ordered pool allocations)
    std::vector<void*> allocs;
    int64_t bytes = 0;
    int32_t *src_begin = nullptr, *tgt_begin = nullptr;
    int32_t *src_loc = nullptr, *src_perm = nullptr, *tgt_loc = nullptr, *tgt_perm = nullptr;
    int32_t* tgt_leaf = nullptr;   // Morton index of each sorted target's leaf
    void* f_sorted = nullptr;
    void* qhat = nullptr;
    void* uhat = nullptr;
    void* Qbox = nullptr;          // per-box total charge (8 B per box)
    void* Cbox = nullptr;          // per-box incoming constant (8 B per box)
    std::vector<int64_t> lvl_off;  // offset (boxes) of level l inside qhat / uhat
    int* status = nullptr;         // device status word written by kernels (LFMM_ETIMEOUT)
    int tc_min_level = kDefaultTcMinLevel;
    double* f_stage = nullptr;     // device copy of a host f
    double* u_stage = nullptr;     // device result before a host copy (3 x n_tgt)
    void* m2l_part = nullptr;      // partial sums of the K-split fused small-level M2L
    int64_t m2l_part_bytes = 0;
    int m2l_part_nvec = 0;         // vectors the buffer has been sized for
    std::unique_ptr<Forest> forest;  // pruned tree or forest (null: uniform tree)
    void* tc_split = nullptr;        // TF32 hi/lo copies of q_hat and the parent u_hat for the tensor cores
    double* un_tmp = nullptr;        // near field per target (caller order) from the concurrent near-field pass
    double* uf_tmp = nullptr;        // far field per target (caller order), before the final sum
    struct AuxStream* aux = nullptr;  // near-field pass runs here, beside the far-field sweeps
    // uniform storage: the targets are bucketed on `aux` while the plan's creation and the
    // evaluation's upward sweep go on; whatever reads them waits for this event
    cudaEvent_t tgt_ready = nullptr;
    int64_t n_boxes = 0;
    // LFMM_FLAG_GRAPH: the recorded evaluation and the device pointers it was recorded for
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    const double* graph_f = nullptr;
    double* graph_out[3] = {nullptr, nullptr, nullptr};
    // lfmm_eval_multi: per-vector sorted charges, leaf charges, near and far parts,
    // and host staging, for up to multi_cap vectors (grown on demand)
    int multi_cap = 0;
    void* m_fsorted = nullptr;
    void* m_qhat = nullptr;
    void* m_uhat = nullptr;
    void* m_Q = nullptr;
    void* m_C = nullptr;
    void* m_split = nullptr;
    double* m_un = nullptr;
    double* m_uf = nullptr;
    int host_cap = 0;
    double* m_fstage = nullptr;
    double* m_ustage = nullptr;
};

// A second stream with its fork / join events, pooled process-wide (plans are often
// short-lived; creating streams and events per plan would cost more than the overlap
// gains on small problems).
struct AuxStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    int device = -1;
};

namespace {

std::mutex g_aux_mu;
std::vector<AuxStream*> g_aux_free;

AuxStream* acquire_aux(int device) {
    {
        std::lock_guard<std::mutex> g(g_aux_mu);
        for (size_t i = 0; i < g_aux_free.size(); ++i)
            if (g_aux_free[i]->device == device) {
                AuxStream* a = g_aux_free[i];
                g_aux_free.erase(g_aux_free.begin() + i);
                return a;
            }
    }
    AuxStream* a = new (std::nothrow) AuxStream();
    if (!a) return nullptr;
    a->device = device;
    if (cudaStreamCreateWithFlags(&a->s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&a->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&a->join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (a->s) cudaStreamDestroy(a->s);
        if (a->fork) cudaEventDestroy(a->fork);
        delete a;
        return nullptr;
    }
    return a;
}

void release_aux(AuxStream* a) {
    if (!a) return;
    cudaStreamSynchronize(a->s);
    std::lock_guard<std::mutex> g(g_aux_mu);
    g_aux_free.push_back(a);
}

// Work on `s` that reads the bucketed targets waits for their bucketing (a no-op once it
// has completed; skipped while `s` is being captured, whose graph is launched behind the
// same wait).
int wait_targets(const lfmm_plan* p, cudaStream_t s) {
    if (!p->tgt_ready) return LFMM_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    LFMM_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    if (cs == cudaStreamCaptureStatusNone) LFMM_CUDA_TRY(cudaStreamWaitEvent(s, p->tgt_ready, 0));
    return LFMM_OK;
}

constexpr int kMaxLevel = 14;  // deepest leaf level searched (pruned storage beyond 4^13 leaves)
constexpr int kMaxTreeLevelForTc = 30;  // opts.tc_min_level above this: no level on the tensor cores

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void setup_pool(int dev) {
    static std::once_flag once;
    std::call_once(once, [dev] {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        cudaGetLastError();
    });
}

int palloc(lfmm_plan* p, void** out, size_t bytes, cudaStream_t s) {
    *out = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = dev_malloc(out, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return fail(LFMM_ENOMEM, std::string("device allocation of ") + std::to_string(bytes) +
                                     " bytes failed: " + cudaGetErrorString(e));
    }
    p->allocs.push_back(*out);
    p->bytes += (int64_t)bytes;
    return LFMM_OK;
}

struct Temp {  // stream-ordered temporary freed on scope exit
    void* ptr = nullptr;
    cudaStream_t s = nullptr;
    void reset_now() {
        if (ptr) cudaFreeAsync(ptr, s);
        ptr = nullptr;
    }
    ~Temp() {
        if (ptr) cudaFreeAsync(ptr, s);
    }
};

int talloc(Temp& t, size_t bytes, cudaStream_t s) {
    t.s = s;
    cudaError_t e = dev_malloc(&t.ptr, bytes ? bytes : 16, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        t.ptr = nullptr;
        return fail(LFMM_ENOMEM, std::string("temporary allocation failed: ") + cudaGetErrorString(e));
    }
    return LFMM_OK;
}

void free_plan_buffers(lfmm_plan* p) {
    for (void* a : p->allocs) cudaFreeAsync(a, p->last_stream);
    p->allocs.clear();
    if (p->forest) p->forest->release(p->last_stream);
}

int validate_opts(const lfmm_opts& o) {
    if (o.precision != LFMM_FP64 && o.precision != LFMM_MIXED && o.precision != LFMM_DF)
        return fail(LFMM_EINVAL, "opts.precision must be LFMM_FP64, LFMM_MIXED or LFMM_DF");
    if (o.p < 2 || o.p > 17) return fail(LFMM_EINVAL, "opts.p must be in [2, 17]");
    if (o.leaf_size < 1) return fail(LFMM_EINVAL, "opts.leaf_size must be >= 1");
    if (o.max_leaf_side < 1 || o.max_leaf_side > kMaxLeafSide ||
        (o.max_leaf_side & (o.max_leaf_side - 1)))
        return fail(LFMM_EINVAL, "opts.max_leaf_side must be a power of 2 in [1, 32]");
    if (o.proxies_per_edge < 8 || o.proxies_per_edge > 1024)
        return fail(LFMM_EINVAL, "opts.proxies_per_edge must be in [8, 1024]");
    if (o.tc_min_level < 0) return fail(LFMM_EINVAL, "opts.tc_min_level must be >= 0");
    if (o.tree != LFMM_TREE_AUTO && o.tree != LFMM_TREE_UNIFORM && o.tree != LFMM_TREE_PRUNED)
        return fail(LFMM_EINVAL, "opts.tree must be LFMM_TREE_AUTO, LFMM_TREE_UNIFORM or LFMM_TREE_PRUNED");
    if (o.flags & ~(LFMM_FLAG_GRAPH | LFMM_FLAG_SERIAL | LFMM_FLAG_PERSISTENT))
        return fail(LFMM_EINVAL, "opts.flags has unknown bits");
    if (o.m2l_tile != 0 && o.m2l_tile != 16 && o.m2l_tile != 32 && o.m2l_tile != 64 && o.m2l_tile != 128)
        return fail(LFMM_EINVAL, "opts.m2l_tile must be 0, 16, 32, 64 or 128");
    if (o.m2l_stages != 0 && (o.m2l_stages < 2 || o.m2l_stages > 4))
        return fail(LFMM_EINVAL, "opts.m2l_stages must be 0, 2, 3 or 4");
    if (o.m2l_split < 0 || o.m2l_split > 9) return fail(LFMM_EINVAL, "opts.m2l_split must be in [0, 9]");
    if (o.reserved != 0) return fail(LFMM_EINVAL, "opts.reserved must be 0");
    return LFMM_OK;
}

// Page-locked host words for the tree build's readbacks (one set per host thread): a
// copy into pageable memory would be staged by the driver and complete later.
int* readback_words() {
    static thread_local int* words = [] {
        void* h = nullptr;
        if (cudaMallocHost(&h, 16 * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            h = nullptr;
        }
        return (int*)h;
    }();
    return words;
}

int ilog2_ceil(int64_t v) {
    int k = 0;
    while (((int64_t)1 << k) < v) ++k;
    return k;
}

// Coordinates usable by the kernels: 8-byte aligned device memory.
int device_coords(lfmm_plan* p, const int32_t* xy, int64_t n, const int32_t** out, cudaStream_t s) {
    const bool dev = is_device_ptr(xy);
    if (dev && ((uintptr_t)xy % 8) == 0) {
        *out = xy;
        return LFMM_OK;
    }
    void* buf;
    int st = palloc(p, &buf, (size_t)n * 8, s);
    if (st) return st;
    cudaError_t e = cudaMemcpyAsync(buf, xy, (size_t)n * 8, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(LFMM_ECUDA, std::string("coordinate copy: ") + cudaGetErrorString(e));
    *out = (const int32_t*)buf;
    return LFMM_OK;
}

// Operators and workspaces of a pruned tree or forest (tree already in p->forest).
int forest_workspaces(lfmm_plan* p, cudaStream_t s) {
    int st;
    Forest& F = *p->forest;
    p->side = F.side;
    p->max_src = F.max_src;
    p->max_tgt = F.max_tgt;
    p->K = 0;
    p->L = 0;
    for (int i = 0; i < F.np; ++i) {
        p->K = std::max(p->K, (int)F.K[i]);
        p->L = std::max(p->L, (int)F.L[i]);
    }
    if (F.np == 1) {
        p->x0 = F.x0[0];
        p->y0 = F.y0[0];
    }
    p->P = 4 * (p->opts.p - 1);
    p->NP = p->P <= 32 ? 32 : 64;
    const int n_levels = std::max(1, F.kmax + 1);
    std::string err;
    ModelOps* mo = get_model_ops(F.side, p->P, p->opts.proxies_per_edge, n_levels, &err);
    if (!mo) return fail(LFMM_EINTERNAL, err);
    p->ops = get_device_ops(mo, p->opts.precision, p->NP, n_levels, s, &err);
    if (!p->ops) return fail(LFMM_ECUDA, err);
    const size_t esz = p->opts.precision == LFMM_MIXED ? sizeof(float) : sizeof(double);
    if ((st = palloc(p, &p->f_sorted, (size_t)p->ns * esz, s))) return st;
    const int64_t boxes = std::max<int64_t>(F.total_boxes, 1);
    p->n_boxes = F.total_boxes;
    if ((st = palloc(p, &p->qhat, (size_t)boxes * p->NP * esz, s))) return st;
    if ((st = palloc(p, &p->uhat, (size_t)boxes * p->NP * esz, s))) return st;
    {  // work-queue counters of the persistent sweeps
        void* c;
        if ((st = palloc(p, &c, 32 * sizeof(unsigned long long), s))) return st;
        F.sweep_ctr = (unsigned long long*)c;
    }
    {  // partial sums of the list M2L levels split along K (few boxes)
        F.m2l_split = p->opts.m2l_split;
        const int64_t sb = forest_m2l_split_bytes(F, p->NP, esz, p->num_sms, F.m2l_split);
        if (sb > 0 && (st = palloc(p, &F.m2l_part, (size_t)sb, s))) return st;
    }
    // tensor-core list M2L of the large levels (mixed path; opts.tc_min_level
    // beyond every tree level keeps them on the CUDA cores): TF32 hi / lo rows
    F.tc_list = p->opts.precision == LFMM_MIXED && p->opts.tc_min_level <= kMaxTreeLevelForTc;
    if (F.tc_list) {
        int64_t need = 0;
        const int nk = (int)F.levels.size();
        for (int k = 0; k < nk && F.kmax >= 0; ++k)
            if (F.levels[k].nb >= kTcListMinBoxes)
                need = std::max(need, m2l_tc_list_split_floats(F.levels[k].nb, k + 1 < nk ? F.levels[k + 1].nb : 0,
                                                               p->NP));
        void* b = nullptr;
        if (need > 0 && (st = palloc(p, &b, (size_t)need * sizeof(float), s))) return st;
        F.tc_split = (float*)b;
    }
    if ((st = palloc(p, &p->Qbox, (size_t)boxes * 8, s))) return st;
    if ((st = palloc(p, &p->Cbox, (size_t)boxes * 8, s))) return st;
    void* stbuf;
    if ((st = palloc(p, &stbuf, 16, s))) return st;
    p->status = (int*)stbuf;
    LFMM_CUDA_TRY(cudaMemsetAsync(p->status, 0, 16, s));  // status word + grid-barrier words
    p->tc_min_level = p->opts.tc_min_level == 0 ? kDefaultTcMinLevel : p->opts.tc_min_level;
    p->bytes += F.bytes;
    return LFMM_OK;
}

int ensure_m2l_part(lfmm_plan* p, int nvec, cudaStream_t s);

int plan_build(lfmm_plan* p, const int32_t* src_xy, const int32_t* tgt_xy, cudaStream_t s) {
    int st;
    LFMM_CUDA_TRY(cudaGetDevice(&p->device));
    LFMM_CUDA_TRY(cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device));
    setup_pool(p->device);
    const int32_t *src, *tgt;
    {
        PhaseTimer pt(LFMM_PHASE_COPY, s);
        if ((st = device_coords(p, src_xy, p->ns, &src, s))) return st;
        if ((st = device_coords(p, tgt_xy, p->nt, &tgt, s))) return st;
    }
    std::unique_ptr<PhaseTimer> tree_timer(new PhaseTimer(LFMM_PHASE_TREE, s));

    // ---- root box (Sec. 6): lower-left corner of all points, side 2^K.  The leaf level
    // is at least the pigeonhole level L_pig, known without the points; unless the
    // leaf-side bound raises it, the first level counted below is L_pig + 1.  That count
    // is launched right behind the bounding box (the kernel reads the root box on the
    // device), so one host round trip returns both; a wrong guess is counted again.
    const int nleaf = p->opts.leaf_size;
    const int64_t nmax = std::max(p->ns, p->nt);
    int L_pig = 0;
    while (((int64_t)nleaf << (2 * L_pig)) < nmax) ++L_pig;
    const int Lf_guess = L_pig + 1;
    Temp t4;
    if ((st = talloc(t4, 10 * sizeof(int), s))) return st;
    int* d4 = (int*)t4.ptr;
    Temp ranks;  // each point's arrival rank in its box of level Lf_last
    if ((st = talloc(ranks, (size_t)(p->ns + p->nt) * sizeof(int32_t), s))) return st;
    Temp guess;  // counts at level Lf_guess: [fine src][fine tgt][coarse src][coarse tgt]
    bool have_guess = Lf_guess <= kMaxLevel;
    const int64_t nf_g = have_guess ? (int64_t)1 << (2 * Lf_guess) : 0, nc_g = nf_g / 4;
    if (have_guess && (st = talloc(guess, (size_t)(2 * nf_g + 2 * nc_g) * sizeof(int32_t), s))) return st;
    // one launch sets the bounding-box words, zeroes the maxima words and the fine counts
    LFMM_CUDA_TRY(launch_init_tree(d4, (int32_t*)guess.ptr, 2 * nf_g, s));
    LFMM_CUDA_TRY(launch_bbox(src, p->ns, tgt, p->nt, d4, s));
    tree_timer->add_launches(2);
    if (have_guess) {
        int32_t* fs = (int32_t*)guess.ptr;
        LFMM_CUDA_TRY(launch_histogram_bbox(src, p->ns, tgt, p->nt, d4, Lf_guess, fs, fs + nf_g,
                                            (int32_t*)ranks.ptr, s));
        LFMM_CUDA_TRY(launch_coarsen(fs, fs + nf_g, nc_g, fs + 2 * nf_g, fs + 2 * nf_g + nc_g, d4 + 4, s));
        tree_timer->add_launches(2);
    }
    int h10[10];
    {
        int* hw = readback_words();
        int* dst = hw ? hw : h10;
        const int nw = have_guess ? 10 : 4;
        LFMM_CUDA_TRY(cudaMemcpyAsync(dst, d4, nw * sizeof(int), cudaMemcpyDeviceToHost, s));
        LFMM_CUDA_TRY(cudaStreamSynchronize(s));
        if (hw) std::copy(hw, hw + nw, h10);
    }
    p->x0 = h10[0];
    p->y0 = h10[1];
    const int64_t ext = std::max((int64_t)h10[2] - h10[0], (int64_t)h10[3] - h10[1]) + 1;
    if (ext > ((int64_t)1 << 30)) return fail(LFMM_EINVAL, "points span more than 2^30 lattice cells");
    p->K = ilog2_ceil(ext);

    // ---- leaf level: coarsest level with <= N_leaf sources and targets per box,
    // leaf side <= max_leaf_side.  Levels below the pigeonhole bound cannot qualify.
    const int L_side = std::max(0, p->K - ilog2_ceil(p->opts.max_leaf_side));
    int L_try = std::max(L_side, L_pig);
    if (L_try > p->K) L_try = p->K;
    int Lf = std::min(p->K, L_try + 1);
    Temp cnt;
    int32_t *cs = nullptr, *ct = nullptr;  // counts at the chosen level
    int32_t *fs_last = nullptr, *ft_last = nullptr;  // counts at the histogram level Lf_last
    int Lf_last = 0;
    int chosen = -1;
    int early_side = 0;    // > 0: pruned storage decided on the way, the builder's first leaf side
    int64_t nonempty = 1;  // leaves holding a source or a target at the chosen level
    for (;;) {
        if (Lf > kMaxLevel)
            return fail(LFMM_EUNSUPPORTED, "tree would need more than 4^14 leaves");
        const int64_t nf = (int64_t)1 << (2 * Lf);
        const int64_t nc = Lf >= 1 ? nf / 4 : 0;
        Temp c2;
        // [max fine src, max fine tgt, max coarse src, max coarse tgt, non-empty fine, non-empty coarse]
        int m4[6] = {(int)std::min<int64_t>(p->ns, INT_MAX), (int)std::min<int64_t>(p->nt, INT_MAX), 0, 0, 1, 1};
        if (have_guess && Lf == Lf_guess) {  // counted with the bounding box
            c2.ptr = guess.ptr;
            c2.s = s;
            guess.ptr = nullptr;
            for (int k = 0; k < 6; ++k) m4[k] = h10[4 + k];
        } else {
            if ((st = talloc(c2, (size_t)(2 * nf + 2 * nc) * sizeof(int32_t), s))) return st;
            int32_t* f0 = (int32_t*)c2.ptr;
            LFMM_CUDA_TRY(cudaMemsetAsync(f0, 0, (size_t)2 * nf * sizeof(int32_t), s));
            LFMM_CUDA_TRY(launch_histogram(src, p->ns, tgt, p->nt, p->x0, p->y0, p->K - Lf, f0, f0 + nf, s,
                                           (int32_t*)ranks.ptr));
            tree_timer->add_launches(1);
            if (Lf >= 1) {
                LFMM_CUDA_TRY(cudaMemsetAsync(d4 + 4, 0, 6 * sizeof(int), s));
                LFMM_CUDA_TRY(launch_coarsen(f0, f0 + nf, nc, f0 + 2 * nf, f0 + 2 * nf + nc, d4 + 4, s));
                tree_timer->add_launches(1);
                LFMM_CUDA_TRY(cudaMemcpyAsync(m4, d4 + 4, sizeof(m4), cudaMemcpyDeviceToHost, s));
                LFMM_CUDA_TRY(cudaStreamSynchronize(s));
            }
        }
        have_guess = false;  // a later pass counts again (and overwrites the ranks)
        int32_t* fs = (int32_t*)c2.ptr;
        int32_t* ft = fs + nf;
        int32_t* ccs = ft + nf;
        int32_t* cct = ccs + nc;
        // Clustered input: more than half of the boxes of the coarse level counted here are
        // empty, hence of every finer level too (a non-empty box has a non-empty parent), so
        // automatic storage is pruned whatever the leaf level turns out to be.  The forest
        // builder finds the leaf side itself, starting at the largest side these counts
        // leave possible; no finer (and larger) dense count is made.
        if (p->opts.tree == LFMM_TREE_AUTO && Lf >= 1 && 2 * (int64_t)m4[5] < nc) {
            if (Lf - 1 >= L_try && std::max(m4[2], m4[3]) <= nleaf) early_side = 1 << (p->K - Lf + 1);
            else if (std::max(m4[0], m4[1]) <= nleaf || Lf == p->K) early_side = 1 << (p->K - Lf);
            else early_side = 1 << std::max(0, p->K - Lf - 1);
            break;
        }
        if (Lf - 1 >= L_try && std::max(m4[2], m4[3]) <= nleaf) {
            chosen = Lf - 1;
            p->max_src = m4[2];
            p->max_tgt = m4[3];
            nonempty = m4[5];
            cs = ccs;
            ct = cct;
        } else if (std::max(m4[0], m4[1]) <= nleaf || Lf == p->K) {
            chosen = Lf;
            p->max_src = m4[0];
            p->max_tgt = m4[1];
            nonempty = m4[4];
            cs = fs;
            ct = ft;
        }
        if (chosen >= 0) {
            cnt.ptr = c2.ptr;  // keep the counts alive
            cnt.s = s;
            c2.ptr = nullptr;
            fs_last = fs;
            ft_last = ft;
            Lf_last = Lf;
            break;
        }
        const int next = std::min({p->K, Lf + 2, kMaxLevel});
        Lf = next > Lf ? next : kMaxLevel + 1;
    }
    p->L = early_side > 0 ? 0 : chosen;
    p->side = early_side > 0 ? early_side : 1 << (p->K - p->L);
    const int64_t n_leaves = (int64_t)1 << (2 * p->L);

    // ---- pruned storage: most leaves empty (or asked for)
    const bool pruned = early_side > 0 || p->opts.tree == LFMM_TREE_PRUNED ||
                        (p->opts.tree == LFMM_TREE_AUTO && 2 * nonempty < n_leaves);
    if (pruned) {
        cnt.reset_now();
        tree_timer.reset();
        PhaseTimer pt(LFMM_PHASE_TREE, s);
        p->forest.reset(new (std::nothrow) Forest());
        if (!p->forest) return fail(LFMM_ENOMEM, "host allocation failed");
        const int64_t so[2] = {0, p->ns}, to[2] = {0, p->nt};
        if ((st = forest_build(*p->forest, src, so, p->ns, tgt, to, p->nt, 1, p->opts.leaf_size, p->side, s, &pt)))
            return st;
        return forest_workspaces(p, s);
    }

    // ---- buckets
    void* buf;
    if ((st = palloc(p, &buf, (size_t)2 * (n_leaves + 1) * sizeof(int32_t), s))) return st;
    p->src_begin = (int32_t*)buf;
    p->tgt_begin = p->src_begin + (n_leaves + 1);
    Temp part;
    if ((st = talloc(part, scan_partials_size(n_leaves) * sizeof(int32_t), s))) return st;
    LFMM_CUDA_TRY(launch_scan2(cs, p->src_begin, ct, p->tgt_begin, p->L, (int32_t*)part.ptr, s));
    tree_timer->add_launches(3);
    if ((st = palloc(p, &buf, (size_t)(2 * (p->ns + p->nt) + p->nt) * sizeof(int32_t), s))) return st;
    p->src_loc = (int32_t*)buf;
    p->src_perm = p->src_loc + p->ns;
    p->tgt_loc = p->src_perm + p->ns;
    p->tgt_perm = p->tgt_loc + p->nt;
    p->tgt_leaf = p->tgt_perm + p->nt;
    // bucket by the histogram ranks (no second atomic pass): the sources on `s`, the targets
    // (read first by the near field and L2P) on the plan's second stream, which then frees
    // the ranks and counts both scatters read
    LFMM_CUDA_TRY(launch_scatter_ranked(src, p->ns, p->x0, p->y0, p->K, p->L, Lf_last, p->src_begin, fs_last,
                                        (const int32_t*)ranks.ptr, p->src_loc, p->src_perm, s));
    cudaStream_t ts = s;
    if (!(p->opts.flags & LFMM_FLAG_SERIAL) && p->L >= 2) {
        if (!p->aux) p->aux = acquire_aux(p->device);
        if (p->aux && cudaEventCreateWithFlags(&p->tgt_ready, cudaEventDisableTiming) == cudaSuccess) {
            LFMM_CUDA_TRY(cudaEventRecord(p->aux->fork, s));
            LFMM_CUDA_TRY(cudaStreamWaitEvent(p->aux->s, p->aux->fork, 0));
            ts = p->aux->s;
        } else {
            cudaGetLastError();
            p->tgt_ready = nullptr;
        }
    }
    LFMM_CUDA_TRY(launch_scatter_ranked(tgt, p->nt, p->x0, p->y0, p->K, p->L, Lf_last, p->tgt_begin, ft_last,
                                        (const int32_t*)ranks.ptr + p->ns, p->tgt_loc, p->tgt_perm, ts, p->tgt_leaf));
    if (ts != s) {
        LFMM_CUDA_TRY(cudaEventRecord(p->tgt_ready, ts));
        ranks.s = ts;  // freed behind the target scatter
        cnt.s = ts;
    }
    tree_timer->add_launches(2);
    tree_timer.reset();
    PhaseTimer op_timer(LFMM_PHASE_OPERATORS, s);

    // ---- operators of the model boxes (cached across plans)
    p->P = 4 * (p->opts.p - 1);
    p->NP = p->P <= 32 ? 32 : 64;
    const int n_levels = std::max(1, p->L - 1);
    std::string err;
    ModelOps* mo = get_model_ops(p->side, p->P, p->opts.proxies_per_edge, n_levels, &err);
    if (!mo) return fail(LFMM_EINTERNAL, err);
    p->ops = get_device_ops(mo, p->opts.precision, p->NP, n_levels, s, &err);
    if (!p->ops) return fail(LFMM_ECUDA, err);

    // ---- workspaces: sorted charges, expansions of levels min(2,L)..L
    const size_t esz = p->opts.precision == LFMM_MIXED ? sizeof(float) : sizeof(double);
    if ((st = palloc(p, &p->f_sorted, (size_t)p->ns * esz, s))) return st;
    p->lvl_off.assign(p->L + 2, 0);
    int64_t boxes = 0;
    for (int l = std::min(2, p->L); l <= p->L; ++l) {
        p->lvl_off[l] = boxes;
        boxes += (int64_t)1 << (2 * l);
    }
    p->n_boxes = boxes;
    if (p->opts.precision == LFMM_MIXED && p->L >= (p->opts.tc_min_level == 0 ? kDefaultTcMinLevel : p->opts.tc_min_level)) {
        // largest tensor-core level: TF32 hi/lo of its q_hat and of its parent's u_hat
        const size_t n = ((size_t)p->NP << (2 * p->L)) * 2 + ((size_t)p->NP << (2 * std::max(0, p->L - 1))) * 2;
        if ((st = palloc(p, &p->tc_split, n * sizeof(float), s))) return st;
    }
    if ((st = palloc(p, &p->qhat, (size_t)boxes * p->NP * esz, s))) return st;
    if ((st = palloc(p, &p->uhat, (size_t)boxes * p->NP * esz, s))) return st;
    if ((st = palloc(p, &p->Qbox, (size_t)boxes * 8, s))) return st;
    if ((st = palloc(p, &p->Cbox, (size_t)boxes * 8, s))) return st;
    if (p->L >= 2) {  // a far field: near and far parts go to these buffers, then one sum
        void* b;
        if ((st = palloc(p, &b, (size_t)2 * p->nt * sizeof(double), s))) return st;
        p->un_tmp = (double*)b;
        p->uf_tmp = p->un_tmp + p->nt;
    }
    void* stbuf;
    if ((st = palloc(p, &stbuf, 16, s))) return st;
    p->status = (int*)stbuf;
    LFMM_CUDA_TRY(cudaMemsetAsync(p->status, 0, 16, s));  // status word + grid-barrier words
    p->tc_min_level = p->opts.tc_min_level == 0 ? kDefaultTcMinLevel : p->opts.tc_min_level;
    // the one-vector partial sums of the K-split coarse-level M2L belong to the plan from
    // the start, so that device_bytes counts them before the first evaluation
    if ((st = ensure_m2l_part(p, 1, s))) return st;
    // no final synchronisation: temporaries are freed in stream order, and the host
    // buffers of copied coordinates were read before the root-box readback
    return LFMM_OK;
}

TreeView tree_view(const lfmm_plan* p) {
    TreeView t;
    t.L = p->L;
    t.side = p->side;
    t.n_leaves = (int64_t)1 << (2 * p->L);
    t.src_begin = p->src_begin;
    t.tgt_begin = p->tgt_begin;
    t.src_loc = p->src_loc;
    t.src_perm = p->src_perm;
    t.tgt_loc = p->tgt_loc;
    t.tgt_perm = p->tgt_perm;
    t.tgt_leaf = p->tgt_leaf;
    t.n_tgt = p->nt;
    t.n_src_all = p->ns;
    t.max_leaf_src = p->max_src;
    t.max_leaf_tgt = p->max_tgt;
    return t;
}

// Expansion arrays of one or more charge vectors: vector v's q_hat / u_hat start v vq
// elements, its Q / C v vQ value pairs after vector 0's.
struct FarBufs {
    void *q, *u, *Q, *C;
    float* split;
    int nvec;
    int64_t vq, vQ;
};

FarBufs plan_far_bufs(lfmm_plan* p) {
    return FarBufs{p->qhat, p->uhat, p->Qbox, p->Cbox, (float*)p->tc_split, 1, 0, 0};
}

// M2M, M2L and L2L of a uniform plan (Sec. 8.2 steps 2-4), from the leaf expansions the
// P2M left in b.q / b.Q to the leaf incoming expansions in b.u / b.C, for b.nvec
// vectors at once (the fused coarse-level kernels and the tensor-core M2L take them in
// one launch; the per-level fallbacks loop).  `before_fine` runs after the cooperative
// coarse-level kernels, before the per-level launches (the near field is forked there).
template <typename T, typename Hook>
int far_sweeps(lfmm_plan* p, const FarBufs& b, cudaStream_t s, Hook before_fine) {
    const DeviceOps& ops = *p->ops;
    const int NP = p->NP;
    const int L = p->L;
    using V8 = char[8];
    auto Qx = [&](int l, int v) { return (T*)b.q + v * b.vq + (size_t)p->lvl_off[l] * NP; };
    auto Ux = [&](int l, int v) { return (T*)b.u + v * b.vq + (size_t)p->lvl_off[l] * NP; };
    auto Qm = [&](int l, int v) { return (void*)((V8*)b.Q + v * b.vQ + (size_t)p->lvl_off[l]); };
    auto Cm = [&](int l, int v) { return (void*)((V8*)b.C + v * b.vQ + (size_t)p->lvl_off[l]); };
    LevelBufs lb;
    for (int l = std::min(2, L); l <= L && l < 16; ++l) {
        lb.q[l] = Qx(l, 0);
        lb.u[l] = Ux(l, 0);
        lb.Q[l] = Qm(l, 0);
        lb.C[l] = Cm(l, 0);
    }
    lb.nvec = b.nvec;
    lb.vq = b.vq;
    lb.vQ = b.vQ;
    lb.part = p->m2l_part;
    lb.part_bytes = p->m2l_part_bytes;
    unsigned* gsync = (unsigned*)(p->status + 1);  // grid-barrier words beside the status word
    {
        PhaseTimer pt(LFMM_PHASE_M2M, s);
        if (L >= 3 && launch_m2m_fused<T>(ops, L, lb, gsync, p->status, p->num_sms, s) == cudaSuccess) {
            pt.add_launches(1);
        } else {
            for (int v = 0; v < b.nvec; ++v)
                for (int l = L - 1; l >= 2; --l) {
                    LFMM_CUDA_TRY(launch_m2m<T>(ops, L - l, l, Qx(l + 1, v), Qm(l + 1, v), Qx(l, v), Qm(l, v), s));
                    pt.add_launches(1);
                }
        }
    }
    int l_first = 2;  // first level left for the per-level M2L launches
    if (L >= 2) {
        PhaseTimer pt(LFMM_PHASE_M2L, s);
        int last = 1;
        if (launch_m2l_fused<T>(ops, L, lb, p->tc_min_level, gsync, p->status, p->num_sms, &last, s,
                                p->opts.m2l_split) == cudaSuccess) {
            pt.add_launches(1);
            l_first = last + 1;
        }
    }
    {
        const int st = before_fine();
        if (st) return st;
    }
    for (int l = l_first; l <= L; ++l) {
        const bool tc = m2l_uses_tc(ops, L - l, l, p->tc_min_level, sizeof(T) == 4);
        PhaseTimer pt(tc ? LFMM_PHASE_M2L_TC : LFMM_PHASE_M2L, s);
        if constexpr (sizeof(T) == 4) {
            if (tc) {
                LFMM_CUDA_TRY(launch_m2l_tma(ops, L - l, l, (const float*)Qx(l, 0), Qm(l, 0),
                                             l >= 3 ? (const float*)Ux(l - 1, 0) : nullptr,
                                             l >= 3 ? Cm(l - 1, 0) : nullptr, (float*)Ux(l, 0), Cm(l, 0), b.split,
                                             p->status, p->num_sms, s, b.nvec, b.vq, b.vQ, p->opts.m2l_tile,
                                             p->opts.m2l_stages));
                pt.add_launches(2);
                continue;
            }
        }
        for (int v = 0; v < b.nvec; ++v) {
            LFMM_CUDA_TRY(launch_m2l<T>(ops, L - l, l, Qx(l, v), Qm(l, v), l >= 3 ? Ux(l - 1, v) : nullptr,
                                        l >= 3 ? Cm(l - 1, v) : nullptr, Ux(l, v), Cm(l, v), s));
            pt.add_launches(1);
        }
    }
    return LFMM_OK;
}

template <typename T>
int eval_impl(lfmm_plan* p, const double* f, double* u, double* un, double* uf, cudaStream_t s) {
    if (p->forest)
        return forest_eval<T>(*p->forest, *p->ops, f, (T*)p->f_sorted, (T*)p->qhat, (T*)p->uhat, p->Qbox, p->Cbox,
                              u, un, uf, p->num_sms, s, p->status, (p->opts.flags & LFMM_FLAG_PERSISTENT) != 0);
    const TreeView t = tree_view(p);
    const DeviceOps& ops = *p->ops;
    const int NP = p->NP;
    const int L = p->L;
    const size_t leaf_off = (size_t)p->lvl_off[L];
    T* q_leaf = (T*)p->qhat + leaf_off * NP;
    T* u_leaf = (T*)p->uhat + leaf_off * NP;
    void* Q_leaf = (char*)p->Qbox + leaf_off * 8;
    void* C_leaf = (char*)p->Cbox + leaf_off * 8;
    {
        PhaseTimer pt(LFMM_PHASE_P2M, s);
        LFMM_CUDA_TRY(launch_p2m<T>(t, ops, f, (T*)p->f_sorted, q_leaf, Q_leaf, s));
        pt.add_launches(1);
    }
    // The near field depends only on the sorted charges and the leaf charges (P2M): it
    // runs on the plan's second stream beside the per-level M2L launches and the L2P
    // (after the cooperative coarse-level kernels, which need the whole device), and
    // one elementwise sum joins the two.  With LFMM_FLAG_SERIAL the same kernels run in
    // the same order on `s` alone.
    const bool split = L >= 2 && p->un_tmp != nullptr;
    if (split && !(p->opts.flags & LFMM_FLAG_SERIAL) && !p->aux) p->aux = acquire_aux(p->device);
    const bool concurrent = split && !(p->opts.flags & LFMM_FLAG_SERIAL) && p->aux != nullptr;
    cudaStream_t near_s = concurrent ? p->aux->s : s;
    auto near = [&]() -> int {
        if (!split) return LFMM_OK;
        if (concurrent) {
            LFMM_CUDA_TRY(cudaEventRecord(p->aux->fork, s));
            LFMM_CUDA_TRY(cudaStreamWaitEvent(p->aux->s, p->aux->fork, 0));
        }
        {
            const int st = wait_targets(p, near_s);
            if (st) return st;
        }
        PhaseTimer pt(LFMM_PHASE_P2P, near_s);
        LFMM_CUDA_TRY(launch_p2p_l2p<T>(t, ops, (const T*)p->f_sorted, nullptr, nullptr, Q_leaf, nullptr, p->un_tmp,
                                        nullptr, p->num_sms, near_s));
        pt.add_launches(1);
        return LFMM_OK;
    };
    {
        const int st = far_sweeps<T>(p, plan_far_bufs(p), s, near);
        if (st) return st;
    }
    if (split) {
        {
            const int st = wait_targets(p, s);
            if (st) return st;
            PhaseTimer pt(LFMM_PHASE_L2P, s);
            LFMM_CUDA_TRY(launch_l2p<T>(t, ops, u_leaf, C_leaf, p->uf_tmp, s));
            pt.add_launches(1);
        }
        if (concurrent) {
            LFMM_CUDA_TRY(cudaEventRecord(p->aux->join, p->aux->s));
            LFMM_CUDA_TRY(cudaStreamWaitEvent(s, p->aux->join, 0));
        }
        PhaseTimer pt(LFMM_PHASE_L2P, s);
        LFMM_CUDA_TRY(launch_combine(p->nt, p->un_tmp, p->uf_tmp, u, un, uf, s));
        pt.add_launches(1);
    } else {
        const int st = wait_targets(p, s);
        if (st) return st;
        PhaseTimer pt(LFMM_PHASE_P2P, s);
        LFMM_CUDA_TRY(launch_p2p_l2p<T>(t, ops, (const T*)p->f_sorted, nullptr, nullptr, Q_leaf, u, un, uf,
                                        p->num_sms, s));
        pt.add_launches(1);
    }
    return LFMM_OK;
}

// Charge vectors evaluated together by lfmm_eval_multi (the per-vector buffers hold
// this many).
constexpr int kMultiGroup = 16;

// k charge vectors on one uniform plan, in groups of up to kMultiGroup: P2M, the
// far-field sweeps and L2P take a group's vectors in one launch each (per-vector
// expansion arrays), the near field four vectors per pass sharing each table lookup,
// and one binary64 sum writes the group's results.  Every vector's arithmetic is that
// of lfmm_eval, so the results are bit-identical.
template <typename T>
int eval_multi_impl(lfmm_plan* p, const double* F, int k, double* U, cudaStream_t s) {
    const int L = p->L;
    {
        const int st = wait_targets(p, s);
        if (st) return st;
    }
    if (p->forest || L < 2 || !p->un_tmp) {  // one vector at a time
        for (int r = 0; r < k; ++r) {
            const int st = eval_impl<T>(p, F + (size_t)r * p->ns, U + (size_t)r * p->nt, nullptr, nullptr, s);
            if (st) return st;
        }
        return LFMM_OK;
    }
    const TreeView t = tree_view(p);
    const DeviceOps& ops = *p->ops;
    const int NP = p->NP;
    const size_t leaf_off = (size_t)p->lvl_off[L];
    const int64_t vq = p->n_boxes * NP, vQ = p->n_boxes;
    T* fs = (T*)p->m_fsorted;
    T* mq = (T*)p->m_qhat;
    T* mu = (T*)p->m_uhat;
    char* mQ = (char*)p->m_Q;
    char* mC = (char*)p->m_C;
    for (int r0 = 0; r0 < k; r0 += kMultiGroup) {
        const int g = std::min(kMultiGroup, k - r0);
        {
            PhaseTimer pt(LFMM_PHASE_P2M, s);
            LFMM_CUDA_TRY(launch_p2m<T>(t, ops, F + (size_t)r0 * p->ns, fs, mq + leaf_off * NP, mQ + leaf_off * 8, s,
                                        g, vq, vQ));
            pt.add_launches(1);
        }
        const FarBufs fb{mq, mu, mQ, mC, (float*)p->m_split, g, vq, vQ};
        const int st = far_sweeps<T>(p, fb, s, [] { return LFMM_OK; });
        if (st) return st;
        {
            PhaseTimer pt(LFMM_PHASE_L2P, s);
            LFMM_CUDA_TRY(launch_l2p<T>(t, ops, mu + leaf_off * NP, mC + leaf_off * 8, p->m_uf, s, g, vq, vQ));
            pt.add_launches(1);
        }
        {
            PhaseTimer pt(LFMM_PHASE_P2P, s);
            LFMM_CUDA_TRY(launch_p2p_multi<T>(t, ops, g, fs, p->ns, mQ + leaf_off * 8, vQ, p->m_un, p->nt,
                                              p->num_sms, s));
            pt.add_launches((g + 3) / 4);
        }
        PhaseTimer pt(LFMM_PHASE_L2P, s);
        LFMM_CUDA_TRY(launch_combine((int64_t)g * p->nt, p->m_un, p->m_uf, U + (size_t)r0 * p->nt, nullptr, nullptr,
                                     s));
        pt.add_launches(1);
    }
    return LFMM_OK;
}

int eval_dispatch(lfmm_plan* p, const double* f, double* const out[3], cudaStream_t s) {
    return p->opts.precision == LFMM_MIXED ? eval_impl<float>(p, f, out[0], out[1], out[2], s)
           : p->opts.precision == LFMM_DF  ? eval_impl<DF>(p, f, out[0], out[1], out[2], s)
                                           : eval_impl<double>(p, f, out[0], out[1], out[2], s);
}

// Graph form of one evaluation.  The launch sequence depends only on the plan and the
// argument pointers, so a graph recorded once replays it exactly.  Recording happens on
// a plan-owned stream (the caller's may be the legacy default stream, which cannot be
// captured); the executable graph is launched on the caller's stream, after whatever
// the caller queued there.
int eval_graph(lfmm_plan* p, const double* f, double* const out[3], cudaStream_t s) {
    const bool same = p->graph && p->graph_f == f && p->graph_out[0] == out[0] && p->graph_out[1] == out[1] &&
                      p->graph_out[2] == out[2];
    if (!same) {
        if (!p->cap_stream) LFMM_CUDA_TRY(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
        LFMM_CUDA_TRY(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
        const int st = eval_dispatch(p, f, out, p->cap_stream);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(p->cap_stream, &g);
        if (st || e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return st ? st : fail(LFMM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        }
        if (p->graph) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(p->graph, g, &info) != cudaSuccess) {
                cudaGetLastError();
                cudaGraphExecDestroy(p->graph);
                p->graph = nullptr;
            }
        }
        if (!p->graph) {
            const cudaError_t ei = cudaGraphInstantiate(&p->graph, g, 0);
            if (ei != cudaSuccess) {
                cudaGraphDestroy(g);
                p->graph = nullptr;
                cudaGetLastError();
                return fail(LFMM_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei));
            }
        }
        cudaGraphDestroy(g);
        p->graph_f = f;
        for (int i = 0; i < 3; ++i) p->graph_out[i] = out[i];
    }
    {
        const int st = wait_targets(p, s);
        if (st) return st;
    }
    LFMM_CUDA_TRY(cudaGraphLaunch(p->graph, s));
    return LFMM_OK;
}

// Room for the partial sums of the K-split fused small-level M2L for nvec vectors
// (plan-owned, allocated before any evaluation or graph capture needs it).
int ensure_m2l_part(lfmm_plan* p, int nvec, cudaStream_t s) {
    if (p->forest || p->L < 2 || !p->ops || nvec <= p->m2l_part_nvec) return LFMM_OK;
    const int64_t need =
        p->opts.precision == LFMM_MIXED
            ? m2l_fused_split_bytes<float>(*p->ops, p->L, p->tc_min_level, p->num_sms, nvec, p->opts.m2l_split)
        : p->opts.precision == LFMM_DF
            ? m2l_fused_split_bytes<DF>(*p->ops, p->L, p->tc_min_level, p->num_sms, nvec, p->opts.m2l_split)
            : m2l_fused_split_bytes<double>(*p->ops, p->L, p->tc_min_level, p->num_sms, nvec, p->opts.m2l_split);
    if (need > p->m2l_part_bytes) {
        void* b;
        const int st = palloc(p, &b, (size_t)need, s);
        if (st) return st;
        p->m2l_part = b;
        p->m2l_part_bytes = need;
    }
    p->m2l_part_nvec = nvec;
    return LFMM_OK;
}

int eval_common(lfmm_plan* p, const double* f, double* u, double* un, double* uf, void* stream) {
    if (!p || !f) return fail(LFMM_EINVAL, "NULL plan or f");
    if (!u && !un && !uf) return fail(LFMM_EINVAL, "no output");
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    {
        const int st = ensure_m2l_part(p, 1, s);
        if (st) return st;
    }
    const double* fd = f;
    if (!is_device_ptr(f)) {
        if (!p->f_stage) {
            void* b;
            int st = palloc(p, &b, (size_t)p->ns * sizeof(double), s);
            if (st) return st;
            p->f_stage = (double*)b;
        }
        PhaseTimer pt(LFMM_PHASE_COPY, s);
        LFMM_CUDA_TRY(cudaMemcpyAsync(p->f_stage, f, (size_t)p->ns * sizeof(double), cudaMemcpyHostToDevice, s));
        fd = p->f_stage;
    }
    double* outs[3] = {u, un, uf};
    double* douts[3] = {u, un, uf};
    bool host_out[3] = {false, false, false};
    for (int i = 0; i < 3; ++i) {
        if (!outs[i] || is_device_ptr(outs[i])) continue;
        if (!p->u_stage) {
            void* b;
            int st = palloc(p, &b, (size_t)3 * p->nt * sizeof(double), s);
            if (st) return st;
            p->u_stage = (double*)b;
        }
        douts[i] = p->u_stage + (size_t)i * p->nt;
        host_out[i] = true;
    }
    const int st = (p->opts.flags & LFMM_FLAG_GRAPH) && !profiling_enabled() ? eval_graph(p, fd, douts, s)
                                                                               : eval_dispatch(p, fd, douts, s);
    if (st) return st;
    bool any_host = false;
    {
        PhaseTimer pt(LFMM_PHASE_COPY, s);
        for (int i = 0; i < 3; ++i)
            if (host_out[i]) {
                LFMM_CUDA_TRY(cudaMemcpyAsync(outs[i], douts[i], (size_t)p->nt * sizeof(double),
                                              cudaMemcpyDeviceToHost, s));
                any_host = true;
            }
    }
    if (any_host) LFMM_CUDA_TRY(cudaStreamSynchronize(s));
    if (profiling_enabled()) profile_flush();
    return LFMM_OK;
}

}  // namespace

extern "C" {

void lfmm_opts_default(lfmm_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = LFMM_MIXED;
    o->p = 8;
    o->leaf_size = 64;
    o->max_leaf_side = 32;
    o->proxies_per_edge = 64;
}

int lfmm_plan_create(lfmm_plan** plan, const int32_t* src_xy, int64_t n_src, const int32_t* tgt_xy,
                     int64_t n_tgt, const lfmm_opts* opts, void* stream) {
    if (!plan) return fail(LFMM_EINVAL, "NULL plan out-pointer");
    *plan = nullptr;
    if (!src_xy || !tgt_xy) return fail(LFMM_EINVAL, "NULL coordinates");
    if (n_src < 1 || n_tgt < 1 || n_src > INT32_MAX / 2 || n_tgt > INT32_MAX / 2)
        return fail(LFMM_EINVAL, "n_src and n_tgt must be in [1, 2^30)");
    lfmm_opts o;
    if (opts) o = *opts;
    else lfmm_opts_default(&o);
    int st = validate_opts(o);
    if (st) return st;
    lfmm_plan* p = new (std::nothrow) lfmm_plan();
    if (!p) return fail(LFMM_ENOMEM, "host allocation failed");
    p->opts = o;
    p->ns = n_src;
    p->nt = n_tgt;
    p->last_stream = (cudaStream_t)stream;
    st = plan_build(p, src_xy, tgt_xy, (cudaStream_t)stream);
    if (st) {
        // the target scatter may still run on the second stream: it ends before the buffers go
        if (p->tgt_ready) cudaEventSynchronize(p->tgt_ready);
        cudaStreamSynchronize((cudaStream_t)stream);
        cudaGetLastError();
        free_plan_buffers(p);
        if (p->tgt_ready) cudaEventDestroy(p->tgt_ready);
        release_aux(p->aux);
        delete p;
        return st;
    }
    set_error("");
    if (profiling_enabled()) profile_flush();
    *plan = p;
    return LFMM_OK;
}

int lfmm_eval(lfmm_plan* plan, const double* f, double* u, void* stream) {
    return eval_common(plan, f, u, nullptr, nullptr, stream);
}

int lfmm_eval_parts(lfmm_plan* plan, const double* f, double* u_near, double* u_far, void* stream) {
    if (!u_near || !u_far) return fail(LFMM_EINVAL, "NULL output");
    return eval_common(plan, f, nullptr, u_near, u_far, stream);
}

int lfmm_plan_destroy(lfmm_plan* plan) {
    if (!plan) return LFMM_OK;
    if (plan->tgt_ready) cudaStreamWaitEvent(plan->last_stream, plan->tgt_ready, 0);
    free_plan_buffers(plan);
    cudaError_t e = cudaStreamSynchronize(plan->last_stream);
    if (plan->tgt_ready) cudaEventDestroy(plan->tgt_ready);
    if (plan->graph) cudaGraphExecDestroy(plan->graph);
    if (plan->cap_stream) cudaStreamDestroy(plan->cap_stream);
    release_aux(plan->aux);
    delete plan;
    if (e != cudaSuccess) return fail(LFMM_ECUDA, std::string("plan destroy: ") + cudaGetErrorString(e));
    return LFMM_OK;
}

int lfmm_solve(const int32_t* src_xy, int64_t n_src, const int32_t* tgt_xy, int64_t n_tgt, const double* f,
               double* u, const lfmm_opts* opts, void* stream) {
    if (!src_xy || !tgt_xy || !f || !u) return fail(LFMM_EINVAL, "NULL argument");
    if (n_src < 1 || n_tgt < 1 || n_src > INT32_MAX / 2 || n_tgt > INT32_MAX / 2)
        return fail(LFMM_EINVAL, "n_src and n_tgt must be in [1, 2^30)");
    cudaStream_t s = (cudaStream_t)stream;
    int device = 0;
    LFMM_CUDA_TRY(cudaGetDevice(&device));
    setup_pool(device);
    std::vector<void*> temps;
    auto release = [&]() {
        for (void* t : temps) cudaFreeAsync(t, s);
    };
    auto upload = [&](const void* h, size_t bytes, cudaStream_t on, void** d) -> int {
        LFMM_CUDA_TRY(dev_malloc(d, bytes, s));
        temps.push_back(*d);
        LFMM_CUDA_TRY(cudaMemcpyAsync(*d, h, bytes, cudaMemcpyHostToDevice, on));
        return LFMM_OK;
    };
    int st = LFMM_OK;
    const int32_t* sd = src_xy;
    const int32_t* td = tgt_xy;
    const double* fd = f;
    AuxStream* aux = nullptr;
    {
        PhaseTimer pt(LFMM_PHASE_COPY, s);
        void* d;
        if (!is_device_ptr(src_xy)) {
            if ((st = upload(src_xy, (size_t)n_src * 2 * sizeof(int32_t), s, &d))) return release(), st;
            sd = (const int32_t*)d;
        }
        if (!is_device_ptr(tgt_xy)) {
            if ((st = upload(tgt_xy, (size_t)n_tgt * 2 * sizeof(int32_t), s, &d))) return release(), st;
            td = (const int32_t*)d;
        }
        if (!is_device_ptr(f)) {
            // f behind the coordinates on a second stream: it lands while the tree is built
            aux = acquire_aux(device);
            cudaStream_t fs = s;
            if (aux) {
                LFMM_CUDA_TRY(cudaEventRecord(aux->fork, s));
                LFMM_CUDA_TRY(cudaStreamWaitEvent(aux->s, aux->fork, 0));
                fs = aux->s;
            }
            if ((st = upload(f, (size_t)n_src * sizeof(double), fs, &d))) {
                release_aux(aux);
                return release(), st;
            }
            fd = (const double*)d;
            if (aux) LFMM_CUDA_TRY(cudaEventRecord(aux->join, aux->s));
        }
    }
    // a host u is written by one copy from a device temporary, so that everything up to
    // the plan's release is queued before the host waits (once, in lfmm_plan_destroy)
    double* ud = u;
    if (!is_device_ptr(u)) {
        void* d;
        const cudaError_t e = dev_malloc(&d, (size_t)n_tgt * sizeof(double), s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (aux) {
                cudaStreamWaitEvent(s, aux->join, 0);
                cudaStreamSynchronize(s);
                release_aux(aux);
            }
            release();
            return fail(LFMM_ENOMEM, std::string("temporary allocation failed: ") + cudaGetErrorString(e));
        }
        temps.push_back(d);
        ud = (double*)d;
    }
    lfmm_plan* plan = nullptr;
    st = lfmm_plan_create(&plan, sd, n_src, td, n_tgt, opts, stream);
    if (!st) {
        if (aux) cudaStreamWaitEvent(s, aux->join, 0);
        st = lfmm_eval(plan, fd, ud, stream);
    }
    if (!st && ud != u) {
        const cudaError_t e = cudaMemcpyAsync(u, ud, (size_t)n_tgt * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            st = fail(LFMM_ECUDA, std::string("result copy: ") + cudaGetErrorString(e));
        }
    }
    if (aux) cudaStreamWaitEvent(s, aux->join, 0);  // the upload is done before its buffer is freed
    release();                                       // in stream order, behind the result copy
    int st2 = LFMM_OK;
    if (plan) {
        st2 = lfmm_plan_destroy(plan);  // frees in stream order, then waits for the stream
    } else {
        const cudaError_t e = cudaStreamSynchronize(s);  // host inputs were read, host output written
        if (e != cudaSuccess) {
            cudaGetLastError();
            st2 = fail(LFMM_ECUDA, std::string("solve: ") + cudaGetErrorString(e));
        }
    }
    release_aux(aux);
    return st ? st : st2;
}

int lfmm_eval_multi(lfmm_plan* p, const double* F, int32_t k, double* U, void* stream) {
    if (!p || !F || !U) return fail(LFMM_EINVAL, "NULL plan, F or U");
    if (k < 1 || k > 4096) return fail(LFMM_EINVAL, "k must be in [1, 4096]");
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    int st;
    const bool uniform = !p->forest && p->L >= 2 && p->un_tmp;
    const int group = std::min(k, kMultiGroup);
    if (uniform && (st = ensure_m2l_part(p, group, s))) return st;
    if (uniform && p->multi_cap < group) {
        // per-vector buffers for one group (allocated once per plan and size)
        const size_t esz = p->opts.precision == LFMM_MIXED ? sizeof(float) : sizeof(double);
        const size_t g = (size_t)group;
        const size_t split = p->tc_split ? ((size_t)p->NP << (2 * p->L)) * 2 + ((size_t)p->NP << (2 * (p->L - 1))) * 2
                                         : 0;
        void *a, *bq, *bu, *bQ, *bC, *c, *d = nullptr;
        if ((st = palloc(p, &a, g * p->ns * esz, s))) return st;
        if ((st = palloc(p, &bq, g * p->n_boxes * p->NP * esz, s))) return st;
        if ((st = palloc(p, &bu, g * p->n_boxes * p->NP * esz, s))) return st;
        if ((st = palloc(p, &bQ, g * p->n_boxes * 8, s))) return st;
        if ((st = palloc(p, &bC, g * p->n_boxes * 8, s))) return st;
        if ((st = palloc(p, &c, (size_t)2 * g * p->nt * sizeof(double), s))) return st;
        if (split && (st = palloc(p, &d, g * split * sizeof(float), s))) return st;
        p->m_fsorted = a;
        p->m_qhat = bq;
        p->m_uhat = bu;
        p->m_Q = bQ;
        p->m_C = bC;
        p->m_split = d;
        p->m_un = (double*)c;
        p->m_uf = p->m_un + g * p->nt;
        p->multi_cap = group;
    }
    const double* Fd = F;
    double* Ud = U;
    const bool host_f = !is_device_ptr(F), host_u = !is_device_ptr(U);
    if ((host_f || host_u) && p->host_cap < k) {
        void *a, *b;
        if ((st = palloc(p, &a, (size_t)k * p->ns * sizeof(double), s))) return st;
        if ((st = palloc(p, &b, (size_t)k * p->nt * sizeof(double), s))) return st;
        p->m_fstage = (double*)a;
        p->m_ustage = (double*)b;
        p->host_cap = k;
    }
    if (host_f) {
        PhaseTimer pt(LFMM_PHASE_COPY, s);
        LFMM_CUDA_TRY(cudaMemcpyAsync(p->m_fstage, F, (size_t)k * p->ns * sizeof(double), cudaMemcpyHostToDevice, s));
        Fd = p->m_fstage;
    }
    if (host_u) Ud = p->m_ustage;
    st = p->opts.precision == LFMM_MIXED ? eval_multi_impl<float>(p, Fd, k, Ud, s)
         : p->opts.precision == LFMM_DF  ? eval_multi_impl<DF>(p, Fd, k, Ud, s)
                                         : eval_multi_impl<double>(p, Fd, k, Ud, s);
    if (st) return st;
    if (host_u) {
        PhaseTimer pt(LFMM_PHASE_COPY, s);
        LFMM_CUDA_TRY(cudaMemcpyAsync(U, Ud, (size_t)k * p->nt * sizeof(double), cudaMemcpyDeviceToHost, s));
        LFMM_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (profiling_enabled()) profile_flush();
    return LFMM_OK;
}

int lfmm_plan_set_flags(lfmm_plan* p, int32_t flags) {
    if (!p) return fail(LFMM_EINVAL, "NULL plan");
    if (flags & ~(LFMM_FLAG_GRAPH | LFMM_FLAG_SERIAL | LFMM_FLAG_PERSISTENT))
        return fail(LFMM_EINVAL, "flags has unknown bits");
    if (flags != p->opts.flags && p->graph) {
        // the recorded launch sequence depends on the flags
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
    }
    p->opts.flags = flags;
    return LFMM_OK;
}

int lfmm_plan_status(lfmm_plan* p, void* stream) {
    if (!p) return fail(LFMM_EINVAL, "NULL plan");
    int h = 0;
    LFMM_CUDA_TRY(cudaMemcpyAsync(&h, p->status, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    LFMM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    if (h != LFMM_OK) {
        // status word and the grid-barrier words (a barrier that gave up may leave them
        // set); the fourth word, the wait budget, stays
        LFMM_CUDA_TRY(cudaMemsetAsync(p->status, 0, 12, (cudaStream_t)stream));
        LFMM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
        return fail(h, "a bounded device-side wait gave up; results of the affected evaluation are invalid");
    }
    return LFMM_OK;
}

int lfmm_plan_set_wait_budget(lfmm_plan* p, int32_t polls) {
    if (!p) return fail(LFMM_EINVAL, "NULL plan");
    if (polls < 0) return fail(LFMM_EINVAL, "polls must be >= 0");
    // the fourth word of the status buffer (status, barrier count, barrier generation, budget)
    LFMM_CUDA_TRY(cudaMemcpyAsync(p->status + 3, &polls, sizeof(int32_t), cudaMemcpyHostToDevice, p->last_stream));
    LFMM_CUDA_TRY(cudaStreamSynchronize(p->last_stream));
    return LFMM_OK;
}

int lfmm_plan_inject_barrier_stall(lfmm_plan* p) {
    if (!p) return fail(LFMM_EINVAL, "NULL plan");
    // an arrival count far beyond any grid: no arrival ever completes the barrier
    const uint32_t far = 0x80000000u;
    LFMM_CUDA_TRY(cudaMemcpyAsync(p->status + 1, &far, sizeof(uint32_t), cudaMemcpyHostToDevice, p->last_stream));
    LFMM_CUDA_TRY(cudaStreamSynchronize(p->last_stream));
    return LFMM_OK;
}

int lfmm_pool_used_bytes(int64_t* bytes) {
    if (!bytes) return fail(LFMM_EINVAL, "NULL argument");
    int dev = 0;
    LFMM_CUDA_TRY(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    LFMM_CUDA_TRY(cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t used = 0;
    LFMM_CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
    *bytes = (int64_t)used;
    return LFMM_OK;
}

int lfmm_fault_inject_alloc(int64_t nth) {
    if (nth < 0) return fail(LFMM_EINVAL, "nth must be >= 0");
    g_alloc_fail_in.store(nth);
    return LFMM_OK;
}

int lfmm_plan_get_info(const lfmm_plan* p, lfmm_plan_info* info) {
    if (!p || !info) return fail(LFMM_EINVAL, "NULL argument");
    info->n_src = p->ns;
    info->n_tgt = p->nt;
    info->x0 = p->x0;
    info->y0 = p->y0;
    info->K = p->K;
    info->L = p->L;
    info->leaf_side = p->side;
    info->P = p->ops ? p->P : 0;
    info->P_pad = p->NP;
    info->precision = p->opts.precision;
    info->max_leaf_src = p->max_src;
    info->max_leaf_tgt = p->max_tgt;
    info->device_bytes = p->bytes;
    info->tree = p->forest ? LFMM_TREE_PRUNED : LFMM_TREE_UNIFORM;
    info->n_problems = p->forest ? p->forest->np : 1;
    info->n_boxes = p->n_boxes;
    return LFMM_OK;
}

int lfmm_forest_create(lfmm_plan** plan, const int32_t* src_xy, const int64_t* src_offsets, const int32_t* tgt_xy,
                       const int64_t* tgt_offsets, int64_t n_problems, const lfmm_opts* opts, void* stream) {
    if (!plan) return fail(LFMM_EINVAL, "NULL plan out-pointer");
    *plan = nullptr;
    if (!src_xy || !tgt_xy || !src_offsets || !tgt_offsets) return fail(LFMM_EINVAL, "NULL argument");
    if (n_problems < 1 || n_problems > (1 << 24)) return fail(LFMM_EINVAL, "n_problems must be in [1, 2^24]");
    if (src_offsets[0] != 0 || tgt_offsets[0] != 0) return fail(LFMM_EINVAL, "offsets must start at 0");
    for (int64_t i = 0; i < n_problems; ++i)
        if (src_offsets[i + 1] <= src_offsets[i] || tgt_offsets[i + 1] <= tgt_offsets[i])
            return fail(LFMM_EINVAL, "every problem needs at least one source and one target (problem " +
                                         std::to_string(i) + ")");
    const int64_t ns = src_offsets[n_problems], nt = tgt_offsets[n_problems];
    if (ns > INT32_MAX / 2 || nt > INT32_MAX / 2) return fail(LFMM_EINVAL, "more than 2^30 points");
    lfmm_opts o;
    if (opts) o = *opts;
    else lfmm_opts_default(&o);
    int st = validate_opts(o);
    if (st) return st;
    lfmm_plan* p = new (std::nothrow) lfmm_plan();
    if (!p) return fail(LFMM_ENOMEM, "host allocation failed");
    p->opts = o;
    p->ns = ns;
    p->nt = nt;
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    auto build = [&]() -> int {
        LFMM_CUDA_TRY(cudaGetDevice(&p->device));
        LFMM_CUDA_TRY(cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device));
        setup_pool(p->device);
        const int32_t *src, *tgt;
        int r;
        {
            PhaseTimer pt(LFMM_PHASE_COPY, s);
            if ((r = device_coords(p, src_xy, ns, &src, s))) return r;
            if ((r = device_coords(p, tgt_xy, nt, &tgt, s))) return r;
        }
        PhaseTimer pt(LFMM_PHASE_TREE, s);
        p->forest.reset(new (std::nothrow) Forest());
        if (!p->forest) return fail(LFMM_ENOMEM, "host allocation failed");
        if ((r = forest_build(*p->forest, src, src_offsets, ns, tgt, tgt_offsets, nt, (int)n_problems, o.leaf_size,
                              o.max_leaf_side, s, &pt)))
            return r;
        return forest_workspaces(p, s);
    };
    st = build();
    if (st) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
        free_plan_buffers(p);
        delete p;
        return st;
    }
    set_error("");
    if (profiling_enabled()) profile_flush();
    *plan = p;
    return LFMM_OK;
}

const char* lfmm_status_string(int status) {
    switch (status) {
        case LFMM_OK: return "ok";
        case LFMM_EINVAL: return "invalid argument";
        case LFMM_ENOMEM: return "out of memory";
        case LFMM_ECUDA: return "CUDA error";
        case LFMM_ETIMEOUT: return "device wait timed out";
        case LFMM_EUNSUPPORTED: return "unsupported";
        case LFMM_EINTERNAL: return "internal error";
        case LFMM_EBUSY: return "refused or shed by the server's overload policy";
        case LFMM_ECANCELED: return "cancelled";
        default: return "unknown status";
    }
}

const char* lfmm_last_error(void) { return lfmm::last_error_cstr(); }

int lfmm_phi_table(int32_t R, double* out) {
    if (!out || R < 1 || R > 256) return fail(LFMM_EINVAL, "R must be in [1, 256]");
    std::vector<double> t = R <= kPhiHostRadius ? phi_host_table() : compute_phi_octant(R);
    std::memcpy(out, t.data(), sizeof(double) * (size_t)(R + 1) * (R + 2) / 2);
    return LFMM_OK;
}

int lfmm_phi(const int64_t* d, int64_t n, double* out) {
    if (!d || !out || n < 0) return fail(LFMM_EINVAL, "bad arguments");
    for (int64_t i = 0; i < n; ++i) out[i] = phi_host(d[2 * i], d[2 * i + 1]);
    return LFMM_OK;
}

int lfmm_model_skeleton(int32_t leaf_side, int32_t p, int32_t ppe, int32_t level, int32_t* xy, int32_t* count) {
    if (!xy || !count || p < 2 || p > 17 || level < 0) return fail(LFMM_EINVAL, "bad arguments");
    std::string err;
    ModelOps* mo = get_model_ops(leaf_side, 4 * (p - 1), ppe, level + 1, &err);
    if (!mo) return fail(LFMM_EINVAL, err);
    std::lock_guard<std::mutex> g(mo->mu);
    const LevelOps& lv = mo->levels[level];
    *count = lv.P;
    for (int i = 0; i < 2 * lv.P; ++i) xy[i] = lv.skel[i];
    return LFMM_OK;
}

int lfmm_model_tofs(int32_t leaf_side, int32_t p, int32_t ppe, double* out) {
    if (!out || p < 2 || p > 17) return fail(LFMM_EINVAL, "bad arguments");
    std::string err;
    ModelOps* mo = get_model_ops(leaf_side, 4 * (p - 1), ppe, 1, &err);
    if (!mo) return fail(LFMM_EINVAL, err);
    std::lock_guard<std::mutex> g(mo->mu);
    std::memcpy(out, mo->tofs.data(), mo->tofs.size() * sizeof(double));
    return LFMM_OK;
}

int lfmm_model_s(int32_t leaf_side, int32_t p, int32_t ppe, int32_t level, double* out) {
    if (!out || p < 2 || p > 17 || level < 1) return fail(LFMM_EINVAL, "bad arguments");
    std::string err;
    ModelOps* mo = get_model_ops(leaf_side, 4 * (p - 1), ppe, level + 1, &err);
    if (!mo) return fail(LFMM_EINVAL, err);
    std::lock_guard<std::mutex> g(mo->mu);
    const LevelOps& lv = mo->levels[level];
    std::memcpy(out, lv.S.data(), lv.S.size() * sizeof(double));
    return LFMM_OK;
}

}  // extern "C"
