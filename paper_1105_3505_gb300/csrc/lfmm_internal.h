// Internal declarations shared by the translation units of liblfmm.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <array>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lfmm.h"

namespace lfmm {

#ifdef __CUDACC__
// ---------------------------------------------------------------- dependent launches
// Kernels of one dependency chain on a stream are launched with programmatic stream
// serialisation: a kernel's blocks may be scheduled while its predecessor's last blocks
// drain, and griddep_wait() - the first statement of every kernel launched this way -
// holds them until the predecessor has completed and its writes are visible.  Launched
// without the attribute (or behind a copy, a memset or an event), the wait returns at once.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                             Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}
#endif

// ---------------------------------------------------------------- float-float numbers
// hi + lo with |lo| <= ulp(hi) / 2: about 48 significant bits in two binary32 values.
// Element type of the LFMM_DF path (and of the compensated total-charge / incoming-
// constant channel of the mixed path); its arithmetic (device_common.h) runs on the
// FP32 pipes.
struct DF {
    float hi, lo;
    DF() = default;
    __host__ __device__ constexpr DF(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ explicit DF(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
int fail(int status, const std::string& msg);

#define LFMM_CUDA_TRY(expr)                                                            \
    do {                                                                               \
        cudaError_t _e = (expr);                                                       \
        if (_e != cudaSuccess)                                                         \
            return ::lfmm::fail(_e == cudaErrorMemoryAllocation ? LFMM_ENOMEM : LFMM_ECUDA, \
                                std::string(#expr) + ": " + cudaGetErrorString(_e));   \
    } while (0)

// Every device allocation of plans, temporaries and staging buffers goes through here
// (the stream-ordered pool); lfmm_fault_inject_alloc can make the n-th call fail with
// cudaErrorMemoryAllocation, as a full device would.
cudaError_t dev_malloc(void** ptr, size_t bytes, cudaStream_t s);

// A failed runtime call that is not a launch (an attribute set, say) also leaves its
// code as the thread's last error, which the next launch check would report again:
// read it off before handing the code back.
inline cudaError_t clear_and_return(cudaError_t e) {
    (void)cudaGetLastError();
    return e;
}

// Raises the dynamic shared-memory limit of kernel `func` to at least `bytes`
// (thread-safe; each kernel's limit only grows).
cudaError_t ensure_dynamic_smem(const void* func, size_t bytes);
// Resident blocks per SM of `func` at this block size and dynamic shared memory
// (cached, thread-safe; at least 1).
int blocks_per_sm(const void* func, int threads, size_t smem);

// ---------------------------------------------------------------- constants
constexpr int kPhiHostRadius = 128;   // host phi table radius; eq. 3.1 beyond
constexpr int kMaxLeafSide = 32;      // largest supported leaf side (P2P table in shared memory)
constexpr int kMaxP = 64;             // largest skeleton size
constexpr int kNumOffsets = 40;       // offsets (ox,oy) in [-3,3]^2 with max(|ox|,|oy|) >= 2

// The 40 interaction offsets, in row-major order over oy then ox, skipping the 3x3 core.
struct OffsetTable {
    int ox[kNumOffsets], oy[kNumOffsets];
    int index[49];  // (oy+3)*7 + (ox+3) -> position in the list, -1 for the 3x3 core
    OffsetTable();
};
const OffsetTable& offsets();

// ---------------------------------------------------------------- Morton codes
__host__ __device__ inline uint32_t spread_bits16(uint32_t v) {
    v &= 0x0000ffffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}
__host__ __device__ inline uint32_t compact_bits16(uint32_t v) {
    v &= 0x55555555u;
    v = (v | (v >> 1)) & 0x33333333u;
    v = (v | (v >> 2)) & 0x0f0f0f0fu;
    v = (v | (v >> 4)) & 0x00ff00ffu;
    v = (v | (v >> 8)) & 0x0000ffffu;
    return v;
}
// Box (bx, by) at a level <= 15 -> Morton index; children of b are 4b + (cx + 2cy).
__host__ __device__ inline uint32_t morton2(uint32_t bx, uint32_t by) {
    return spread_bits16(bx) | (spread_bits16(by) << 1);
}
__host__ __device__ inline void unmorton2(uint32_t m, uint32_t& bx, uint32_t& by) {
    bx = compact_bits16(m);
    by = compact_bits16(m >> 1);
}

// ---------------------------------------------------------------- phi (host)
// Gauss-Legendre nodes and weights on [-1, 1].
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);
// Library phi on the packed octant |m|_inf <= R by Remark 3.1 quadrature.
std::vector<double> compute_phi_octant(int R);
const std::vector<double>& phi_host_table();  // R = kPhiHostRadius, computed once
double phi_asym_host(double m1, double m2);  // eq. 3.1 without the remainder
double phi_host(int64_t dx, int64_t dy);     // table or eq. 3.1

// ---------------------------------------------------------------- model-box operators
struct LevelOps {
    int side = 0;               // box side at this level
    int P = 0;                  // skeleton size
    std::vector<int> skel;      // 2*P coordinates relative to the box corner
    std::vector<double> S;      // P x (4*P_child), row-major (levels above the leaf)
};

struct DeviceOps;  // per precision device copies

struct ModelOps {
    int leaf_side = 0, P_target = 0, ppe = 0;
    std::vector<double> tofs;     // P0 x leaf_side^2, row-major
    std::vector<LevelOps> levels; // 0 = leaf, k = k levels above
    std::mutex mu;                // guards growth and device uploads
    std::unique_ptr<DeviceOps> dev[3][2];  // [precision][NP==64]
};

// Returns the cached operators for (leaf_side, P, ppe) with at least n_levels levels.
ModelOps* get_model_ops(int leaf_side, int P, int ppe, int n_levels, std::string* err);

// phi(skel_p - skel_q - o*side) for offset o, P x P row-major.
void tifo_matrix(const LevelOps& lv, int o, std::vector<double>& out);

// ---------------------------------------------------------------- device operators
// Layout per level k (levels above the leaf), element type T, padded length NP:
//   m2m  [4NP][NP]   m2m[c*NP+q][p] = S_k[p][c*P_{k-1}+q]     (q-hat_parent = sum)
//   l2l  [4][NP][NP] l2l[c][q][p]   = S_k[q][c*P_{k-1}+p]     (u-hat_child += ...)
//   tifo [40][NP][NP] tifo[o][q][p] = phi(skel_p - skel_q - o*side) - c_o
//   mono [2][40]      c_o = phi(o*side) split as (hi, lo) of the element type
// Leaf: tofsT [s^2][NP] tofsT[J][p] = T_ofs[p][J];
//   P2P table [(2H+1)][W] of phi(dx,dy) - phi0, then phi0 = phi(s, 0) as (hi, lo).
struct DeviceOps {
    int NP = 0, precision = 0, n_levels = 0, leaf_side = 0;
    int tab_H = 0, tab_W = 0;             // P2P table half width and row width
    void* base = nullptr;                 // one allocation
    size_t bytes = 0;
    void* tofsT = nullptr;
    void* p2p_table = nullptr;
    std::vector<void*> m2m, l2l, tifo;    // per level k
    std::vector<void*> mono;              // per level k: deflation constants (hi[40], lo[40])
    std::vector<void*> tc;                // per level k (mixed, NP = 32): tensor-core B tiles,
                                          // [40 offsets + 4 L2L classes][hi, lo][32 x 32 fp32]
    std::vector<void*> retired;           // earlier, smaller uploads (kept alive)
};

const DeviceOps* get_device_ops(ModelOps* mo, int precision, int NP, int n_levels,
                                cudaStream_t stream, std::string* err);

// ---------------------------------------------------------------- tracing
// Counts every kernel launch; when profiling is on, brackets phases with CUDA events.
void count_launches(int n);
class PhaseTimer {
   public:
    PhaseTimer(int phase, cudaStream_t s);
    ~PhaseTimer();
    void add_launches(int n) { launches_ += n; count_launches(n); }

   private:
    int phase_;
    cudaStream_t s_;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
    int launches_ = 0;
};
// Reads and accumulates the events recorded since the last flush (synchronises).
void profile_flush();
bool profiling_enabled();

// ---------------------------------------------------------------- kernels (launchers)
struct TreeView {
    int L = 0;                 // leaf level
    int side = 0;              // leaf side
    int64_t n_leaves = 0;      // 4^L
    const int32_t* src_begin = nullptr;  // n_leaves + 1, row-major leaf order
    const int32_t* tgt_begin = nullptr;
    const int32_t* src_loc = nullptr;    // (lx | ly << 16) within the leaf
    const int32_t* src_perm = nullptr;   // caller index of each sorted source
    const int32_t* tgt_loc = nullptr;
    const int32_t* tgt_perm = nullptr;
    const int32_t* tgt_leaf = nullptr;   // Morton index of each sorted target's leaf
    int64_t n_tgt = 0;         // targets
    int64_t n_src_all = 0;     // sources
    int max_leaf_src = 0;      // largest leaf occupancies (size the P2P staging)
    int max_leaf_tgt = 0;
};

// ---------------------------------------------------------------- pruned trees / forests
// Stream-ordered temporary, freed on scope exit.
struct DevTemp {
    void* ptr = nullptr;
    cudaStream_t s = nullptr;
    void reset(cudaStream_t st) {
        if (ptr) cudaFreeAsync(ptr, s);
        ptr = nullptr;
        s = st;
    }
    ~DevTemp() {
        if (ptr) cudaFreeAsync(ptr, s);
    }
};

// Boxes of level k (k = levels above the leaves) over all problems of a pruned tree or
// forest.  Compact ids number the non-empty boxes (a source or target below them) in
// parity-class order (class c = (x & 1) + 2 (y & 1), then problem, then the (x >> 1,
// y >> 1) grid row by row), so each parity class is one contiguous range.
struct ForestLevel {
    int64_t nb = 0;            // compact boxes
    int64_t cls[5] = {0};      // class ranges of the compact ids (host)
    int64_t* d_cls = nullptr;  // same on the device
    int64_t box_off = 0;       // offset of this level in the expansion arrays (boxes)
    int32_t* bp = nullptr;     // [nb] problem of each box
    int32_t* bxy = nullptr;    // [nb] x | y << 16 at the box's level
    int32_t* par = nullptr;    // [nb] parent's compact id at k + 1, or -1
    int32_t* il = nullptr;     // [nb][27] interaction list (slot order of the box's class)
    int32_t* ch = nullptr;     // [nb][4] children's compact ids at k - 1 (k >= 1), -1 if empty
    int32_t* rl = nullptr;     // k = 0: [nb] the leaf's index in the row-major leaf list
};

// Near-field staging of the pruned / forest strip kernel: leaves per strip and staged
// sources and targets per block.
constexpr int kStripMaxSW = 32;
constexpr int kStripCapSrc = 2048;
constexpr int kStripCapTgt = 1536;

struct Forest {
    int np = 0;
    int64_t ns = 0, nt = 0;
    int ls = 0, side = 1;                   // common leaf side 2^ls
    std::vector<int32_t> x0, y0, K, L;      // per problem: root corner, root 2^K, leaf level
    int kb = 1;                             // bits per coordinate in packed box keys
    int kmax = -1;                          // deepest k with expansions (levels >= 2)
    int max_src = 0, max_tgt = 0;           // largest leaf occupancies
    int SW = 1;                             // leaves per near-field strip
    int64_t total_boxes = 0;                // expansion rows over all levels
    std::vector<ForestLevel> levels;        // k = 0 .. max(kmax, 0)
    // device
    int32_t* d_L = nullptr;                 // [np] leaf level of each problem
    // occupied leaves in row-major order per problem, keys (p << 2 kb) | (y << kb) | x:
    // first sorted source and target of each ([n_leaves] = totals) and compact id
    int64_t n_leaves = 0;
    uint64_t* rl_key = nullptr;
    int32_t *rl_s = nullptr, *rl_t = nullptr, *rl_id = nullptr;
    int32_t *sloc = nullptr, *sperm = nullptr, *tloc = nullptr, *tperm = nullptr;
    int4* strips = nullptr;                     // (problem, leaf row, first column, 0)
    // per strip, the leaves of its three neighbour-row segments (columns first - 1 ..
    // first + SW): [j0, j1) in the occupied-leaf list for each row, -1 outside the tree;
    // 2 int4 per strip {j0 r0, j1 r0, j0 r1, j1 r1}, {j0 r2, j1 r2, 0, 0}
    int4* strip_rows = nullptr;
    int32_t* n_strips_d = nullptr;
    std::vector<void*> owned;
    int64_t bytes = 0;
    void* m2l_part = nullptr;               // partial sums of K-split list M2L levels (plan-owned)
    int m2l_split = 0;                      // opts.m2l_split (0: chunks by the number of tiles)
    unsigned long long* sweep_ctr = nullptr;  // work-queue counters of the persistent sweeps (2 x 16)
    bool tc_list = false;                   // list M2L of large levels on the tensor cores (mixed path)
    float* tc_split = nullptr;              // TF32 hi / lo rows of those levels (plan-owned)
    void release(cudaStream_t s);
};

// K chunks of the list M2L of a level whose largest parity class has maxc boxes: more
// than one (up to 7) while its 32-box tiles are fewer than three per SM.
int m2l_list_chunks(int64_t maxc, int num_sms, int split = 0);
// Bytes of partial sums the K-split list M2L levels of F need (0: none split).
int64_t forest_m2l_split_bytes(const Forest& F, int NP, size_t esz, int num_sms, int split = 0);

// Builds the tree of every problem (offsets: n_problems + 1 entries, host memory).
// Leaf side: the largest power of two <= max_leaf_side at which no leaf holds more than
// leaf_size sources or targets.  Synchronises the stream.
int forest_build(Forest& F, const int32_t* src, const int64_t* soff_h, int64_t ns, const int32_t* tgt,
                 const int64_t* toff_h, int64_t nt, int np, int leaf_size, int max_leaf_side, cudaStream_t s,
                 PhaseTimer* timer);
// status: the plan's status word (grid-barrier words beside it; timed-out waits are
// recorded there); persistent: run each sweep as one persistent cooperative launch
// (LFMM_FLAG_PERSISTENT), else one launch per level, the list M2L of levels with at
// least kTcListMinBoxes boxes on the tensor cores when F.tc_list is set.
template <typename T>
int forest_eval(const Forest& F, const DeviceOps& ops, const double* f, T* f_sorted, T* qhat, T* uhat, void* Qbox,
                void* Cbox, double* u, double* un, double* uf, int num_sms, cudaStream_t s, int* status,
                bool persistent);
// Tensor-core M2L + L2L over the compact box lists of one pruned / forest level (mixed
// path, P_pad 32 or 64): splits the level's expansions (nb rows) and the parent level's
// incoming expansions (nb_parent rows, none without L2L) into TF32 hi / lo rows in
// `split` (m2l_tc_list_split_floats(nb, nb_parent, NP) floats), then one persistent launch
// over tiles of 128 boxes of one parity class whose A operand is gathered by list;
// cls_start on the device, cls_host its host copy; a timed-out wait is reported in *status.
constexpr int64_t kTcListMinBoxes = 1024;
int64_t m2l_tc_list_split_floats(int64_t nb, int64_t nb_parent, int NP);
cudaError_t launch_m2l_tc_list(const DeviceOps& ops, int k, const int64_t* cls_start, const int64_t* cls_host,
                               const int32_t* il, const int32_t* par, const float* q_level, int64_t nb,
                               const void* Q_level, const float* u_parent, int64_t nb_parent, const void* C_parent,
                               float* u_level, void* C_level, float* split, int* status, int num_sms,
                               cudaStream_t s);

// words[0..3] = {INT_MAX, INT_MAX, INT_MIN, INT_MIN}, words[4..9] = 0, zero[0..n_zero) = 0
// (zero 16-byte aligned), in one launch.
cudaError_t launch_init_tree(int* words, int32_t* zero, int64_t n_zero, cudaStream_t s);
cudaError_t launch_set4(int* p, int a, int b, int c, int d, cudaStream_t s);
cudaError_t launch_bbox(const int32_t* a, int64_t na, const int32_t* b, int64_t nb, int* out4,
                        cudaStream_t s);
// Morton counts of sources and targets per box of the level K - shift; rank (optional,
// ns + nt entries, sources first) receives each point's arrival rank in its box.
cudaError_t launch_histogram(const int32_t* src, int64_t ns, const int32_t* tgt, int64_t nt,
                             int64_t x0, int64_t y0, int shift, int32_t* cnt_src,
                             int32_t* cnt_tgt, cudaStream_t s, int32_t* rank = nullptr);
// Leaf buckets from histogram ranks taken at level Lf (L or L + 1; fine = that level's
// Morton counts): no atomics.
cudaError_t launch_scatter_ranked(const int32_t* xy, int64_t n, int64_t x0, int64_t y0, int K, int L, int Lf,
                                  const int32_t* begin, const int32_t* fine, const int32_t* rank, int32_t* loc,
                                  int32_t* perm, cudaStream_t s, int32_t* leaf_of_slot = nullptr);
// Sums 2x2 blocks of two Morton count arrays; max4[0..3] receive (atomic max) the
// largest fine source / target count and the largest coarse ones, max4[4..5] (atomic
// add) the number of non-empty fine and coarse boxes.  max4 must be zeroed first.
// Counts at level Lf with the root box taken from the device bbox words {min x, min y,
// max x, max y} (no host round trip); ranks always recorded; nothing counted if K < Lf.
cudaError_t launch_histogram_bbox(const int32_t* src, int64_t ns, const int32_t* tgt, int64_t nt, const int* bbox4,
                                  int Lf, int32_t* cs, int32_t* ct, int32_t* rank, cudaStream_t s);
cudaError_t launch_coarsen(const int32_t* fs, const int32_t* ft, int64_t n_coarse, int32_t* cs,
                           int32_t* ct, int* max4, cudaStream_t s);
// Exclusive scan over the 4^L leaves in row-major order of two Morton-indexed count
// arrays; out has 4^L + 1 entries.
cudaError_t launch_scan2(const int32_t* in_a, int32_t* out_a, const int32_t* in_b,
                         int32_t* out_b, int L, int32_t* partials, cudaStream_t s);
size_t scan_partials_size(int64_t n);
// Buckets points by leaf in row-major leaf order (leaf = by * 2^L + bx).
cudaError_t launch_scatter(const int32_t* xy, int64_t n, int64_t x0, int64_t y0, int shift,
                           int leaf_side, int L, const int32_t* begin, int32_t* cursor, int32_t* loc,
                           int32_t* perm, cudaStream_t s);

// Per-box scalars Q (total charge) and C (incoming constant) are 8 bytes per box:
// a float (hi, lo) pair on the mixed path, a double on the binary64 path.
template <typename T>
// nvec charge vectors: vector v reads f + v n_src, writes f_sorted + v n_src and the
// leaf expansions / charges v vq / v vQ elements after vector 0's.
cudaError_t launch_p2m(const TreeView& t, const DeviceOps& ops, const double* f, T* f_sorted,
                       T* qhat_leaf, void* Q_leaf, cudaStream_t s, int nvec = 1, int64_t vq = 0, int64_t vQ = 0);
// Far field of every target (L2P + incoming constant), binary64, caller order.
template <typename T>
// (nvec vectors: uhat / Cleaf of vector v at v vq / v vQ elements, uf at v n_tgt.)
cudaError_t launch_l2p(const TreeView& t, const DeviceOps& ops, const T* uhat_leaf, const void* Cleaf, double* uf,
                       cudaStream_t s, int nvec = 1, int64_t vq = 0, int64_t vQ = 0);
// u = un + uf elementwise (and the parts, where requested; any output may be null).
cudaError_t launch_combine(int64_t n, const double* un, const double* uf, double* u, double* u_near, double* u_far,
                           cudaStream_t s);
template <typename T>
cudaError_t launch_m2m(const DeviceOps& ops, int k, int level, const T* q_child, const void* Q_child,
                       T* q_parent, void* Q_parent, cudaStream_t s);
// Device buffers of every level of a uniform tree (index = level; null where absent).
struct LevelBufs {
    void* q[16] = {nullptr};
    void* u[16] = {nullptr};
    void* Q[16] = {nullptr};
    void* C[16] = {nullptr};
    // charge vectors evaluated together: vector v's arrays start v vq elements (q, u)
    // and v vQ elements (Q, C) after vector 0's
    int nvec = 1;
    int64_t vq = 0, vQ = 0;
    // partial sums of the fused small-level M2L split along K (m2l_fused_split_bytes)
    void* part = nullptr;
    int64_t part_bytes = 0;
};
// Bytes of partial sums launch_m2l_fused needs for nvec charge vectors (0: no K split;
// the split depends on the plan, not on nvec, so one and several vectors sum alike).
template <typename T>
int64_t m2l_fused_split_bytes(const DeviceOps& ops, int L, int tc_min_level, int num_sms, int nvec, int split = 0);
// The same from the plan's shape alone (has_tc: the mixed path's tensor-core tiles exist,
// i.e. binary32 with NP = 32), for footprints computed before any operator is uploaded.
template <typename T>
int64_t m2l_fused_split_bytes_shape(int NP, bool has_tc, int L, int tc_min_level, int num_sms, int nvec,
                                    int split = 0);
// M2M of levels L-1 .. 2 in one cooperative launch (grid barriers between levels).
// sync: two zero device words (barrier state).  Returns an error (nothing launched)
// when a cooperative launch is not possible; the caller then runs the per-level path.
template <typename T>
cudaError_t launch_m2m_fused(const DeviceOps& ops, int L, const LevelBufs& b, unsigned* sync, int* status,
                             int num_sms, cudaStream_t s);
// M2L + L2L of the small levels 2 .. *last_level (those the per-level path runs on the
// split-K kernel) in one cooperative launch; the caller continues at *last_level + 1.
template <typename T>
cudaError_t launch_m2l_fused(const DeviceOps& ops, int L, const LevelBufs& b, int tc_min_level, unsigned* sync,
                             int* status, int num_sms, int* last_level, cudaStream_t s, int split = 0);

// First tree level whose M2L runs on the tensor cores when opts.tc_min_level is 0
// (levels of 4^6 boxes and more: on uniform_1m level 6 there took the step from 0.478 to
// 0.468 ms at p = 8 and from 0.778 to 0.686 ms at p = 16; level 5 was slower again).
constexpr int kDefaultTcMinLevel = 6;
// Whether level `level` (k levels above the leaves) runs M2L + L2L on the tensor cores:
// fp32 arithmetic, P <= 32, tiles present, level >= tc_min_level.
inline bool m2l_uses_tc(const DeviceOps& ops, int k, int level, int tc_min_level, bool fp32) {
    return fp32 && (ops.NP == 32 || ops.NP == 64) && ops.tc.size() > (size_t)k && ops.tc[k] != nullptr &&
           level >= tc_min_level;
}
// M2L + L2L of one level; mixed-path levels >= tc_min_level (P <= 32) run on the
// tensor cores, which report a timed-out wait in *status.
template <typename T>
cudaError_t launch_m2l(const DeviceOps& ops, int k, int level, const T* q_level, const void* Q_level,
                       const T* u_parent, const void* C_parent, T* u_level, void* C_level, cudaStream_t s);
// Tensor-core M2L + L2L of one level (Morton-ordered q_hat / u_hat in and out):
// splits the level's expansions and the parent's into TF32 hi / lo layouts in `split`
// (8 np^2 + 2 np^2 rows of 32 floats, np = 2^(level-1)), then one persistent launch fed
// by tiled TMA loads; a timed-out wait is reported in *status.
// nvec charge vectors at once: vector v's arrays start v vq floats (q, u) and v vQ
// value pairs (Q, C) after vector 0's; `split` then holds nvec times the rows.
cudaError_t launch_m2l_tma(const DeviceOps& ops, int k, int level, const float* q_level, const void* Q_level,
                           const float* u_parent, const void* C_parent, float* u_level, void* C_level, float* split,
                           int* status, int num_sms, cudaStream_t s, int nvec = 1, int64_t vq = 0, int64_t vQ = 0,
                           int tile = 0, int stages = 0);
// Near field of k charge vectors (vector r: f_sorted + r f_stride, Qleaf + r q_stride,
// out u_near + r u_stride), four vectors per pass sharing each table lookup.
template <typename T>
cudaError_t launch_p2p_multi(const TreeView& t, const DeviceOps& ops, int k, const T* f_sorted, int64_t f_stride,
                             const void* Qleaf, int64_t q_stride, double* u_near, int64_t u_stride, int num_sms,
                             cudaStream_t s);
template <typename T>
cudaError_t launch_p2p_l2p(const TreeView& t, const DeviceOps& ops, const T* f_sorted,
                           const T* uhat_leaf, const void* C_leaf, const void* Q_leaf, double* u,
                           double* u_near, double* u_far, int num_sms, cudaStream_t s);

}  // namespace lfmm
