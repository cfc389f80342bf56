// lfmm_plan_shape_noalloc: the tree shape and device footprint a plan would have,
// computed without allocating memory (declared in include/lfmm.h).
//
// Who needs this: code that cannot call cudaMalloc at the moment it must decide
// about a problem - an admission controller that has to size a request before it
// commits memory to it (allocating in order to find out how much to allocate defeats
// the purpose), host code running while a CUDA stream is being captured into a graph
// (allocation calls are not allowed there), and processes whose device memory is
// owned by another allocator that forbids outside cudaMalloc/cudaFree.
//
// The bounding-box and leaf-count kernels of the plan builder run on a scratch area
// that is a file-scope static device array (one per GPU that loads the library, held
// until the process exits).  Host code cannot use the array's symbol as a device
// address, so the first call on each device looks the address up with
// cudaGetSymbolAddress while that device is current; make that first call outside
// any stream capture.  All calls share the array: each call clears what it counts
// into, and calls that overlap on the GPU (different streams, or different host
// threads) race on it and must be serialised by the caller.
#include <climits>
#include <cstring>
#include <mutex>

#include "lfmm_internal.h"

namespace lfmm {

namespace {

// Finest counting level supported: 4^10 boxes per count array.
constexpr int kNoAllocMaxLevel = 10;
constexpr int64_t kNoAllocFine = (int64_t)1 << (2 * kNoAllocMaxLevel);
// [fine src][fine tgt][coarse src][coarse tgt][8 ints for box / maxima]
constexpr int64_t kNoAllocInts = 2 * kNoAllocFine + 2 * (kNoAllocFine / 4) + 64;

static __device__ __align__(256) int32_t g_noalloc_scratch[kNoAllocInts];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
int32_t* g_addr[kMaxDevices] = {nullptr};

int scratch_address(int dev, int32_t** out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(LFMM_EUNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> g(g_addr_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return fail(LFMM_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_addr[dev] = (int32_t*)p;
    }
    *out = g_addr[dev];
    return LFMM_OK;
}

bool device_resident(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int ceil_log2(int64_t v) {
    int k = 0;
    while (((int64_t)1 << k) < v) ++k;
    return k;
}

}  // namespace

}  // namespace lfmm

using namespace lfmm;

extern "C" int lfmm_plan_shape_noalloc(const int32_t* src_xy, int64_t n_src, const int32_t* tgt_xy, int64_t n_tgt,
                                       const lfmm_opts* opts, lfmm_plan_info* info, void* stream) {
    if (!src_xy || !tgt_xy || !info) return fail(LFMM_EINVAL, "NULL argument");
    if (n_src < 1 || n_tgt < 1 || n_src > INT32_MAX / 2 || n_tgt > INT32_MAX / 2)
        return fail(LFMM_EINVAL, "n_src and n_tgt must be in [1, 2^30)");
    lfmm_opts o;
    if (opts) o = *opts;
    else lfmm_opts_default(&o);
    if (o.precision != LFMM_FP64 && o.precision != LFMM_MIXED && o.precision != LFMM_DF)
        return fail(LFMM_EINVAL, "bad opts.precision");
    if (o.p < 2 || o.p > 17 || o.leaf_size < 1 || o.max_leaf_side < 1 || o.max_leaf_side > kMaxLeafSide ||
        (o.max_leaf_side & (o.max_leaf_side - 1)))
        return fail(LFMM_EINVAL, "bad opts");
    // Coordinates are read in place: they must be 8-byte aligned device memory (copying host
    // data would need a device buffer).
    if (!device_resident(src_xy) || !device_resident(tgt_xy) || ((uintptr_t)src_xy % 8) ||
        ((uintptr_t)tgt_xy % 8))
        return fail(LFMM_EINVAL, "lfmm_plan_shape_noalloc needs 8-byte aligned device coordinates");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    LFMM_CUDA_TRY(cudaGetDevice(&dev));
    int32_t* scratch = nullptr;
    int st = scratch_address(dev, &scratch);
    if (st) return st;
    int* d4 = scratch + (kNoAllocInts - 64);

    // root box: lower-left corner of all points, side 2^K
    LFMM_CUDA_TRY(launch_set4(d4, INT_MAX, INT_MAX, INT_MIN, INT_MIN, s));
    LFMM_CUDA_TRY(launch_bbox(src_xy, n_src, tgt_xy, n_tgt, d4, s));
    int h4[4];
    LFMM_CUDA_TRY(cudaMemcpyAsync(h4, d4, sizeof(h4), cudaMemcpyDeviceToHost, s));
    LFMM_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t ext = std::max((int64_t)h4[2] - h4[0], (int64_t)h4[3] - h4[1]) + 1;
    if (ext > ((int64_t)1 << 30)) return fail(LFMM_EINVAL, "points span more than 2^30 lattice cells");
    const int K = ceil_log2(ext);

    // leaf level: coarsest level with <= leaf_size sources and targets per box
    const int L_side = std::max(0, K - ceil_log2(o.max_leaf_side));
    int L_pig = 0;
    while (((int64_t)o.leaf_size << (2 * L_pig)) < std::max(n_src, n_tgt)) ++L_pig;
    int L_try = std::min(K, std::max(L_side, L_pig));
    int Lf = std::min(K, L_try + 1);
    int L = -1, msrc = 0, mtgt = 0;
    int64_t nonempty = 1;
    for (;;) {
        if (Lf > kNoAllocMaxLevel)
            return fail(LFMM_EINVAL, "tree needs counting on level " + std::to_string(Lf) +
                                         "; lfmm_plan_shape_noalloc supports levels up to " +
                                         std::to_string(kNoAllocMaxLevel) + " (scratch of " +
                                         std::to_string(kNoAllocInts * 4) + " bytes)");
        const int64_t nf = (int64_t)1 << (2 * Lf), nc = Lf >= 1 ? nf / 4 : 0;
        int32_t *fs = scratch, *ft = scratch + nf, *cs = ft + nf, *ct = cs + nc;
        LFMM_CUDA_TRY(cudaMemsetAsync(fs, 0, (size_t)2 * nf * sizeof(int32_t), s));
        LFMM_CUDA_TRY(launch_histogram(src_xy, n_src, tgt_xy, n_tgt, h4[0], h4[1], K - Lf, fs, ft, s));
        int m4[6] = {(int)n_src, (int)n_tgt, 0, 0, 1, 1};
        if (Lf >= 1) {
            LFMM_CUDA_TRY(cudaMemsetAsync(d4 + 4, 0, 6 * sizeof(int), s));
            LFMM_CUDA_TRY(launch_coarsen(fs, ft, nc, cs, ct, d4 + 4, s));
            LFMM_CUDA_TRY(cudaMemcpyAsync(m4, d4 + 4, sizeof(m4), cudaMemcpyDeviceToHost, s));
            LFMM_CUDA_TRY(cudaStreamSynchronize(s));
        }
        if (Lf - 1 >= L_try && std::max(m4[2], m4[3]) <= o.leaf_size) {
            L = Lf - 1;
            msrc = m4[2];
            mtgt = m4[3];
            nonempty = m4[5];
        } else if (std::max(m4[0], m4[1]) <= o.leaf_size || Lf == K) {
            L = Lf;
            msrc = m4[0];
            mtgt = m4[1];
            nonempty = m4[4];
        }
        if (L >= 0) break;
        Lf = std::min(K, Lf + 2);
    }

    // device memory the plan would own (inputs read in place)
    const int P = 4 * (o.p - 1), NP = P <= 32 ? 32 : 64;
    const int64_t esz = o.precision == LFMM_MIXED ? 4 : 8;
    const int64_t n_leaves = (int64_t)1 << (2 * L);
    int64_t boxes = 0;
    for (int l = std::min(2, L); l <= L; ++l) boxes += (int64_t)1 << (2 * l);
    auto a = [](int64_t b) { return b == 0 ? (int64_t)16 : b; };
    const int tc_min = o.tc_min_level == 0 ? kDefaultTcMinLevel : o.tc_min_level;
    const int64_t split = (o.precision == LFMM_MIXED && L >= tc_min)
                              ? a(((int64_t)NP << (2 * L)) * 2 * 4 + ((int64_t)NP << (2 * std::max(0, L - 1))) * 2 * 4)
                              : 0;  // TF32 hi/lo copies for the tensor-core M2L
    const int64_t un_tmp = L >= 2 ? a(2 * n_tgt * 8) : 0;  // near and far parts before the final sum
    // one vector's partial sums of the coarse-level M2L split along K (sized from the shape)
    int num_sms = 0;
    LFMM_CUDA_TRY(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
    const bool has_tc = o.precision == LFMM_MIXED;
    const int64_t part = L < 2 ? 0
                         : o.precision == LFMM_MIXED ? m2l_fused_split_bytes_shape<float>(NP, has_tc, L, tc_min, num_sms, 1, o.m2l_split)
                         : o.precision == LFMM_DF    ? m2l_fused_split_bytes_shape<DF>(NP, has_tc, L, tc_min, num_sms, 1, o.m2l_split)
                                                     : m2l_fused_split_bytes_shape<double>(NP, has_tc, L, tc_min, num_sms, 1, o.m2l_split);
    const int64_t bytes = a(2 * (n_leaves + 1) * 4) + a((2 * (n_src + n_tgt) + n_tgt) * 4) + a(n_src * esz) + split +
                          un_tmp + part +
                          2 * a(boxes * NP * esz) + 2 * a(boxes * 8) + 16 /* status word */;

    std::memset(info, 0, sizeof(*info));
    info->n_src = n_src;
    info->n_tgt = n_tgt;
    info->x0 = h4[0];
    info->y0 = h4[1];
    info->K = K;
    info->L = L;
    info->leaf_side = 1 << (K - L);
    info->P = P;
    info->P_pad = NP;
    info->precision = o.precision;
    info->max_leaf_src = msrc;
    info->max_leaf_tgt = mtgt;
    info->device_bytes = bytes;
    info->tree = (o.tree == LFMM_TREE_PRUNED || (o.tree == LFMM_TREE_AUTO && 2 * nonempty < n_leaves))
                     ? LFMM_TREE_PRUNED
                     : LFMM_TREE_UNIFORM;
    info->n_problems = 1;
    info->n_boxes = boxes;
    return LFMM_OK;
}
