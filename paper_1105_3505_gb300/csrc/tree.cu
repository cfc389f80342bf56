// Uniform quadtree build on the GPU (Sec. 6): root box, leaf level, points bucketed
// by leaf in Morton order.
//
// The leaf level L is the coarsest level at which no box holds more than N_leaf
// sources or N_leaf targets.  Counting runs on one fine level (one atomic per point
// into a per-box counter, Morton-indexed so coarser boxes are contiguous ranges) and
// one coarsening pass; an exclusive scan turns leaf counts into bucket offsets, and a
// scatter places every point in its leaf bucket (order inside a bucket is the
// arrival order of the atomics; nothing downstream depends on it beyond rounding).
#include <algorithm>

#include "lfmm_internal.h"

namespace lfmm {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int warp_min(int v) {
    for (int o = 16; o; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ int warp_max(int v) {
    for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// out4 = {min x, min y, max x, max y} over both point sets; out4 preset by the host.
// Warp and block reductions first: one set of atomics per block.
__global__ void bbox_kernel(const int2* __restrict__ a, int64_t na, const int2* __restrict__ b,
                            int64_t nb, int* __restrict__ out4) {
    griddep_wait();
    __shared__ int sh[4][kThreads / 32];
    int mnx = INT_MAX, mny = INT_MAX, mxx = INT_MIN, mxy = INT_MIN;
    const int64_t n = na + nb;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    auto at = [&](int64_t i) { return i < na ? a[i] : b[i - na]; };
    auto take = [&](int2 p) {
        mnx = min(mnx, p.x);
        mny = min(mny, p.y);
        mxx = max(mxx, p.x);
        mxy = max(mxy, p.y);
    };
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // four independent loads in flight per thread (the input is read cold from DRAM)
    for (; i + 3 * stride < n; i += 4 * stride) {
        const int2 p0 = at(i), p1 = at(i + stride), p2 = at(i + 2 * stride), p3 = at(i + 3 * stride);
        take(p0);
        take(p1);
        take(p2);
        take(p3);
    }
    for (; i < n; i += stride) take(at(i));
    mnx = warp_min(mnx);
    mny = warp_min(mny);
    mxx = warp_max(mxx);
    mxy = warp_max(mxy);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][wid] = mnx;
        sh[1][wid] = mny;
        sh[2][wid] = mxx;
        sh[3][wid] = mxy;
    }
    __syncthreads();
    if (wid == 0) {
        const bool ok = lane < kThreads / 32;
        mnx = warp_min(ok ? sh[0][lane] : INT_MAX);
        mny = warp_min(ok ? sh[1][lane] : INT_MAX);
        mxx = warp_max(ok ? sh[2][lane] : INT_MIN);
        mxy = warp_max(ok ? sh[3][lane] : INT_MIN);
        if (lane == 0) {
            atomicMin(out4 + 0, mnx);
            atomicMin(out4 + 1, mny);
            atomicMax(out4 + 2, mxx);
            atomicMax(out4 + 3, mxy);
        }
    }
}

__device__ __forceinline__ uint32_t box_of(int2 p, int64_t x0, int64_t y0, int shift) {
    const uint32_t bx = (uint32_t)(((int64_t)p.x - x0) >> shift);
    const uint32_t by = (uint32_t)(((int64_t)p.y - y0) >> shift);
    return morton2(bx, by);
}

// Counts points per box; with `rank` set, also records each point's arrival rank in
// its box (the value its atomic increment returned), which places it in its bucket
// later without a second atomic pass.
__global__ void histogram_kernel(const int2* __restrict__ src, int64_t ns,
                                 const int2* __restrict__ tgt, int64_t nt, int64_t x0,
                                 int64_t y0, int shift, int32_t* __restrict__ cs,
                                 int32_t* __restrict__ ct, int32_t* __restrict__ rank) {
    griddep_wait();
    const int64_t n = ns + nt;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int r = i < ns ? atomicAdd(cs + box_of(src[i], x0, y0, shift), 1)
                             : atomicAdd(ct + box_of(tgt[i - ns], x0, y0, shift), 1);
        if (rank) rank[i] = r;
    }
}

// The same counts at level Lf before the host has read the bounding box: the root box
// (corner and side 2^K, K the smallest with 2^K >= the larger extent) comes from the
// bbox words the previous kernel wrote.  Nothing is counted when K < Lf (the host then
// finds that level Lf was the wrong guess and counts again).
__global__ void histogram_bbox_kernel(const int2* __restrict__ src, int64_t ns, const int2* __restrict__ tgt,
                                      int64_t nt, const int* __restrict__ bbox4, int Lf, int32_t* __restrict__ cs,
                                      int32_t* __restrict__ ct, int32_t* __restrict__ rank) {
    griddep_wait();
    const int64_t x0 = bbox4[0], y0 = bbox4[1];
    const int64_t ext = max((int64_t)bbox4[2] - x0, (int64_t)bbox4[3] - y0) + 1;
    if (ext < 1) return;
    const int K = ext <= 1 ? 0 : 64 - __clzll((unsigned long long)(ext - 1));
    if (K < Lf) return;
    const int shift = K - Lf;
    const int64_t n = ns + nt;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int r = i < ns ? atomicAdd(cs + box_of(src[i], x0, y0, shift), 1)
                             : atomicAdd(ct + box_of(tgt[i - ns], x0, y0, shift), 1);
        rank[i] = r;
    }
}

// Buckets points by leaf (row-major leaf order at level L) from the ranks the histogram
// recorded at level Lf (= L or L + 1, Morton counts `fine` of that level): a point's
// slot is its leaf's start, plus the counts of its box's earlier siblings when Lf = L + 1,
// plus its rank.
__global__ void scatter_ranked_kernel(const int2* __restrict__ xy, int64_t n, int64_t x0, int64_t y0, int K, int L,
                                      int Lf, const int32_t* __restrict__ begin, const int32_t* __restrict__ fine,
                                      const int32_t* __restrict__ rank, int32_t* __restrict__ loc,
                                      int32_t* __restrict__ perm, int32_t* __restrict__ leaf_of_slot) {
    griddep_wait();
    const int shift = K - L, lside = 1 << shift;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int2 p = xy[i];
        const int64_t rx = (int64_t)p.x - x0, ry = (int64_t)p.y - y0;
        const int64_t leaf = ((ry >> shift) << L) | (rx >> shift);
        int slot = begin[leaf] + rank[i];
        if (Lf == L + 1) {
            const uint32_t mf = morton2((uint32_t)(rx >> (shift - 1)), (uint32_t)(ry >> (shift - 1)));
            const uint32_t base = mf & ~3u;
            for (uint32_t c = base; c < mf; ++c) slot += fine[c];
        }
        loc[slot] = (int)(rx & (lside - 1)) | ((int)(ry & (lside - 1)) << 16);
        perm[slot] = (int32_t)i;
        if (leaf_of_slot) leaf_of_slot[slot] = (int32_t)morton2((uint32_t)(rx >> shift), (uint32_t)(ry >> shift));
    }
}

// coarse[b] = sum of fine[4b..4b+3]; max4 = {max fine src, max fine tgt, max coarse src,
// max coarse tgt}.
__global__ void coarsen_kernel(const int4* __restrict__ fs, const int4* __restrict__ ft,
                               int64_t n_coarse, int32_t* __restrict__ cs,
                               int32_t* __restrict__ ct, int* __restrict__ max4) {
    griddep_wait();
    int m0 = 0, m1 = 0, m2 = 0, m3 = 0, nf = 0, nc = 0;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n_coarse;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int4 s = fs[b], t = ft[b];
        const int ss = s.x + s.y + s.z + s.w, tt = t.x + t.y + t.z + t.w;
        cs[b] = ss;
        ct[b] = tt;
        m0 = max(m0, max(max(s.x, s.y), max(s.z, s.w)));
        m1 = max(m1, max(max(t.x, t.y), max(t.z, t.w)));
        m2 = max(m2, ss);
        m3 = max(m3, tt);
        nf += (s.x + t.x > 0) + (s.y + t.y > 0) + (s.z + t.z > 0) + (s.w + t.w > 0);
        nc += ss + tt > 0;
    }
    m0 = warp_max(m0);
    m1 = warp_max(m1);
    m2 = warp_max(m2);
    m3 = warp_max(m3);
    for (int o = 16; o; o >>= 1) {
        nf += __shfl_xor_sync(0xffffffffu, nf, o);
        nc += __shfl_xor_sync(0xffffffffu, nc, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(max4 + 0, m0);
        atomicMax(max4 + 1, m1);
        atomicMax(max4 + 2, m2);
        atomicMax(max4 + 3, m3);
        atomicAdd(max4 + 4, nf);
        atomicAdd(max4 + 5, nc);
    }
}

// ---- exclusive scan of two int32 arrays of length n into out[0..n] (out[n] = total)
constexpr int kScanItems = 8;
constexpr int kScanTile = kThreads * kScanItems;

__device__ __forceinline__ int block_exclusive_scan(int v, int* sh, int& total) {
    // sh: kThreads/32 ints
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = lane < kThreads / 32 ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kThreads / 32) sh[lane] = w;
    }
    __syncthreads();
    const int warp_off = wid ? sh[wid - 1] : 0;
    total = sh[kThreads / 32 - 1];
    __syncthreads();
    return warp_off + x - v;
}

// Counts are stored Morton-indexed; the scan runs over leaves in row-major order
// (index i = by * 2^L + bx), gathering count[morton(bx, by)].
__device__ __forceinline__ int32_t count_rm(const int32_t* in, int64_t i, int L) {
    const uint32_t bx = (uint32_t)(i & ((1 << L) - 1)), by = (uint32_t)(i >> L);
    return in[morton2(bx, by)];
}

__global__ void scan_tile_sums(const int32_t* __restrict__ a, const int32_t* __restrict__ b,
                               int64_t n, int L, int32_t* __restrict__ partials) {
    griddep_wait();
    __shared__ int sh[kThreads / 32];
    const int32_t* in = blockIdx.y ? b : a;
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
        if (i < n) s += count_rm(in, i, L);
    }
    int total;
    block_exclusive_scan(s, sh, total);
    if (threadIdx.x == 0) partials[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = total;
}

__global__ void scan_partials(int32_t* __restrict__ partials, int n_tiles) {
    griddep_wait();
    __shared__ int sh[kThreads / 32];
    int32_t* p = partials + (int64_t)blockIdx.x * n_tiles;
    int carry = 0;
    for (int base = 0; base < n_tiles; base += kThreads) {
        const int i = base + threadIdx.x;
        const int v = i < n_tiles ? p[i] : 0;
        int total;
        const int ex = block_exclusive_scan(v, sh, total);
        if (i < n_tiles) p[i] = carry + ex;
        carry += total;
    }
}

__global__ void scan_tiles(const int32_t* __restrict__ a, int32_t* __restrict__ oa,
                           const int32_t* __restrict__ b, int32_t* __restrict__ ob, int64_t n, int L,
                           const int32_t* __restrict__ partials) {
    griddep_wait();
    __shared__ int sh[kThreads / 32];
    const int32_t* in = blockIdx.y ? b : a;
    int32_t* out = blockIdx.y ? ob : oa;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + k;
        v[k] = i < n ? count_rm(in, i, L) : 0;
        s += v[k];
    }
    int total;
    int run = block_exclusive_scan(s, sh, total) + partials[(int64_t)blockIdx.y * gridDim.x + blockIdx.x];
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + k;
        if (i < n) out[i] = run;
        run += v[k];
        if (i == n - 1) out[n] = run;
    }
}

__global__ void scatter_kernel(const int2* __restrict__ xy, int64_t n, int64_t x0, int64_t y0,
                               int shift, int leaf_side, int n_side, const int32_t* __restrict__ begin,
                               int32_t* __restrict__ cursor, int32_t* __restrict__ loc,
                               int32_t* __restrict__ perm) {
    griddep_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int2 p = xy[i];
        const int64_t rx = (int64_t)p.x - x0, ry = (int64_t)p.y - y0;
        const uint32_t L = (uint32_t)__popc((unsigned)(n_side - 1));
        const uint32_t leaf = ((uint32_t)(ry >> shift) << L) | (uint32_t)(rx >> shift);
        const int slot = begin[leaf] + atomicAdd(cursor + leaf, 1);
        const int lx = (int)(rx & (leaf_side - 1)), ly = (int)(ry & (leaf_side - 1));
        loc[slot] = lx | (ly << 16);
        perm[slot] = (int32_t)i;
    }
}

__global__ void set4_kernel(int* p, int a, int b, int c, int d) {
    p[0] = a;
    p[1] = b;
    p[2] = c;
    p[3] = d;
}

// words[0..3] = {INT_MAX, INT_MAX, INT_MIN, INT_MIN} (bounding box to be reduced),
// words[4..9] = 0 (maxima and counts of coarsen_kernel), zero[0..n_zero) = 0
__global__ void init_tree_kernel(int* __restrict__ words, int32_t* __restrict__ zero, int64_t n_zero) {
    griddep_wait();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 10) words[t] = t < 2 ? INT_MAX : (t < 4 ? INT_MIN : 0);
    for (int64_t i = t; i < n_zero / 4; i += (int64_t)gridDim.x * blockDim.x)
        reinterpret_cast<int4*>(zero)[i] = make_int4(0, 0, 0, 0);
    for (int64_t i = n_zero / 4 * 4 + t; i < n_zero; i += (int64_t)gridDim.x * blockDim.x) zero[i] = 0;
}

int grid_for(int64_t n, int threads, int cap = 152 * 16) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

}  // namespace

cudaError_t launch_set4(int* p, int a, int b, int c, int d, cudaStream_t s) {
    set4_kernel<<<1, 1, 0, s>>>(p, a, b, c, d);
    return cudaGetLastError();
}

cudaError_t launch_init_tree(int* words, int32_t* zero, int64_t n_zero, cudaStream_t s) {
    (void)launch_dependent(init_tree_kernel, dim3(grid_for(std::max<int64_t>(n_zero / 4, 10), kThreads)), dim3(kThreads), 0, s, words, zero, n_zero);
    return cudaGetLastError();
}

cudaError_t launch_bbox(const int32_t* a, int64_t na, const int32_t* b, int64_t nb, int* out4,
                        cudaStream_t s) {
    return launch_dependent(bbox_kernel, dim3(grid_for((na + nb + 7) / 8, kThreads, 152 * 8)), dim3(kThreads), 0, s,
                            (const int2*)a, na, (const int2*)b, nb, out4);
}

cudaError_t launch_histogram(const int32_t* src, int64_t ns, const int32_t* tgt, int64_t nt,
                             int64_t x0, int64_t y0, int shift, int32_t* cs, int32_t* ct,
                             cudaStream_t s, int32_t* rank) {
    (void)launch_dependent(histogram_kernel, dim3(grid_for(ns + nt, kThreads)), dim3(kThreads), 0, s,
        (const int2*)src, ns, (const int2*)tgt, nt, x0, y0, shift, cs, ct, rank);
    return cudaGetLastError();
}

cudaError_t launch_histogram_bbox(const int32_t* src, int64_t ns, const int32_t* tgt, int64_t nt, const int* bbox4,
                                  int Lf, int32_t* cs, int32_t* ct, int32_t* rank, cudaStream_t s) {
    return launch_dependent(histogram_bbox_kernel, dim3(grid_for(ns + nt, kThreads)), dim3(kThreads), 0, s,
                            (const int2*)src, ns, (const int2*)tgt, nt, bbox4, Lf, cs, ct, rank);
}

cudaError_t launch_scatter_ranked(const int32_t* xy, int64_t n, int64_t x0, int64_t y0, int K, int L, int Lf,
                                  const int32_t* begin, const int32_t* fine, const int32_t* rank, int32_t* loc,
                                  int32_t* perm, cudaStream_t s, int32_t* leaf_of_slot) {
    return launch_dependent(scatter_ranked_kernel, dim3(grid_for(n, kThreads)), dim3(kThreads), 0, s,
                            (const int2*)xy, n, x0, y0, K, L, Lf, begin, fine, rank, loc, perm, leaf_of_slot);
}

cudaError_t launch_coarsen(const int32_t* fs, const int32_t* ft, int64_t n_coarse, int32_t* cs,
                           int32_t* ct, int* max4, cudaStream_t s) {
    return launch_dependent(coarsen_kernel, dim3(grid_for(n_coarse, kThreads)), dim3(kThreads), 0, s,
                            (const int4*)fs, (const int4*)ft, n_coarse, cs, ct, max4);
}

size_t scan_partials_size(int64_t n) {
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    return (size_t)(2 * (tiles < 1 ? 1 : tiles));
}

cudaError_t launch_scan2(const int32_t* a, int32_t* oa, const int32_t* b, int32_t* ob, int L,
                         int32_t* partials, cudaStream_t s) {
    const int64_t n = (int64_t)1 << (2 * L);
    int tiles = (int)((n + kScanTile - 1) / kScanTile);
    if (tiles < 1) tiles = 1;
    dim3 g(tiles, 2);
    cudaError_t e = launch_dependent(scan_tile_sums, g, dim3(kThreads), 0, s, a, b, n, L, partials);
    if (e == cudaSuccess) e = launch_dependent(scan_partials, dim3(2), dim3(kThreads), 0, s, partials, tiles);
    if (e == cudaSuccess) e = launch_dependent(scan_tiles, g, dim3(kThreads), 0, s, a, oa, b, ob, n, L, partials);
    return e;
}

cudaError_t launch_scatter(const int32_t* xy, int64_t n, int64_t x0, int64_t y0, int shift,
                           int leaf_side, int L, const int32_t* begin, int32_t* cursor, int32_t* loc,
                           int32_t* perm, cudaStream_t s) {
    (void)launch_dependent(scatter_kernel, dim3(grid_for(n, kThreads)), dim3(kThreads), 0, s, (const int2*)xy, n, x0, y0, shift,
                                                             leaf_side, 1 << L, begin, cursor, loc, perm);
    return cudaGetLastError();
}

}  // namespace lfmm
