// Construction of pruned quadtrees and forests (Sec. 6, Def. 6.1) in O(N log N) work:
// every structure comes from sorted packed box keys or, for forests of small problems,
// from counts on each problem's dense leaf grid - never from dense maps of a deep level.
//
// A box of problem p at coordinates (x, y) of its level packs into the 64-bit key
// (p << 2 kb) | (y << kb) | x, kb = bits of the deepest leaf level, so a sorted key array
// lists the boxes of each problem row by row.  The builder
//   1. picks the common leaf side (the largest power of two <= max_leaf_side at which no
//      leaf holds more than leaf_size sources or targets): on the problems' dense leaf
//      grids when their cells are few (occupancy counts), else from sorted leaf keys of
//      the points (a run of equal keys is one leaf);
//   2. puts the points in row-major leaf order per problem (a counting sort on the dense
//      grids, else the sorted keys), so the sources of a leaf row segment are one
//      contiguous range, and lists the occupied leaves with their first source and
//      target;
//   3. builds the boxes of every level at once: each leaf emits its level-k key where it
//      heads its level-k row segment, one sort and one unique pass give every level's
//      boxes; a second sort numbers each level's boxes in parity-class order (class,
//      problem, (y >> 1, x >> 1) row by row: each class one contiguous range of compact
//      ids), and one kernel finds parents, children and interaction lists by binary
//      search;
//   4. lists the near-field strips (SW consecutive leaves of a row holding a target) and
//      the occupied leaves of each strip's three neighbour-row segments.
// The sorts are a stable least-significant-digit radix sort (8-bit digits, per-block
// digit counts, one exclusive scan, ranked scatter).  When targets equal sources (same
// offsets and coordinates) one order serves both.
#include <algorithm>
#include <climits>

#include "device_common.h"

namespace lfmm {

namespace {

constexpr int kT = 256;

int grid_of(int64_t n, int threads = kT, int cap = 152 * 16) {
    int64_t g = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

// ------------------------------------------------------------------------- exclusive scan
constexpr int kScanBlock = 1024;

__global__ void scan_reduce_kernel(const int32_t* __restrict__ in, int64_t n, int32_t* __restrict__ sums) {
    __shared__ int32_t w[kT / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    int32_t v = 0;
    for (int i = threadIdx.x; i < kScanBlock; i += blockDim.x)
        if (base + i < n) v += in[base + i];
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += w[i];
        sums[blockIdx.x] = t;
    }
}

// exclusive scan of the block totals in place (one block); total to sums[nb]
__global__ void scan_sums_kernel(int32_t* __restrict__ sums, int nb) {
    __shared__ int32_t carry_s, w[1024 / 32];
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int32_t v = i < nb ? sums[i] : 0;
        int32_t x = v;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) w[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int32_t s = lane < (int)(blockDim.x >> 5) ? w[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(kFull, s, o);
                if (lane >= o) s += y;
            }
            w[lane] = s;
        }
        __syncthreads();
        const int32_t incl = x + (wid > 0 ? w[wid - 1] : 0);
        const int32_t carry = carry_s;
        if (i < nb) sums[i] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry_s = carry + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[nb] = carry_s;
}

__global__ void scan_apply_kernel(const int32_t* __restrict__ in, int64_t n, const int32_t* __restrict__ sums,
                                  int32_t* __restrict__ out) {
    __shared__ int32_t w[kT / 32];
    constexpr int PER = kScanBlock / kT;  // 4 consecutive items per thread
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * PER;
    int32_t v[PER], t = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        v[j] = base + j < n ? in[base + j] : 0;
        t += v[j];
    }
    int32_t x = t;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) w[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int32_t s = lane < (int)(blockDim.x >> 5) ? w[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        w[lane] = s;
    }
    __syncthreads();
    int32_t run = sums[blockIdx.x] + x - t + (wid > 0 ? w[wid - 1] : 0);
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        if (base + j < n) out[base + j] = run;
        run += v[j];
    }
    const int64_t nblk = (n + kScanBlock - 1) / kScanBlock;
    if (blockIdx.x == nblk - 1 && threadIdx.x == blockDim.x - 1) out[n] = sums[nblk];
}

int64_t scan_tmp_ints(int64_t n) { return (n + kScanBlock - 1) / kScanBlock + 1; }

// out[0..n] = exclusive prefix sums of in[0..n) (out[n] = total); sums: scan_tmp_ints(n)
cudaError_t exscan(const int32_t* in, int32_t* out, int64_t n, int32_t* sums, cudaStream_t s) {
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    if (nb == 0) return cudaMemsetAsync(out, 0, sizeof(int32_t), s);
    scan_reduce_kernel<<<(unsigned)nb, kT, 0, s>>>(in, n, sums);
    scan_sums_kernel<<<1, 1024, 0, s>>>(sums, (int)nb);
    scan_apply_kernel<<<(unsigned)nb, kT, 0, s>>>(in, n, sums, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------- radix sort
constexpr int kRadix = 256;
constexpr int kItems = 8;
constexpr int kTile = kT * kItems;  // keys per block

// hist[d * nblocks + b] = keys of tile b whose digit (bits shift .. shift + 7) is d
__global__ void radix_hist_kernel(const uint64_t* __restrict__ keys, int64_t n, int shift, int nblocks,
                                  int32_t* __restrict__ hist) {
    __shared__ int32_t h[kRadix];
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) h[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int i = threadIdx.x; i < kTile; i += blockDim.x)
        if (base + i < n) atomicAdd(&h[(int)((keys[base + i] >> shift) & (kRadix - 1))], 1);
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) hist[(int64_t)d * nblocks + blockIdx.x] = h[d];
}

// Stable scatter of tile b: keys go to offs[d * nblocks + b] + (keys of digit d before them
// in the tile).  Warp w takes the tile's keys [w 256, w 256 + 256) in 8 rounds of 32; a
// key's rank among its warp's keys of the same digit comes from the lanes that share its
// digit in the round (match) and the warp's running count; warps are then offset by the
// counts of the warps before them.
__global__ void __launch_bounds__(kT) radix_scatter_kernel(const uint64_t* __restrict__ kin,
                                                           const uint32_t* __restrict__ vin,
                                                           uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                           int64_t n, int shift, int nblocks,
                                                           const int32_t* __restrict__ offs) {
    __shared__ int32_t wc[kT / 32][kRadix];
    __shared__ int32_t boff[kRadix];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < (kT / 32) * kRadix; i += kT) (&wc[0][0])[i] = 0;
    for (int d = threadIdx.x; d < kRadix; d += kT) boff[d] = offs[(int64_t)d * nblocks + blockIdx.x];
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)warp * (32 * kItems);
    uint64_t k[kItems];
    uint32_t v[kItems];
    int dg[kItems], rk[kItems];
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const int64_t i = base + it * 32 + lane;
        const bool ok = i < n;
        k[it] = ok ? kin[i] : 0ull;
        v[it] = (ok && vin) ? vin[i] : 0u;
        const int d = ok ? (int)((k[it] >> shift) & (kRadix - 1)) : kRadix;  // kRadix: no key
        const unsigned peers = __match_any_sync(kFull, d);
        const int leader = __ffs(peers) - 1;
        int start = 0;
        if (lane == leader && ok) {
            start = wc[warp][d];
            wc[warp][d] = start + __popc(peers);
        }
        start = __shfl_sync(kFull, start, leader);
        dg[it] = d;
        rk[it] = start + __popc(peers & ((1u << lane) - 1u));
        __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kT) {
        int run = 0;
        for (int w = 0; w < kT / 32; ++w) {
            const int t = wc[w][d];
            wc[w][d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        if (dg[it] < kRadix) {
            const int64_t pos = (int64_t)boff[dg[it]] + wc[warp][dg[it]] + rk[it];
            kout[pos] = k[it];
            if (vout) vout[pos] = v[it];
        }
    }
}

// Device scratch of one sorting job: second key / value buffers and the digit counts.
struct SortBufs {
    uint64_t* k2 = nullptr;
    uint32_t* v2 = nullptr;
    int32_t* hist = nullptr;  // 256 nblocks + 1 ints
    int32_t* sums = nullptr;  // scan_tmp_ints(256 nblocks)
};

int64_t sort_hist_ints(int64_t n) { return (int64_t)kRadix * ((n + kTile - 1) / kTile) + 1; }

// Sorts n keys (and values, when v is set) by their low `bits` bits (bits <= 64; the
// keys hold no higher bits), stably, in place: the passes alternate between (k, v) and
// the scratch, and after an odd number of them one copy brings the result back.
cudaError_t radix_sort(uint64_t* k, uint32_t* v, int64_t n, int bits, SortBufs& b, cudaStream_t s) {
    if (n <= 1) return cudaSuccess;
    const int nblocks = (int)((n + kTile - 1) / kTile);
    const int passes = std::max(1, (bits + 7) / 8);
    uint64_t *ki = k, *ko = b.k2;
    uint32_t *vi = v, *vo = v ? b.v2 : nullptr;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        radix_hist_kernel<<<nblocks, kT, 0, s>>>(ki, n, shift, nblocks, b.hist);
        cudaError_t e = exscan(b.hist, b.hist, (int64_t)kRadix * nblocks, b.sums, s);
        if (e != cudaSuccess) return e;
        radix_scatter_kernel<<<nblocks, kT, 0, s>>>(ki, vi, ko, vo, n, shift, nblocks, b.hist);
        std::swap(ki, ko);
        std::swap(vi, vo);
    }
    if (passes & 1) {
        cudaError_t e = cudaMemcpyAsync(k, ki, (size_t)n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess && v) e = cudaMemcpyAsync(v, vi, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------- keys and runs
__device__ __forceinline__ uint64_t pack_key(int p, int y, int x, int kb) {
    return ((uint64_t)p << (2 * kb)) | ((uint64_t)y << kb) | (uint64_t)x;
}
__device__ __forceinline__ void unpack_key(uint64_t key, int kb, int& p, int& y, int& x) {
    const uint64_t m = ((uint64_t)1 << kb) - 1;
    x = (int)(key & m);
    y = (int)((key >> kb) & m);
    p = (int)(key >> (2 * kb));
}
__device__ __forceinline__ int64_t lower_bound_key(const uint64_t* __restrict__ a, int64_t n, uint64_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// [first, end) of every box row of A (level k, problem p, row y; its entry is
// row_off[k np + p] + y); rows without boxes keep {0, 0}
__global__ void row_range_kernel(const uint64_t* __restrict__ A, int64_t na, int kb, int kbits, int np,
                                 const int64_t* __restrict__ row_off, int2* __restrict__ rows) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < na; j += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = A[j], rk = key >> kb;
        const bool head = j == 0 || (A[j - 1] >> kb) != rk;
        const bool tail = j == na - 1 || (A[j + 1] >> kb) != rk;
        if (!head && !tail) continue;
        int p, y, x;
        unpack_key(key & (((uint64_t)1 << kbits) - 1), kb, p, y, x);
        const int64_t r = row_off[(key >> kbits) * np + p] + y;
        if (head) rows[r].x = (int)j;
        if (tail) rows[r].y = (int)(j + 1);
    }
}

// First entry of A at or after key v = (k, p, y, x) within its row (the row's end if none;
// `end` is set to the row's end), or, without a row table, within all of A.
__device__ __forceinline__ int64_t find_in_row(const uint64_t* __restrict__ A, int64_t na,
                                               const int2* __restrict__ rows, const int64_t* __restrict__ row_off,
                                               int np, int k, int p, int y, uint64_t v, int64_t& end) {
    int64_t lo = 0, hi = na;
    if (rows) {
        const int2 rr = rows[row_off[(int64_t)k * np + p] + y];
        lo = rr.x;
        hi = rr.y;
    }
    end = hi;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (A[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void pid_kernel(const int64_t* __restrict__ off, int np, int32_t* __restrict__ pid) {
    for (int p = blockIdx.x; p < np; p += gridDim.x)
        for (int64_t i = off[p] + threadIdx.x; i < off[p + 1]; i += blockDim.x) pid[i] = p;
}

// bounding box of each problem's sources and targets, one block per problem
__global__ void bbox_forest_kernel(const int2* __restrict__ src, const int64_t* __restrict__ soff,
                                   const int2* __restrict__ tgt, const int64_t* __restrict__ toff, int np,
                                   int4* __restrict__ bb) {
    __shared__ int red[4][kT / 32];
    for (int p = blockIdx.x; p < np; p += gridDim.x) {
        int x0 = INT_MAX, y0 = INT_MAX, x1 = INT_MIN, y1 = INT_MIN;
        for (int64_t i = soff[p] + threadIdx.x; i < soff[p + 1]; i += blockDim.x) {
            const int2 v = src[i];
            x0 = min(x0, v.x), y0 = min(y0, v.y), x1 = max(x1, v.x), y1 = max(y1, v.y);
        }
        for (int64_t i = toff[p] + threadIdx.x; i < toff[p + 1]; i += blockDim.x) {
            const int2 v = tgt[i];
            x0 = min(x0, v.x), y0 = min(y0, v.y), x1 = max(x1, v.x), y1 = max(y1, v.y);
        }
        for (int o = 16; o; o >>= 1) {
            x0 = min(x0, __shfl_xor_sync(kFull, x0, o));
            y0 = min(y0, __shfl_xor_sync(kFull, y0, o));
            x1 = max(x1, __shfl_xor_sync(kFull, x1, o));
            y1 = max(y1, __shfl_xor_sync(kFull, y1, o));
        }
        const int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) red[0][w] = x0, red[1][w] = y0, red[2][w] = x1, red[3][w] = y1;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
                x0 = min(x0, red[0][i]), y0 = min(y0, red[1][i]);
                x1 = max(x1, red[2][i]), y1 = max(y1, red[3][i]);
            }
            bb[p] = make_int4(x0, y0, x1, y1);
        }
        __syncthreads();
    }
}

// leaf key of every point at leaf side 2^ls (value: the point's index)
__global__ void leaf_key_kernel(const int2* __restrict__ xy, int64_t n, const int32_t* __restrict__ pid,
                                const int32_t* __restrict__ x0, const int32_t* __restrict__ y0, int ls, int kb,
                                uint64_t* __restrict__ key, uint32_t* __restrict__ idx) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int p = pid[i];
        const int2 v = xy[i];
        const int bx = (int)(((int64_t)v.x - x0[p]) >> ls), by = (int)(((int64_t)v.y - y0[p]) >> ls);
        key[i] = pack_key(p, by, bx, kb);
        idx[i] = (uint32_t)i;
    }
}

// flag[i] = 1 where a run of equal keys starts (and key is not the skip value)
__global__ void run_start_kernel(const uint64_t* __restrict__ key, int64_t n, uint64_t skip,
                                 int32_t* __restrict__ flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = (key[i] != skip && (i == 0 || key[i] != key[i - 1])) ? 1 : 0;
}

// out[pos[i]] = key[i] and first[pos[i]] = i at run starts; first[m] = n (m runs)
__global__ void run_compact_kernel(const uint64_t* __restrict__ key, int64_t n, const int32_t* __restrict__ flag,
                                   const int32_t* __restrict__ pos, uint64_t* __restrict__ out,
                                   int32_t* __restrict__ first) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (flag[i]) {
            out[pos[i]] = key[i];
            if (first) first[pos[i]] = (int32_t)i;
        }
        if (i == 0 && first) first[pos[n]] = (int32_t)n;
    }
}

// *mx = longest run (first[j + 1] - first[j]) over j < m
__global__ void max_run_kernel(const int32_t* __restrict__ first, int64_t m, int* __restrict__ mx) {
    int best = 0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        best = max(best, first[j + 1] - first[j]);
    for (int o = 16; o; o >>= 1) best = max(best, __shfl_xor_sync(kFull, best, o));
    if ((threadIdx.x & 31) == 0) atomicMax(mx, best);
}

// sorted points: perm = the caller's index, loc = lx | ly << 16 inside the leaf
__global__ void point_order_kernel(const int2* __restrict__ xy, int64_t n, const uint32_t* __restrict__ idx,
                                   const int32_t* __restrict__ pid, const int32_t* __restrict__ x0,
                                   const int32_t* __restrict__ y0, int ls, int32_t* __restrict__ loc,
                                   int32_t* __restrict__ perm) {
    const int mask = (1 << ls) - 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = idx[i];
        const int p = pid[j];
        const int2 v = xy[j];
        const int lx = (int)(((int64_t)v.x - x0[p]) & mask), ly = (int)(((int64_t)v.y - y0[p]) & mask);
        loc[i] = lx | (ly << 16);
        perm[i] = (int32_t)j;
    }
}

// first sorted source / target of every occupied leaf (lower bound of its key); entry m
// holds the totals
__global__ void leaf_ranges_kernel(const uint64_t* __restrict__ leaves, int64_t m, const uint64_t* __restrict__ sk,
                                   int64_t ns, const uint64_t* __restrict__ tk, int64_t nt, int32_t* __restrict__ rs,
                                   int32_t* __restrict__ rt) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= m; j += (int64_t)gridDim.x * blockDim.x) {
        if (j == m) {
            rs[j] = (int32_t)ns;
            rt[j] = (int32_t)nt;
        } else {
            rs[j] = (int32_t)lower_bound_key(sk, ns, leaves[j]);
            rt[j] = (int32_t)lower_bound_key(tk, nt, leaves[j]);
        }
    }
}

// Boxes of every level from the occupied leaves.  A box of level k (k levels above the
// leaves) of problem p is the key (k << kbits) | (p, y >> k, x >> k) of any leaf below it;
// the levels of p are k = 1 .. L_p - 2 (levels >= 2 of its own tree).  Leaf j emits its
// level-k key only when it heads its level-k row segment (the previous leaf lies in
// another problem, row or level-k column), which leaves at most the 2^k leaf rows of a
// box to remove as duplicates.  Entry (k - 1) m + j.
__global__ void head_flag_kernel(const uint64_t* __restrict__ leaves, int64_t m, int kmax, const int32_t* __restrict__ L,
                                 int kb, int32_t* __restrict__ flag) {
    const int64_t n = m * kmax;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(i / m) + 1;
        const int64_t j = i - (int64_t)(k - 1) * m;
        int p, y, x;
        unpack_key(leaves[j], kb, p, y, x);
        bool head = L[p] - k >= 2;
        if (head && j > 0) {
            int pp, yy, xx;
            unpack_key(leaves[j - 1], kb, pp, yy, xx);
            head = !(pp == p && yy == y && (xx >> k) == (x >> k));
        }
        flag[i] = head ? 1 : 0;
    }
}

__global__ void head_key_kernel(const uint64_t* __restrict__ leaves, int64_t m, int kmax, int kb, int kbits,
                                const int32_t* __restrict__ flag, const int32_t* __restrict__ pos,
                                uint64_t* __restrict__ out) {
    const int64_t n = m * kmax;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[i]) continue;
        const int k = (int)(i / m) + 1;
        const int64_t j = i - (int64_t)(k - 1) * m;
        int p, y, x;
        unpack_key(leaves[j], kb, p, y, x);
        out[pos[i]] = ((uint64_t)k << kbits) | pack_key(p, y >> k, x >> k, kb);
    }
}

// class-major key (k, class, problem, y >> 1, x >> 1) of every box of every level (value:
// its position in the level-major row-major key array A)
__global__ void class_key_kernel(const uint64_t* __restrict__ A, int64_t n, int kb, int kbits,
                                 uint64_t* __restrict__ ck, uint32_t* __restrict__ idx) {
    const uint64_t low = ((uint64_t)1 << kbits) - 1;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = A[g];
        const uint64_t k = key >> kbits;
        int p, y, x;
        unpack_key(key & low, kb, p, y, x);
        const uint64_t c = (uint64_t)((x & 1) | ((y & 1) << 1));
        ck[g] = (k << (kbits + 2)) | (c << kbits) | pack_key(p, y >> 1, x >> 1, kb);
        idx[g] = (uint32_t)g;
    }
}

// first class-major position of class c of level k (entry 4 k + c; entry 4 nk: all boxes)
__global__ void class_starts_kernel(const uint64_t* __restrict__ ck, int64_t n, int nk, int kbits,
                                    int64_t* __restrict__ cstart) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > 4 * nk) return;
    if (t == 4 * nk) {
        cstart[t] = n;
        return;
    }
    const uint64_t v = ((uint64_t)(t >> 2) << (kbits + 2)) | ((uint64_t)(t & 3) << kbits);
    cstart[t] = lower_bound_key(ck, n, v);
}

// Box b of the class-major order (all levels, level-major) <- its row-major entry cm[b]
// of A: problem, coordinates, the level-local compact id of each entry of A, and the
// row-major leaf index of each level-0 box.
__global__ void box_records_kernel(const uint64_t* __restrict__ A, const uint64_t* __restrict__ ck,
                                   const uint32_t* __restrict__ cm, int64_t n, const int64_t* __restrict__ cstart, int kb,
                                   int kbits, int32_t* __restrict__ bp, int32_t* __restrict__ bxy,
                                   int32_t* __restrict__ local_of, int32_t* __restrict__ leaf_rl) {
    const uint64_t low = ((uint64_t)1 << kbits) - 1;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(ck[b] >> (kbits + 2));
        const uint32_t g = cm[b];
        int p, y, x;
        unpack_key(A[g] & low, kb, p, y, x);
        bp[b] = p;
        bxy[b] = x | (y << 16);
        const int64_t local = b - cstart[4 * k];
        local_of[g] = (int32_t)local;
        if (k == 0) leaf_rl[local] = (int32_t)g;
    }
}

// Parent, children and interaction list (Def. 6.1, slot order of the box's class) of
// every box, by search in A (sorted by level, problem, row, column).  A list's 27 boxes
// lie in the six rows y - 2 - (y & 1) .. y + 3 - (y & 1), six columns wide: one search
// per row, then a scan of at most six keys; s_slot maps an offset to its slot.
__global__ void links_kernel(int64_t n, const uint64_t* __restrict__ ck, const uint64_t* __restrict__ A, int64_t na,
                             const int32_t* __restrict__ local_of, const int32_t* __restrict__ bp,
                             const int32_t* __restrict__ bxy, const int32_t* __restrict__ L, int kb, int kbits, int kmax,
                             const int2* __restrict__ rows, const int64_t* __restrict__ row_off, int np,
                             int32_t* __restrict__ par, int32_t* __restrict__ ch, int32_t* __restrict__ il) {
    __shared__ signed char s_slot[4][36];
    for (int t = threadIdx.x; t < 4 * 36; t += blockDim.x) (&s_slot[0][0])[t] = -1;
    __syncthreads();
    for (int t = threadIdx.x; t < 4 * 27; t += blockDim.x) {
        const int c = t / 27, st = t % 27, px = c & 1, py = c >> 1;
        int dx, dy;
        interaction_slot(px, py, st, dx, dy);
        s_slot[c][(dy + 2 + py) * 6 + dx + 2 + px] = (signed char)st;
    }
    __syncthreads();
    const uint64_t cmask = ((uint64_t)1 << kb) - 1;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(ck[b] >> (kbits + 2));
        const int p = bp[b];
        const int x = bxy[b] & 0xffff, y = bxy[b] >> 16;
        const int l = L[p] - k;
        const int nn = 1 << l;
        const int px = x & 1, py = y & 1, c = px | (py << 1);
        // parent at level k + 1 (a level >= 2 of the problem's tree)
        int pr = -1;
        if (k + 1 <= kmax && l - 1 >= 2) {
            const uint64_t v = ((uint64_t)(k + 1) << kbits) | pack_key(p, y >> 1, x >> 1, kb);
            int64_t e;
            const int64_t j = find_in_row(A, na, rows, row_off, np, k + 1, p, y >> 1, v, e);
            if (j < e && A[j] == v) pr = local_of[j];
        }
        par[b] = pr;
        // children at level k - 1, two per row
        if (k >= 1) {
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const uint64_t v = ((uint64_t)(k - 1) << kbits) | pack_key(p, 2 * y + r, 2 * x, kb);
                int64_t e;
                int64_t j = find_in_row(A, na, rows, row_off, np, k - 1, p, 2 * y + r, v, e);
                int c0 = -1, c1 = -1;
                if (j < e && A[j] == v) {
                    c0 = local_of[j];
                    ++j;
                }
                if (j < e && A[j] == v + 1) c1 = local_of[j];
                ch[b * 4 + 2 * r] = c0;
                ch[b * 4 + 2 * r + 1] = c1;
            }
        }
        // interaction list
        int32_t* out = il + b * 27;
        for (int st = 0; st < 27; ++st) out[st] = -1;
        const uint64_t lev = (uint64_t)k << kbits;
        const int xlo = max(x - 2 - px, 0), xhi = min(x + 3 - px, nn - 1);
        for (int dy = -2 - py; dy <= 3 - py; ++dy) {
            const int yy = y + dy;
            if (yy < 0 || yy >= nn) continue;
            const uint64_t vhi = lev | pack_key(p, yy, xhi, kb);
            int64_t e;
            for (int64_t j = find_in_row(A, na, rows, row_off, np, k, p, yy, lev | pack_key(p, yy, xlo, kb), e);
                 j < e && A[j] <= vhi; ++j) {
                const int dx = (int)(A[j] & cmask) - x;
                const int sl = s_slot[c][(dy + 2 + py) * 6 + dx + 2 + px];
                if (sl >= 0) out[sl] = local_of[j];
            }
        }
    }
}

// leaf occupancy of every problem's dense leaf grid at side 2^ls (L: leaf levels at that
// side, cell_off: first cell of each problem)
__global__ void dense_count_kernel(const int2* __restrict__ xy, int64_t n, const int32_t* __restrict__ pid,
                                   const int32_t* __restrict__ x0, const int32_t* __restrict__ y0,
                                   const int32_t* __restrict__ L, const int64_t* __restrict__ cell_off, int ls,
                                   int32_t* __restrict__ cnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int p = pid[i];
        const int2 v = xy[i];
        const int64_t bx = ((int64_t)v.x - x0[p]) >> ls, by = ((int64_t)v.y - y0[p]) >> ls;
        atomicAdd(cnt + cell_off[p] + (by << L[p]) + bx, 1);
    }
}

// Counting sort on the dense leaf grids: each point takes the next slot of its leaf
// (cursor = the leaf's first slot, advanced atomically), so points come out row-major by
// leaf per problem, in arrival order inside a leaf; loc = lx | ly << 16, perm = the
// caller's index.
__global__ void dense_scatter_kernel(const int2* __restrict__ xy, int64_t n, const int32_t* __restrict__ pid,
                                     const int32_t* __restrict__ x0, const int32_t* __restrict__ y0,
                                     const int32_t* __restrict__ L, const int64_t* __restrict__ cell_off, int ls,
                                     int32_t* __restrict__ cursor, int32_t* __restrict__ loc,
                                     int32_t* __restrict__ perm) {
    const int mask = (1 << ls) - 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int p = pid[i];
        const int2 v = xy[i];
        const int64_t dx = (int64_t)v.x - x0[p], dy = (int64_t)v.y - y0[p];
        const int pos = atomicAdd(cursor + cell_off[p] + ((dy >> ls) << L[p]) + (dx >> ls), 1);
        loc[pos] = (int)(dx & mask) | ((int)(dy & mask) << 16);
        perm[pos] = (int32_t)i;
    }
}

// 1 where a dense leaf holds a source or a target
__global__ void occupied_flag_kernel(const int32_t* __restrict__ cs, const int32_t* __restrict__ ct, int64_t cells,
                                     int32_t* __restrict__ flag) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += (int64_t)gridDim.x * blockDim.x)
        flag[c] = (cs[c] + (ct ? ct[c] : 0)) > 0 ? 1 : 0;
}

// occupied leaf j (dense cell c, pos[c] = j): key, first source and first target
__global__ void occupied_compact_kernel(const int32_t* __restrict__ flag, const int32_t* __restrict__ pos,
                                        int64_t cells, const int64_t* __restrict__ cell_off, int np,
                                        const int32_t* __restrict__ L, int kb, const int32_t* __restrict__ ss,
                                        const int32_t* __restrict__ ts, uint64_t* __restrict__ key,
                                        int32_t* __restrict__ rs, int32_t* __restrict__ rt) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[c]) continue;
        int lo = 0, hi = np;  // problem p: cell_off[p] <= c < cell_off[p + 1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (cell_off[mid] <= c) lo = mid;
            else hi = mid;
        }
        const int64_t r = c - cell_off[lo];
        const int j = pos[c];
        key[j] = pack_key(lo, (int)(r >> L[lo]), (int)(r & (((int64_t)1 << L[lo]) - 1)), kb);
        rs[j] = ss[c];
        rt[j] = ts[c];
    }
}

// *mx = max(*mx, largest count)
__global__ void max_count_kernel(const int32_t* __restrict__ cnt, int64_t n, int* __restrict__ mx) {
    int best = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        best = max(best, cnt[i]);
    for (int o = 16; o; o >>= 1) best = max(best, __shfl_xor_sync(kFull, best, o));
    if ((threadIdx.x & 31) == 0) atomicMax(mx, best);
}

// *diff = 1 if the two point lists differ anywhere
__global__ void same_points_kernel(const int2* __restrict__ a, const int2* __restrict__ b, int64_t n,
                                   int* __restrict__ diff) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int2 u = a[i], v = b[i];
        if (u.x != v.x || u.y != v.y) *diff = 1;
    }
}

// strip key (problem, leaf row, column / SW) of each occupied leaf with a target, the
// skip value for the others (non-decreasing over the target leaves: leaves are row-major)
__global__ void strip_key_kernel(const uint64_t* __restrict__ leaves, const int32_t* __restrict__ rt, int64_t m,
                                 int kb, int SW, uint64_t skip, uint64_t* __restrict__ out) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        int p, y, x;
        unpack_key(leaves[j], kb, p, y, x);
        out[j] = rt[j + 1] > rt[j] ? pack_key(p, y, x / SW, kb) : skip;
    }
}

// strip records (problem, leaf row, first column, 0)
__global__ void strip_record_kernel(const uint64_t* __restrict__ sk, int64_t m, int kb, int SW,
                                    int4* __restrict__ strips) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        int p, y, x;
        unpack_key(sk[j], kb, p, y, x);
        strips[j] = make_int4(p, y, x * SW, 0);
    }
}

// Leaves of the three row segments a strip's near field reads (rows by - 1 .. by + 1,
// columns max(bx0 - 1, 0) .. min(bx0 + SW, n - 1)): index ranges [j0, j1) in the sorted
// occupied-leaf keys, found by binary search.  The end key is column c_hi + 1 taken as a
// sum, so that one past the row's last column carries into the next row.
__global__ void strip_rows_kernel(const int4* __restrict__ strips, int64_t nstr, const uint64_t* __restrict__ leaves,
                                  int64_t m, const int32_t* __restrict__ L, int kb, int SW,
                                  int4* __restrict__ rows) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nstr; i += (int64_t)gridDim.x * blockDim.x) {
        const int4 q = strips[i];
        const int p = q.x, by = q.y, bx0 = q.z;
        const int n = 1 << L[p];
        const int bx1 = min(bx0 + SW, n);
        const int c_lo = max(bx0 - 1, 0), c_hi = min(bx1, n - 1);
        int j[6];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int yy = by + r - 1;
            if (yy >= 0 && yy < n) {
                const uint64_t row = ((uint64_t)p << (2 * kb)) + ((uint64_t)yy << kb);
                j[2 * r] = (int)lower_bound_key(leaves, m, row + (uint64_t)c_lo);
                j[2 * r + 1] = (int)lower_bound_key(leaves, m, row + (uint64_t)c_hi + 1);
            } else {
                j[2 * r] = j[2 * r + 1] = -1;
            }
        }
        rows[2 * i] = make_int4(j[0], j[1], j[2], j[3]);
        rows[2 * i + 1] = make_int4(j[4], j[5], 0, 0);
    }
}

int ceil_log2(int64_t v) {
    int k = 0;
    while (((int64_t)1 << k) < v) ++k;
    return k;
}

struct DevBuf {  // stream-ordered temporary freed on scope exit
    void* ptr = nullptr;
    cudaStream_t s = nullptr;
    ~DevBuf() {
        if (ptr) cudaFreeAsync(ptr, s);
    }
    int get(size_t bytes, cudaStream_t st) {
        s = st;
        const cudaError_t e = dev_malloc(&ptr, bytes ? bytes : 16, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ptr = nullptr;
            return fail(LFMM_ENOMEM, "tree build: device allocation of " + std::to_string(bytes) + " bytes failed");
        }
        return LFMM_OK;
    }
};

int alloc(Forest& F, void** out, size_t n, cudaStream_t s) {
    *out = nullptr;
    const cudaError_t e = dev_malloc(out, n ? n : 16, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return fail(LFMM_ENOMEM, "device allocation of " + std::to_string(n) + " bytes failed");
    }
    F.owned.push_back(*out);
    F.bytes += (int64_t)(n ? n : 16);
    return LFMM_OK;
}

// Unique keys of a sorted array (skipping `skip`): out[0..m), first[0..m] (first[m] = n),
// m on the host.  flag / pos: n + 1 ints of scratch; sums: scan_tmp_ints(n).
int unique_runs(const uint64_t* key, int64_t n, uint64_t skip, uint64_t* out, int32_t* first, int32_t* flag,
                int32_t* pos, int32_t* sums, int* m_host, cudaStream_t s) {
    if (n == 0) {
        *m_host = 0;
        if (first) LFMM_CUDA_TRY(cudaMemsetAsync(first, 0, sizeof(int32_t), s));
        return LFMM_OK;
    }
    run_start_kernel<<<grid_of(n), kT, 0, s>>>(key, n, skip, flag);
    LFMM_CUDA_TRY(exscan(flag, pos, n, sums, s));
    run_compact_kernel<<<grid_of(n), kT, 0, s>>>(key, n, flag, pos, out, first);
    LFMM_CUDA_TRY(cudaGetLastError());
    int32_t h = 0;
    LFMM_CUDA_TRY(cudaMemcpyAsync(&h, pos + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LFMM_CUDA_TRY(cudaStreamSynchronize(s));
    *m_host = h;
    return LFMM_OK;
}

}  // namespace

int forest_build(Forest& F, const int32_t* src, const int64_t* soff_h, int64_t ns, const int32_t* tgt,
                 const int64_t* toff_h, int64_t nt, int np, int leaf_size, int max_leaf_side, cudaStream_t s,
                 PhaseTimer* timer) {
    int st;
    F.np = np;
    F.ns = ns;
    F.nt = nt;
    if (ns > INT32_MAX / 2 || nt > INT32_MAX / 2) return fail(LFMM_EINVAL, "forest too large");
    void* v;
    // targets = sources (same counts, offsets and coordinates): one sort serves both sides
    bool same = ns == nt && std::equal(soff_h, soff_h + np + 1, toff_h);
    // problem offsets and per-point problem ids (temporaries)
    DevBuf offs, pids;
    if ((st = offs.get((size_t)2 * (np + 1) * sizeof(int64_t) + 16, s))) return st;
    int64_t* soff = (int64_t*)offs.ptr;
    int64_t* toff = soff + (np + 1);
    int* word = (int*)(toff + (np + 1));  // the coordinate comparison's flag
    LFMM_CUDA_TRY(cudaMemcpyAsync(soff, soff_h, (np + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    LFMM_CUDA_TRY(cudaMemcpyAsync(toff, toff_h, (np + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    LFMM_CUDA_TRY(cudaMemsetAsync(word, 0, sizeof(int), s));
    if (same && src != tgt) same_points_kernel<<<grid_of(ns), kT, 0, s>>>((const int2*)src, (const int2*)tgt, ns, word);
    // bounding boxes first (int4: 16-byte aligned at the allocation's start), then the ids
    if ((st = pids.get((size_t)np * sizeof(int4) + (size_t)(ns + nt) * sizeof(int32_t), s))) return st;
    int4* bb = (int4*)pids.ptr;
    int32_t* spid = (int32_t*)(bb + np);
    int32_t* tpid = spid + ns;
    if (np == 1) {
        LFMM_CUDA_TRY(cudaMemsetAsync(spid, 0, (size_t)(ns + nt) * sizeof(int32_t), s));
        LFMM_CUDA_TRY(launch_set4((int*)bb, INT_MAX, INT_MAX, INT_MIN, INT_MIN, s));
        LFMM_CUDA_TRY(launch_bbox(src, ns, tgt, nt, (int*)bb, s));
    } else {
        pid_kernel<<<std::min(np, 152 * 8), kT, 0, s>>>(soff, np, spid);
        pid_kernel<<<std::min(np, 152 * 8), kT, 0, s>>>(toff, np, tpid);
        bbox_forest_kernel<<<std::min(np, 152 * 8), kT, 0, s>>>((const int2*)src, soff, (const int2*)tgt, toff, np,
                                                               bb);
    }
    LFMM_CUDA_TRY(cudaGetLastError());
    timer->add_launches(5);
    std::vector<int4> hbb(np);
    int hdiff = 0;
    LFMM_CUDA_TRY(cudaMemcpyAsync(hbb.data(), bb, np * sizeof(int4), cudaMemcpyDeviceToHost, s));
    LFMM_CUDA_TRY(cudaMemcpyAsync(&hdiff, word, sizeof(int), cudaMemcpyDeviceToHost, s));
    LFMM_CUDA_TRY(cudaStreamSynchronize(s));
    same = same && hdiff == 0;
    F.x0.resize(np);
    F.y0.resize(np);
    F.K.resize(np);
    int Kmax = 0;
    for (int p = 0; p < np; ++p) {
        const int4 b = hbb[p];
        if (b.x > b.z) return fail(LFMM_EINVAL, "forest problem " + std::to_string(p) + " has no points");
        F.x0[p] = b.x;
        F.y0[p] = b.y;
        const int64_t ext = std::max((int64_t)b.z - b.x, (int64_t)b.w - b.y) + 1;
        if (ext > ((int64_t)1 << 30)) return fail(LFMM_EINVAL, "points span more than 2^30 lattice cells");
        F.K[p] = ceil_log2(ext);
        Kmax = std::max(Kmax, F.K[p]);
    }
    const int pbits = ceil_log2(std::max(np, 1));
    if ((st = alloc(F, &v, (size_t)3 * np * sizeof(int32_t), s))) return st;
    int32_t* dx0 = (int32_t*)v;
    int32_t* dy0 = dx0 + np;
    int32_t* dL = dy0 + np;
    F.d_L = dL;
    LFMM_CUDA_TRY(cudaMemcpyAsync(dx0, F.x0.data(), np * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    LFMM_CUDA_TRY(cudaMemcpyAsync(dy0, F.y0.data(), np * sizeof(int32_t), cudaMemcpyHostToDevice, s));

    // sorting scratch, sized for the largest sort of this phase (the union of source and
    // target leaves)
    const int64_t nmax = std::max<int64_t>({ns, nt, 1});
    const int64_t nsort = 2 * nmax;
    DevBuf kv, sb, runs;
    // sorted source keys / values, target keys / values, and one spare pair of 2 nmax
    if ((st = kv.get((size_t)4 * nmax * (sizeof(uint64_t) + sizeof(uint32_t)), s))) return st;
    uint64_t* sk = (uint64_t*)kv.ptr;      // source keys
    uint64_t* tk = sk + nmax;              // target keys
    uint64_t* kspare = sk + 2 * nmax;      // 2 nmax
    uint32_t* sv = (uint32_t*)(sk + 4 * nmax);
    uint32_t* tv = sv + nmax;
    SortBufs sbuf;
    const int64_t hist_ints = sort_hist_ints(nsort);
    if ((st = sb.get((size_t)(nsort * (sizeof(uint64_t) + sizeof(uint32_t))) +
                         (size_t)(hist_ints + scan_tmp_ints(hist_ints)) * sizeof(int32_t), s)))
        return st;
    sbuf.k2 = (uint64_t*)sb.ptr;
    sbuf.v2 = (uint32_t*)(sbuf.k2 + nsort);
    sbuf.hist = (int32_t*)(sbuf.v2 + nsort);
    sbuf.sums = sbuf.hist + hist_ints;
    // run scratch: flags, positions, firsts (n + 1 each), scan sums, two words, unique keys
    if ((st = runs.get((size_t)(3 * (nsort + 1) + scan_tmp_ints(nsort) + 2) * sizeof(int32_t) +
                           (size_t)(nsort + 1) * sizeof(uint64_t) + 16, s)))
        return st;
    int32_t* flag = (int32_t*)runs.ptr;
    int32_t* pos = flag + (nsort + 1);
    int32_t* first = pos + (nsort + 1);
    int32_t* ssum = first + (nsort + 1);
    int* mx = (int*)(ssum + scan_tmp_ints(nsort));
    uint64_t* ukeys = (uint64_t*)(((uintptr_t)(mx + 2) + 15) & ~(uintptr_t)15);  // unique keys

    // ---- 1. leaf side: the largest power of two <= max_leaf_side (and <= every root that
    // needs splitting) at which no leaf of any problem holds more than leaf_size points.
    // A candidate is checked on each problem's dense leaf grid when the grids are small,
    // else on sorted leaf keys (runs of equal keys are leaves), which then serve as the
    // point order.
    int ls = ceil_log2(max_leaf_side);
    if ((1 << ls) > max_leaf_side) --ls;
    ls = std::min(ls, Kmax);
    int maxs = 0, maxt = 0, kb = 1;
    bool dense = false;             // the final side was checked on dense grids (kept in cbk)
    DevBuf cbk;
    int64_t cells_k = 0;
    auto sort_side = [&](bool is_src, int bits, int* maxrun) -> int {
        const int64_t n = is_src ? ns : nt;
        uint64_t* k = is_src ? sk : tk;
        uint32_t* vv = is_src ? sv : tv;
        leaf_key_kernel<<<grid_of(n), kT, 0, s>>>((const int2*)(is_src ? src : tgt), n, is_src ? spid : tpid, dx0, dy0,
                                                  ls, kb, k, vv);
        LFMM_CUDA_TRY(cudaGetLastError());
        LFMM_CUDA_TRY(radix_sort(k, vv, n, bits, sbuf, s));
        timer->add_launches(1 + 5 * ((bits + 7) / 8));
        if (!maxrun) return LFMM_OK;
        int m = 0;
        int r;
        if ((r = unique_runs(k, n, ~0ull, ukeys, first, flag, pos, ssum, &m, s))) return r;
        LFMM_CUDA_TRY(cudaMemsetAsync(mx, 0, sizeof(int), s));
        max_run_kernel<<<grid_of(m), kT, 0, s>>>(first, m, mx);
        LFMM_CUDA_TRY(cudaMemcpyAsync(maxrun, mx, sizeof(int), cudaMemcpyDeviceToHost, s));
        LFMM_CUDA_TRY(cudaStreamSynchronize(s));
        timer->add_launches(5);
        return LFMM_OK;
    };
    for (;;) {
        F.L.assign(np, 0);
        int Lmax = 0;
        int64_t cells = 0;
        std::vector<int64_t> cell_off(np + 1, 0);
        for (int p = 0; p < np; ++p) {
            F.L[p] = std::max(0, F.K[p] - ls);
            Lmax = std::max(Lmax, F.L[p]);
            cell_off[p] = cells;
            cells += (int64_t)1 << (2 * F.L[p]);
        }
        cell_off[np] = cells;
        kb = std::max(1, Lmax);
        if (Lmax > 20 || pbits + 2 * kb + 7 > 63)
            return fail(LFMM_EUNSUPPORTED, "forest problem needs more than 2^20 leaves per side");
        LFMM_CUDA_TRY(cudaMemcpyAsync(dL, F.L.data(), np * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        const int bits = pbits + 2 * kb;
        dense = cells <= std::max<int64_t>(2 * (ns + nt), (int64_t)1 << 22);
        DevBuf cb;
        if (dense) {
            if ((st = cb.get((size_t)(np + 1) * sizeof(int64_t) + (size_t)2 * cells * sizeof(int32_t) + 16, s))) return st;
            int64_t* doff = (int64_t*)cb.ptr;
            int32_t* cnt = (int32_t*)(doff + np + 1);
            LFMM_CUDA_TRY(cudaMemcpyAsync(doff, cell_off.data(), (np + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
            LFMM_CUDA_TRY(cudaMemsetAsync(cnt, 0, (size_t)2 * cells * sizeof(int32_t), s));
            LFMM_CUDA_TRY(cudaMemsetAsync(mx, 0, 2 * sizeof(int), s));
            dense_count_kernel<<<grid_of(ns), kT, 0, s>>>((const int2*)src, ns, spid, dx0, dy0, dL, doff, ls, cnt);
            max_count_kernel<<<grid_of(cells), kT, 0, s>>>(cnt, cells, mx);
            if (!same) {
                dense_count_kernel<<<grid_of(nt), kT, 0, s>>>((const int2*)tgt, nt, tpid, dx0, dy0, dL, doff, ls,
                                                             cnt + cells);
                max_count_kernel<<<grid_of(cells), kT, 0, s>>>(cnt + cells, cells, mx + 1);
            }
            LFMM_CUDA_TRY(cudaGetLastError());
            int h[2] = {0, 0};
            LFMM_CUDA_TRY(cudaMemcpyAsync(h, mx, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
            LFMM_CUDA_TRY(cudaStreamSynchronize(s));
            timer->add_launches(4);
            maxs = h[0];
            maxt = same ? h[0] : h[1];
        } else {
            if ((st = sort_side(true, bits, &maxs))) return st;
            if (same) maxt = maxs;
            else if ((st = sort_side(false, bits, &maxt))) return st;
        }
        if (std::max(maxs, maxt) <= leaf_size || ls == 0) {
            if (dense) {  // keep the grids' offsets and counts for the counting sort
                std::swap(cbk.ptr, cb.ptr);
                cbk.s = s;
                cells_k = cells;
            }
            break;
        }
        --ls;
    }
    F.ls = ls;
    F.side = 1 << ls;
    F.kb = kb;
    F.max_src = maxs;
    F.max_tgt = maxt;
    const int kbits = pbits + 2 * kb;          // bits of a packed key
    int Lmax = 0;
    for (int p = 0; p < np; ++p) Lmax = std::max(Lmax, F.L[p]);
    // ---- 2. points in leaf order, occupied leaves with their first source and target
    void* vp;
    if ((st = alloc(F, &vp, (size_t)2 * (ns + (same ? 0 : nt)) * sizeof(int32_t), s))) return st;
    F.sloc = (int32_t*)vp;
    F.sperm = F.sloc + ns;
    F.tloc = same ? F.sloc : F.sperm + ns;
    F.tperm = same ? F.sperm : F.tloc + nt;
    int M = 0;
    if (dense) {
        // counting sort on the grids: first slot of every leaf by one exclusive scan of the
        // counts, points placed by atomic cursors; occupied leaves by one compaction
        const int64_t cells = cells_k;
        if (cells > INT32_MAX / 2) return fail(LFMM_EUNSUPPORTED, "forest leaf grids too large");
        int64_t* doff = (int64_t*)cbk.ptr;
        int32_t* cs = (int32_t*)(doff + np + 1);
        int32_t* ct = same ? nullptr : cs + cells;
        DevBuf gb;
        const int64_t sc = scan_tmp_ints(cells);
        if ((st = gb.get((size_t)(4 * (cells + 1) + 2 * sc) * sizeof(int32_t), s))) return st;
        int32_t* ss = (int32_t*)gb.ptr;      // [cells + 1] first source of each leaf
        int32_t* ts = ss + (cells + 1);      // [cells + 1] first target (targets != sources)
        int32_t* gflag = ts + (cells + 1);
        int32_t* gpos = gflag + (cells + 1);
        int32_t* gsum = gpos + (cells + 1);
        // occupied leaves before the counts turn into cursors
        occupied_flag_kernel<<<grid_of(cells), kT, 0, s>>>(cs, ct, cells, gflag);
        LFMM_CUDA_TRY(exscan(gflag, gpos, cells, gsum, s));
        LFMM_CUDA_TRY(exscan(cs, ss, cells, gsum + sc, s));
        if (!same) LFMM_CUDA_TRY(exscan(ct, ts, cells, gsum + sc, s));
        LFMM_CUDA_TRY(cudaMemcpyAsync(&M, gpos + cells, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LFMM_CUDA_TRY(cudaStreamSynchronize(s));
        if ((st = alloc(F, &vp, (size_t)(M + 1) * sizeof(uint64_t), s))) return st;
        F.rl_key = (uint64_t*)vp;
        if ((st = alloc(F, &vp, (size_t)(same ? 2 : 3) * (M + 1) * sizeof(int32_t), s))) return st;
        F.rl_s = (int32_t*)vp;
        F.rl_id = F.rl_s + (M + 1);
        F.rl_t = same ? F.rl_s : F.rl_id + (M + 1);
        occupied_compact_kernel<<<grid_of(cells), kT, 0, s>>>(gflag, gpos, cells, doff, np, dL, kb, ss, same ? ss : ts,
                                                              F.rl_key, F.rl_s, F.rl_t);
        LFMM_CUDA_TRY(cudaMemcpyAsync(F.rl_s + M, ss + cells, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        if (!same) LFMM_CUDA_TRY(cudaMemcpyAsync(F.rl_t + M, ts + cells, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        // the counts become cursors (each leaf's first slot), then the points are placed
        LFMM_CUDA_TRY(cudaMemcpyAsync(cs, ss, (size_t)cells * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        dense_scatter_kernel<<<grid_of(ns), kT, 0, s>>>((const int2*)src, ns, spid, dx0, dy0, dL, doff, ls, cs, F.sloc,
                                                        F.sperm);
        if (!same) {
            LFMM_CUDA_TRY(cudaMemcpyAsync(ct, ts, (size_t)cells * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
            dense_scatter_kernel<<<grid_of(nt), kT, 0, s>>>((const int2*)tgt, nt, tpid, dx0, dy0, dL, doff, ls, ct,
                                                            F.tloc, F.tperm);
        }
        LFMM_CUDA_TRY(cudaGetLastError());
        timer->add_launches(16);
    } else {
        point_order_kernel<<<grid_of(ns), kT, 0, s>>>((const int2*)src, ns, sv, spid, dx0, dy0, ls, F.sloc, F.sperm);
        if (!same)
            point_order_kernel<<<grid_of(nt), kT, 0, s>>>((const int2*)tgt, nt, tv, tpid, dx0, dy0, ls, F.tloc, F.tperm);
        LFMM_CUDA_TRY(cudaGetLastError());
        if (same) {
            if ((st = alloc(F, &vp, (size_t)(ns + 1) * sizeof(uint64_t), s))) return st;
            F.rl_key = (uint64_t*)vp;
            if ((st = unique_runs(sk, ns, ~0ull, F.rl_key, nullptr, flag, pos, ssum, &M, s))) return st;
        } else {
            // unique source leaves and unique target leaves, merged by one more sort
            int mm = 0, mt = 0;
            if ((st = unique_runs(sk, ns, ~0ull, kspare, nullptr, flag, pos, ssum, &mm, s))) return st;
            if ((st = unique_runs(tk, nt, ~0ull, kspare + mm, nullptr, flag, pos, ssum, &mt, s))) return st;
            LFMM_CUDA_TRY(radix_sort(kspare, nullptr, (int64_t)mm + mt, kbits, sbuf, s));
            if ((st = alloc(F, &vp, (size_t)(mm + mt + 1) * sizeof(uint64_t), s))) return st;
            F.rl_key = (uint64_t*)vp;
            if ((st = unique_runs(kspare, (int64_t)mm + mt, ~0ull, F.rl_key, nullptr, flag, pos, ssum, &M, s))) return st;
        }
        if ((st = alloc(F, &vp, (size_t)(same ? 2 : 3) * (M + 1) * sizeof(int32_t), s))) return st;
        F.rl_s = (int32_t*)vp;
        F.rl_id = F.rl_s + (M + 1);
        F.rl_t = same ? F.rl_s : F.rl_id + (M + 1);
        leaf_ranges_kernel<<<grid_of(M + 1), kT, 0, s>>>(F.rl_key, M, sk, ns, same ? sk : tk, same ? ns : nt, F.rl_s,
                                                         F.rl_t);
        LFMM_CUDA_TRY(cudaGetLastError());
        timer->add_launches(12);
    }
    F.n_leaves = M;

    // ---- 3. boxes of every level: A = the leaves (k = 0), then the boxes of levels
    // k = 1 .. kmax, sorted by (k, problem, row, column); compact ids number each level's
    // boxes in class-major order; links by search in A
    F.kmax = Lmax - 2;  // may be negative: no far field anywhere
    const int nk = std::max(F.kmax, 0) + 1;
    const int lbits = ceil_log2(nk);
    const int kmx = std::max(F.kmax, 0);
    int E = 0, U = 0;
    DevBuf ebuf, abuf;
    // level >= 1 keys of the row-segment heads
    const int64_t nh = (int64_t)M * kmx;
    if (nh > INT32_MAX / 2) return fail(LFMM_EUNSUPPORTED, "tree too deep for the box lists");
    {
        DevBuf hb;
        if ((st = hb.get((size_t)(2 * (nh + 1) + scan_tmp_ints(nh)) * sizeof(int32_t), s))) return st;
        int32_t* hflag = (int32_t*)hb.ptr;
        int32_t* hpos = hflag + (nh + 1);
        int32_t* hsum = hpos + (nh + 1);
        if (nh > 0) {
            head_flag_kernel<<<grid_of(nh), kT, 0, s>>>(F.rl_key, M, kmx, dL, kb, hflag);
            LFMM_CUDA_TRY(exscan(hflag, hpos, nh, hsum, s));
            LFMM_CUDA_TRY(cudaMemcpyAsync(&E, hpos + nh, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            LFMM_CUDA_TRY(cudaStreamSynchronize(s));
        }
        // A (M + E keys at most) and, past it, the emitted keys
        if ((st = abuf.get((size_t)(M + 2 * (int64_t)E + 1) * sizeof(uint64_t), s))) return st;
        if (E > 0) {
            head_key_kernel<<<grid_of(nh), kT, 0, s>>>(F.rl_key, M, kmx, kb, kbits, hflag, hpos,
                                                       (uint64_t*)abuf.ptr + M + E);
            LFMM_CUDA_TRY(cudaGetLastError());
        }
        timer->add_launches(5);
    }
    uint64_t* A = (uint64_t*)abuf.ptr;
    LFMM_CUDA_TRY(cudaMemcpyAsync(A, F.rl_key, (size_t)M * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    // scratch of the level sorts: E keys, then the class sort of all boxes
    const int64_t nlev = std::max<int64_t>((int64_t)M + E, 1);
    SortBufs lsb;
    const int64_t lh = sort_hist_ints(nlev);
    if ((st = ebuf.get((size_t)nlev * (2 * sizeof(uint64_t) + 2 * sizeof(uint32_t) + sizeof(int32_t)) +
                           (size_t)(lh + scan_tmp_ints(lh) + 3 * (nlev + 1) + scan_tmp_ints(nlev) + 8) * sizeof(int32_t),
                       s)))
        return st;
    uint64_t* ck = (uint64_t*)ebuf.ptr;
    lsb.k2 = ck + nlev;
    uint32_t* cidx = (uint32_t*)(lsb.k2 + nlev);
    lsb.v2 = cidx + nlev;
    int32_t* local_of = (int32_t*)(lsb.v2 + nlev);
    lsb.hist = local_of + nlev;
    lsb.sums = lsb.hist + lh;
    int32_t* lflag = lsb.sums + scan_tmp_ints(lh);
    int32_t* lpos = lflag + (nlev + 1);
    int32_t* lsum = lpos + (nlev + 1);
    if (E > 0) {
        uint64_t* ek = A + M + E;
        LFMM_CUDA_TRY(radix_sort(ek, nullptr, E, kbits + lbits, lsb, s));
        if ((st = unique_runs(ek, E, ~0ull, A + M, nullptr, lflag, lpos, lsum, &U, s))) return st;
        timer->add_launches(4 + 5 * ((kbits + lbits + 7) / 8));
    }
    const int64_t NB = (int64_t)M + U;
    // class-major order of every level
    class_key_kernel<<<grid_of(NB), kT, 0, s>>>(A, NB, kb, kbits, ck, cidx);
    LFMM_CUDA_TRY(cudaGetLastError());
    LFMM_CUDA_TRY(radix_sort(ck, cidx, NB, kbits + 2 + lbits, lsb, s));
    // per-box records of all levels in one allocation (level k at box_off[k])
    if ((st = alloc(F, &vp, (size_t)NB * (3 + 27 + 4) * sizeof(int32_t) + (size_t)M * sizeof(int32_t) +
                                (size_t)(4 * nk + 1 + 5 * nk) * sizeof(int64_t) + 16, s)))
        return st;
    int64_t* cstart = (int64_t*)vp;                 // 4 nk + 1
    int64_t* dcls = cstart + (4 * nk + 1);          // 5 nk, level-local class starts
    int32_t* bp_all = (int32_t*)(dcls + 5 * nk);
    int32_t* bxy_all = bp_all + NB;
    int32_t* par_all = bxy_all + NB;
    int32_t* il_all = par_all + NB;
    int32_t* ch_all = il_all + 27 * NB;
    int32_t* leaf_rl = ch_all + 4 * NB;
    class_starts_kernel<<<(4 * nk + 1 + kT - 1) / kT, kT, 0, s>>>(ck, NB, nk, kbits, cstart);
    box_records_kernel<<<grid_of(NB), kT, 0, s>>>(A, ck, cidx, NB, cstart, kb, kbits, bp_all, bxy_all, local_of, leaf_rl);
    // the [first, end) of every box row of A, so that the links' searches (parent, two child
    // rows, six neighbour rows per box) cover one row instead of all of A; without it (a
    // table far larger than the boxes) they search all of A
    DevBuf rowbuf;
    const int2* rows = nullptr;
    const int64_t* row_off = nullptr;
    {
        std::vector<int64_t> ro((size_t)nk * np + 1, 0);
        int64_t R = 0;
        for (int k = 0; k < nk; ++k)
            for (int p = 0; p < np; ++p) {
                ro[(size_t)k * np + p] = R;
                if (F.L[p] >= k) R += (int64_t)1 << (F.L[p] - k);
            }
        ro[(size_t)nk * np] = R;
        if (R <= 8 * NB + ((int64_t)1 << 20)) {
            if ((st = rowbuf.get((size_t)R * sizeof(int2) + ro.size() * sizeof(int64_t) + 16, s))) return st;
            int2* rt = (int2*)rowbuf.ptr;
            int64_t* ro_d = (int64_t*)(rt + R);
            LFMM_CUDA_TRY(cudaMemsetAsync(rt, 0, (size_t)R * sizeof(int2), s));
            LFMM_CUDA_TRY(cudaMemcpyAsync(ro_d, ro.data(), ro.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
            row_range_kernel<<<grid_of(NB), kT, 0, s>>>(A, NB, kb, kbits, np, ro_d, rt);
            rows = rt;
            row_off = ro_d;
            timer->add_launches(1);
        }
    }
    links_kernel<<<grid_of(NB), kT, 0, s>>>(NB, ck, A, NB, local_of, bp_all, bxy_all, dL, kb, kbits, F.kmax, rows,
                                            row_off, np, par_all, ch_all, il_all);
    LFMM_CUDA_TRY(cudaGetLastError());
    LFMM_CUDA_TRY(cudaMemcpyAsync(F.rl_id, local_of, (size_t)M * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    timer->add_launches(4 + 5 * ((kbits + 2 + lbits + 7) / 8));
    // class ranges of every level
    {
        std::vector<int64_t> hc((size_t)4 * nk + 1);
        LFMM_CUDA_TRY(cudaMemcpyAsync(hc.data(), cstart, hc.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        LFMM_CUDA_TRY(cudaStreamSynchronize(s));
        F.levels.assign(nk, ForestLevel());
        std::vector<int64_t> hl((size_t)5 * nk);
        for (int k = 0; k < nk; ++k) {
            ForestLevel& lv = F.levels[k];
            lv.box_off = hc[4 * k];
            lv.nb = hc[4 * k + 4] - hc[4 * k];
            for (int c = 0; c <= 4; ++c) lv.cls[c] = hc[4 * k + c] - lv.box_off;
            for (int c = 0; c <= 4; ++c) hl[5 * k + c] = lv.cls[c];
            lv.d_cls = dcls + 5 * k;
            lv.bp = bp_all + lv.box_off;
            lv.bxy = bxy_all + lv.box_off;
            lv.par = par_all + lv.box_off;
            lv.il = il_all + 27 * lv.box_off;
            lv.ch = k >= 1 ? ch_all + 4 * lv.box_off : nullptr;
            lv.rl = k == 0 ? leaf_rl : nullptr;
        }
        F.total_boxes = NB;
        LFMM_CUDA_TRY(cudaMemcpyAsync(dcls, hl.data(), hl.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        LFMM_CUDA_TRY(cudaStreamSynchronize(s));  // hl is a local
    }

    // ---- 4. strips of the near-field sweep
    const int msr = std::max(1, maxs), mtg = std::max(1, maxt);
    const int SW = std::min({kStripMaxSW, kStripCapSrc / (3 * msr) - 2, kStripCapTgt / mtg});
    if (SW < 1) return fail(LFMM_EUNSUPPORTED, "leaves too full for the near-field staging (" + std::to_string(msr) +
                                                   " sources / " + std::to_string(mtg) + " targets)");
    F.SW = SW;
    {
        // strip keys of the target leaves (the others: the skip value, sorted to the end)
        const uint64_t skip = 1ull << kbits;  // above every key
        strip_key_kernel<<<grid_of(M), kT, 0, s>>>(F.rl_key, F.rl_t, M, kb, SW, skip, kspare);
        LFMM_CUDA_TRY(cudaGetLastError());
        LFMM_CUDA_TRY(radix_sort(kspare, nullptr, M, kbits + 1, sbuf, s));
        int nstr = 0;
        if ((st = unique_runs(kspare, M, skip, ukeys, nullptr, flag, pos, ssum, &nstr, s))) return st;
        const size_t n4 = (size_t)std::max(nstr, 1);
        if ((st = alloc(F, &vp, 3 * n4 * sizeof(int4) + 16, s))) return st;
        F.strips = (int4*)vp;
        F.strip_rows = F.strips + n4;
        F.n_strips_d = (int32_t*)(F.strip_rows + 2 * n4);
        const int32_t ns32 = nstr;
        LFMM_CUDA_TRY(cudaMemcpyAsync(F.n_strips_d, &ns32, sizeof(int32_t), cudaMemcpyHostToDevice, s));
        strip_record_kernel<<<grid_of(nstr), kT, 0, s>>>(ukeys, nstr, kb, SW, F.strips);
        strip_rows_kernel<<<grid_of(nstr), kT, 0, s>>>(F.strips, nstr, F.rl_key, M, dL, kb, SW, F.strip_rows);
        LFMM_CUDA_TRY(cudaGetLastError());
        timer->add_launches(7 + 5 * ((kbits + 8) / 8));
    }
    return LFMM_OK;  // temporaries are freed in stream order
}

}  // namespace lfmm
