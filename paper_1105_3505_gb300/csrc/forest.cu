// Pruned quadtrees and forests: trees whose boxes are listed explicitly instead of
// filling every cell of a level, and the sweeps of Sec. 8.2 driven by those lists.
//
// A forest is a set of independent problems (sources, targets) that share one leaf
// side s; problem p has its own root box (lower-left corner of its points, side
// s 2^L_p) and its own leaf level L_p.  A single clustered problem is a forest of one
// whose empty boxes are dropped.  Boxes are grouped by k = levels above the leaves
// (k = 0: leaves), because the model-box operators of Sec. 8.1 depend on k only.
//
// Level k over all problems is described by a dense map in parity-plane order: for
// each parity class c = (x & 1) + 2 (y & 1), the problems in turn, and inside a
// problem the (x >> 1, y >> 1) grid of that class row by row.  Non-empty boxes
// (any source or target below them) get compact ids by an exclusive scan of that
// map, so compact ids come grouped by parity class - what the M2L kernels need, since
// a class fixes the 27 operators of a box's interaction list (Def. 6.1).  Per compact
// box the builder stores its problem, coordinates, parent, children and interaction
// list (27 compact ids in slot order, -1 where the box is empty or outside).
//
// Points are bucketed per problem into row-major leaves, as on the uniform tree, so
// the sources of a leaf's 3 x 3 neighbourhood are three contiguous ranges and the
// near-field strip kernel carries over; it walks a list of the strips that hold
// targets.
#include <algorithm>
#include <climits>
#include <type_traits>

#include "device_common.h"
#include "lfmm_internal.h"

namespace lfmm {

namespace {

constexpr int kThreads = 256;

int grid_for(int64_t n, int threads, int cap = 152 * 16) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// last index p in [0, n) with a[p] <= v (a non-decreasing, a[0] <= v)
template <typename I>
__device__ __forceinline__ int upper_index(const I* a, int n, int64_t v) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if ((int64_t)a[mid] <= v) lo = mid;
        else hi = mid;
    }
    return lo;
}

// position of box (x, y) of level l of a problem starting at off_p in each class
// segment of length S (parity-plane order)
__device__ __forceinline__ int64_t plane_entry(int64_t S, int64_t off_p, int l, int x, int y) {
    const int c = (x & 1) | ((y & 1) << 1);
    const int64_t h = l >= 1 ? ((int64_t)1 << (l - 1)) : 1;
    return (int64_t)c * S + off_p + (int64_t)(y >> 1) * h + (x >> 1);
}

// ------------------------------------------------------------------------- tree build
__global__ void pid_kernel(const int64_t* __restrict__ off, int np, int32_t* __restrict__ pid) {
    griddep_wait();
    for (int p = blockIdx.x; p < np; p += gridDim.x)
        for (int64_t i = off[p] + threadIdx.x; i < off[p + 1]; i += blockDim.x) pid[i] = p;
}

// bounding box of each problem's sources and targets, one block per problem
__global__ void bbox_forest_kernel(const int2* __restrict__ src, const int64_t* __restrict__ soff,
                                   const int2* __restrict__ tgt, const int64_t* __restrict__ toff, int np,
                                   int4* __restrict__ bb) {
    griddep_wait();
    __shared__ int red[4][kThreads / 32];
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

struct ProblemGeo {
    const int32_t* pid;       // problem of each point
    const int32_t* x0;        // [np] root corner
    const int32_t* y0;
    const int32_t* L;         // [np] leaf level
    const int64_t* leaf_off;  // [np + 1] first absolute leaf of each problem
};

__device__ __forceinline__ int64_t leaf_of(const ProblemGeo& g, int p, int2 v, int ls, int& lx, int& ly) {
    const int64_t rx = (int64_t)v.x - g.x0[p], ry = (int64_t)v.y - g.y0[p];
    const int n = 1 << g.L[p];
    const int bx = (int)(rx >> ls), by = (int)(ry >> ls);
    lx = (int)(rx & ((1 << ls) - 1));
    ly = (int)(ry & ((1 << ls) - 1));
    return g.leaf_off[p] + (int64_t)by * n + bx;
}

// leaf counts; rank[i] = the point's arrival rank in its leaf (its slot offset later)
__global__ void count_forest_kernel(const int2* __restrict__ xy, int64_t n, ProblemGeo g, int ls,
                                    int32_t* __restrict__ cnt, int32_t* __restrict__ rank) {
    griddep_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int lx, ly;
        rank[i] = atomicAdd(cnt + leaf_of(g, g.pid[i], xy[i], ls, lx, ly), 1);
    }
}

__global__ void max2_kernel(const int32_t* __restrict__ a, const int32_t* __restrict__ b, int64_t n,
                            int* __restrict__ out2) {
    griddep_wait();
    int ma = 0, mb = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        ma = max(ma, a[i]);
        mb = max(mb, b[i]);
    }
    for (int o = 16; o; o >>= 1) {
        ma = max(ma, __shfl_xor_sync(kFull, ma, o));
        mb = max(mb, __shfl_xor_sync(kFull, mb, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out2, ma);
        atomicMax(out2 + 1, mb);
    }
}

__global__ void scatter_forest_kernel(const int2* __restrict__ xy, int64_t n, ProblemGeo g, int ls,
                                      const int32_t* __restrict__ begin, const int32_t* __restrict__ rank,
                                      int32_t* __restrict__ loc, int32_t* __restrict__ perm) {
    griddep_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int lx, ly;
        const int64_t leaf = leaf_of(g, g.pid[i], xy[i], ls, lx, ly);
        const int slot = begin[leaf] + rank[i];
        loc[slot] = lx | (ly << 16);
        perm[slot] = (int32_t)i;
    }
}

// ---- exclusive scan of int32 (blocks of 1024, one block for the block totals)
constexpr int kScanBlock = 1024;

__global__ void scan_reduce_kernel(const int32_t* __restrict__ in, int64_t n, int32_t* __restrict__ sums) {
    griddep_wait();
    __shared__ int32_t w[kThreads / 32];
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
    griddep_wait();
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
    griddep_wait();
    __shared__ int32_t w[kThreads / 32];
    constexpr int PER = kScanBlock / kThreads;  // 4 consecutive items per thread
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

// ---- levels
struct LevelGeo {
    int k;
    int np;
    int64_t S;                // entries per class segment
    const int64_t* off;       // [np] start of each problem in a class segment
    const int64_t* size;      // [np] entries per class of each problem (0: absent)
};

// flags of the leaves (k = 0): box non-empty if it holds a source or a target
__global__ void flag_leaves_kernel(const int32_t* __restrict__ cs, const int32_t* __restrict__ ct, int64_t NL,
                                   ProblemGeo g, int np, LevelGeo lv, int32_t* __restrict__ flags) {
    griddep_wait();
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < NL; a += (int64_t)gridDim.x * blockDim.x) {
        if (cs[a] + ct[a] == 0) continue;
        const int p = upper_index(g.leaf_off, np, a);
        const int L = g.L[p];
        const int64_t r = a - g.leaf_off[p];
        const int x = (int)(r & ((1 << L) - 1)), y = (int)(r >> L);
        flags[plane_entry(lv.S, lv.off[p], L, x, y)] = 1;
    }
}

// flags of level k >= 1 from the compact map of level k-1 (any child present)
__global__ void flag_parents_kernel(ProblemGeo g, LevelGeo lv, LevelGeo lc, const int32_t* __restrict__ map_child,
                                    int32_t* __restrict__ flags) {
    griddep_wait();
    const int64_t n = 4 * lv.S;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / lv.S);
        const int64_t r = e - (int64_t)c * lv.S;
        const int p = upper_index(lv.off, lv.np, r);
        const int64_t rr = r - lv.off[p];
        if (rr >= lv.size[p]) {
            flags[e] = 0;
            continue;
        }
        const int l = g.L[p] - lv.k;
        const int h = 1 << (l - 1);
        const int x = 2 * (int)(rr % h) + (c & 1), y = 2 * (int)(rr / h) + (c >> 1);
        int any = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b)
            any |= map_child[plane_entry(lc.S, lc.off[p], l + 1, 2 * x + (b & 1), 2 * y + (b >> 1))] >= 0;
        flags[e] = any;
    }
}

// map[e] = compact id or -1; box records of the compact ids
__global__ void compact_kernel(ProblemGeo g, LevelGeo lv, const int32_t* __restrict__ scan, int32_t* __restrict__ map,
                               int32_t* __restrict__ bp, int32_t* __restrict__ bxy) {
    griddep_wait();
    const int64_t n = 4 * lv.S;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const bool on = scan[e + 1] != scan[e];
        if (!on) {
            map[e] = -1;
            continue;
        }
        const int cid = scan[e];
        map[e] = cid;
        if (bp) {
            const int c = (int)(e / lv.S);
            const int64_t r = e - (int64_t)c * lv.S;
            const int p = upper_index(lv.off, lv.np, r);
            const int64_t rr = r - lv.off[p];
            const int l = g.L[p] - lv.k;
            const int h = l >= 1 ? 1 << (l - 1) : 1;
            const int x = 2 * (int)(rr % h) + (c & 1), y = 2 * (int)(rr / h) + (c >> 1);
            bp[cid] = p;
            bxy[cid] = x | (y << 16);
        }
    }
}

// parent, children and interaction list of every compact box of level k
__global__ void links_kernel(ProblemGeo g, LevelGeo lv, int64_t nb, const int32_t* __restrict__ bp,
                             const int32_t* __restrict__ bxy, const int32_t* __restrict__ map,
                             LevelGeo lpar, const int32_t* __restrict__ map_par, LevelGeo lch,
                             const int32_t* __restrict__ map_ch, int32_t* __restrict__ par, int32_t* __restrict__ ch,
                             int32_t* __restrict__ il) {
    griddep_wait();
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
        const int p = bp[b];
        const int x = bxy[b] & 0xffff, y = bxy[b] >> 16;
        const int l = g.L[p] - lv.k;
        const int n = 1 << l;
        if (par) {
            int v = -1;
            if (map_par && l - 1 >= 2 && lpar.size[p] > 0)
                v = map_par[plane_entry(lpar.S, lpar.off[p], l - 1, x >> 1, y >> 1)];
            par[b] = v;
        }
        if (ch) {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                ch[b * 4 + c] = map_ch[plane_entry(lch.S, lch.off[p], l + 1, 2 * x + (c & 1), 2 * y + (c >> 1))];
        }
        if (il) {
            for (int st = 0; st < 27; ++st) {
                int dx, dy;
                interaction_slot(x & 1, y & 1, st, dx, dy);
                const int sx = x + dx, sy = y + dy;
                int v = -1;
                if (sx >= 0 && sx < n && sy >= 0 && sy < n) v = map[plane_entry(lv.S, lv.off[p], l, sx, sy)];
                il[b * 27 + st] = v;
            }
        }
    }
}

// strips of SW leaves of one leaf row holding at least one target
__global__ void strip_flag_kernel(ProblemGeo g, int np, const int64_t* __restrict__ strip_off, int SW,
                                  const int32_t* __restrict__ tbeg, int32_t* __restrict__ flags) {
    griddep_wait();
    const int64_t n = strip_off[np];
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int p = upper_index(strip_off, np, q);
        const int L = g.L[p];
        const int nn = 1 << L, nseg = (nn + SW - 1) / SW;
        const int64_t r = q - strip_off[p];
        const int by = (int)(r / nseg), bx0 = (int)(r % nseg) * SW, bx1 = min(bx0 + SW, nn);
        const int64_t row = g.leaf_off[p] + (int64_t)by * nn;
        flags[q] = tbeg[row + bx1] != tbeg[row + bx0];
    }
}

__global__ void strip_compact_kernel(ProblemGeo g, int np, const int64_t* __restrict__ strip_off, int SW,
                                     const int32_t* __restrict__ scan, int4* __restrict__ strips) {
    griddep_wait();
    const int64_t n = strip_off[np];
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        if (scan[q + 1] == scan[q]) continue;
        const int p = upper_index(strip_off, np, q);
        const int nn = 1 << g.L[p], nseg = (nn + SW - 1) / SW;
        const int64_t r = q - strip_off[p];
        strips[scan[q]] = make_int4(p, (int)(r / nseg), (int)(r % nseg) * SW, 0);
    }
}

__global__ void gather_kernel(const int32_t* __restrict__ a, const int64_t* __restrict__ idx, int n,
                              int32_t* __restrict__ out) {
    griddep_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[idx[i]];
}

// ------------------------------------------------------------------------- sweeps
// P2M: one warp per compact leaf.
template <typename T, int NP>
__device__ __forceinline__ void p2m_list_warp(int64_t b, int lane, const int32_t* __restrict__ bp,
                                              const int32_t* __restrict__ bxy, const ProblemGeo& g,
                                              const int32_t* __restrict__ begin, const int32_t* __restrict__ loc,
                                              const int32_t* __restrict__ perm, const double* __restrict__ f,
                                              T* __restrict__ f_sorted, const T* __restrict__ tofsT, int side,
                                              T* __restrict__ qhat, typename Mono<T>::V* __restrict__ Q) {
    using M = Mono<T>;
    constexpr int PL = NP / 32;
    const int p = bp[b];
    const int x = bxy[b] & 0xffff, y = bxy[b] >> 16;
    const int64_t leaf = g.leaf_off[p] + ((int64_t)y << g.L[p]) + x;
    const int s0 = begin[leaf], s1 = begin[leaf + 1];
    T acc[PL];
#pragma unroll
    for (int i = 0; i < PL; ++i) acc[i] = T(0);
    typename M::V qsum = M::zero();
    for (int j0 = s0; j0 < s1; j0 += 32) {
        const int j = j0 + lane;
        T fj = T(0);
        int J = 0;
        if (j < s1) {
            const int l = loc[j];
            J = (l & 0xffff) + side * (l >> 16);
            const double fd = f[perm[j]];
            fj = (T)fd;
            f_sorted[j] = fj;
            qsum = M::add(qsum, M::from_double(fd));
        }
        const int cnt = min(32, s1 - j0);
        for (int kk = 0; kk < cnt; ++kk) {
            const T fk = shfl(fj, kk);
            const T* row = tofsT + (size_t)shfl(J, kk) * NP;
#pragma unroll
            for (int i = 0; i < PL; ++i) acc[i] = fma(ldg(row + lane + 32 * i), fk, acc[i]);
        }
    }
#pragma unroll
    for (int i = 0; i < PL; ++i) qhat[(size_t)b * NP + lane + 32 * i] = acc[i];
#pragma unroll
    for (int off = 16; off; off >>= 1) qsum = M::add(qsum, shfl_xor_v(qsum, off));
    if (lane == 0) Q[b] = qsum;
}

template <typename T, int NP>
__global__ void __launch_bounds__(256) p2m_list_kernel(int64_t nb, const int32_t* __restrict__ bp,
                                                       const int32_t* __restrict__ bxy, ProblemGeo g,
                                                       const int32_t* __restrict__ begin,
                                                       const int32_t* __restrict__ loc,
                                                       const int32_t* __restrict__ perm,
                                                       const double* __restrict__ f, T* __restrict__ f_sorted,
                                                       const T* __restrict__ tofsT, int side, T* __restrict__ qhat,
                                                       typename Mono<T>::V* __restrict__ Q) {
    griddep_wait();
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nb; b += nw)
        p2m_list_warp<T, NP>(b, lane, bp, bxy, g, begin, loc, perm, f, f_sorted, tofsT, side, qhat, Q);
}

// M2M: one warp per compact parent; children by compact id (-1: empty).
// The same M2M for levels with few parents: one block per parent, warp c computing the
// 32 products of input chunk c; the chunks are added in order, as in m2m_list_kernel,
// so both give bit-identical results.
template <typename T, int NP>
__global__ void __launch_bounds__(4 * NP) m2m_list_block_kernel(int64_t nb, const int32_t* __restrict__ ch,
                                                               const T* __restrict__ qc, const T* __restrict__ m2m,
                                                               const typename Mono<T>::V* __restrict__ Qin,
                                                               T* __restrict__ qp,
                                                               typename Mono<T>::V* __restrict__ Qout) {
    griddep_wait();
    using M = Mono<T>;
    constexpr int CL = 4 * NP / 32, PL = NP / 32;
    __shared__ T red[CL][PL][32];
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const int child = ch[b * 4 + (32 * c) / NP];
        const T xv = child >= 0 ? qc[(size_t)child * NP + (32 * c) % NP + lane] : T(0);
        T acc[PL];
#pragma unroll
        for (int i = 0; i < PL; ++i) acc[i] = T(0);
#pragma unroll 4
        for (int l = 0; l < 32; ++l) {
            const T v = shfl(xv, l);
            const T* row = m2m + (size_t)(32 * c + l) * NP;
#pragma unroll
            for (int i = 0; i < PL; ++i) acc[i] = fma(ldg(row + lane + 32 * i), v, acc[i]);
        }
#pragma unroll
        for (int i = 0; i < PL; ++i) red[c][i][lane] = acc[i];
        __syncthreads();
        if (c == 0) {
#pragma unroll
            for (int i = 0; i < PL; ++i) {
                T a = red[0][i][lane];
#pragma unroll
                for (int cc = 1; cc < CL; ++cc) a += red[cc][i][lane];
                qp[(size_t)b * NP + lane + 32 * i] = a;
            }
            typename M::V qv = M::zero();
            if (lane < 4) {
                const int cb = ch[b * 4 + lane];
                if (cb >= 0) qv = Qin[cb];
            }
            qv = M::add(qv, shfl_xor_v(qv, 1));
            qv = M::add(qv, shfl_xor_v(qv, 2));
            if (lane == 0) Qout[b] = qv;
        }
        __syncthreads();
    }
}

// One parent per warp (lanes own outputs).  CG: children read through L2 only (they
// were written by other blocks of the same cooperative launch).
template <typename T, int NP, bool CG>
__device__ __forceinline__ void m2m_list_warp(int64_t b, int lane, const int32_t* __restrict__ ch,
                                              const T* __restrict__ qc, const T* __restrict__ m2m,
                                              const typename Mono<T>::V* __restrict__ Qin, T* __restrict__ qp,
                                              typename Mono<T>::V* __restrict__ Qout) {
    using M = Mono<T>;
    constexpr int CL = 4 * NP / 32, PL = NP / 32;
    T xv[CL];
#pragma unroll
    for (int c = 0; c < CL; ++c) {
        const int child = ch[b * 4 + (32 * c) / NP];
        const T* src = qc + (size_t)child * NP + (32 * c) % NP + lane;
        xv[c] = child >= 0 ? (CG ? ldcg(src) : *src) : T(0);
    }
    T acc[CL][PL];
#pragma unroll
    for (int c = 0; c < CL; ++c)
#pragma unroll
        for (int i = 0; i < PL; ++i) acc[c][i] = T(0);
#pragma unroll 4
    for (int l = 0; l < 32; ++l) {
#pragma unroll
        for (int c = 0; c < CL; ++c) {
            const T v = shfl(xv[c], l);
            const T* row = m2m + (size_t)(32 * c + l) * NP;
#pragma unroll
            for (int i = 0; i < PL; ++i) acc[c][i] = fma(ldg(row + lane + 32 * i), v, acc[c][i]);
        }
    }
#pragma unroll
    for (int i = 0; i < PL; ++i) {
        T a = acc[0][i];
#pragma unroll
        for (int c = 1; c < CL; ++c) a += acc[c][i];
        qp[(size_t)b * NP + lane + 32 * i] = a;
    }
    typename M::V qv = M::zero();
    if (lane < 4) {
        const int child = ch[b * 4 + lane];
        if (child >= 0) qv = CG ? ldcg(Qin + child) : Qin[child];
    }
    qv = M::add(qv, shfl_xor_v(qv, 1));
    qv = M::add(qv, shfl_xor_v(qv, 2));
    if (lane == 0) Qout[b] = qv;
}

template <typename T, int NP>
__global__ void __launch_bounds__(256) m2m_list_kernel(int64_t nb, const int32_t* __restrict__ ch,
                                                       const T* __restrict__ qc, const T* __restrict__ m2m,
                                                       const typename Mono<T>::V* __restrict__ Qin,
                                                       T* __restrict__ qp, typename Mono<T>::V* __restrict__ Qout) {
    griddep_wait();
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nb; b += nw)
        m2m_list_warp<T, NP, false>(b, lane, ch, qc, m2m, Qin, qp, Qout);
}

// M2L + L2L over compact boxes of one level.  A block takes 32 boxes of one parity
// class and splits the 27 (+1 L2L) K-steps over its 8 warps; per step a warp stages
// the NP x 32 operator block and the 32 source rows (gathered through the interaction
// lists) in shared memory, each lane owns one box and 32 outputs; the warps' partials
// are added in shared memory.  The constant channel (C = C_parent + sum c_o Q) is
// accumulated per warp over its own steps in compensated arithmetic.
constexpr int kLWarps = 8;

template <typename T, int NP>
struct LCfg {
    static constexpr int WARPS = (sizeof(T) == 8 && NP == 64) ? 6 : kLWarps;
    static constexpr int ROWS = 32 * NP + 32;
    static constexpr size_t SMEM = (size_t)WARPS * (NP * 32 + ROWS) * sizeof(T);
};

// The work of one block: 32 boxes (tile bx) of class cls, K chunk z of n_chunks.  CG: the
// parent level's expansions and constants read through L2 only (written by other blocks
// of the same cooperative launch).
template <typename T, int NP, bool CG>
__device__ __forceinline__ void m2l_list_block(
    int64_t bx, int cls, int z, int n_chunks, const int64_t* __restrict__ cls_start, const int32_t* __restrict__ il,
    const int32_t* __restrict__ par, const T* __restrict__ q, const T* __restrict__ u_par, const T* __restrict__ ops,
    const T* __restrict__ l2l, const T* __restrict__ mono, const typename Mono<T>::V* __restrict__ Qin,
    const typename Mono<T>::V* __restrict__ Cpar, T* __restrict__ out, typename Mono<T>::V* __restrict__ Cout,
    int64_t nb, T* __restrict__ part, typename Mono<T>::V* __restrict__ cpart) {
    using M = Mono<T>;
    using V = typename M::V;
    constexpr int W = LCfg<T, NP>::WARPS;
    // K split over n_chunks chunks (levels with few boxes): chunk z takes the steps
    // [z per, (z + 1) per) and writes its partial sums to part / cpart (chunk-major);
    // the reduction adds the chunks in order.
    constexpr int kRows = LCfg<T, NP>::ROWS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sop = reinterpret_cast<T*>(smem_raw);
    T* red = sop + W * NP * 32;
    __shared__ int s_op[27];
    __shared__ V s_cpart[W][32];
    const int64_t c0 = cls_start[cls], c1 = cls_start[cls + 1];
    if (bx * 32 >= c1 - c0) return;  // block-uniform
    const int px = cls & 1, py = cls >> 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < 27) {
        int dx, dy;
        interaction_slot(px, py, threadIdx.x, dx, dy);
        s_op[threadIdx.x] = offset_index(dx, dy);
    }
    __syncthreads();
    const int64_t box = c0 + bx * 32 + lane;
    const bool valid = box < c1;
    const int pbox = (valid && par) ? par[box] : -1;
    const bool has_l2l = u_par != nullptr;
    const int n_steps = 27 + (has_l2l ? 1 : 0);
    T* my_op = sop + warp * NP * 32;
    T* my_rows = red + (size_t)warp * kRows;
    V cacc = M::zero();
    const int per = (n_steps + n_chunks - 1) / n_chunks;
    const int st0 = z * per, st1 = min(n_steps, st0 + per);
    for (int half = 0; half < NP / 32; ++half) {
        T acc[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = T(0);
        for (int st = st0 + warp; st < st1; st += W) {
            const T* op;
            const T* src = nullptr;
            if (st < 27) {
                const int o = s_op[st];
                op = ops + (size_t)o * NP * NP;
                const int sb = valid ? il[box * 27 + st] : -1;
                if (sb >= 0) {
                    src = q + (size_t)sb * NP;
                    if (half == 0) cacc = M::add(cacc, M::mul(M::make(mono[o], mono[kNumOffsets + o]), Qin[sb]));
                }
            } else {
                op = l2l + (size_t)cls * NP * NP;
                if (pbox >= 0) src = u_par + (size_t)pbox * NP;
            }
            __syncwarp();
            {
                constexpr int V4 = (int)(16 / sizeof(T));
                constexpr int PER = NP * 32 / V4 / 32;
                uint4 buf[PER];
#pragma unroll
                for (int c = 0; c < PER; ++c) {
                    const int i = (c * 32 + lane) * V4;
                    const int k = i >> 5, j = i & 31;
                    buf[c] = __ldg(reinterpret_cast<const uint4*>(op + (size_t)k * NP + 32 * half + j));
                }
#pragma unroll
                for (int c = 0; c < PER; ++c) reinterpret_cast<uint4*>(my_op)[c * 32 + lane] = buf[c];
            }
            {
                constexpr int V4 = (int)(16 / sizeof(T));
                constexpr int CPR = NP / V4;
                constexpr int RPI = 32 / CPR;
                const int ch = lane % CPR;
                // the parent's incoming expansion (step 27) may come from an earlier level of
                // the same cooperative launch: through L2 only; source expansions (from the
                // upward sweep) through the read-only cache, where the neighbouring target
                // boxes of an SM share them.  Loads go out four at a time before their stores.
                const bool cg = CG && st >= 27;
                constexpr int NI = 32 / RPI, G = NI < 4 ? NI : 4;
#pragma unroll
                for (int i0 = 0; i0 < NI; i0 += G) {
                    uint4 vals[G];
                    if (cg) {
#pragma unroll
                        for (int i = 0; i < G; ++i) {
                            const T* rs = reinterpret_cast<const T*>(__shfl_sync(
                                kFull, reinterpret_cast<unsigned long long>(src), lane / CPR + RPI * (i0 + i)));
                            vals[i] = rs ? __ldcg(reinterpret_cast<const uint4*>(rs) + ch) : make_uint4(0, 0, 0, 0);
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < G; ++i) {
                            const T* rs = reinterpret_cast<const T*>(__shfl_sync(
                                kFull, reinterpret_cast<unsigned long long>(src), lane / CPR + RPI * (i0 + i)));
                            vals[i] = rs ? __ldg(reinterpret_cast<const uint4*>(rs) + ch) : make_uint4(0, 0, 0, 0);
                        }
                    }
#pragma unroll
                    for (int i = 0; i < G; ++i) {
                        const int r = lane / CPR + RPI * (i0 + i);
                        const T* ve = reinterpret_cast<const T*>(&vals[i]);
#pragma unroll
                        for (int e = 0; e < V4; ++e) {
                            const int k = ch * V4 + e;
                            my_rows[r * NP + ((k + r) & (NP - 1))] = ve[e];
                        }
                    }
                }
            }
            __syncwarp();
            if (src) {
                const T* rowp = my_rows + lane * NP;
#pragma unroll 4
                for (int k = 0; k < NP; ++k) {
                    const T a = rowp[(k + lane) & (NP - 1)];
                    // the 32 operator values of row k (broadcast) in 16-byte loads
                    constexpr int E = (int)(16 / sizeof(T));
                    const uint4* b16 = reinterpret_cast<const uint4*>(my_op + k * 32);
#pragma unroll
                    for (int c = 0; c < 32 / E; ++c) {
                        const uint4 raw = b16[c];
                        const T* e = reinterpret_cast<const T*>(&raw);
#pragma unroll
                        for (int t = 0; t < E; ++t) acc[c * E + t] = fma(a, e[t], acc[c * E + t]);
                    }
                }
            }
            __syncwarp();
        }
        T* my_red = my_rows;
#pragma unroll
        for (int j = 0; j < 32; ++j) my_red[lane * 33 + j] = acc[j];
        if (half == 0) s_cpart[warp][lane] = cacc;
        __syncthreads();
        for (int i = threadIdx.x; i < 32 * 32; i += blockDim.x) {
            const int b = i >> 5, j = i & 31;
            T v = T(0);
#pragma unroll
            for (int w = 0; w < W; ++w) v += red[(size_t)w * kRows + b * 33 + j];
            const int64_t bb = c0 + bx * 32 + b;
            if (bb < c1) {
                if (n_chunks == 1) out[(size_t)bb * NP + 32 * half + j] = v;
                else part[((size_t)z * nb + bb) * NP + 32 * half + j] = v;
            }
        }
        __syncthreads();
    }
    if (warp == 0 && valid) {
        if (n_chunks == 1) {
            V sacc = pbox >= 0 ? (CG ? ldcg(Cpar + pbox) : Cpar[pbox]) : M::zero();
#pragma unroll
            for (int w = 0; w < W; ++w) sacc = M::add(sacc, s_cpart[w][lane]);
            Cout[box] = sacc;
        } else {
            V sacc = M::zero();
#pragma unroll
            for (int w = 0; w < W; ++w) sacc = M::add(sacc, s_cpart[w][lane]);
            cpart[(size_t)z * nb + box] = sacc;
        }
    }
}

template <typename T, int NP>
__global__ void __launch_bounds__(LCfg<T, NP>::WARPS * 32) m2l_list_kernel(
    const int64_t* __restrict__ cls_start, const int32_t* __restrict__ il, const int32_t* __restrict__ par,
    const T* __restrict__ q, const T* __restrict__ u_par, const T* __restrict__ ops, const T* __restrict__ l2l,
    const T* __restrict__ mono, const typename Mono<T>::V* __restrict__ Qin,
    const typename Mono<T>::V* __restrict__ Cpar, T* __restrict__ out, typename Mono<T>::V* __restrict__ Cout,
    int64_t nb, T* __restrict__ part, typename Mono<T>::V* __restrict__ cpart) {
    griddep_wait();
    m2l_list_block<T, NP, false>(blockIdx.x, blockIdx.y, blockIdx.z, gridDim.z, cls_start, il, par, q, u_par, ops,
                                 l2l, mono, Qin, Cpar, out, Cout, nb, part, cpart);
}

// The chunks of a K-split list M2L added in chunk order: out = sum_z part[z], and
// Cout = Cpar[parent] + sum_z cpart[z].  Grid-stride over (tid, stride); CG: inputs
// written by other blocks of the same cooperative launch are read through L2 only.
template <typename T, int NP, bool CG>
__device__ __forceinline__ void m2l_list_reduce(int64_t tid, int64_t stride, int64_t nb, int n_chunks,
                                                const T* __restrict__ part,
                                                const typename Mono<T>::V* __restrict__ cpart,
                                                const int32_t* __restrict__ par,
                                                const typename Mono<T>::V* __restrict__ Cpar, T* __restrict__ out,
                                                typename Mono<T>::V* __restrict__ Cout) {
    using M = Mono<T>;
    for (int64_t i = tid; i < nb * NP; i += stride) {
        T v = CG ? ldcg(part + i) : part[i];
        for (int z = 1; z < n_chunks; ++z) v += CG ? ldcg(part + (size_t)z * nb * NP + i) : part[(size_t)z * nb * NP + i];
        out[i] = v;
    }
    for (int64_t b = tid; b < nb; b += stride) {
        const int pb = (par && Cpar) ? par[b] : -1;
        typename M::V sacc = pb >= 0 ? (CG ? ldcg(Cpar + pb) : Cpar[pb]) : M::zero();
        for (int z = 0; z < n_chunks; ++z) sacc = M::add(sacc, CG ? ldcg(cpart + (size_t)z * nb + b) : cpart[(size_t)z * nb + b]);
        Cout[b] = sacc;
    }
}

template <typename T, int NP>
__global__ void m2l_list_reduce_kernel(int64_t nb, int n_chunks, const T* __restrict__ part,
                                       const typename Mono<T>::V* __restrict__ cpart, const int32_t* __restrict__ par,
                                       const typename Mono<T>::V* __restrict__ Cpar, T* __restrict__ out,
                                       typename Mono<T>::V* __restrict__ Cout) {
    griddep_wait();
    m2l_list_reduce<T, NP, false>((int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x, nb,
                                  n_chunks, part, cpart, par, Cpar, out, Cout);
}

// ------------------------------------------------------------------------- fused sweeps
// The upward sweep (P2M of every leaf of every problem, then M2M level by level) and the
// downward sweep (M2L + L2L level by level, coarse to fine) of the whole forest, each in
// one persistent cooperative launch: the blocks walk the work of a level (leaves, parents,
// 32-box tiles x K chunks) with a grid stride, and a bounded grid barrier separates the
// levels.  Every box's arithmetic is that of the per-level kernels, so the results are
// bit-identical to them.
constexpr int kMaxForestLevels = 16;

template <typename T>
struct UpSweep {
    using V = typename Mono<T>::V;
    int64_t nb0;  // P2M: compact leaves (k = 0)
    const int32_t *bp, *bxy, *begin, *loc, *perm;
    ProblemGeo g;
    const double* f;
    T* f_sorted;
    const T* tofsT;
    int side;
    int nk;  // levels k = 0 .. nk - 1
    int64_t nb[kMaxForestLevels];
    const int32_t* ch[kMaxForestLevels];
    const T* m2m[kMaxForestLevels];
    T* q[kMaxForestLevels];
    V* Q[kMaxForestLevels];
};

// Work queue: a warp takes kUpChunk consecutive boxes of a level at a time from the
// level's counter (ctr[k], zero before the launch), so that uneven boxes balance out.
constexpr int kUpChunk = 4;

template <typename T, int NP>
__global__ void __launch_bounds__(256) forest_up_kernel(const UpSweep<T> U, unsigned* sync, int* status,
                                                        unsigned long long* ctr) {
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < U.nk; ++k) {
        if (k > 0) grid_barrier(sync, sync + 1, status);
        const int64_t nb = k == 0 ? U.nb0 : U.nb[k];
        for (;;) {
            unsigned long long c0 = 0;
            if (lane == 0) c0 = atomicAdd(ctr + k, (unsigned long long)kUpChunk);
            c0 = __shfl_sync(kFull, c0, 0);
            if ((int64_t)c0 >= nb) break;
            const int64_t c1 = min((int64_t)c0 + kUpChunk, nb);
            for (int64_t b = (int64_t)c0; b < c1; ++b) {
                if (k == 0)
                    p2m_list_warp<T, NP>(b, lane, U.bp, U.bxy, U.g, U.begin, U.loc, U.perm, U.f, U.f_sorted, U.tofsT,
                                         U.side, U.q[0], U.Q[0]);
                else
                    m2m_list_warp<T, NP, true>(b, lane, U.ch[k], U.q[k - 1], U.m2m[k], U.Q[k - 1], U.q[k], U.Q[k]);
            }
        }
    }
}

template <typename T>
struct DownLevel {
    using V = typename Mono<T>::V;
    const int64_t* cls;
    const int32_t *il, *par;
    const T *q, *u_par, *tifo, *l2l, *mono;
    const V *Qin, *Cpar;
    T* out;
    V* Cout;
    int64_t nb;
    int tiles;  // 32-box tiles of the largest class
    int nc;     // K chunks (partial sums in the sweep's part / cpart when > 1)
};

template <typename T>
struct DownSweep {
    int n;  // levels in processing order (coarse to fine)
    DownLevel<T> lv[kMaxForestLevels];
    T* part;
    typename Mono<T>::V* cpart;
};

// Work queue: a block takes one item (tile, class, K chunk) of a level at a time from the
// level's counter (ctr[i], zero before the launch).
template <typename T, int NP>
__global__ void __launch_bounds__(LCfg<T, NP>::WARPS * 32, sizeof(T) == 4 ? 2 : 1)
    forest_m2l_kernel(const DownSweep<T> D, unsigned* sync, int* status, unsigned long long* ctr) {
    using V = typename Mono<T>::V;
    __shared__ long long s_item;
    for (int i = 0; i < D.n; ++i) {
        const DownLevel<T>& L = D.lv[i];
        const int tiles = L.tiles, nc = L.nc;
        const int64_t items = (int64_t)4 * tiles * nc;
        T* part = nc > 1 ? D.part : nullptr;
        V* cpart = nc > 1 ? (V*)(D.part + (size_t)nc * L.nb * NP) : nullptr;
        for (;;) {
            if (threadIdx.x == 0) s_item = (long long)atomicAdd(ctr + i, 1ull);
            __syncthreads();
            const int64_t it = s_item;
            __syncthreads();
            if (it >= items) break;
            const int64_t bx = it % tiles;
            const int64_t r = it / tiles;
            m2l_list_block<T, NP, true>(bx, (int)(r & 3), (int)(r >> 2), nc, L.cls, L.il, L.par, L.q, L.u_par, L.tifo,
                                        L.l2l, L.mono, L.Qin, L.Cpar, L.out, L.Cout, L.nb, part, cpart);
        }
        if (nc > 1) {
            grid_barrier(sync, sync + 1, status);
            m2l_list_reduce<T, NP, true>((int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                                         (int64_t)gridDim.x * blockDim.x, L.nb, nc, part, cpart, L.par, L.Cpar, L.out,
                                         L.Cout);
        }
        if (i + 1 < D.n) grid_barrier(sync, sync + 1, status);
    }
}

// P2P + L2P over a list of strips (problem, leaf row, first leaf column): the
// uniform-tree strip kernel with per-problem leaf grids and compact-id lookups.
template <typename T>
struct LStripCfg {
    static constexpr int WARPS = 8;
    static constexpr int CAPS = sizeof(T) == 4 ? 4096 : 2048;
    static constexpr int CAPT = 2048;
    static constexpr int MAXSW = 32;
};

struct LeafMap {  // compact leaf ids through the k = 0 map
    const int32_t* map;
    const int64_t* off;
    int64_t S;
    __device__ __forceinline__ int operator()(int p, int L, int x, int y) const {
        return map[plane_entry(S, off[p], L, x, y)];
    }
};

template <typename T, int NP>
__global__ void __launch_bounds__(LStripCfg<T>::WARPS * 32) p2p_list_kernel(
    const int4* __restrict__ strips, const int32_t* __restrict__ n_strips_d, ProblemGeo g, LeafMap lm, int side,
    int SW, const int32_t* __restrict__ sbeg, const int32_t* __restrict__ sloc, const int32_t* __restrict__ tbeg,
    const int32_t* __restrict__ tloc, const int32_t* __restrict__ tperm, const T* __restrict__ f_sorted,
    const T* __restrict__ table, int tab_H, int tab_W, const T* __restrict__ uhat,
    const typename Mono<T>::V* __restrict__ Cleaf, const typename Mono<T>::V* __restrict__ Qleaf,
    const T* __restrict__ tofsT, double* __restrict__ u, double* __restrict__ u_near, double* __restrict__ u_far) {
    griddep_wait();
    using M = Mono<T>;
    using V = typename M::V;
    using Cfg = LStripCfg<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tab_n = (2 * tab_H + 1) * tab_W;
    T* tab = reinterpret_cast<T*>(smem_raw);
    SrcEntry<T>* s_src = reinterpret_cast<SrcEntry<T>*>(tab + tab_n);
    T* s_uhat = reinterpret_cast<T*>(s_src + Cfg::CAPS);      // [MAXSW][NP]
    V* s_q = reinterpret_cast<V*>(s_uhat + Cfg::MAXSW * NP);  // [3][MAXSW+2]
    V* s_c = s_q + 3 * (Cfg::MAXSW + 2);                      // [MAXSW]
    int* s_tloc = reinterpret_cast<int*>(s_c + Cfg::MAXSW);   // [CAPT]
    int* s_tperm = s_tloc + Cfg::CAPT;                        // [CAPT]
    int* s_sb = s_tperm + Cfg::CAPT;                          // [3][MAXSW+3]
    int* s_tb = s_sb + 3 * (Cfg::MAXSW + 3);                  // [MAXSW+1]
    __shared__ int s_rs[4];
    __shared__ int s_ra[Cfg::MAXSW][3], s_rl[Cfg::MAXSW][3];
    __shared__ double s_nc[Cfg::MAXSW];
    __shared__ int s_has[Cfg::MAXSW];

    for (int i = threadIdx.x; i < tab_n; i += blockDim.x) tab[i] = table[i];
    const V phi0 = M::make(table[tab_n], table[tab_n + 1]);
    const T* tab_c = tab + (tab_H + tab_H * tab_W);
    const int n_strips = *n_strips_d;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    for (int strip = blockIdx.x; strip < n_strips; strip += gridDim.x) {
        const int4 sd = strips[strip];
        const int p = sd.x, by = sd.y, bx0 = sd.z;
        const int L = g.L[p];
        const int n = 1 << L;
        const int64_t lo_leaf = g.leaf_off[p];
        const int bx1 = min(bx0 + SW, n);
        const int c_lo = max(bx0 - 1, 0), c_hi = min(bx1, n - 1);
        const int ncol = c_hi - c_lo + 1;
        __syncthreads();
        for (int i = threadIdx.x; i < 3 * (ncol + 1); i += blockDim.x) {
            const int r = i / (ncol + 1), c = i % (ncol + 1);
            const int yy = by + r - 1;
            s_sb[r * (Cfg::MAXSW + 3) + c] = (yy >= 0 && yy < n) ? sbeg[lo_leaf + (int64_t)yy * n + c_lo + c] : 0;
        }
        for (int i = threadIdx.x; i <= bx1 - bx0; i += blockDim.x) s_tb[i] = tbeg[lo_leaf + (int64_t)by * n + bx0 + i];
        for (int i = threadIdx.x; i < 3 * ncol; i += blockDim.x) {
            const int r = i / ncol, c = i % ncol;
            const int yy = by + r - 1;
            V qv = M::zero();
            if (yy >= 0 && yy < n) {
                const int cid = lm(p, L, c_lo + c, yy);
                if (cid >= 0) qv = Qleaf[cid];
            }
            s_q[r * (Cfg::MAXSW + 2) + c] = qv;
        }
        for (int i = threadIdx.x; i < bx1 - bx0; i += blockDim.x) {
            const int cid = lm(p, L, bx0 + i, by);
            s_has[i] = cid;
            s_c[i] = (Cleaf && cid >= 0) ? Cleaf[cid] : M::zero();
        }
        __syncthreads();
        for (int i = threadIdx.x; i < (bx1 - bx0) * NP; i += blockDim.x) {
            const int c = i / NP, pp = i % NP;
            const int cid = s_has[c];
            s_uhat[i] = (uhat && cid >= 0) ? uhat[(size_t)cid * NP + pp] : T(0);
        }
        for (int li = threadIdx.x; li < bx1 - bx0; li += blockDim.x) {
            const int bx = bx0 + li;
            const int ca = max(bx - 1, 0) - c_lo, cb = min(bx + 1, n - 1) - c_lo + 1;
            int rs = 0;
            V qn = M::zero();
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const int* sb = s_sb + r * (Cfg::MAXSW + 3);
                s_ra[li][r] = rs + (sb[ca] - sb[0]);
                s_rl[li][r] = sb[cb] - sb[ca];
                rs += sb[ncol] - sb[0];
                for (int c = ca; c < cb; ++c) qn = M::add(qn, s_q[r * (Cfg::MAXSW + 2) + c]);
            }
            s_nc[li] = M::to_double(M::mul(phi0, qn));
        }
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int r = 0; r < 3; ++r) {
                s_rs[r] = acc;
                acc += s_sb[r * (Cfg::MAXSW + 3) + ncol] - s_sb[r * (Cfg::MAXSW + 3)];
            }
            s_rs[3] = acc;
        }
        __syncthreads();
        const int ns_strip = s_rs[3];
        for (int v = threadIdx.x; v < ns_strip; v += blockDim.x) {
            const int r = (v >= s_rs[1]) + (v >= s_rs[2]);
            const int* sb = s_sb + r * (Cfg::MAXSW + 3);
            const int j = sb[0] + (v - s_rs[r]);
            int lo = 0, hi = ncol;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (sb[mid] <= j) lo = mid;
                else hi = mid;
            }
            const int l = sloc[j];
            SrcEntry<T> e;
            e.off = (c_lo + lo - bx0) * side + (l & 0xffff) + tab_W * ((r - 1) * side + (l >> 16));
            e.f = f_sorted[j];
            s_src[v] = e;
        }
        const int tb0 = s_tb[0], nt_strip = s_tb[bx1 - bx0] - tb0;
        for (int v = threadIdx.x; v < nt_strip; v += blockDim.x) {
            int lo = 0, hi = bx1 - bx0;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (s_tb[mid] - tb0 <= v) lo = mid;
                else hi = mid;
            }
            s_tloc[v] = tloc[tb0 + v] | (lo << 8);
            s_tperm[v] = tperm[tb0 + v];
        }
        __syncthreads();

        const int n_chunks = (nt_strip + 31) >> 5;
        for (int chunk = warp; chunk < n_chunks; chunk += Cfg::WARPS) {
            const int v = chunk * 32 + lane;
            const bool active = v < nt_strip;
            const int n_act = min(32, nt_strip - chunk * 32);
            const int tl = s_tloc[active ? v : chunk * 32];
            const int li = (tl >> 8) & 0xff, tx = tl & 0xff, ty = tl >> 16;
            const T* tp = tab_c + (tx + tab_W * ty + li * side);
            T acc = T(0), cmp = T(0);
            auto add = [&](T term) {
                if constexpr (sizeof(T) == 4) {
                    const T y = term - cmp;
                    const T s2 = acc + y;
                    cmp = (s2 - acc) - y;
                    acc = s2;
                } else {
                    acc += term;
                }
            };
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const SrcEntry<T>* src = s_src + s_ra[li][r];
                const int len = active ? s_rl[li][r] : 0;
                int j = 0;
                for (; j + 4 <= len; j += 4) {
                    const SrcEntry<T> e0 = src[j], e1 = src[j + 1], e2 = src[j + 2], e3 = src[j + 3];
                    T b = tp[-e0.off] * e0.f;
                    b = fma(tp[-e1.off], e1.f, b);
                    b = fma(tp[-e2.off], e2.f, b);
                    b = fma(tp[-e3.off], e3.f, b);
                    add(b);
                }
                if (j < len) {
                    T b = T(0);
                    for (; j < len; ++j) {
                        const SrcEntry<T> e = src[j];
                        b = fma(tp[-e.off], e.f, b);
                    }
                    add(b);
                }
            }
            acc -= cmp;
            T far = T(0);
            if (uhat) {
                constexpr int PL = NP / 32;
                const int myJ = tx + side * ty;
                T part[32];
#pragma unroll
                for (int qq = 0; qq < 32; ++qq) {
                    const int Jq = shfl(myJ, qq), lq = shfl(li, qq);
                    T w = T(0);
                    if (qq < n_act) {
                        const T* row = tofsT + (size_t)Jq * NP;
                        const T* uq = s_uhat + lq * NP;
#pragma unroll
                        for (int i = 0; i < PL; ++i) w = fma(ldg(row + lane + 32 * i), uq[lane + 32 * i], w);
                    }
                    part[qq] = w;
                }
                far = reduce_scatter32(part);
            }
            if (active) {
                const int dst = s_tperm[v];
                const double dn = (double)acc + s_nc[li];
                const double df = (double)far + M::to_double(s_c[li]);
                if (u) u[dst] = dn + df;
                if (u_near) u_near[dst] = dn;
                if (u_far) u_far[dst] = df;
            }
        }
    }
}

}  // namespace

// ------------------------------------------------------------------------- host side
namespace {

int alloc(std::vector<void*>& owned, int64_t& bytes, void** out, size_t n, cudaStream_t s) {
    *out = nullptr;
    cudaError_t e = dev_malloc(out, n ? n : 16, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return fail(LFMM_ENOMEM, std::string("device allocation of ") + std::to_string(n) + " bytes failed: " +
                                     cudaGetErrorString(e));
    }
    owned.push_back(*out);
    bytes += (int64_t)(n ? n : 16);
    return LFMM_OK;
}

cudaError_t exscan(const int32_t* in, int32_t* out, int64_t n, int32_t* sums, cudaStream_t s) {
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    if (nb == 0) return cudaMemsetAsync(out, 0, sizeof(int32_t), s);
    (void)launch_dependent(scan_reduce_kernel, dim3((unsigned)nb), dim3(kThreads), 0, s, in, n, sums);
    (void)launch_dependent(scan_sums_kernel, dim3(1), dim3(1024), 0, s, sums, (int)nb);
    (void)launch_dependent(scan_apply_kernel, dim3((unsigned)nb), dim3(kThreads), 0, s, in, n, sums, out);
    return cudaGetLastError();
}

int64_t exscan_tmp_ints(int64_t n) { return (n + kScanBlock - 1) / kScanBlock + 1; }

int ceil_log2(int64_t v) {
    int k = 0;
    while (((int64_t)1 << k) < v) ++k;
    return k;
}

}  // namespace

void Forest::release(cudaStream_t s) {
    for (void* a : owned) cudaFreeAsync(a, s);
    owned.clear();
    levels.clear();
}

int m2l_list_chunks(int64_t maxc, int num_sms, int split) {
    if (split > 0) return std::min(split, 7);  // chosen by the caller (opts.m2l_split)
    const int64_t blocks = 4 * ((maxc + 31) / 32);
    if (blocks == 0 || blocks >= 3 * (int64_t)num_sms) return 1;
    return (int)std::min<int64_t>(7, (3 * (int64_t)num_sms + blocks - 1) / blocks);
}

int64_t forest_m2l_split_bytes(const Forest& F, int NP, size_t esz, int num_sms, int split) {
    int64_t need = 0;
    for (const ForestLevel& lv : F.levels) {
        int64_t maxc = 0;
        for (int c = 0; c < 4; ++c) maxc = std::max(maxc, lv.cls[c + 1] - lv.cls[c]);
        const int nc = m2l_list_chunks(maxc, num_sms, split);
        if (nc > 1) need = std::max<int64_t>(need, (int64_t)nc * lv.nb * ((int64_t)NP * (int64_t)esz + 8));
    }
    return need;
}

int forest_build(Forest& F, const int32_t* src, const int64_t* soff_h, int64_t ns, const int32_t* tgt,
                 const int64_t* toff_h, int64_t nt, int np, int leaf_size, int max_leaf_side, cudaStream_t s,
                 PhaseTimer* timer) {
    int st;
    F.np = np;
    F.ns = ns;
    F.nt = nt;
    if (ns > INT32_MAX / 2 || nt > INT32_MAX / 2) return fail(LFMM_EINVAL, "forest too large");
    auto A = [&](void** p, size_t n) { return alloc(F.owned, F.bytes, p, n, s); };
    void* v;
    // problem offsets and per-point problem ids
    if ((st = A(&v, (size_t)2 * (np + 1) * sizeof(int64_t)))) return st;
    int64_t* soff = (int64_t*)v;
    int64_t* toff = soff + (np + 1);
    LFMM_CUDA_TRY(cudaMemcpyAsync(soff, soff_h, (np + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    LFMM_CUDA_TRY(cudaMemcpyAsync(toff, toff_h, (np + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    if ((st = A(&v, (size_t)(ns + nt) * sizeof(int32_t)))) return st;
    F.spid = (int32_t*)v;
    F.tpid = F.spid + ns;
    if (np == 1) {
        LFMM_CUDA_TRY(cudaMemsetAsync(F.spid, 0, (size_t)(ns + nt) * sizeof(int32_t), s));
    } else {
        (void)launch_dependent(pid_kernel, dim3(std::min(np, 152 * 8)), dim3(kThreads), 0, s, soff, np, F.spid);
        (void)launch_dependent(pid_kernel, dim3(std::min(np, 152 * 8)), dim3(kThreads), 0, s, toff, np, F.tpid);
    }
    // bounding boxes
    if ((st = A(&v, (size_t)np * sizeof(int4)))) return st;
    int4* bb = (int4*)v;
    if (np == 1) {
        LFMM_CUDA_TRY(launch_set4((int*)bb, INT_MAX, INT_MAX, INT_MIN, INT_MIN, s));
        LFMM_CUDA_TRY(launch_bbox(src, ns, tgt, nt, (int*)bb, s));
    } else {
        (void)launch_dependent(bbox_forest_kernel, dim3(std::min(np, 152 * 8)), dim3(kThreads), 0, s, (const int2*)src, soff, (const int2*)tgt,
                                                                       toff, np, bb);
    }
    LFMM_CUDA_TRY(cudaGetLastError());
    timer->add_launches(4);
    std::vector<int4> hbb(np);
    LFMM_CUDA_TRY(cudaMemcpyAsync(hbb.data(), bb, np * sizeof(int4), cudaMemcpyDeviceToHost, s));
    LFMM_CUDA_TRY(cudaStreamSynchronize(s));
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
    if ((st = A(&v, (size_t)3 * np * sizeof(int32_t)))) return st;
    int32_t* dx0 = (int32_t*)v;
    int32_t* dy0 = dx0 + np;
    int32_t* dL = dy0 + np;
    F.d_L = dL;
    LFMM_CUDA_TRY(cudaMemcpyAsync(dx0, F.x0.data(), np * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    LFMM_CUDA_TRY(cudaMemcpyAsync(dy0, F.y0.data(), np * sizeof(int32_t), cudaMemcpyHostToDevice, s));

    // common leaf side: the largest power of two <= max_leaf_side (and <= every root
    // that needs splitting) at which no leaf of any problem holds more than leaf_size
    // sources or targets
    int ls = ceil_log2(max_leaf_side);
    if ((1 << ls) > max_leaf_side) --ls;
    ls = std::min(ls, Kmax);
    DevTemp counts;  // dense leaf counts of the accepted side
    DevTemp ranks;   // each point's arrival rank in its leaf (sources, then targets)
    LFMM_CUDA_TRY(dev_malloc(&ranks.ptr, (size_t)(ns + nt) * sizeof(int32_t), s));
    ranks.s = s;
    int32_t* rank_s = (int32_t*)ranks.ptr;
    int32_t* rank_t = rank_s + ns;
    std::vector<int64_t> leaf_off(np + 1);
    int maxs = 0, maxt = 0;
    for (;;) {
        F.L.assign(np, 0);
        leaf_off[0] = 0;
        for (int p = 0; p < np; ++p) {
            F.L[p] = std::max(0, F.K[p] - ls);
            if (F.L[p] > 14) return fail(LFMM_EUNSUPPORTED, "forest problem needs more than 4^14 leaves");
            leaf_off[p + 1] = leaf_off[p] + ((int64_t)1 << (2 * F.L[p]));
        }
        const int64_t NL = leaf_off[np];
        if (NL > ((int64_t)1 << 28)) return fail(LFMM_EUNSUPPORTED, "forest has more than 2^28 leaves");
        counts.reset(s);
        LFMM_CUDA_TRY(dev_malloc(&counts.ptr, (size_t)(2 * NL + 2) * sizeof(int32_t) + (np + 1) * sizeof(int64_t), s));
        counts.s = s;
        int32_t* cs = (int32_t*)counts.ptr;
        int32_t* ct = cs + NL;
        int32_t* mx = ct + NL;
        int64_t* dlo = (int64_t*)(mx + 2);
        LFMM_CUDA_TRY(cudaMemsetAsync(cs, 0, (size_t)(2 * NL + 2) * sizeof(int32_t), s));
        LFMM_CUDA_TRY(cudaMemcpyAsync(dL, F.L.data(), np * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        LFMM_CUDA_TRY(cudaMemcpyAsync(dlo, leaf_off.data(), (np + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        ProblemGeo g{F.spid, dx0, dy0, dL, dlo};
        (void)launch_dependent(count_forest_kernel, dim3(grid_for(ns, kThreads)), dim3(kThreads), 0, s, (const int2*)src, ns, g, ls, cs, rank_s);
        g.pid = F.tpid;
        (void)launch_dependent(count_forest_kernel, dim3(grid_for(nt, kThreads)), dim3(kThreads), 0, s, (const int2*)tgt, nt, g, ls, ct, rank_t);
        (void)launch_dependent(max2_kernel, dim3(grid_for(NL, kThreads)), dim3(kThreads), 0, s, cs, ct, NL, mx);
        LFMM_CUDA_TRY(cudaGetLastError());
        timer->add_launches(3);
        int hm[2];
        LFMM_CUDA_TRY(cudaMemcpyAsync(hm, mx, sizeof(hm), cudaMemcpyDeviceToHost, s));
        LFMM_CUDA_TRY(cudaStreamSynchronize(s));
        maxs = hm[0];
        maxt = hm[1];
        if (std::max(maxs, maxt) <= leaf_size || ls == 0) break;
        --ls;
    }
    F.ls = ls;
    F.side = 1 << ls;
    F.max_src = maxs;
    F.max_tgt = maxt;
    F.leaf_off = leaf_off;
    const int64_t NL = leaf_off[np];
    F.NL = NL;
    if ((st = A(&v, (size_t)(np + 1) * sizeof(int64_t)))) return st;
    F.d_leaf_off = (int64_t*)v;
    LFMM_CUDA_TRY(cudaMemcpyAsync(F.d_leaf_off, leaf_off.data(), (np + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    ProblemGeo g{F.spid, dx0, dy0, dL, F.d_leaf_off};
    F.geo_x0 = dx0;
    F.geo_y0 = dy0;
    int32_t* cs = (int32_t*)counts.ptr;
    int32_t* ct = cs + NL;

    // buckets
    if ((st = A(&v, (size_t)2 * (NL + 1) * sizeof(int32_t)))) return st;
    F.sbeg = (int32_t*)v;
    F.tbeg = F.sbeg + (NL + 1);
    DevTemp tmp;
    const int64_t big = std::max<int64_t>(NL, 1);
    LFMM_CUDA_TRY(dev_malloc(&tmp.ptr, (size_t)exscan_tmp_ints(big) * sizeof(int32_t), s));
    tmp.s = s;
    int32_t* sums = (int32_t*)tmp.ptr;
    LFMM_CUDA_TRY(exscan(cs, F.sbeg, NL, sums, s));
    LFMM_CUDA_TRY(exscan(ct, F.tbeg, NL, sums, s));
    if ((st = A(&v, (size_t)2 * (ns + nt) * sizeof(int32_t)))) return st;
    F.sloc = (int32_t*)v;
    F.sperm = F.sloc + ns;
    F.tloc = F.sperm + ns;
    F.tperm = F.tloc + nt;
    g.pid = F.spid;
    (void)launch_dependent(scatter_forest_kernel, dim3(grid_for(ns, kThreads)), dim3(kThreads), 0, s, (const int2*)src, ns, g, ls, F.sbeg, rank_s,
                                                                       F.sloc, F.sperm);
    g.pid = F.tpid;
    (void)launch_dependent(scatter_forest_kernel, dim3(grid_for(nt, kThreads)), dim3(kThreads), 0, s, (const int2*)tgt, nt, g, ls, F.tbeg, rank_t,
                                                                       F.tloc, F.tperm);
    LFMM_CUDA_TRY(cudaGetLastError());
    timer->add_launches(8);

    // levels k = 0 .. kmax
    int Lmax = 0;
    for (int p = 0; p < np; ++p) Lmax = std::max(Lmax, F.L[p]);
    F.kmax = Lmax - 2;  // may be negative: no far field anywhere
    const int nk = std::max(F.kmax, 0) + 1;
    F.levels.assign(nk, ForestLevel());
    std::vector<std::vector<int64_t>> hoff(nk), hsize(nk);
    int64_t flag_total = 0;
    for (int k = 0; k < nk; ++k) {
        ForestLevel& lv = F.levels[k];
        hoff[k].assign(np, 0);
        hsize[k].assign(np, 0);
        int64_t S = 0;
        for (int p = 0; p < np; ++p) {
            const int l = F.L[p] - k;
            const bool present = (k == 0) || (l >= 2);
            hoff[k][p] = S;
            if (present) hsize[k][p] = l >= 1 ? ((int64_t)1 << (2 * (l - 1))) : 1;
            S += hsize[k][p];
        }
        lv.S = S;
        flag_total += 4 * S + 1;
    }
    // device: per level off/size, map, scan
    std::vector<int32_t*> scan(nk);
    DevTemp lt;
    {
        int64_t ints = 0;
        for (int k = 0; k < nk; ++k) ints += 4 * F.levels[k].S + 1;
        LFMM_CUDA_TRY(dev_malloc(&lt.ptr, (size_t)(ints + 1) * sizeof(int32_t), s));
        lt.s = s;
        int32_t* q = (int32_t*)lt.ptr;
        for (int k = 0; k < nk; ++k) {
            scan[k] = q;
            q += 4 * F.levels[k].S + 1;
        }
    }
    int64_t maxflags = 1;
    for (int k = 0; k < nk; ++k) maxflags = std::max(maxflags, 4 * F.levels[k].S);
    DevTemp ssum;
    LFMM_CUDA_TRY(dev_malloc(&ssum.ptr, (size_t)exscan_tmp_ints(maxflags) * sizeof(int32_t), s));
    ssum.s = s;
    for (int k = 0; k < nk; ++k) {
        ForestLevel& lv = F.levels[k];
        if ((st = A(&v, (size_t)2 * np * sizeof(int64_t)))) return st;
        lv.off = (int64_t*)v;
        lv.size = lv.off + np;
        LFMM_CUDA_TRY(cudaMemcpyAsync(lv.off, hoff[k].data(), np * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        LFMM_CUDA_TRY(cudaMemcpyAsync(lv.size, hsize[k].data(), np * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        if ((st = A(&v, (size_t)4 * lv.S * sizeof(int32_t)))) return st;
        lv.map = (int32_t*)v;
        LevelGeo lg{k, np, lv.S, lv.off, lv.size};
        if (k == 0) {
            LFMM_CUDA_TRY(cudaMemsetAsync(lv.map, 0, (size_t)4 * lv.S * sizeof(int32_t), s));
            g.pid = F.spid;
            (void)launch_dependent(flag_leaves_kernel, dim3(grid_for(NL, kThreads)), dim3(kThreads), 0, s, cs, ct, NL, g, np, lg, lv.map);
        } else {
            const ForestLevel& lc = F.levels[k - 1];
            LevelGeo lcg{k - 1, np, lc.S, lc.off, lc.size};
            (void)launch_dependent(flag_parents_kernel, dim3(grid_for(4 * lv.S, kThreads)), dim3(kThreads), 0, s, g, lg, lcg, lc.map, lv.map);
        }
        LFMM_CUDA_TRY(exscan(lv.map, scan[k], 4 * lv.S, (int32_t*)ssum.ptr, s));
        (void)launch_dependent(compact_kernel, dim3(grid_for(4 * lv.S, kThreads)), dim3(kThreads), 0, s, g, lg, scan[k], lv.map, nullptr, nullptr);
        LFMM_CUDA_TRY(cudaGetLastError());
        timer->add_launches(5);
    }
    // compact counts and class starts
    std::vector<int64_t> idx;
    for (int k = 0; k < nk; ++k)
        for (int c = 0; c <= 4; ++c) idx.push_back((int64_t)(scan[k] - scan[0]) + c * F.levels[k].S);
    DevTemp gi;
    LFMM_CUDA_TRY(dev_malloc(&gi.ptr, idx.size() * (sizeof(int64_t) + sizeof(int32_t)), s));
    gi.s = s;
    int64_t* didx = (int64_t*)gi.ptr;
    int32_t* dval = (int32_t*)(didx + idx.size());
    LFMM_CUDA_TRY(cudaMemcpyAsync(didx, idx.data(), idx.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    (void)launch_dependent(gather_kernel, dim3((unsigned)((idx.size() + 127) / 128)), dim3(128), 0, s, scan[0], didx, (int)idx.size(), dval);
    LFMM_CUDA_TRY(cudaGetLastError());
    std::vector<int32_t> hval(idx.size());
    LFMM_CUDA_TRY(cudaMemcpyAsync(hval.data(), dval, hval.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LFMM_CUDA_TRY(cudaStreamSynchronize(s));
    F.total_boxes = 0;
    for (int k = 0; k < nk; ++k) {
        ForestLevel& lv = F.levels[k];
        for (int c = 0; c <= 4; ++c) lv.cls[c] = hval[k * 5 + c];
        lv.nb = lv.cls[4];
        lv.box_off = F.total_boxes;
        F.total_boxes += lv.nb;
        if ((st = A(&v, (size_t)5 * sizeof(int64_t)))) return st;
        lv.d_cls = (int64_t*)v;
        LFMM_CUDA_TRY(cudaMemcpyAsync(lv.d_cls, lv.cls, 5 * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        // box records, links
        const size_t per = 2 + 1 + (k >= 1 ? 4 : 0) + 27;
        if ((st = A(&v, (size_t)std::max<int64_t>(lv.nb, 1) * per * sizeof(int32_t)))) return st;
        lv.bp = (int32_t*)v;
        lv.bxy = lv.bp + lv.nb;
        lv.par = lv.bxy + lv.nb;
        lv.il = lv.par + lv.nb;
        lv.ch = k >= 1 ? lv.il + lv.nb * 27 : nullptr;
        LevelGeo lg{k, np, lv.S, lv.off, lv.size};
        (void)launch_dependent(compact_kernel, dim3(grid_for(4 * lv.S, kThreads)), dim3(kThreads), 0, s, g, lg, scan[k], lv.map, lv.bp, lv.bxy);
        LFMM_CUDA_TRY(cudaGetLastError());
        timer->add_launches(1);
    }
    for (int k = 0; k < nk; ++k) {
        ForestLevel& lv = F.levels[k];
        if (lv.nb == 0) continue;
        LevelGeo lg{k, np, lv.S, lv.off, lv.size};
        const bool has_par = k + 1 < nk;
        LevelGeo lpar = has_par ? LevelGeo{k + 1, np, F.levels[k + 1].S, F.levels[k + 1].off, F.levels[k + 1].size}
                                : lg;
        LevelGeo lch = k >= 1 ? LevelGeo{k - 1, np, F.levels[k - 1].S, F.levels[k - 1].off, F.levels[k - 1].size}
                              : lg;
        (void)launch_dependent(links_kernel, dim3(grid_for(lv.nb, kThreads)), dim3(kThreads), 0, s,
            g, lg, lv.nb, lv.bp, lv.bxy, lv.map, lpar, has_par ? F.levels[k + 1].map : nullptr, lch,
            k >= 1 ? F.levels[k - 1].map : nullptr, lv.par, lv.ch, lv.il);
        LFMM_CUDA_TRY(cudaGetLastError());
        timer->add_launches(1);
    }

    // strips of the near-field sweep
    const int ms = std::max(1, maxs), mt = std::max(1, maxt);
    int SW = std::min({LStripCfg<float>::MAXSW, LStripCfg<double>::CAPS / (3 * ms) - 2, LStripCfg<float>::CAPT / mt});
    if (SW < 1) return fail(LFMM_EUNSUPPORTED, "leaves too full for the near-field staging (" + std::to_string(ms) +
                                                   " sources / " + std::to_string(mt) + " targets)");
    F.SW = SW;
    std::vector<int64_t> soffs(np + 1, 0);
    for (int p = 0; p < np; ++p) {
        const int64_t nn = (int64_t)1 << F.L[p];
        soffs[p + 1] = soffs[p] + nn * ((nn + SW - 1) / SW);
    }
    const int64_t ncand = soffs[np];
    DevTemp sf;
    LFMM_CUDA_TRY(dev_malloc(&sf.ptr, (size_t)(np + 1) * sizeof(int64_t) +
                                               (size_t)(2 * ncand + 2 + exscan_tmp_ints(ncand)) * sizeof(int32_t), s));
    sf.s = s;
    int64_t* dsoff = (int64_t*)sf.ptr;
    int32_t* sflag = (int32_t*)(dsoff + np + 1);
    int32_t* sscan = sflag + ncand + 1;
    int32_t* ssums = sscan + ncand + 1;
    LFMM_CUDA_TRY(cudaMemcpyAsync(dsoff, soffs.data(), (np + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    (void)launch_dependent(strip_flag_kernel, dim3(grid_for(ncand, kThreads)), dim3(kThreads), 0, s, g, np, dsoff, SW, F.tbeg, sflag);
    LFMM_CUDA_TRY(exscan(sflag, sscan, ncand, ssums, s));
    if ((st = A(&v, (size_t)std::max<int64_t>(ncand, 1) * sizeof(int4) + 16))) return st;
    F.strips = (int4*)v;
    F.n_strips_d = (int32_t*)(F.strips + std::max<int64_t>(ncand, 1));
    (void)launch_dependent(strip_compact_kernel, dim3(grid_for(ncand, kThreads)), dim3(kThreads), 0, s, g, np, dsoff, SW, sscan, F.strips);
    LFMM_CUDA_TRY(cudaMemcpyAsync(F.n_strips_d, sscan + ncand, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    LFMM_CUDA_TRY(cudaGetLastError());
    timer->add_launches(5);
    return LFMM_OK;  // temporaries are freed in stream order
}

// Cooperative launch through the capturable launch API (the fused sweeps).
static cudaError_t launch_coop(const void* fn, int grid, int threads, size_t smem, void** args, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelExC(&cfg, fn, args);
    if (e != cudaSuccess) cudaGetLastError();
    return e;
}

template <typename T>
int forest_eval(const Forest& F, const DeviceOps& ops, const double* f, T* f_sorted, T* qhat, T* uhat, void* Qbox,
                void* Cbox, double* u, double* un, double* uf, int num_sms, cudaStream_t s, int* status) {
    using V = typename Mono<T>::V;
    const int NP = ops.NP;
    const int nk = (int)F.levels.size();
    ProblemGeo g{F.spid, F.geo_x0, F.geo_y0, F.d_L, F.d_leaf_off};
    auto Qx = [&](int k) { return qhat + (size_t)F.levels[k].box_off * NP; };
    auto Ux = [&](int k) { return uhat + (size_t)F.levels[k].box_off * NP; };
    auto Qm = [&](int k) { return (V*)Qbox + F.levels[k].box_off; };
    auto Cm = [&](int k) { return (V*)Cbox + F.levels[k].box_off; };
    const bool far = F.kmax >= 0;
    unsigned* sync = status ? (unsigned*)(status + 1) : nullptr;  // grid-barrier words beside the status word
    // ---- upward sweep in one persistent launch (P2M, then M2M level by level)
    bool up_done = false;
    if (sync && F.sweep_ctr && nk <= kMaxForestLevels && F.levels[0].nb > 0) {
        PhaseTimer pt(LFMM_PHASE_M2M, s);
        UpSweep<T> U;
        U.nb0 = F.levels[0].nb;
        U.bp = F.levels[0].bp;
        U.bxy = F.levels[0].bxy;
        U.begin = F.sbeg;
        U.loc = F.sloc;
        U.perm = F.sperm;
        U.g = g;
        U.f = f;
        U.f_sorted = f_sorted;
        U.tofsT = (const T*)ops.tofsT;
        U.side = F.side;
        U.nk = far ? nk : 1;
        for (int k = 0; k < kMaxForestLevels; ++k) {
            const bool on = k < U.nk;
            U.nb[k] = on ? F.levels[k].nb : 0;
            U.ch[k] = on ? F.levels[k].ch : nullptr;
            U.m2m[k] = on && k >= 1 ? (const T*)ops.m2m[k] : nullptr;
            U.q[k] = on ? Qx(k) : nullptr;
            U.Q[k] = on ? Qm(k) : nullptr;
        }
        const void* fn = NP == 32 ? (const void*)forest_up_kernel<T, 32> : (const void*)forest_up_kernel<T, 64>;
        const int grid = num_sms * std::max(1, blocks_per_sm(fn, 256, 0));
        unsigned long long* ctr = F.sweep_ctr;
        void* args[] = {&U, &sync, &status, &ctr};
        if (cudaMemsetAsync(ctr, 0, 2 * kMaxForestLevels * sizeof(unsigned long long), s) == cudaSuccess &&
            launch_coop(fn, grid, 256, 0, args, s) == cudaSuccess) {
            pt.add_launches(1);
            up_done = true;
        }
    }
    if (!up_done) {
        PhaseTimer pt(LFMM_PHASE_P2M, s);
        const ForestLevel& l0 = F.levels[0];
        if (l0.nb > 0) {
            int64_t blocks = std::min<int64_t>((l0.nb * 32 + 255) / 256, 152 * 64);
            if (NP == 32)
                (void)launch_dependent(p2m_list_kernel<T, 32>, dim3((int)blocks), dim3(256), 0, s, l0.nb, l0.bp, l0.bxy, g, F.sbeg, F.sloc, F.sperm,
                                                                    f, f_sorted, (const T*)ops.tofsT, F.side, Qx(0),
                                                                    Qm(0));
            else
                (void)launch_dependent(p2m_list_kernel<T, 64>, dim3((int)blocks), dim3(256), 0, s, l0.nb, l0.bp, l0.bxy, g, F.sbeg, F.sloc, F.sperm,
                                                                    f, f_sorted, (const T*)ops.tofsT, F.side, Qx(0),
                                                                    Qm(0));
            LFMM_CUDA_TRY(cudaGetLastError());
            pt.add_launches(1);
        }
    }
    if (far && !up_done) {
        PhaseTimer pt(LFMM_PHASE_M2M, s);
        for (int k = 1; k < nk; ++k) {
            const ForestLevel& lv = F.levels[k];
            if (lv.nb == 0) continue;
            if (lv.nb < (int64_t)num_sms * 16) {  // few parents: one block each
                const int64_t nbk = std::min<int64_t>(lv.nb, (int64_t)num_sms * 16);
                if (NP == 32)
                    (void)launch_dependent(m2m_list_block_kernel<T, 32>, dim3((unsigned)nbk), dim3(128), 0, s, lv.nb,
                                           lv.ch, Qx(k - 1), (const T*)ops.m2m[k], Qm(k - 1), Qx(k), Qm(k));
                else
                    (void)launch_dependent(m2m_list_block_kernel<T, 64>, dim3((unsigned)nbk), dim3(256), 0, s, lv.nb,
                                           lv.ch, Qx(k - 1), (const T*)ops.m2m[k], Qm(k - 1), Qx(k), Qm(k));
                LFMM_CUDA_TRY(cudaGetLastError());
                pt.add_launches(1);
                continue;
            }
            int64_t blocks = std::min<int64_t>((lv.nb * 32 + 255) / 256, 152 * 8);
            if (NP == 32)
                (void)launch_dependent(m2m_list_kernel<T, 32>, dim3((int)blocks), dim3(256), 0, s, lv.nb, lv.ch, Qx(k - 1), (const T*)ops.m2m[k],
                                                                    Qm(k - 1), Qx(k), Qm(k));
            else
                (void)launch_dependent(m2m_list_kernel<T, 64>, dim3((int)blocks), dim3(256), 0, s, lv.nb, lv.ch, Qx(k - 1), (const T*)ops.m2m[k],
                                                                    Qm(k - 1), Qx(k), Qm(k));
            LFMM_CUDA_TRY(cudaGetLastError());
            pt.add_launches(1);
        }
    }
    // ---- downward sweep in one persistent launch (M2L + L2L, coarse to fine)
    bool down_done = false;
    if (far && up_done && nk <= kMaxForestLevels) {  // its counters were zeroed with the upward sweep's
        PhaseTimer pt(LFMM_PHASE_M2L, s);
        DownSweep<T> D;
        D.n = 0;
        D.part = (T*)F.m2l_part;
        D.cpart = nullptr;
        bool ok = true;
        for (int k = nk - 1; k >= 0; --k) {
            const ForestLevel& lv = F.levels[k];
            if (lv.nb == 0) continue;
            int64_t maxc = 0;
            for (int c = 0; c < 4; ++c) maxc = std::max(maxc, lv.cls[c + 1] - lv.cls[c]);
            if (maxc == 0) continue;
            const bool l2l = k + 1 < nk;
            DownLevel<T>& L = D.lv[D.n++];
            L.cls = lv.d_cls;
            L.il = lv.il;
            L.par = l2l ? lv.par : nullptr;
            L.q = Qx(k);
            L.u_par = l2l ? Ux(k + 1) : nullptr;
            L.tifo = (const T*)ops.tifo[k];
            L.l2l = l2l ? (const T*)ops.l2l[k + 1] : nullptr;
            L.mono = (const T*)ops.mono[k];
            L.Qin = Qm(k);
            L.Cpar = l2l ? Cm(k + 1) : nullptr;
            L.out = Ux(k);
            L.Cout = Cm(k);
            L.nb = lv.nb;
            L.tiles = (int)((maxc + 31) / 32);
            L.nc = F.m2l_part ? m2l_list_chunks(maxc, num_sms, F.m2l_split) : 1;
            if (L.nc > 1 && !F.m2l_part) ok = false;
        }
        if (ok && D.n > 0) {
            auto go = [&](auto np_tag) -> cudaError_t {
                constexpr int NPc = decltype(np_tag)::value;
                const void* fn = (const void*)forest_m2l_kernel<T, NPc>;
                constexpr size_t smem = LCfg<T, NPc>::SMEM;
                constexpr int threads = LCfg<T, NPc>::WARPS * 32;
                cudaError_t e = ensure_dynamic_smem(fn, smem);
                if (e != cudaSuccess) return e;
                const int grid = num_sms * std::max(1, blocks_per_sm(fn, threads, smem));
                unsigned long long* ctr = F.sweep_ctr + kMaxForestLevels;  // zeroed with the upward sweep's
                void* args[] = {&D, &sync, &status, &ctr};
                return launch_coop(fn, grid, threads, smem, args, s);
            };
            if ((NP == 32 ? go(std::integral_constant<int, 32>()) : go(std::integral_constant<int, 64>())) ==
                cudaSuccess) {
                pt.add_launches(1);
                down_done = true;
            }
        }
    }
    if (far && !down_done) {
        PhaseTimer pt(LFMM_PHASE_M2L, s);
        for (int k = nk - 1; k >= 0; --k) {
            const ForestLevel& lv = F.levels[k];
            if (lv.nb == 0) continue;
            const bool l2l = k + 1 < nk;
            int64_t maxc = 0;
            for (int c = 0; c < 4; ++c) maxc = std::max(maxc, lv.cls[c + 1] - lv.cls[c]);
            if (maxc == 0) continue;
            const int nc = F.m2l_part ? m2l_list_chunks(maxc, num_sms, F.m2l_split) : 1;
            dim3 grid((unsigned)((maxc + 31) / 32), 4, (unsigned)nc);
            T* part = nc > 1 ? (T*)F.m2l_part : nullptr;
            V* cpart = nc > 1 ? (V*)(part + (size_t)nc * lv.nb * NP) : nullptr;
            auto go = [&](auto np_tag) -> cudaError_t {
                constexpr int NPc = decltype(np_tag)::value;
                constexpr size_t smem = LCfg<T, NPc>::SMEM;
                {
                    cudaError_t e = ensure_dynamic_smem((const void*)m2l_list_kernel<T, NPc>, smem);
                    if (e != cudaSuccess) return e;
                }
                (void)launch_dependent(m2l_list_kernel<T, NPc>, dim3(grid), dim3(LCfg<T, NPc>::WARPS * 32), smem, s,
                    lv.d_cls, lv.il, l2l ? lv.par : nullptr, Qx(k), l2l ? Ux(k + 1) : nullptr,
                    (const T*)ops.tifo[k], l2l ? (const T*)ops.l2l[k + 1] : nullptr, (const T*)ops.mono[k], Qm(k),
                    l2l ? Cm(k + 1) : nullptr, Ux(k), Cm(k), lv.nb, part, cpart);
                if (nc > 1) {
                    const int64_t rb = std::min<int64_t>((lv.nb * NPc + 255) / 256, (int64_t)num_sms * 8);
                    (void)launch_dependent(m2l_list_reduce_kernel<T, NPc>, dim3((unsigned)std::max<int64_t>(rb, 1)),
                                           dim3(256), 0, s, lv.nb, nc, (const T*)part, (const V*)cpart,
                                           l2l ? (const int32_t*)lv.par : nullptr, l2l ? (const V*)Cm(k + 1) : nullptr,
                                           Ux(k), (V*)Cm(k));
                }
                return cudaGetLastError();
            };
            cudaError_t e = NP == 32 ? go(std::integral_constant<int, 32>()) : go(std::integral_constant<int, 64>());
            if (e != cudaSuccess) return fail(LFMM_ECUDA, std::string("m2l_list_kernel: ") + cudaGetErrorString(e));
            pt.add_launches(nc > 1 ? 2 : 1);
        }
    }
    {
        PhaseTimer pt(LFMM_PHASE_P2P, s);
        using Cfg = LStripCfg<T>;
        const size_t tab_bytes = (size_t)(2 * ops.tab_H + 1) * ops.tab_W * sizeof(T);
        const size_t smem = tab_bytes + (size_t)Cfg::CAPS * sizeof(SrcEntry<T>) +
                            (size_t)Cfg::MAXSW * NP * sizeof(T) +
                            (size_t)(3 * (Cfg::MAXSW + 2) + Cfg::MAXSW) * sizeof(V) + (size_t)2 * Cfg::CAPT * sizeof(int) +
                            (size_t)(3 * (Cfg::MAXSW + 3) + Cfg::MAXSW + 1) * sizeof(int);
        const ForestLevel& l0 = F.levels[0];
        LeafMap lm{l0.map, l0.off, l0.S};
        auto go = [&](auto np_tag) -> cudaError_t {
            constexpr int NPc = decltype(np_tag)::value;
            {
                cudaError_t e = ensure_dynamic_smem((const void*)p2p_list_kernel<T, NPc>, smem);
                if (e != cudaSuccess) return e;
            }
            const int per_sm = blocks_per_sm((const void*)p2p_list_kernel<T, NPc>, Cfg::WARPS * 32, smem);
            (void)launch_dependent(p2p_list_kernel<T, NPc>, dim3(num_sms * per_sm), dim3(Cfg::WARPS * 32), smem, s,
                F.strips, F.n_strips_d, g, lm, F.side, F.SW, F.sbeg, F.sloc, F.tbeg, F.tloc, F.tperm, f_sorted,
                (const T*)ops.p2p_table, ops.tab_H, ops.tab_W, far ? Ux(0) : nullptr, far ? Cm(0) : nullptr, Qm(0),
                (const T*)ops.tofsT, u, un, uf);
            return cudaGetLastError();
        };
        cudaError_t e = NP == 32 ? go(std::integral_constant<int, 32>()) : go(std::integral_constant<int, 64>());
        if (e != cudaSuccess) return fail(LFMM_ECUDA, std::string("p2p_list_kernel: ") + cudaGetErrorString(e));
        pt.add_launches(1);
    }
    return LFMM_OK;
}

template int forest_eval<float>(const Forest&, const DeviceOps&, const double*, float*, float*, float*, void*, void*,
                                double*, double*, double*, int, cudaStream_t, int*);
template int forest_eval<double>(const Forest&, const DeviceOps&, const double*, double*, double*, double*, void*,
                                 void*, double*, double*, double*, int, cudaStream_t, int*);
template int forest_eval<DF>(const Forest&, const DeviceOps&, const double*, DF*, DF*, DF*, void*, void*, double*,
                             double*, double*, int, cudaStream_t, int*);

}  // namespace lfmm
