// Device helpers shared by the kernel translation units: compensated float pairs,
// the element-type traits of the total-charge / incoming-constant channel, warp
// shuffles and reductions, asynchronous copies, the interaction-offset numbering and
// the staged-source record of the near-field kernels.  Everything has internal
// linkage (each translation unit gets its own copy).
#pragma once

#include <cstdint>

#include "lfmm_internal.h"

namespace lfmm {
namespace {

using ::fma;  // the float / double overloads stay visible beside the DF one below

constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------------------- compensated scalars
// Error-free transformations (Knuth two-sum, FMA two-product) on float pairs.
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = a + b;
    const float bp = s - a;
    const float ap = s - bp;
    return {s, (a - ap) + (b - bp)};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    DF s = two_sum(a.hi, b.hi);
    DF t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    return fast_two_sum(p, e);
}

// ---- DF as a number (element type of the LFMM_DF path)
__device__ __forceinline__ DF operator-(DF a) { return DF{-a.hi, -a.lo}; }
__device__ __forceinline__ DF operator+(DF a, DF b) { return df_add(a, b); }
__device__ __forceinline__ DF operator-(DF a, DF b) { return df_add(a, -b); }
__device__ __forceinline__ DF operator*(DF a, DF b) { return df_mul(a, b); }
__device__ __forceinline__ DF& operator+=(DF& a, DF b) { return a = df_add(a, b); }
__device__ __forceinline__ DF& operator-=(DF& a, DF b) { return a = df_add(a, -b); }
// a * b + c: the exact product (FMA two-product, 4 operations) added to c by two-sum
// (6) with the low parts (2) and one renormalisation (3): 15 binary32 operations
__device__ __forceinline__ DF fma(DF a, DF b, DF c) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float s = p + c.hi;
    const float bb = s - p;
    const float err = (p - (s - bb)) + (c.hi - bb);
    const float t = (err + c.lo) + e;
    const float hi = s + t;
    return DF{hi, t - (hi - s)};
}

// N elements of T loaded and stored as one unit (16-byte aligned from 16 bytes up)
template <typename T, int N>
struct alignas(sizeof(T) * N > 16 ? 16 : sizeof(T) * N) VecT {
    T v[N];
};

// read-only loads of any element type
template <typename T>
__device__ __forceinline__ T ldg(const T* p) {
    return __ldg(p);
}
__device__ __forceinline__ DF ldg(const DF* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return DF{v.x, v.y};
}

// loads that bypass L1 (cache at L2 only): for data another block of the same launch
// wrote before a grid barrier, which a stale L1 line could otherwise hide
template <typename T>
__device__ __forceinline__ T ldcg(const T* p) {
    return __ldcg(p);
}
__device__ __forceinline__ DF ldcg(const DF* p) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return DF{v.x, v.y};
}

template <typename T>
struct Mono;
template <>
struct Mono<float> {
    using V = DF;
    __device__ static V zero() { return {0.f, 0.f}; }
    __device__ static V from_double(double x) {
        const float h = (float)x;
        return {h, (float)(x - (double)h)};
    }
    __device__ static V make(float hi, float lo) { return {hi, lo}; }
    __device__ static V add(V a, V b) { return df_add(a, b); }
    __device__ static V mul(V a, V b) { return df_mul(a, b); }
    __device__ static double to_double(V a) { return (double)a.hi + (double)a.lo; }
};
template <>
struct Mono<DF> {
    using V = DF;
    __device__ static V zero() { return {0.f, 0.f}; }
    __device__ static V from_double(double x) { return DF(x); }
    __device__ static V make(DF hi, DF lo) { return df_add(hi, lo); }
    __device__ static V add(V a, V b) { return df_add(a, b); }
    __device__ static V mul(V a, V b) { return df_mul(a, b); }
    __device__ static double to_double(V a) { return (double)a.hi + (double)a.lo; }
};
template <>
struct Mono<double> {
    using V = double;
    __device__ static V zero() { return 0.0; }
    __device__ static V from_double(double x) { return x; }
    __device__ static V make(double hi, double lo) { return hi + lo; }
    __device__ static V add(V a, V b) { return a + b; }
    __device__ static V mul(V a, V b) { return a * b; }
    __device__ static double to_double(V a) { return a; }
};

template <typename T>
__device__ __forceinline__ T shfl(T v, int src) {
    return __shfl_sync(kFull, v, src);
}
__device__ __forceinline__ DF shfl(DF v, int src) {
    return DF{__shfl_sync(kFull, v.hi, src), __shfl_sync(kFull, v.lo, src)};
}
__device__ __forceinline__ DF shfl_xor_v(DF v, int m) {
    return {__shfl_xor_sync(kFull, v.hi, m), __shfl_xor_sync(kFull, v.lo, m)};
}
__device__ __forceinline__ double shfl_xor_v(double v, int m) { return __shfl_xor_sync(kFull, v, m); }
__device__ __forceinline__ float shfl_xor_v(float v, int m) { return __shfl_xor_sync(kFull, v, m); }

// v[i] summed over the warp lands in lane i (31 shuffles for 32 values).
template <typename T>
__device__ __forceinline__ T reduce_scatter32(T (&v)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < off; ++i) {
            const T send = upper ? v[i] : v[i + off];
            const T keep = upper ? v[i + off] : v[i];
            v[i] = keep + shfl_xor_v(send, off);
        }
    }
    return v[0];
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Block-wide copy of n16 16-byte words from global to shared memory (both 16-byte
// aligned): each thread issues U loads before their stores, so a block staging a table
// pays about n16 / (U blockDim) load latencies instead of n16 / blockDim.
template <int U = 8>
__device__ __forceinline__ void block_stage16(uint4* __restrict__ dst, const uint4* __restrict__ src, int n16) {
    for (int i0 = threadIdx.x; i0 < n16; i0 += U * blockDim.x) {
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * (int)blockDim.x;
            if (i < n16) v[u] = __ldg(src + i);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * (int)blockDim.x;
            if (i < n16) dst[i] = v[u];
        }
    }
}
// n elements of T (dst and src 16-byte aligned): the 16-byte words as above, then the tail
template <typename T>
__device__ __forceinline__ void block_stage(T* __restrict__ dst, const T* __restrict__ src, int n) {
    const int n16 = (int)((size_t)n * sizeof(T) / 16);
    block_stage16(reinterpret_cast<uint4*>(dst), reinterpret_cast<const uint4*>(src), n16);
    for (int i = (int)((size_t)n16 * 16 / sizeof(T)) + threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// Position of offset (ox, oy) in the list of 40: row-major over [-3,3]^2 minus the core.
__device__ __forceinline__ int offset_index(int ox, int oy) {
    const int raw = (oy + 3) * 7 + (ox + 3);
    int inner_before;
    if (oy < -1) inner_before = 0;
    else if (oy > 1) inner_before = 9;
    else inner_before = 3 * (oy + 1) + (ox > 1 ? 3 : 0);
    return raw - inner_before;
}

template <typename T>
struct SrcEntry;
template <>
struct alignas(8) SrcEntry<float> {
    int off;
    float f;
};
template <>
struct alignas(16) SrcEntry<double> {
    int off, pad;
    double f;
};
template <>
struct alignas(16) SrcEntry<DF> {
    int off, pad;
    DF f;
};

// Staging of a near-field strip (a run of leaves of one leaf row): its sources are the
// contiguous source ranges of three leaf rows (row r from sorted index sb_r[0], leaf
// column boundaries sb_r[0..ncol], rows concatenated at rs[r]).  Each staged source gets
// its table offset relative to the strip's first leaf bx0.  A thread takes U sources at a
// time and issues their loads before the searches and stores.
template <typename T, int U = 4>
__device__ __forceinline__ void stage_strip_sources(SrcEntry<T>* __restrict__ s_src, int ns_strip,
                                                    const int* __restrict__ rs, const int* __restrict__ s_sb,
                                                    int sb_stride, int ncol, int c_lo, int bx0, int side, int tab_W,
                                                    const int32_t* __restrict__ sloc,
                                                    const T* __restrict__ f_sorted) {
    for (int v0 = threadIdx.x; v0 < ns_strip; v0 += U * blockDim.x) {
        int lv[U];
        T fv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int v = v0 + u * (int)blockDim.x;
            if (v < ns_strip) {
                const int r = (v >= rs[1]) + (v >= rs[2]);
                const int j = s_sb[r * sb_stride] + (v - rs[r]);
                lv[u] = sloc[j];
                fv[u] = f_sorted[j];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int v = v0 + u * (int)blockDim.x;
            if (v < ns_strip) {
                const int r = (v >= rs[1]) + (v >= rs[2]);
                const int* sb = s_sb + r * sb_stride;
                const int j = sb[0] + (v - rs[r]);
                int lo = 0, hi = ncol;  // leaf column c with sb[c] <= j < sb[c+1]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (sb[mid] <= j) lo = mid;
                    else hi = mid;
                }
                const int l = lv[u];
                SrcEntry<T> e;
                e.off = (c_lo + lo - bx0) * side + (l & 0xffff) + tab_W * ((r - 1) * side + (l >> 16));
                e.f = fv[u];
                s_src[v] = e;
            }
        }
    }
}

// The strip's targets (sorted indices tb0 .. tb0 + nt_strip - 1; leaf i of the strip starts
// at s_tb[i]), with the leaf's index in the strip packed into bits 8..15 of the local
// position (x < 256; leaf sides are at most 32).
template <int U = 4>
__device__ __forceinline__ void stage_strip_targets(int* __restrict__ s_tloc, int* __restrict__ s_tperm,
                                                    int nt_strip, const int* __restrict__ s_tb, int nleaf, int tb0,
                                                    const int32_t* __restrict__ tloc,
                                                    const int32_t* __restrict__ tperm) {
    for (int v0 = threadIdx.x; v0 < nt_strip; v0 += U * blockDim.x) {
        int lv[U], pv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int v = v0 + u * (int)blockDim.x;
            if (v < nt_strip) {
                lv[u] = tloc[tb0 + v];
                pv[u] = tperm[tb0 + v];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int v = v0 + u * (int)blockDim.x;
            if (v < nt_strip) {
                int lo = 0, hi = nleaf;  // leaf li with s_tb[li] <= tb0 + v < s_tb[li + 1]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (s_tb[mid] - tb0 <= v) lo = mid;
                    else hi = mid;
                }
                s_tloc[v] = lv[u] | (lo << 8);
                s_tperm[v] = pv[u];
            }
        }
    }
}

// The 27 interaction-list slots of a box of parity class (px, py): offsets (dx, dy) of
// the parent's neighbours' children that are not adjacent, in row-major order over the
// 6 x 6 block of the parent's 3 x 3 neighbourhood.  Slot order is shared by the list
// builder and every M2L kernel.
__host__ __device__ inline void interaction_slot(int px, int py, int slot, int& dx, int& dy) {
    int n = 0;
    for (int d = 0; d < 36; ++d) {
        const int ex = (d % 6) - 2 - px, ey = (d / 6) - 2 - py;
        if (ex >= -1 && ex <= 1 && ey >= -1 && ey <= 1) continue;
        if (n == slot) {
            dx = ex;
            dy = ey;
            return;
        }
        ++n;
    }
    dx = dy = 0;
}

// Grid-wide barrier of a cooperative launch.  count and gen are plan-owned device words
// (zero before the first use, and back to that state after every barrier); status[3]
// holds the plan's wait budget in polls (0: 2^24 polls, about a second).  The wait is
// bounded; on expiry the block records LFMM_ETIMEOUT and goes on (results invalid, no
// hang).
__device__ __forceinline__ void grid_barrier(unsigned* count, unsigned* gen, int* status) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = gen;
        const unsigned g = *vgen;
        const unsigned b = (unsigned)((volatile int*)status)[3];
        const unsigned budget = b ? b : (1u << 24);
        __threadfence();
        if (atomicAdd(count, 1u) + 1 == gridDim.x) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            unsigned it = 0;
            while (*vgen == g) {
                if (++it > budget) {
                    atomicExch(status, LFMM_ETIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
}


}  // namespace
}  // namespace lfmm
