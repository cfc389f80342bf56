// Pruned quadtrees and forests: trees whose boxes are listed explicitly instead of
// filling every cell of a level, and the sweeps of Sec. 8.2 driven by those lists.
//
// A forest is a set of independent problems (sources, targets) that share one leaf
// side s; problem p has its own root box (lower-left corner of its points, side
// s 2^L_p) and its own leaf level L_p.  A single clustered problem is a forest of one
// whose empty boxes are dropped.  Boxes are grouped by k = levels above the leaves
// (k = 0: leaves), because the model-box operators of Sec. 8.1 depend on k only.
//
// The builder (forest_tree.cu) numbers the non-empty boxes of each level (a source or
// target below them) in parity-class order - class c = (x & 1) + 2 (y & 1), then
// problem, then the (x >> 1, y >> 1) grid row by row - so compact ids come grouped by
// class, which is what the M2L kernels need: a class fixes the 27 operators of a box's
// interaction list (Def. 6.1).  Per compact box it stores its problem, coordinates,
// parent, children and interaction list (27 compact ids in slot order, -1 where the box
// is empty or outside).
//
// Points are sorted per problem into row-major leaves, as on the uniform tree, so the
// sources of a leaf's 3 x 3 neighbourhood are three contiguous ranges and the
// near-field strip kernel carries over; it walks a list of the strips that hold
// targets, each with the occupied leaves of its three neighbour-row segments.
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

// ------------------------------------------------------------------------- sweeps
// P2M of compact leaves b0 .. b0 + 3 (those below nb): a quarter warp per leaf, lane h
// of a quarter owning expansion entries [h PL, h PL + PL), PL = NP / 8; leaf b's sources
// are [rl_s[j], rl_s[j + 1]), j = the leaf's row-major index.
template <typename T, int NP>
__device__ __forceinline__ void p2m_list_quad(int64_t b0, int64_t nb, int lane, const int32_t* __restrict__ leaf_rl,
                                              const int32_t* __restrict__ rl_s, const int32_t* __restrict__ loc,
                                              const int32_t* __restrict__ perm, const double* __restrict__ f,
                                              T* __restrict__ f_sorted, const T* __restrict__ tofsT, int side,
                                              T* __restrict__ qhat, typename Mono<T>::V* __restrict__ Q) {
    using M = Mono<T>;
    constexpr int G = 8, PL = NP / G;
    using Row = VecT<T, PL>;
    const int grp = lane >> 3, hl = lane & (G - 1);
    const int64_t b = b0 + grp;
    const bool lv = b < nb;
    int s0 = 0, s1 = 0;
    if (lv) {
        const int j = leaf_rl[b];
        s0 = rl_s[j];
        s1 = rl_s[j + 1];
    }
    const int cnt = s1 - s0;
    int cmax = max(cnt, __shfl_xor_sync(kFull, cnt, 8));
    cmax = max(cmax, __shfl_xor_sync(kFull, cmax, 16));
    T acc[PL];
#pragma unroll
    for (int i = 0; i < PL; ++i) acc[i] = T(0);
    typename M::V qsum = M::zero();
    for (int j0 = 0; j0 < cmax; j0 += G) {
        T fj = T(0);
        int J = 0;
        if (j0 + hl < cnt) {
            const int j = s0 + j0 + hl;
            const int l = loc[j];
            J = (l & 0xffff) + side * (l >> 16);
            const double fd = f[perm[j]];
            fj = (T)fd;
            f_sorted[j] = fj;
            qsum = M::add(qsum, M::from_double(fd));
        }
        const int cc = min(G, cmax - j0);
        for (int k = 0; k < cc; ++k) {
            // lanes of a quarter with fewer sources multiply row 0 by zero
            const T fk = shfl(fj, (grp << 3) + k);
            const int Jk = __shfl_sync(kFull, J, (grp << 3) + k);
            const Row r = *reinterpret_cast<const Row*>(tofsT + (size_t)Jk * NP + hl * PL);
#pragma unroll
            for (int i = 0; i < PL; ++i) acc[i] = fma(r.v[i], fk, acc[i]);
        }
    }
    if (lv) {
        Row o;
#pragma unroll
        for (int i = 0; i < PL; ++i) o.v[i] = acc[i];
        *reinterpret_cast<Row*>(qhat + (size_t)b * NP + hl * PL) = o;
    }
#pragma unroll
    for (int off = 4; off; off >>= 1) qsum = M::add(qsum, shfl_xor_v(qsum, off));
    if (lv && hl == 0) Q[b] = qsum;
}

template <typename T, int NP>
__global__ void __launch_bounds__(256) p2m_list_kernel(int64_t nb, const int32_t* __restrict__ leaf_rl,
                                                       const int32_t* __restrict__ rl_s,
                                                       const int32_t* __restrict__ loc,
                                                       const int32_t* __restrict__ perm,
                                                       const double* __restrict__ f, T* __restrict__ f_sorted,
                                                       const T* __restrict__ tofsT, int side, T* __restrict__ qhat,
                                                       typename Mono<T>::V* __restrict__ Q) {
    griddep_wait();
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; 4 * w < nb; w += nw)
        p2m_list_quad<T, NP>(4 * w, nb, lane, leaf_rl, rl_s, loc, perm, f, f_sorted, tofsT, side, qhat, Q);
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

// M2M of a level with many parents (binary32, NP = 32, 256 threads): tiles of 64
// consecutive compact parents, their children's expansions gathered through the child
// lists into shared memory (row stride 132 floats; an empty child's row is zero), the
// operator staged once per block; thread t computes parents 2 (t / 8) + {0, 1} of the
// tile at outputs 4 (t % 8) + {0..3}, so every step of the 128-long contraction is two
// broadcast words, one 16-byte operator word and eight multiply-adds.  Per output the
// products are summed as in m2m_list_warp (one chain per child in ascending input
// order, the chains added child by child) and the parent's charge is the same pairwise
// sum, so both give bit-identical results.
constexpr int kListM2MTile = 64;
constexpr int kListM2MStride = 132;
constexpr int64_t kListM2MTileMin = 4096;  // fewer parents: a warp or a block per parent
constexpr size_t kListM2MSmem = (size_t)(128 * 32 + kListM2MTile * kListM2MStride) * sizeof(float);

__global__ void __launch_bounds__(256) m2m_list_tiles_kernel(int64_t nb, const int32_t* __restrict__ ch,
                                                             const float* __restrict__ qc,
                                                             const float* __restrict__ m2m, const DF* __restrict__ Qin,
                                                             float* __restrict__ qp, DF* __restrict__ Qout) {
    griddep_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* sop = reinterpret_cast<float*>(smem_raw);  // [128 inputs][32 outputs]
    float* sin = sop + 128 * 32;                      // [64 parents][132]
    __shared__ int s_ch[kListM2MTile * 4];
    block_stage16<4>(reinterpret_cast<uint4*>(sop), reinterpret_cast<const uint4*>(m2m), 128 * 32 / 4);
    const int g = threadIdx.x >> 3, cq = threadIdx.x & 7;
    const int64_t n_tiles = (nb + kListM2MTile - 1) / kListM2MTile;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t b0 = tile * kListM2MTile;
        __syncthreads();  // the operator is staged; the previous tile's reads are done
        s_ch[threadIdx.x] = b0 + (threadIdx.x >> 2) < nb ? ch[b0 * 4 + threadIdx.x] : -1;
        __syncthreads();
        {
            // 64 parents x 4 children x 8 float4, eight per thread, the loads first
            float4 x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = threadIdx.x + 256 * u, it = i >> 5, k4 = i & 31;
                const int child = s_ch[it * 4 + (k4 >> 3)];
                x[u] = child >= 0 ? __ldg(reinterpret_cast<const float4*>(qc + (size_t)child * 32) + (k4 & 7))
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = threadIdx.x + 256 * u, it = i >> 5, k4 = i & 31;
                *reinterpret_cast<float4*>(sin + it * kListM2MStride + 4 * k4) = x[u];
            }
        }
        if (threadIdx.x < kListM2MTile && b0 + threadIdx.x < nb) {
            DF q[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int child = s_ch[threadIdx.x * 4 + c];
                q[c] = child >= 0 ? Qin[child] : DF{0.f, 0.f};
            }
            Qout[b0 + threadIdx.x] = df_add(df_add(q[0], q[1]), df_add(q[2], q[3]));
        }
        __syncthreads();
        const float* x0p = sin + (2 * g) * kListM2MStride;
        const float* x1p = x0p + kListM2MStride;
        float r0[4], r1[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float a0[4] = {0.f, 0.f, 0.f, 0.f}, a1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
            for (int l = 0; l < 32; ++l) {
                const int k = 32 * c + l;
                const float4 o = *reinterpret_cast<const float4*>(sop + k * 32 + 4 * cq);
                const float x0 = x0p[k], x1 = x1p[k];
                a0[0] = fmaf(o.x, x0, a0[0]);
                a0[1] = fmaf(o.y, x0, a0[1]);
                a0[2] = fmaf(o.z, x0, a0[2]);
                a0[3] = fmaf(o.w, x0, a0[3]);
                a1[0] = fmaf(o.x, x1, a1[0]);
                a1[1] = fmaf(o.y, x1, a1[1]);
                a1[2] = fmaf(o.z, x1, a1[2]);
                a1[3] = fmaf(o.w, x1, a1[3]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                r0[j] = c == 0 ? a0[j] : r0[j] + a0[j];
                r1[j] = c == 0 ? a1[j] : r1[j] + a1[j];
            }
        }
        const int64_t p0 = b0 + 2 * g;
        if (p0 < nb)
            *reinterpret_cast<float4*>(qp + (size_t)p0 * 32 + 4 * cq) = make_float4(r0[0], r0[1], r0[2], r0[3]);
        if (p0 + 1 < nb)
            *reinterpret_cast<float4*>(qp + (size_t)(p0 + 1) * 32 + 4 * cq) = make_float4(r1[0], r1[1], r1[2], r1[3]);
    }
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
    const int32_t *leaf_rl, *rl_s, *loc, *perm;
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
// level's counter (ctr[k], zero before the launch), so that uneven boxes balance out;
// P2M takes the chunk's four leaves at once (p2m_list_quad, as the per-level kernel).
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
            if (k == 0) {  // the chunk's four leaves, a quarter warp each
                p2m_list_quad<T, NP>((int64_t)c0, nb, lane, U.leaf_rl, U.rl_s, U.loc, U.perm, U.f, U.f_sorted,
                                     U.tofsT, U.side, U.q[0], U.Q[0]);
                continue;
            }
            const int64_t c1 = min((int64_t)c0 + kUpChunk, nb);
            for (int64_t b = (int64_t)c0; b < c1; ++b)
                m2m_list_warp<T, NP, true>(b, lane, U.ch[k], U.q[k - 1], U.m2m[k], U.Q[k - 1], U.q[k], U.Q[k]);
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
// Six warps per block and staging for 2,048 sources and 1,536 targets: four blocks per SM
// at binary32 (forest_4096, mixed p = 7: 2.25 ms with eight warps and room for 4,096
// sources and 2,048 targets, three blocks per SM; 2.22 ms with eight warps and these
// caps; 2.73 / 2.23 / 2.00 / 1.95 ms with two / three / four / six warps).  Forest strips
// are short (rows of 8 to 32 leaves of ~16 targets), so fewer warps per strip idle less
// at the strip's barriers.
template <typename T>
struct LStripCfg {
    static constexpr int WARPS = 6;
    static constexpr int CAPS = 2048;
    static constexpr int CAPT = 1536;
    static constexpr int MAXSW = 32;
    // the builder sizes strips with the smallest of these (kStripCapSrc: the binary64 case)
    static_assert(MAXSW == kStripMaxSW && CAPT == kStripCapTgt && CAPS >= kStripCapSrc, "strip staging caps");
};

template <typename T, int NP>
__global__ void __launch_bounds__(LStripCfg<T>::WARPS * 32) p2p_list_kernel(
    const int4* __restrict__ strips, const int4* __restrict__ strip_rows, const int32_t* __restrict__ n_strips_d,
    const int32_t* __restrict__ Lp, const uint64_t* __restrict__ rl_key, const int32_t* __restrict__ rl_s,
    const int32_t* __restrict__ rl_t, const int32_t* __restrict__ rl_id, int kb, int side, int SW,
    const int32_t* __restrict__ sloc, const int32_t* __restrict__ tloc, const int32_t* __restrict__ tperm,
    const T* __restrict__ f_sorted,
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
    __shared__ int s_rj[3][2];                 // leaf-list range [j0, j1) of each row (-1: outside)
    __shared__ int s_lc[3][Cfg::MAXSW + 2];    // column - c_lo of each listed leaf (ascending)

    block_stage(tab, table, tab_n);
    const V phi0 = M::make(table[tab_n], table[tab_n + 1]);
    const T* tab_c = tab + (tab_H + tab_H * tab_W);
    const int n_strips = *n_strips_d;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    for (int strip = blockIdx.x; strip < n_strips; strip += gridDim.x) {
        const int4 sd = strips[strip];
        const int p = sd.x, by = sd.y, bx0 = sd.z;
        const int n = 1 << Lp[p];
        const int bx1 = min(bx0 + SW, n);
        const int c_lo = max(bx0 - 1, 0), c_hi = min(bx1, n - 1);
        const int ncol = c_hi - c_lo + 1;
        __syncthreads();
        // the occupied leaves of the three row segments: short ascending lists, so each
        // column below is a search in shared memory
        if (threadIdx.x < 6) {
            const int4 q = strip_rows[2 * (int64_t)strip + (threadIdx.x >> 2)];
            const int e = threadIdx.x & 3;
            s_rj[threadIdx.x >> 1][threadIdx.x & 1] = e == 0 ? q.x : e == 1 ? q.y : e == 2 ? q.z : q.w;
        }
        __syncthreads();
        const uint64_t kmask = ((uint64_t)1 << kb) - 1;
        for (int i = threadIdx.x; i < 3 * (Cfg::MAXSW + 2); i += blockDim.x) {
            const int r = i / (Cfg::MAXSW + 2), q = i % (Cfg::MAXSW + 2);
            const int j0 = s_rj[r][0];
            if (j0 >= 0 && j0 + q < s_rj[r][1]) s_lc[r][q] = (int)(rl_key[j0 + q] & kmask) - c_lo;
        }
        __syncthreads();
        // first listed leaf of row r at column >= c (the row's count if none)
        auto first_at = [&](int r, int c) {
            int lo = 0, hi = s_rj[r][1] - s_rj[r][0];
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s_lc[r][mid] < c) lo = mid + 1;
                else hi = mid;
            }
            return lo;
        };
        // int items: the first source at or after column c of each row (past its last
        // column: the first source of the next occupied leaf, as in a dense bucket array)
        // and the target boundaries of the strip's leaves; V items: the leaf charges of the
        // three rows and the strip leaves' incoming constants, through each leaf's compact
        // id.  A thread takes one item of each kind and issues its loads before the stores.
        {
            const int nA = 3 * (ncol + 1), nI = nA + (bx1 - bx0 + 1);
            const int nC = 3 * ncol, nV = nC + (bx1 - bx0);
            for (int i = threadIdx.x; i < max(nI, nV); i += blockDim.x) {
                int iv = 0;
                if (i < nA) {
                    const int r = i / (ncol + 1), c = i % (ncol + 1);
                    const int j0 = s_rj[r][0];
                    if (j0 >= 0) iv = rl_s[j0 + first_at(r, c)];
                } else if (i < nI) {
                    iv = rl_t[s_rj[1][0] + first_at(1, bx0 + (i - nA) - c_lo)];
                }
                int cid = -1;
                if (i < nC) {
                    const int r = i / ncol, c = i % ncol;
                    const int j0 = s_rj[r][0];
                    if (j0 >= 0) {
                        const int q = first_at(r, c);
                        if (j0 + q < s_rj[r][1] && s_lc[r][q] == c) cid = rl_id[j0 + q];
                    }
                } else if (i < nV) {
                    const int cc = bx0 + (i - nC) - c_lo;
                    const int q = first_at(1, cc);
                    if (s_rj[1][0] + q < s_rj[1][1] && s_lc[1][q] == cc) cid = rl_id[s_rj[1][0] + q];
                }
                V vv = M::zero();
                if (i < nC) {
                    if (cid >= 0) vv = Qleaf[cid];
                } else if (i < nV) {
                    if (Cleaf && cid >= 0) vv = Cleaf[cid];
                }
                if (i < nA) s_sb[(i / (ncol + 1)) * (Cfg::MAXSW + 3) + i % (ncol + 1)] = iv;
                else if (i < nI) s_tb[i - nA] = iv;
                if (i < nC) {
                    s_q[(i / ncol) * (Cfg::MAXSW + 2) + i % ncol] = vv;
                } else if (i < nV) {
                    s_has[i - nC] = cid;
                    s_c[i - nC] = vv;
                }
            }
        }
        __syncthreads();
        // the strip's leaf expansions (four loads in flight per thread)
        for (int i0 = threadIdx.x; i0 < (bx1 - bx0) * NP; i0 += 4 * blockDim.x) {
            T vals[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int i = i0 + k * (int)blockDim.x;
                const int cid = i < (bx1 - bx0) * NP ? s_has[i / NP] : -1;
                vals[k] = (uhat && cid >= 0) ? uhat[(size_t)cid * NP + i % NP] : T(0);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int i = i0 + k * (int)blockDim.x;
                if (i < (bx1 - bx0) * NP) s_uhat[i] = vals[k];
            }
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
        stage_strip_sources<T>(s_src, ns_strip, s_rs, s_sb, Cfg::MAXSW + 3, ncol, c_lo, bx0, side, tab_W, sloc,
                               f_sorted);
        const int tb0 = s_tb[0], nt_strip = s_tb[bx1 - bx0] - tb0;
        stage_strip_targets(s_tloc, s_tperm, nt_strip, s_tb, bx1 - bx0, tb0, tloc, tperm);
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
#pragma unroll 2
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
void Forest::release(cudaStream_t s) {
    for (void* a : owned) cudaFreeAsync(a, s);
    owned.clear();
    levels.clear();
}

// K chunks of a list M2L level: 1 for levels whose 32-box tiles fill the grid three
// times over; for the others the caller's choice (opts.m2l_split), else enough chunks to
// fill it (at most 7).
int m2l_list_chunks(int64_t maxc, int num_sms, int split) {
    const int64_t blocks = 4 * ((maxc + 31) / 32);
    if (blocks == 0 || blocks >= 3 * (int64_t)num_sms) return 1;
    if (split > 0) return std::min(split, 7);
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
                void* Cbox, double* u, double* un, double* uf, int num_sms, cudaStream_t s, int* status_word,
                bool persistent) {
    int* status = persistent ? status_word : nullptr;
    using V = typename Mono<T>::V;
    const int NP = ops.NP;
    const int nk = (int)F.levels.size();
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
        U.leaf_rl = F.levels[0].rl;
        U.rl_s = F.rl_s;
        U.loc = F.sloc;
        U.perm = F.sperm;
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
            int64_t blocks = std::min<int64_t>((l0.nb * 8 + 255) / 256, 152 * 64);  // four leaves per warp
            if (NP == 32)
                (void)launch_dependent(p2m_list_kernel<T, 32>, dim3((int)blocks), dim3(256), 0, s, l0.nb, l0.rl, F.rl_s,
                                       F.sloc, F.sperm, f, f_sorted, (const T*)ops.tofsT, F.side, Qx(0), Qm(0));
            else
                (void)launch_dependent(p2m_list_kernel<T, 64>, dim3((int)blocks), dim3(256), 0, s, l0.nb, l0.rl, F.rl_s,
                                       F.sloc, F.sperm, f, f_sorted, (const T*)ops.tofsT, F.side, Qx(0), Qm(0));
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
            if constexpr (std::is_same<T, float>::value) {
                if (NP == 32 && lv.nb >= kListM2MTileMin) {  // many parents: 64-parent tiles
                    const void* fn = (const void*)m2m_list_tiles_kernel;
                    LFMM_CUDA_TRY(ensure_dynamic_smem(fn, kListM2MSmem));
                    const int64_t tiles = (lv.nb + kListM2MTile - 1) / kListM2MTile;
                    const int64_t grid =
                        std::min<int64_t>(tiles, (int64_t)num_sms * std::max(1, blocks_per_sm(fn, 256, kListM2MSmem)));
                    (void)launch_dependent(m2m_list_tiles_kernel, dim3((unsigned)grid), dim3(256), kListM2MSmem, s,
                                           lv.nb, lv.ch, Qx(k - 1), (const float*)ops.m2m[k], Qm(k - 1), Qx(k),
                                           Qm(k));
                    LFMM_CUDA_TRY(cudaGetLastError());
                    pt.add_launches(1);
                    continue;
                }
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
    // ---- downward sweep (M2L + L2L, coarse to fine): one persistent launch for the levels
    // k >= k_pers, then one tensor-core launch per finer level (binary32 levels of at
    // least kTcListMinBoxes boxes; the boxes per level do not grow with k, so these are
    // the finest ones)
    auto tc_level = [&](int k) -> bool {
        if constexpr (std::is_same<T, float>::value)
            return F.tc_list && F.tc_split && F.levels[k].nb >= kTcListMinBoxes && status_word != nullptr;
        return false;
    };
    bool down_done = false;
    int k_pers = 0;
    if (far && up_done && nk <= kMaxForestLevels) {  // its counters were zeroed with the upward sweep's
        while (k_pers < nk && tc_level(k_pers)) ++k_pers;
        PhaseTimer pt(LFMM_PHASE_M2L, s);
        DownSweep<T> D;
        D.n = 0;
        D.part = (T*)F.m2l_part;
        D.cpart = nullptr;
        bool ok = true;
        for (int k = nk - 1; k >= k_pers; --k) {
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
        } else if (ok) {
            down_done = true;  // every level with boxes runs on the tensor cores
        }
    }
    if (far) {
        for (int k = (down_done ? k_pers : nk) - 1; k >= 0; --k) {
            const ForestLevel& lv = F.levels[k];
            if (lv.nb == 0) continue;
            const bool l2l = k + 1 < nk;
            int64_t maxc = 0;
            for (int c = 0; c < 4; ++c) maxc = std::max(maxc, lv.cls[c + 1] - lv.cls[c]);
            if (maxc == 0) continue;
            if constexpr (std::is_same<T, float>::value) {
                if (F.tc_list && F.tc_split && lv.nb >= kTcListMinBoxes && status_word) {
                    PhaseTimer pt(LFMM_PHASE_M2L_TC, s);
                    const cudaError_t e = launch_m2l_tc_list(
                        ops, k, lv.d_cls, lv.cls, lv.il, l2l ? lv.par : nullptr, Qx(k), lv.nb, Qm(k),
                        l2l ? Ux(k + 1) : nullptr, l2l ? F.levels[k + 1].nb : 0, l2l ? Cm(k + 1) : nullptr, Ux(k), Cm(k),
                        F.tc_split, status_word, num_sms, s);
                    if (e != cudaSuccess) return fail(LFMM_ECUDA, std::string("m2l_tc_list_kernel: ") + cudaGetErrorString(e));
                    pt.add_launches(l2l ? 3 : 2);
                    continue;
                }
            }
            PhaseTimer pt(LFMM_PHASE_M2L, s);
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
        auto go = [&](auto np_tag) -> cudaError_t {
            constexpr int NPc = decltype(np_tag)::value;
            {
                cudaError_t e = ensure_dynamic_smem((const void*)p2p_list_kernel<T, NPc>, smem);
                if (e != cudaSuccess) return e;
            }
            const int per_sm = blocks_per_sm((const void*)p2p_list_kernel<T, NPc>, Cfg::WARPS * 32, smem);
            (void)launch_dependent(p2p_list_kernel<T, NPc>, dim3(num_sms * per_sm), dim3(Cfg::WARPS * 32), smem, s,
                F.strips, F.strip_rows, F.n_strips_d, F.d_L, F.rl_key, F.rl_s, F.rl_t, F.rl_id, F.kb, F.side, F.SW,
                F.sloc, F.tloc, F.tperm, f_sorted,
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
                                double*, double*, double*, int, cudaStream_t, int*, bool);
template int forest_eval<double>(const Forest&, const DeviceOps&, const double*, double*, double*, double*, void*,
                                 void*, double*, double*, double*, int, cudaStream_t, int*, bool);
template int forest_eval<DF>(const Forest&, const DeviceOps&, const double*, DF*, DF*, DF*, void*, void*, double*,
                             double*, double*, int, cudaStream_t, int*, bool);

}  // namespace lfmm
