// The five sweeps of the lattice FMM application (Sec. 8.2) on a uniform quadtree.
//
//   P2M  q_hat^tau = T_ofs(:, J^tau) f(J^tau)                   step 1, Remark 8.2
//   M2M  q_hat^tau = sum_children T_ofo^{tau,sigma} q_hat^sigma   step 2 (T_ofo = blocks of S)
//   M2L  u_hat^tau = sum_{sigma in int(tau)} T_ifo^{tau,sigma} q_hat^sigma
//                    + T_ifi^{tau,parent} u_hat^parent           steps 3-4 fused
//   L2P  u^tau = T_tfi(J^tau, :) u_hat^tau = T_ofs(:, J^tau)^T u_hat^tau      step 5
//   P2P  u^tau += sum over the own and adjacent leaves of phi(x - y) f(y)     step 5
//
// Element type T is float (mixed path) or double (plain path); NP is the padded
// expansion length (32 or 64).  Expansions of level l are stored Morton-ordered,
// [4^l][NP]; points are bucketed by leaf in row-major leaf order, so the sources of
// a leaf's 3x3 neighbourhood are three contiguous ranges.
//
// Monopole channel.  phi has a large constant part (about -1.4 to -1.9 at the box
// distances here) and the charges sum to zero, so the far field is a cancelling sum
// of large terms.  The M2L operators are stored deflated, T_ifo - c_o 1 1^T with
// c_o = phi(o*side); every box also carries its total charge Q (exact sum of f) and
// the incoming constant C = C_parent + sum_list c_o Q_sigma in compensated arithmetic
// (double-float pairs on the mixed path).  Interpolation reproduces constants
// (T_ofs^T 1 = 1 and T_ifi 1 = 1 to the expansion accuracy), so C bypasses L2L/L2P
// and joins the binary64 final sum.
#include <cstring>
#include <type_traits>

#include "device_common.h"
#include "lfmm_internal.h"

namespace lfmm {

namespace {

// ------------------------------------------------------------------------- P2M
// A quarter warp per leaf (row-major leaf index; a leaf holds ~16 sources at the usual
// leaf sizes).  Lane h of a quarter owns expansion entries [h PL, h PL + PL), PL = NP/8;
// each source's row of T_ofs^T is one or two 16-byte loads per lane, so a source step
// of the warp serves four leaves.  Writes the sorted charges in T, the outgoing
// expansion and the leaf's total charge (Morton index).

template <typename T, int NP>
__global__ void __launch_bounds__(256) p2m_kernel(int L, const int32_t* __restrict__ begin,
                                                  const int32_t* __restrict__ loc,
                                                  const int32_t* __restrict__ perm,
                                                  const double* __restrict__ f,
                                                  T* __restrict__ f_sorted,
                                                  const T* __restrict__ tofsT, int side,
                                                  T* __restrict__ qhat,
                                                  typename Mono<T>::V* __restrict__ Q, int nvec, int64_t ns,
                                                  int64_t vq, int64_t vQ) {
    griddep_wait();
    using M = Mono<T>;
    constexpr int G = 8, PL = NP / G;
    using Row = VecT<T, PL>;
    const int lane = threadIdx.x & 31, grp = lane >> 3, hl = lane & (G - 1);
    const int64_t n_leaves = (int64_t)1 << (2 * L);
    const int64_t n_quads = (n_leaves + 3) >> 2;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // (charge vector, four leaves): vector v reads f + v ns, writes f_sorted + v ns,
    // qhat + v vq and Q + v vQ
    for (int64_t pv = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; pv < n_quads * nvec; pv += nw) {
        const int64_t v = pv / n_quads, quad = pv - v * n_quads;
        const double* fv = f + v * ns;
        T* fsv = f_sorted + v * ns;
        const int64_t leaf = 4 * quad + grp;
        const bool lv = leaf < n_leaves;
        const int b = lv ? begin[leaf] : 0, cnt = lv ? begin[leaf + 1] - b : 0;
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
                const int j = b + j0 + hl;
                const int l = loc[j];
                J = (l & 0xffff) + side * (l >> 16);
                const double fd = fv[perm[j]];
                fj = (T)fd;
                fsv[j] = fj;
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
            const uint32_t mort = morton2((uint32_t)(leaf & ((1 << L) - 1)), (uint32_t)(leaf >> L));
            Row o;
#pragma unroll
            for (int i = 0; i < PL; ++i) o.v[i] = acc[i];
            *reinterpret_cast<Row*>(qhat + v * vq + (size_t)mort * NP + hl * PL) = o;
        }
        // sum of the compensated partial charges over the quarter
#pragma unroll
        for (int off = 4; off; off >>= 1) qsum = M::add(qsum, shfl_xor_v(qsum, off));
        if (lv && hl == 0) Q[v * vQ + morton2((uint32_t)(leaf & ((1 << L) - 1)), (uint32_t)(leaf >> L))] = qsum;
    }
}

// ------------------------------------------------------------------------- M2M / M2L
// One block: BB target rows, all NP outputs, a K loop of NP-wide steps.  Per step the
// gathered source rows (A, [BB][AS]) and the operator block (B, [NP][NP], k-major) are
// staged with cp.async, double buffered; each lane owns MB rows x MP outputs.
//   M2M: rows = parents b of level l (row-major over the parent grid); steps c = 0..3
//        take child 4b+c with operator block c of S.  Also Q_b = sum of children's Q.
//   M2L: rows = boxes of parity class (px, py) = blockIdx.y; steps = the class's 27
//        interaction offsets (Def. 6.1) with deflated T_ifo, then (level >= 3) the
//        parent's incoming expansion with T_ifi block (px + 2py).  Also the incoming
//        constant C (see the monopole channel above).
template <typename T, int NP>
struct TrCfg {
    static constexpr int MB = 4, MP = 8;
    static constexpr int NPG = NP / MP;
    static constexpr int NBG = 32 / NPG;
    static constexpr int WB = MB * NBG;
    static constexpr int WARPS = 4;
    static constexpr int THREADS = 32 * WARPS;
    static constexpr int BB = WB * WARPS;
    static constexpr int AS = NP + 16 / (int)sizeof(T);
    static constexpr int A_ELEMS = BB * AS;
    static constexpr int B_ELEMS = NP * NP;
    static constexpr int STAGE = A_ELEMS + B_ELEMS;
    static constexpr size_t SMEM = 2 * (size_t)STAGE * sizeof(T);
};

constexpr int kModeM2M = 0, kModeM2L = 1;

template <typename T, int NP, int MODE>
__global__ void __launch_bounds__(128) translate_kernel(int level, const T* __restrict__ q,
                                                        const T* __restrict__ u_par,
                                                        const T* __restrict__ ops,
                                                        const T* __restrict__ l2l,
                                                        const T* __restrict__ mono,
                                                        const typename Mono<T>::V* __restrict__ Qin,
                                                        const typename Mono<T>::V* __restrict__ Cpar,
                                                        T* __restrict__ out,
                                                        typename Mono<T>::V* __restrict__ Qout,
                                                        typename Mono<T>::V* __restrict__ Cout) {
    griddep_wait();
    using C = TrCfg<T, NP>;
    using M = Mono<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_off[27][3];
    T* smem = reinterpret_cast<T*>(smem_raw);
    const int cls = MODE == kModeM2L ? (int)blockIdx.y : 0;
    const int px = cls & 1, py = cls >> 1;
    // M2M: grid of parents at `level` (2^level per axis); M2L: parents at level-1
    const int lg = MODE == kModeM2L ? level - 1 : level;
    const int np_side = 1 << lg;
    const int64_t n_rows = (int64_t)1 << (2 * lg);
    const int64_t tile0 = (int64_t)blockIdx.x * C::BB;
    const int side = 1 << level;
    const bool has_l2l = MODE == kModeM2L && u_par != nullptr;
    const int n_steps = MODE == kModeM2M ? 4 : 27 + (has_l2l ? 1 : 0);

    if (MODE == kModeM2L && threadIdx.x == 0) {
        int n = 0;
        for (int d = 0; d < 36; ++d) {
            const int dx = (d % 6) - 2 - px, dy = (d / 6) - 2 - py;
            if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
            s_off[n][0] = dx;
            s_off[n][1] = dy;
            s_off[n][2] = offset_index(dx, dy);
            ++n;
        }
    }
    __syncthreads();

    auto row_ij = [&](int64_t r, int& i, int& j) {
        i = (int)(r & (np_side - 1));
        j = (int)(r >> lg);
    };

    auto stage = [&](int step, int buf) {
        T* As = smem + (size_t)buf * C::STAGE;
        T* Bs = As + C::A_ELEMS;
        const T* op;
        int ox = 0, oy = 0;
        if (MODE == kModeM2M) {
            op = ops + (size_t)step * NP * NP;
        } else if (step < 27) {
            ox = s_off[step][0];
            oy = s_off[step][1];
            op = ops + (size_t)s_off[step][2] * NP * NP;
        } else {
            op = l2l + (size_t)cls * NP * NP;
        }
        constexpr int B_CHUNKS = C::B_ELEMS * (int)sizeof(T) / 16;
        for (int c = threadIdx.x; c < B_CHUNKS; c += C::THREADS)
            cp_async16(reinterpret_cast<char*>(Bs) + 16 * c,
                       reinterpret_cast<const char*>(op) + 16 * c, 16);
        constexpr int RC = NP * (int)sizeof(T) / 16;
        for (int c = threadIdx.x; c < C::BB * RC; c += C::THREADS) {
            const int r = c / RC, ch = c % RC;
            const int64_t pr = tile0 + r;
            const T* src = q;
            int bytes = 0;
            if (pr < n_rows) {
                int i, j;
                row_ij(pr, i, j);
                if (MODE == kModeM2M) {
                    src = q + ((size_t)morton2(i, j) * 4 + step) * NP;
                    bytes = 16;
                } else if (step < 27) {
                    const int sx = 2 * i + px + ox, sy = 2 * j + py + oy;
                    if (sx >= 0 && sx < side && sy >= 0 && sy < side) {
                        src = q + (size_t)morton2(sx, sy) * NP;
                        bytes = 16;
                    }
                } else {
                    src = u_par + (size_t)morton2(i, j) * NP;
                    bytes = 16;
                }
            }
            cp_async16(reinterpret_cast<char*>(As + (size_t)r * C::AS) + 16 * ch,
                       reinterpret_cast<const char*>(src) + 16 * ch, bytes);
        }
    };

    stage(0, 0);
    cp_async_commit();

    // scalar channel, one thread per row, overlapped with the first copies
    if (threadIdx.x < C::BB) {
        const int64_t pr = tile0 + threadIdx.x;
        if (pr < n_rows) {
            int i, j;
            row_ij(pr, i, j);
            if (MODE == kModeM2M) {
                const uint32_t b = morton2(i, j);
                typename M::V s = Qin[4 * b];
#pragma unroll
                for (int c = 1; c < 4; ++c) s = M::add(s, Qin[4 * b + c]);
                Qout[b] = s;
            } else {
                typename M::V s = has_l2l ? Cpar[morton2(i, j)] : M::zero();
                // nine loads in flight at a time
                for (int c0 = 0; c0 < 27; c0 += 9) {
                    typename M::V qv[9];
#pragma unroll
                    for (int k = 0; k < 9; ++k) {
                        const int sx = 2 * i + px + s_off[c0 + k][0], sy = 2 * j + py + s_off[c0 + k][1];
                        const bool in = sx >= 0 && sx < side && sy >= 0 && sy < side;
                        qv[k] = in ? Qin[morton2(sx, sy)] : M::zero();
                    }
#pragma unroll
                    for (int k = 0; k < 9; ++k) {
                        const int o = s_off[c0 + k][2];
                        s = M::add(s, M::mul(M::make(mono[o], mono[kNumOffsets + o]), qv[k]));
                    }
                }
                Cout[morton2(2 * i + px, 2 * j + py)] = s;
            }
        }
    }

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bg = lane % C::NBG, pg = lane / C::NBG;
    const int wbox = warp * C::WB;
    T acc[C::MB][C::MP];
#pragma unroll
    for (int i = 0; i < C::MB; ++i)
#pragma unroll
        for (int j = 0; j < C::MP; ++j) acc[i][j] = T(0);

    for (int step = 0; step < n_steps; ++step) {
        if (step + 1 < n_steps) {
            stage(step + 1, (step + 1) & 1);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const T* As = smem + (size_t)(step & 1) * C::STAGE;
        const T* Bs = As + C::A_ELEMS;
#pragma unroll 4
        for (int k = 0; k < NP; ++k) {
            T a[C::MB], b[C::MP];
#pragma unroll
            for (int i = 0; i < C::MB; ++i) a[i] = As[(size_t)(wbox + bg + C::NBG * i) * C::AS + k];
#pragma unroll
            for (int j = 0; j < C::MP; ++j) b[j] = Bs[k * NP + pg * C::MP + j];
#pragma unroll
            for (int i = 0; i < C::MB; ++i)
#pragma unroll
                for (int j = 0; j < C::MP; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < C::MB; ++i) {
        const int64_t pr = tile0 + wbox + bg + C::NBG * i;
        if (pr >= n_rows) continue;
        int ii, jj;
        row_ij(pr, ii, jj);
        const uint32_t dst_box = MODE == kModeM2M ? morton2(ii, jj) : morton2(2 * ii + px, 2 * jj + py);
        T* dst = out + (size_t)dst_box * NP + pg * C::MP;
#pragma unroll
        for (int j = 0; j < C::MP; ++j) dst[j] = acc[i][j];
    }
}

// ------------------------------------------------------------------------- small levels
// Levels with few boxes are latency-bound in the tiled kernel (each block walks all
// 28 K-steps in sequence).  Here a block takes 32 target boxes of one parity class and
// splits the K-steps over its W warps (warp w: steps w, w+W, ...).  Per step a warp
// stages the NP x 32 operator block and the 32 source rows in its own shared memory,
// each lane takes one box and 32 outputs, so every operator value loaded is used by 32
// boxes; the W warps' partial sums are added in shared memory.
// Shared memory per warp: the operator slice (NP x 32) and the 32 source rows, the
// rows padded by 32 elements; the padded row area doubles as the warp's 32 x 33 block of
// partial sums once its K-steps are done.  Binary64 with 64 coefficients uses 6 warps
// so that the block fits in 227 KB.
template <typename T, int NP>
struct SkCfg {
    static constexpr int WARPS = (sizeof(T) == 8 && NP == 64) ? 6 : 8;
    static constexpr int ROWS = 32 * NP + 32;  // per-warp row area (>= 32 * 33)
    static constexpr size_t SMEM = (size_t)WARPS * (NP * 32 + ROWS) * sizeof(T);
};

// One 32-box tile of parity class cls at `level` (shared by the per-level kernel and
// the fused small-level kernel).  u_par == nullptr: no L2L step and C starts at 0.
// Only the K-steps [st_begin, st_end) are taken (all by default).
template <typename T, int NP, int W>
__device__ __forceinline__ void m2l_splitk_tile(int level, int cls, int64_t tile, const T* __restrict__ q,
                                                const T* __restrict__ u_par, const T* __restrict__ ops,
                                                const T* __restrict__ l2l, const T* __restrict__ mono,
                                                const typename Mono<T>::V* __restrict__ Qin,
                                                const typename Mono<T>::V* __restrict__ Cpar, T* __restrict__ out,
                                                typename Mono<T>::V* __restrict__ Cout, int st_begin = 0,
                                                int st_end = 1 << 30) {
    using M = Mono<T>;
    using V = typename M::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int kSkWarps = W;
    constexpr int kRows = SkCfg<T, NP>::ROWS;
    T* sop = reinterpret_cast<T*>(smem_raw);            // [warps][NP][32] operator slice
    T* red = sop + kSkWarps * NP * 32;                  // [warps][kRows]: rows, then 32 x 33 sums
    __shared__ int s_off[27][3];
    __syncthreads();  // the previous tile of this block is done with the shared buffers
    const int px = cls & 1, py = cls >> 1;
    const int lg = level - 1;
    const int np_side = 1 << lg;
    const int64_t n_rows = (int64_t)1 << (2 * lg);
    const int side = 1 << level;
    const bool has_l2l = u_par != nullptr;
    const int n_steps = 27 + (has_l2l ? 1 : 0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        int nn = 0;
        for (int d = 0; d < 36; ++d) {
            const int dx = (d % 6) - 2 - px, dy = (d / 6) - 2 - py;
            if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
            s_off[nn][0] = dx;
            s_off[nn][1] = dy;
            s_off[nn][2] = offset_index(dx, dy);
            ++nn;
        }
    }
    __syncthreads();
    const int64_t row = tile * 32 + lane;
    const bool valid = row < n_rows;
    const int ri = valid ? (int)(row & (np_side - 1)) : 0, rj = valid ? (int)(row >> lg) : 0;
    T* my_op = sop + warp * NP * 32;
    // per-warp source rows, skewed so that column reads across rows hit distinct banks:
    // element k of row r at r * NP + ((k + r) mod NP)
    T* my_rows = red + (size_t)warp * kRows;
    // incoming constant: each warp adds c_o Q(source) of its own K-steps (compensated),
    // the partials are combined after the loop
    __shared__ V s_cpart[kSkWarps][32];
    V cacc = M::zero();
    for (int half = 0; half < NP / 32; ++half) {  // 32 outputs per pass
        T acc[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = T(0);
        for (int st = st_begin + warp; st < min(n_steps, st_end); st += kSkWarps) {
            const T* op;
            const T* src = nullptr;
            if (st < 27) {
                const int o = s_off[st][2];
                op = ops + (size_t)o * NP * NP;
                const int sx = 2 * ri + px + s_off[st][0], sy = 2 * rj + py + s_off[st][1];
                if (valid && sx >= 0 && sx < side && sy >= 0 && sy < side) {
                    const uint32_t sb = morton2(sx, sy);
                    src = q + (size_t)sb * NP;
                    if (half == 0) cacc = M::add(cacc, M::mul(M::make(mono[o], mono[kNumOffsets + o]), Qin[sb]));
                }
            } else {
                op = l2l + (size_t)cls * NP * NP;
                if (valid) src = u_par + (size_t)morton2(ri, rj) * NP;
            }
            // operator slice: my_op[k][j] = op[k][32*half + j]   (op is k-major [q][p]);
            // 16-byte loads, all issued before the stores
            __syncwarp();
            {
                constexpr int V4 = (int)(16 / sizeof(T));        // elements per 16 bytes
                constexpr int PER = NP * 32 / V4 / 32;           // 16-byte chunks per lane
                uint4 buf[PER];
#pragma unroll
                for (int c = 0; c < PER; ++c) {
                    const int i = (c * 32 + lane) * V4;
                    const int k = i >> 5, j = i & 31;
                    buf[c] = __ldg(reinterpret_cast<const uint4*>(op + (size_t)k * NP + 32 * half + j));
                }
#pragma unroll
                for (int c = 0; c < PER; ++c)
                    reinterpret_cast<uint4*>(my_op)[c * 32 + lane] = buf[c];
            }
            __syncwarp();
            // coalesced copy of the 32 source rows of this warp (lane l: 16-byte chunk
            // l % CPR of rows l / CPR + (32 / CPR) i)
            {
                constexpr int V4 = (int)(16 / sizeof(T));
                constexpr int CPR = NP / V4;          // 16-byte chunks per row
                constexpr int RPI = 32 / CPR;         // rows per instruction
                const int ch = lane % CPR;
#pragma unroll
                for (int i = 0; i < 32 / RPI; ++i) {
                    const int r = lane / CPR + RPI * i;
                    const T* rs = reinterpret_cast<const T*>(
                        __shfl_sync(kFull, reinterpret_cast<unsigned long long>(src), r));
                    uint4 v = make_uint4(0, 0, 0, 0);
                    if (rs) v = __ldg(reinterpret_cast<const uint4*>(rs) + ch);
                    const T* ve = reinterpret_cast<const T*>(&v);
#pragma unroll
                    for (int e = 0; e < V4; ++e) {
                        const int k = ch * V4 + e;
                        my_rows[r * NP + ((k + r) & (NP - 1))] = ve[e];
                    }
                }
                __syncwarp();
            }
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
        // reduce the warps' partial sums
        T* my_red = my_rows;  // this warp is done with its rows
#pragma unroll
        for (int j = 0; j < 32; ++j) my_red[lane * 33 + j] = acc[j];
        if (half == 0) s_cpart[warp][lane] = cacc;
        __syncthreads();
        for (int i = threadIdx.x; i < 32 * 32; i += blockDim.x) {
            const int b = i >> 5, j = i & 31;
            T v = T(0);
#pragma unroll
            for (int w = 0; w < kSkWarps; ++w) v += red[(size_t)w * kRows + b * 33 + j];
            const int64_t r = tile * 32 + b;
            if (r < n_rows) {
                const int ii = (int)(r & (np_side - 1)), jj = (int)(r >> lg);
                out[(size_t)morton2(2 * ii + px, 2 * jj + py) * NP + 32 * half + j] = v;
            }
        }
        __syncthreads();
    }
    // incoming constant: parent's constant plus the warps' partials, one box per lane
    if (warp == 0 && valid) {
        V sacc = has_l2l ? Cpar[morton2(ri, rj)] : M::zero();
#pragma unroll
        for (int w = 0; w < kSkWarps; ++w) sacc = M::add(sacc, s_cpart[w][lane]);
        Cout[morton2(2 * ri + px, 2 * rj + py)] = sacc;
    }
}

template <typename T, int NP>
__global__ void __launch_bounds__(SkCfg<T, NP>::WARPS * 32) m2l_splitk_kernel(int level, const T* __restrict__ q,
                                                                   const T* __restrict__ u_par,
                                                                   const T* __restrict__ ops,
                                                                   const T* __restrict__ l2l,
                                                                   const T* __restrict__ mono,
                                                                   const typename Mono<T>::V* __restrict__ Qin,
                                                                   const typename Mono<T>::V* __restrict__ Cpar,
                                                                   T* __restrict__ out,
                                                                   typename Mono<T>::V* __restrict__ Cout) {
    griddep_wait();
    m2l_splitk_tile<T, NP, SkCfg<T, NP>::WARPS>(level, blockIdx.y, blockIdx.x, q, u_par, ops, l2l, mono, Qin, Cpar,
                                                 out, Cout);
}

// M2M with one warp per parent: lanes own outputs, children's expansions broadcast by
// shuffles, the operator [4NP][NP] staged in shared memory when it fits (else L1/L2).
// M2M of the parents [warp_id, n_parent) with stride n_warps: one warp per parent,
// lanes own outputs, the children's expansions broadcast by shuffles; op is the
// operator [4NP][NP] in shared memory (staged by the caller) or global memory.
template <typename T, int NP>
__device__ __forceinline__ void m2m_parents(int level, const T* __restrict__ qc, const T* __restrict__ op,
                                            const typename Mono<T>::V* __restrict__ Qin, T* __restrict__ qp,
                                            typename Mono<T>::V* __restrict__ Qout, int64_t warp_id,
                                            int64_t n_warps, int nvec = 1, int64_t vq = 0, int64_t vQ = 0) {
    using M = Mono<T>;
    constexpr int CL = 4 * NP / 32, PL = NP / 32;
    const int lane = threadIdx.x & 31;
    const int64_t n_parent = (int64_t)1 << (2 * level);
    const int64_t n_items = n_parent * nvec;  // (charge vector, parent); vector v's arrays at v vq / v vQ
    // software pipeline: the next parent's children and charges are loaded while this
    // parent is computed
    T nx[CL];
    typename M::V nq = M::zero();
    if (warp_id < n_items) {
        const int64_t v = warp_id / n_parent, pr = warp_id - v * n_parent;
#pragma unroll
        for (int c = 0; c < CL; ++c) nx[c] = ldcg(qc + v * vq + (size_t)pr * 4 * NP + lane + 32 * c);
        if (lane < 4) nq = ldcg(Qin + v * vQ + 4 * pr + lane);
    }
    for (int64_t item = warp_id; item < n_items; item += n_warps) {
        const int64_t vv = item / n_parent, par = item - vv * n_parent;
        T xv[CL];
#pragma unroll
        for (int c = 0; c < CL; ++c) xv[c] = nx[c];
        typename M::V qv = nq;
        const int64_t nxt = item + n_warps;
        if (nxt < n_items) {
            const int64_t v = nxt / n_parent, pr = nxt - v * n_parent;
#pragma unroll
            for (int c = 0; c < CL; ++c) nx[c] = ldcg(qc + v * vq + (size_t)pr * 4 * NP + lane + 32 * c);
            if (lane < 4) nq = ldcg(Qin + v * vQ + 4 * pr + lane);
        }
        // one accumulator chain per 32-wide input chunk, added at the end
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
                const T* row = op + (size_t)(32 * c + l) * NP;
#pragma unroll
                for (int i = 0; i < PL; ++i) acc[c][i] = fma(row[lane + 32 * i], v, acc[c][i]);
            }
        }
#pragma unroll
        for (int i = 0; i < PL; ++i) {
            T a = acc[0][i];
#pragma unroll
            for (int c = 1; c < CL; ++c) a += acc[c][i];
            qp[vv * vq + (size_t)par * NP + lane + 32 * i] = a;
        }
        // total charge of the parent: lanes 0..3 hold the children's, all lanes shuffle
        qv = M::add(qv, shfl_xor_v(qv, 1));
        qv = M::add(qv, shfl_xor_v(qv, 2));
        if (lane == 0) Qout[vv * vQ + par] = qv;
    }
}

// M2M of one level in tiles of 64 parents (binary32, NP = 32, 256 threads): a tile's
// children expansions (64 x 128 floats, contiguous in Morton order) are staged in
// shared memory with a row stride of 132 floats, and thread t computes parents
// 2 (t / 8) + {0, 1} of the tile at outputs 4 (t % 8) + {0..3}, so every step of the
// 128-long contraction is two broadcast words, one 16-byte operator word and eight
// multiply-adds.  Per output the products are summed exactly as in m2m_parents (one
// chain per child in ascending input order, the chains added child by child), and the
// parent's charge is the same pairwise sum, so both give bit-identical results.
constexpr int kM2MTile = 64;
constexpr int kM2MTileStride = 132;
constexpr int64_t kM2MTileMinItems = 4096;  // fewer parents: the warp-per-parent path
constexpr size_t kM2MTileSmem = (size_t)kM2MTile * kM2MTileStride * sizeof(float);

__device__ __forceinline__ void m2m_tiles_f32(int level, const float* __restrict__ qc, const float* __restrict__ op,
                                              const DF* __restrict__ Qin, float* __restrict__ qp,
                                              DF* __restrict__ Qout, int nvec, int64_t vq, int64_t vQ,
                                              float* __restrict__ sin) {
    const int64_t n_parent = (int64_t)1 << (2 * level);  // a multiple of 64 (level >= 3)
    const int64_t n_tiles = n_parent * nvec / kM2MTile;
    const int g = threadIdx.x >> 3, cq = threadIdx.x & 7;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t item0 = tile * kM2MTile;
        const int64_t v = item0 / n_parent, pr0 = item0 - v * n_parent;
        const float* src = qc + v * vq + pr0 * 128;
        __syncthreads();  // the previous tile's reads are done
        for (int i = threadIdx.x; i < kM2MTile * 32; i += blockDim.x) {
            const int it = i >> 5, k4 = i & 31;
            const float4 x = __ldcg(reinterpret_cast<const float4*>(src + (size_t)it * 128) + k4);
            *reinterpret_cast<float4*>(sin + it * kM2MTileStride + 4 * k4) = x;
        }
        if (threadIdx.x < kM2MTile) {
            const DF* qi = Qin + v * vQ + 4 * (pr0 + threadIdx.x);
            const DF q0 = ldcg(qi), q1 = ldcg(qi + 1), q2 = ldcg(qi + 2), q3 = ldcg(qi + 3);
            Qout[v * vQ + pr0 + threadIdx.x] = df_add(df_add(q0, q1), df_add(q2, q3));
        }
        __syncthreads();
        const float* x0p = sin + (2 * g) * kM2MTileStride;
        const float* x1p = x0p + kM2MTileStride;
        float r0[4], r1[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float a0[4] = {0.f, 0.f, 0.f, 0.f}, a1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
            for (int l = 0; l < 32; ++l) {
                const int k = 32 * c + l;
                const float4 o = *reinterpret_cast<const float4*>(op + k * 32 + 4 * cq);
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
        float* dst = qp + v * vq + (pr0 + 2 * g) * 32 + 4 * cq;
        *reinterpret_cast<float4*>(dst) = make_float4(r0[0], r0[1], r0[2], r0[3]);
        *reinterpret_cast<float4*>(dst + 32) = make_float4(r1[0], r1[1], r1[2], r1[3]);
    }
}

template <typename T, int NP, bool SMEM_OP>
__global__ void __launch_bounds__(256) m2m_warp_kernel(int level, const T* __restrict__ qc,
                                                       const T* __restrict__ m2m,
                                                       const typename Mono<T>::V* __restrict__ Qin,
                                                       T* __restrict__ qp,
                                                       typename Mono<T>::V* __restrict__ Qout) {
    griddep_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sop = reinterpret_cast<T*>(smem_raw);
    if (SMEM_OP) {
        constexpr int N4 = 4 * NP * NP * (int)sizeof(T) / 16;
        for (int i = threadIdx.x; i < N4; i += blockDim.x)
            reinterpret_cast<uint4*>(sop)[i] = __ldg(reinterpret_cast<const uint4*>(m2m) + i);
        __syncthreads();
    }
    m2m_parents<T, NP>(level, qc, SMEM_OP ? sop : m2m, Qin, qp, Qout,
                       ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5, ((int64_t)gridDim.x * blockDim.x) >> 5);
}

// ------------------------------------------------------------------------- P2P + L2P
// One warp per target leaf (row-major).  The sources of the leaf's 3x3 neighbourhood
// (three contiguous ranges) are staged in shared memory as (table offset, charge).
// For a batch of nt <= 32 targets the lanes are split into G = 32/nt groups: lane l
// takes target l % nt and every G-th source of its group, so each near-field pair is
// one table load and one multiply-add; the G partial sums are combined with shuffles.
// The table holds phi(dx, dy) - phi0 for |dx|, |dy| <= 2s-1 with row width W, so
// idx(target) - idx(source) addresses it directly; phi0 times the block's charge (sum
// of the nine leaf charges Q) is added in the compensated channel.  On the mixed path
// each lane sums its products with Kahan compensation: the near field of a target is
// a sum of up to 9 N_leaf terms whose constant parts cancel.
constexpr int kP2PWarps = 8;
constexpr int kP2PCap = 9 * 64;  // staged sources per warp per chunk

template <typename T, int NP>
__global__ void __launch_bounds__(kP2PWarps * 32) p2p_leaf_kernel(
    int L, int side, const int32_t* __restrict__ sbeg, const int32_t* __restrict__ sloc,
    const int32_t* __restrict__ tbeg, const int32_t* __restrict__ tloc,
    const int32_t* __restrict__ tperm, const T* __restrict__ f_sorted, const T* __restrict__ table,
    int tab_H, int tab_W, const T* __restrict__ uhat, const typename Mono<T>::V* __restrict__ Cleaf,
    const typename Mono<T>::V* __restrict__ Qleaf, const T* __restrict__ tofsT,
    double* __restrict__ u, double* __restrict__ u_near, double* __restrict__ u_far) {
    griddep_wait();
    using M = Mono<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tab_n = (2 * tab_H + 1) * tab_W;
    T* tab = reinterpret_cast<T*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    SrcEntry<T>* s_src = reinterpret_cast<SrcEntry<T>*>(tab + tab_n) + warp * kP2PCap;
    T* s_uhat = reinterpret_cast<T*>(reinterpret_cast<SrcEntry<T>*>(tab + tab_n) + kP2PWarps * kP2PCap) +
                warp * NP;
    block_stage(tab, table, tab_n);
    const typename M::V phi0 = M::make(table[tab_n], table[tab_n + 1]);
    __syncthreads();
    const T* tab_c = tab + (tab_H + tab_H * tab_W);  // centre: phi(0, 0) - phi0
    const int n = 1 << L;
    const int64_t n_leaves = (int64_t)n * n;
    const int64_t nwarps = (int64_t)gridDim.x * kP2PWarps;

    for (int64_t leaf = (int64_t)blockIdx.x * kP2PWarps + warp; leaf < n_leaves; leaf += nwarps) {
        const int tb = tbeg[leaf], te = tbeg[leaf + 1];
        if (tb == te) continue;
        const int bx = (int)(leaf & (n - 1)), by = (int)(leaf >> L);
        const int c0 = max(bx - 1, 0), c1 = min(bx + 1, n - 1);
        // three row ranges [rb, re) with column boundaries
        int rb[3], rm1[3], rm2[3], re[3], rdy[3];
        int ns = 0;
        // charge of the 3x3 block (lanes 0..8 each read one leaf)
        typename M::V qn = M::zero();
        {
            const int dx = lane % 3 - 1, dy = lane / 3 - 1;
            const int nx = bx + dx, ny = by + dy;
            if (lane < 9 && nx >= 0 && nx < n && ny >= 0 && ny < n) qn = Qleaf[morton2(nx, ny)];
#pragma unroll
            for (int off = 16; off; off >>= 1) qn = M::add(qn, shfl_xor_v(qn, off));
        }
        const double near_const = M::to_double(M::mul(phi0, qn));
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int yy = by + r - 1;
            rdy[r] = r - 1;
            if (yy < 0 || yy >= n) {
                rb[r] = rm1[r] = rm2[r] = re[r] = 0;
                continue;
            }
            const int base = yy * n;
            rb[r] = sbeg[base + c0];
            rm1[r] = sbeg[base + c0 + 1];
            rm2[r] = c1 - c0 >= 2 ? sbeg[base + c0 + 2] : sbeg[base + c1 + 1];
            re[r] = sbeg[base + c1 + 1];
            ns += re[r] - rb[r];
        }
        if (uhat) {
            const uint32_t mort = morton2(bx, by);
            for (int i = lane; i < NP; i += 32) s_uhat[i] = uhat[(size_t)mort * NP + i];
        }
        __syncwarp();
        const int n_chunks = (ns + kP2PCap - 1) / kP2PCap;
        auto fill = [&](int v0) {
            const int cn = min(kP2PCap, ns - v0);
            int skip = v0;
            int w = 0;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const int len = re[r] - rb[r];
                int a = min(skip, len);
                skip -= a;
                const int take = min(len - a, cn - w);
                const int ybase = tab_W * (rdy[r] * side);
                for (int v = lane; v < take; v += 32) {
                    const int j = rb[r] + a + v;
                    const int col = c0 + (j >= rm1[r]) + (j >= rm2[r]);
                    const int l = sloc[j];
                    SrcEntry<T> e;
                    e.off = (col - bx) * side + (l & 0xffff) + ybase + tab_W * (l >> 16);
                    e.f = f_sorted[j];
                    s_src[w + v] = e;
                }
                w += take;
            }
            __syncwarp();
            return cn;
        };
        int cn = n_chunks == 1 ? fill(0) : 0;
        const typename M::V cl = Cleaf ? Cleaf[morton2(bx, by)] : M::zero();
        for (int t0 = tb; t0 < te; t0 += 32) {
            const int nt = min(32, te - t0);
            const int G = 32 / nt;
            const int t = lane % nt, g = lane / nt;
            const bool active = g < G;
            const int tl = tloc[t0 + t];
            const int tx = tl & 0xffff, ty = tl >> 16;
            const T* tp = tab_c + (tx + tab_W * ty);
            T acc = T(0), cmp = T(0);  // Kahan sum and its compensation (mixed path)
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
            for (int ch = 0; ch < n_chunks; ++ch) {
                if (n_chunks > 1) {
                    __syncwarp();
                    cn = fill(ch * kP2PCap);
                }
                if (active) {
                    int j = g;
                    for (; j + G < cn; j += 2 * G) {
                        const SrcEntry<T> e0 = s_src[j], e1 = s_src[j + G];
                        const T p0 = tp[-e0.off] * e0.f;
                        const T p1 = tp[-e1.off] * e1.f;
                        add(p0);
                        add(p1);
                    }
                    if (j < cn) {
                        const SrcEntry<T> e0 = s_src[j];
                        add(tp[-e0.off] * e0.f);
                    }
                }
            }
            // combine the G groups into lane t (compensations folded in)
            acc -= cmp;
            for (int k = 1; k < G; ++k) {
                const T v = shfl(acc, t + k * nt);
                if (g == 0) add(v);
            }
            acc -= cmp;
            if (lane < nt) {
                T far = T(0);
                if (uhat) {
                    const T* row = tofsT + (size_t)(tx + side * ty) * NP;
#pragma unroll 8
                    for (int p = 0; p < NP; ++p) far = fma(ldg(row + p), s_uhat[p], far);
                }
                const int dst = tperm[t0 + lane];
                const double dn = (double)acc + near_const;
                const double df = (double)far + M::to_double(cl);
                if (u) u[dst] = dn + df;
                if (u_near) u_near[dst] = dn;
                if (u_far) u_far[dst] = df;
            }
        }
        __syncwarp();
    }
}

// Strip variant (the normal case).  A block takes a strip of SW consecutive leaves
// of one leaf row.  Their 3x3 neighbourhoods lie in three contiguous source ranges
// (rows by-1, by, by+1, columns bx0-1 .. bx0+SW), which are staged once with
// coalesced loads; each staged source gets its table offset relative to the strip's
// first leaf, so a target in leaf bx reads phi through a pointer shifted by
// (bx - bx0) * s and the pair loop stays one load and one multiply-add per pair.
// Targets and leaf charges of the strip are staged alongside.  The strip form computes
// the near field alone (the far field has its own L2P kernel).  The host picks SW so
// the staged data fit (3 (SW+2) max_leaf_src <= CAPS).  Twelve warps per block, three
// blocks per SM at binary32 (uniform_1m, mixed p = 8: 117 us against 127 us with eight
// warps and 145 us with sixteen, two blocks per SM).
template <typename T>
struct StripCfg {
    static constexpr int WARPS = 12;
    static constexpr int CAPS = sizeof(T) == 4 ? 4096 : 2048;  // staged sources
    static constexpr int CAPT = 2048;                          // staged targets
    static constexpr int MAXSW = 32;
};

template <typename T, int NP>
__global__ void __launch_bounds__(StripCfg<T>::WARPS * 32) p2p_strip_kernel(
    int L, int side, int SW, const int32_t* __restrict__ sbeg, const int32_t* __restrict__ sloc,
    const int32_t* __restrict__ tbeg, const int32_t* __restrict__ tloc, const int32_t* __restrict__ tperm,
    const T* __restrict__ f_sorted, const T* __restrict__ table, int tab_H, int tab_W,
    const typename Mono<T>::V* __restrict__ Cleaf, const typename Mono<T>::V* __restrict__ Qleaf,
    double* __restrict__ u, double* __restrict__ u_near, double* __restrict__ u_far) {
    using M = Mono<T>;
    using V = typename M::V;
    using Cfg = StripCfg<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tab_n = (2 * tab_H + 1) * tab_W;
    T* tab = reinterpret_cast<T*>(smem_raw);
    SrcEntry<T>* s_src = reinterpret_cast<SrcEntry<T>*>(tab + tab_n);
    V* s_q = reinterpret_cast<V*>(s_src + Cfg::CAPS);                    // [3][MAXSW+2]
    V* s_c = s_q + 3 * (Cfg::MAXSW + 2);                                 // [MAXSW]
    int* s_tloc = reinterpret_cast<int*>(s_c + Cfg::MAXSW);              // [CAPT]
    int* s_tperm = s_tloc + Cfg::CAPT;                                   // [CAPT]
    int* s_sb = s_tperm + Cfg::CAPT;                                     // [3][MAXSW+3]
    int* s_tb = s_sb + 3 * (Cfg::MAXSW + 3);                             // [MAXSW+1]
    __shared__ int s_rs[4];
    __shared__ int s_ra[Cfg::MAXSW][3], s_rl[Cfg::MAXSW][3];  // per-leaf source ranges
    __shared__ double s_nc[Cfg::MAXSW];                       // per-leaf phi0 * Q_near

    block_stage(tab, table, tab_n);
    const V phi0 = M::make(table[tab_n], table[tab_n + 1]);
    const T* tab_c = tab + (tab_H + tab_H * tab_W);
    const int n = 1 << L;
    const int n_seg = (n + SW - 1) / SW;
    const int64_t n_strips = (int64_t)n * n_seg;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    for (int64_t strip = blockIdx.x; strip < n_strips; strip += gridDim.x) {
        const int by = (int)(strip / n_seg);
        const int bx0 = (int)(strip % n_seg) * SW;
        const int bx1 = min(bx0 + SW, n);  // exclusive
        const int c_lo = max(bx0 - 1, 0), c_hi = min(bx1, n - 1);
        const int ncol = c_hi - c_lo + 1;
        __syncthreads();  // previous strip done with the staging buffers
        // leaf boundaries of the three source rows and the target row (int items), leaf
        // charges and incoming constants (V items): a thread loads one of each, then stores
        {
            const int nA = 3 * (ncol + 1), nI = nA + (bx1 - bx0 + 1);
            const int nC = 3 * ncol, nV = nC + (bx1 - bx0);
            for (int i = threadIdx.x; i < max(nI, nV); i += blockDim.x) {
                int iv = 0;
                V vv = M::zero();
                if (i < nA) {
                    const int r = i / (ncol + 1), c = i % (ncol + 1);
                    const int yy = by + r - 1;
                    if (yy >= 0 && yy < n) iv = sbeg[(int64_t)yy * n + c_lo + c];
                } else if (i < nI) {
                    iv = tbeg[(int64_t)by * n + bx0 + (i - nA)];
                }
                if (i < nC) {
                    const int r = i / ncol, c = i % ncol;
                    const int yy = by + r - 1;
                    if (yy >= 0 && yy < n) vv = Qleaf[morton2(c_lo + c, yy)];
                } else if (i < nV && Cleaf) {
                    vv = Cleaf[morton2(bx0 + (i - nC), by)];
                }
                if (i < nA) s_sb[(i / (ncol + 1)) * (Cfg::MAXSW + 3) + i % (ncol + 1)] = iv;
                else if (i < nI) s_tb[i - nA] = iv;
                if (i < nC) s_q[(i / ncol) * (Cfg::MAXSW + 2) + i % ncol] = vv;
                else if (i < nV) s_c[i - nC] = vv;
            }
        }
        __syncthreads();
        // per-leaf source ranges (three staged rows) and near-field constant phi0 * Q_near
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
        // sources: coalesced copy + strip-relative table offset; targets with their leaf
        // in the strip
        stage_strip_sources<T>(s_src, ns_strip, s_rs, s_sb, Cfg::MAXSW + 3, ncol, c_lo, bx0, side, tab_W, sloc,
                               f_sorted);
        const int tb0 = s_tb[0], nt_strip = s_tb[bx1 - bx0] - tb0;
        stage_strip_targets(s_tloc, s_tperm, nt_strip, s_tb, bx1 - bx0, tb0, tloc, tperm);
        __syncthreads();

        // pairs: a warp takes 32 consecutive targets of the strip (one per lane, from up
        // to three leaves); each lane walks its leaf's three source ranges.  Products are
        // summed by plain multiply-adds in blocks of four, and the block sums are added
        // with compensation (fp32) so the long sums keep fp32-level relative accuracy.
        const int n_chunks = (nt_strip + 31) >> 5;
        for (int chunk = warp; chunk < n_chunks; chunk += Cfg::WARPS) {
            const int v = chunk * 32 + lane;
            const bool active = v < nt_strip;
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
            if (active) {
                const int dst = s_tperm[v];
                const double dn = (double)acc + s_nc[li];
                const double df = M::to_double(s_c[li]);
                if (u) u[dst] = dn + df;
                if (u_near) u_near[dst] = dn;
                if (u_far) u_far[dst] = df;
            }
        }
    }
}

// Near field for KR charge vectors at once (lfmm_eval_multi): the strip kernel's
// staging and pair loop, with each staged source carrying its KR charges (one 16-byte
// vector for KR = 4 in binary32) so that every table word serves KR multiply-adds.
// Per charge vector the operations and their order are those of p2p_strip_kernel, so
// each result equals the single-vector one bit for bit.  Vector r of the pass reads
// f_sorted + r * f_stride and Qleaf + r * q_stride and writes u_near + r * u_stride
// (binary64, caller order); nr <= KR vectors are active.
template <typename T, int KR>
struct StripMultiCfg {
    static constexpr int WARPS = 8;
    static constexpr int CAPS = (sizeof(T) == 4 ? 4096 : 2048) / (KR > 1 ? 2 : 1);
    static constexpr int CAPT = 2048;
    static constexpr int MAXSW = 32;
};

template <typename T, int KR>
__global__ void __launch_bounds__(StripMultiCfg<T, KR>::WARPS * 32) p2p_strip_multi_kernel(
    int L, int side, int SW, int nr, const int32_t* __restrict__ sbeg, const int32_t* __restrict__ sloc,
    const int32_t* __restrict__ tbeg, const int32_t* __restrict__ tloc, const int32_t* __restrict__ tperm,
    const T* __restrict__ f_sorted, int64_t f_stride, const T* __restrict__ table, int tab_H, int tab_W,
    const typename Mono<T>::V* __restrict__ Qleaf, int64_t q_stride, double* __restrict__ u_near,
    int64_t u_stride) {
    griddep_wait();
    using M = Mono<T>;
    using V = typename M::V;
    using Cfg = StripMultiCfg<T, KR>;
    using FV = VecT<T, KR>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tab_n = (2 * tab_H + 1) * tab_W;
    T* tab = reinterpret_cast<T*>(smem_raw);
    FV* s_f = reinterpret_cast<FV*>(reinterpret_cast<unsigned char*>(smem_raw) +
                                    (((size_t)tab_n * sizeof(T) + 15) & ~(size_t)15));   // [CAPS]
    int* s_off = reinterpret_cast<int*>(s_f + Cfg::CAPS);                              // [CAPS]
    V* s_q = reinterpret_cast<V*>(s_off + Cfg::CAPS);                                  // [KR][3][MAXSW+2]
    int* s_tloc = reinterpret_cast<int*>(s_q + KR * 3 * (Cfg::MAXSW + 2));             // [CAPT]
    int* s_tperm = s_tloc + Cfg::CAPT;                                                 // [CAPT]
    int* s_sb = s_tperm + Cfg::CAPT;                                                   // [3][MAXSW+3]
    int* s_tb = s_sb + 3 * (Cfg::MAXSW + 3);                                           // [MAXSW+1]
    __shared__ int s_rs[4];
    __shared__ int s_ra[Cfg::MAXSW][3], s_rl[Cfg::MAXSW][3];
    __shared__ double s_nc[KR][Cfg::MAXSW];

    block_stage(tab, table, tab_n);
    const V phi0 = M::make(table[tab_n], table[tab_n + 1]);
    const T* tab_c = tab + (tab_H + tab_H * tab_W);
    const int n = 1 << L;
    const int n_seg = (n + SW - 1) / SW;
    const int64_t n_strips = (int64_t)n * n_seg;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    for (int64_t strip = blockIdx.x; strip < n_strips; strip += gridDim.x) {
        const int by = (int)(strip / n_seg);
        const int bx0 = (int)(strip % n_seg) * SW;
        const int bx1 = min(bx0 + SW, n);
        const int c_lo = max(bx0 - 1, 0), c_hi = min(bx1, n - 1);
        const int ncol = c_hi - c_lo + 1;
        __syncthreads();
        for (int i = threadIdx.x; i < 3 * (ncol + 1); i += blockDim.x) {
            const int r = i / (ncol + 1), c = i % (ncol + 1);
            const int yy = by + r - 1;
            s_sb[r * (Cfg::MAXSW + 3) + c] = (yy >= 0 && yy < n) ? sbeg[(int64_t)yy * n + c_lo + c] : 0;
        }
        for (int i = threadIdx.x; i <= bx1 - bx0; i += blockDim.x) s_tb[i] = tbeg[(int64_t)by * n + bx0 + i];
        for (int i = threadIdx.x; i < KR * 3 * ncol; i += blockDim.x) {
            const int k = i / (3 * ncol), rc = i % (3 * ncol);
            const int r = rc / ncol, c = rc % ncol;
            const int yy = by + r - 1;
            s_q[(k * 3 + r) * (Cfg::MAXSW + 2) + c] =
                (k < nr && yy >= 0 && yy < n) ? Qleaf[(size_t)k * q_stride + morton2(c_lo + c, yy)] : M::zero();
        }
        __syncthreads();
        for (int li = threadIdx.x; li < bx1 - bx0; li += blockDim.x) {
            const int bx = bx0 + li;
            const int ca = max(bx - 1, 0) - c_lo, cb = min(bx + 1, n - 1) - c_lo + 1;
            int rs = 0;
            V qn[KR];
#pragma unroll
            for (int k = 0; k < KR; ++k) qn[k] = M::zero();
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const int* sb = s_sb + r * (Cfg::MAXSW + 3);
                s_ra[li][r] = rs + (sb[ca] - sb[0]);
                s_rl[li][r] = sb[cb] - sb[ca];
                rs += sb[ncol] - sb[0];
                for (int c = ca; c < cb; ++c)
#pragma unroll
                    for (int k = 0; k < KR; ++k) qn[k] = M::add(qn[k], s_q[(k * 3 + r) * (Cfg::MAXSW + 2) + c]);
            }
#pragma unroll
            for (int k = 0; k < KR; ++k) s_nc[k][li] = M::to_double(M::mul(phi0, qn[k]));
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
            s_off[v] = (c_lo + lo - bx0) * side + (l & 0xffff) + tab_W * ((r - 1) * side + (l >> 16));
            FV fv;
#pragma unroll
            for (int k = 0; k < KR; ++k) fv.v[k] = k < nr ? f_sorted[(size_t)k * f_stride + j] : T(0);
            s_f[v] = fv;
        }
        const int tb0 = s_tb[0], nt_strip = s_tb[bx1 - bx0] - tb0;
        stage_strip_targets(s_tloc, s_tperm, nt_strip, s_tb, bx1 - bx0, tb0, tloc, tperm);
        __syncthreads();

        const int n_chunks = (nt_strip + 31) >> 5;
        for (int chunk = warp; chunk < n_chunks; chunk += Cfg::WARPS) {
            const int v = chunk * 32 + lane;
            const bool active = v < nt_strip;
            const int tl = s_tloc[active ? v : chunk * 32];
            const int li = (tl >> 8) & 0xff, tx = tl & 0xff, ty = tl >> 16;
            const T* tp = tab_c + (tx + tab_W * ty + li * side);
            T acc[KR], cmp[KR];
#pragma unroll
            for (int k = 0; k < KR; ++k) acc[k] = cmp[k] = T(0);
            auto add = [&](int k, T term) {
                if constexpr (sizeof(T) == 4) {
                    const T y = term - cmp[k];
                    const T s2 = acc[k] + y;
                    cmp[k] = (s2 - acc[k]) - y;
                    acc[k] = s2;
                } else {
                    acc[k] += term;
                }
            };
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const int* so = s_off + s_ra[li][r];
                const FV* sf = s_f + s_ra[li][r];
                const int len = active ? s_rl[li][r] : 0;
                int j = 0;
#pragma unroll 2
                for (; j + 4 <= len; j += 4) {
                    const T p0 = tp[-so[j]], p1 = tp[-so[j + 1]], p2 = tp[-so[j + 2]], p3 = tp[-so[j + 3]];
                    const FV f0 = sf[j], f1 = sf[j + 1], f2 = sf[j + 2], f3 = sf[j + 3];
#pragma unroll
                    for (int k = 0; k < KR; ++k) {
                        T b = p0 * f0.v[k];
                        b = fma(p1, f1.v[k], b);
                        b = fma(p2, f2.v[k], b);
                        b = fma(p3, f3.v[k], b);
                        add(k, b);
                    }
                }
                if (j < len) {
                    T b[KR];
#pragma unroll
                    for (int k = 0; k < KR; ++k) b[k] = T(0);
                    for (; j < len; ++j) {
                        const T pj = tp[-so[j]];
                        const FV fj = sf[j];
#pragma unroll
                        for (int k = 0; k < KR; ++k) b[k] = fma(pj, fj.v[k], b[k]);
                    }
#pragma unroll
                    for (int k = 0; k < KR; ++k) add(k, b[k]);
                }
            }
            if (active) {
                const int dst = s_tperm[v];
#pragma unroll
                for (int k = 0; k < KR; ++k)
                    if (k < nr) u_near[(size_t)k * u_stride + dst] = (double)(acc[k] - cmp[k]) + s_nc[k][li];
            }
        }
    }
}

// ------------------------------------------------------------------------- fused small levels
// The coarse levels hold few boxes, so one launch per level is mostly launch and
// latency.  Two cooperative kernels (all blocks co-resident) cover them instead:
//   upward:   M2M of every level from L-1 up to 2, one grid barrier between levels;
//   downward: the M2L part (27 K-steps, no parent term) of every small level at once,
//             then the L2L chain u_hat_l += T_ifi u_hat_parent and C_l += C_parent from
//             level 3 down to the last small level, one barrier per level.
// The result equals the per-level sweeps (the parent term is added after instead of
// beside the interaction-list terms).
constexpr int kMaxLevels = 16;

template <typename T>
struct LevelPtrs {
    using V = typename Mono<T>::V;
    T* q[kMaxLevels];            // outgoing expansions of level l
    T* u[kMaxLevels];            // incoming expansions of level l
    V* Q[kMaxLevels];            // total charges
    V* C[kMaxLevels];            // incoming constants
    const T* tifo[kMaxLevels];   // deflated T_ifo of level l's boxes
    const T* mono[kMaxLevels];   // deflation constants
    const T* l2l[kMaxLevels];    // [4][NP][NP] from level l-1 to level l
    const T* m2m[kMaxLevels];    // [4NP][NP] from level l+1 to level l
    int64_t item_off[kMaxLevels + 1];  // downward: first M2L work item of level l0 + i
    int nvec;                          // charge vectors; vector v's arrays at v vq (q, u) / v vQ (Q, C)
    int64_t vq, vQ;
    // fused small-level M2L split along K: chunk c of vector v writes its partial sums
    // to part + ((v nch + c) part_stride + box over the levels) NP (then the constants)
    T* part;
    int nch;
    int64_t part_stride;
};

template <typename T, int NP, bool SMEM_OP>
__global__ void __launch_bounds__(256) m2m_up_kernel(LevelPtrs<T> P, int l_top, int l_bot, unsigned* sync,
                                                     int* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sop = reinterpret_cast<T*>(smem_raw);
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int l = l_top; l >= l_bot; --l) {
        const T* op = P.m2m[l];
        if (SMEM_OP) {
            constexpr int N4 = 4 * NP * NP * (int)sizeof(T) / 16;
            __syncthreads();
            for (int i = threadIdx.x; i < N4; i += blockDim.x)
                reinterpret_cast<uint4*>(sop)[i] = __ldg(reinterpret_cast<const uint4*>(op) + i);
            __syncthreads();
            op = sop;
        }
        bool tiled = false;
        if constexpr (std::is_same<T, float>::value && NP == 32 && SMEM_OP) {
            if (((int64_t)P.nvec << (2 * l)) >= kM2MTileMinItems) {
                m2m_tiles_f32(l, P.q[l + 1], op, P.Q[l + 1], P.q[l], P.Q[l], P.nvec, P.vq, P.vQ,
                              sop + 4 * NP * NP);
                tiled = true;
            }
        }
        if (!tiled)
            m2m_parents<T, NP>(l, P.q[l + 1], op, P.Q[l + 1], P.q[l], P.Q[l], wid, nw, P.nvec, P.vq, P.vQ);
        if (l > l_bot) grid_barrier(sync, sync + 1, status);
    }
}

// L2L of one child box b of level l (charge vector vv) by one warp: lanes own outputs,
// the parent's expansion broadcast by shuffles; adds to the box's M2L result and carries
// the incoming constant down.
template <typename T, int NP>
__device__ __forceinline__ void l2l_box(const LevelPtrs<T>& P, int l, int64_t vv, int64_t b, int lane) {
    using M = Mono<T>;
    constexpr int PL = NP / 32;
    const int64_t par = b >> 2;
    const int c = (int)(b & 3);  // Morton: child index = parity class (cx + 2 cy)
    const T* op = P.l2l[l] + (size_t)c * NP * NP;
    T* ul = P.u[l] + vv * P.vq;
    typename M::V* Cl = P.C[l] + vv * P.vQ;
    T pv[PL], acc[PL];
#pragma unroll
    for (int i = 0; i < PL; ++i) {
        pv[i] = ldcg(P.u[l - 1] + vv * P.vq + (size_t)par * NP + lane + 32 * i);
        acc[i] = ldcg(ul + (size_t)b * NP + lane + 32 * i);
    }
#pragma unroll
    for (int i = 0; i < PL; ++i)
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            const T v = shfl(pv[i], kk);
            const T* row = op + (size_t)(32 * i + kk) * NP;
#pragma unroll
            for (int o = 0; o < PL; ++o) acc[o] = fma(ldg(row + lane + 32 * o), v, acc[o]);
        }
#pragma unroll
    for (int i = 0; i < PL; ++i) ul[(size_t)b * NP + lane + 32 * i] = acc[i];
    if (lane == 0) Cl[b] = M::add(ldcg(Cl + b), ldcg(P.C[l - 1] + vv * P.vQ + par));
}

// The fused kernel's tiles have 27 K-steps (no parent term): 9 warps take 3 each (3 warps
// x 9 for binary64-width elements with 64 coefficients, to fit shared memory).
template <typename T, int NP>
struct FusedCfg {
    static constexpr int WARPS = (sizeof(T) == 8 && NP == 64) ? 3 : 9;
    static constexpr size_t SMEM = (size_t)WARPS * (NP * 32 + SkCfg<T, NP>::ROWS) * sizeof(T);
};

template <typename T, int NP>
__global__ void __launch_bounds__(FusedCfg<T, NP>::WARPS * 32) m2l_small_kernel(LevelPtrs<T> P, int l0, int l1,
                                                                                unsigned* sync, int* status) {
    using M = Mono<T>;
    constexpr int PL = NP / 32;
    const int nl = l1 - l0 + 1;
    const int64_t n_items = P.item_off[nl];
    const int nch = P.nch;
    using V = typename M::V;
    V* cpart = nch > 1 ? reinterpret_cast<V*>(P.part + (int64_t)P.nvec * nch * P.part_stride * NP) : nullptr;
    // M2L part of every level: work item = (K chunk, charge vector, level, class, 32-box
    // tile); with several chunks each writes partial sums, added below in chunk order
    for (int64_t it = blockIdx.x; it < n_items * P.nvec * nch; it += gridDim.x) {
        const int ch = (int)(it / (n_items * P.nvec));
        const int64_t rest = it - (int64_t)ch * n_items * P.nvec;
        const int64_t v = rest / n_items, item = rest - v * n_items;
        int i = 0;
        while (item >= P.item_off[i + 1]) ++i;
        const int l = l0 + i;
        const int64_t tiles = (((int64_t)1 << (2 * (l - 1))) + 31) / 32;
        const int64_t local = item - P.item_off[i];
        if (nch == 1) {
            m2l_splitk_tile<T, NP, FusedCfg<T, NP>::WARPS>(l, (int)(local / tiles), local % tiles, P.q[l] + v * P.vq,
                                                           nullptr, P.tifo[l], nullptr, P.mono[l], P.Q[l] + v * P.vQ,
                                                           nullptr, P.u[l] + v * P.vq, P.C[l] + v * P.vQ);
        } else {
            const int per = (27 + nch - 1) / nch;
            int64_t loff = 0;  // boxes of the levels before l
            for (int ll = l0; ll < l; ++ll) loff += (int64_t)1 << (2 * ll);
            const int64_t base = (v * nch + ch) * P.part_stride + loff;
            m2l_splitk_tile<T, NP, FusedCfg<T, NP>::WARPS>(l, (int)(local / tiles), local % tiles, P.q[l] + v * P.vq,
                                                           nullptr, P.tifo[l], nullptr, P.mono[l], P.Q[l] + v * P.vQ,
                                                           nullptr, P.part + base * NP, cpart + base, ch * per,
                                                           ch * per + per);
        }
    }
    if (nch > 1) {  // expansions and constants = the chunks' partial sums, in chunk order
        grid_barrier(sync, sync + 1, status);
        const int64_t nt = (int64_t)gridDim.x * blockDim.x;
        const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        const int64_t per_v = P.part_stride * NP;
        for (int64_t e = t0; e < P.nvec * per_v; e += nt) {
            const int64_t v = e / per_v, r = e - v * per_v, gb = r / NP;
            const int j = (int)(r - gb * NP);
            int l = l0;
            int64_t b = gb;
            while (b >= ((int64_t)1 << (2 * l))) b -= (int64_t)1 << (2 * l++);
            T acc = P.part[((v * nch) * P.part_stride + gb) * NP + j];
            for (int c = 1; c < nch; ++c) acc += P.part[((v * nch + c) * P.part_stride + gb) * NP + j];
            P.u[l][v * P.vq + b * NP + j] = acc;
        }
        for (int64_t e = t0; e < P.nvec * P.part_stride; e += nt) {
            const int64_t v = e / P.part_stride, gb = e - v * P.part_stride;
            int l = l0;
            int64_t b = gb;
            while (b >= ((int64_t)1 << (2 * l))) b -= (int64_t)1 << (2 * l++);
            V acc = M::zero();
            for (int c = 0; c < nch; ++c) acc = M::add(acc, cpart[(v * nch + c) * P.part_stride + gb]);
            P.C[l][v * P.vQ + b] = acc;
        }
    }
    if (nl == 1) return;
    grid_barrier(sync, sync + 1, status);
    // L2L chain: one warp per child box, lanes own outputs, the parent's expansion
    // broadcast by shuffles.  Levels below l_sub level by level with a grid barrier
    // between them; the last three levels by subtrees (one block per box of level l_sub
    // and its children and grandchildren, block barriers only).
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int l_sub = l1 - l0 >= 3 ? l1 - 2 : l1 + 1;
    for (int l = l0 + 1; l < l_sub; ++l) {
        const int64_t nb = (int64_t)1 << (2 * l);
        const int64_t n_box_items = nb * P.nvec;  // (charge vector, child box)
        // software pipeline over the boxes: the next box's rows load during this one
        T npv[PL], nacc[PL];
        if (wid < n_box_items) {
            const int64_t v = wid / nb, bb = wid - v * nb;
#pragma unroll
            for (int i = 0; i < PL; ++i) {
                npv[i] = ldcg(P.u[l - 1] + v * P.vq + (size_t)(bb >> 2) * NP + lane + 32 * i);
                nacc[i] = ldcg(P.u[l] + v * P.vq + (size_t)bb * NP + lane + 32 * i);
            }
        }
        for (int64_t item = wid; item < n_box_items; item += nw) {
            const int64_t vv = item / nb, b = item - vv * nb;
            const int64_t par = b >> 2;
            const int c = (int)(b & 3);  // Morton: child index = parity class (cx + 2 cy)
            const T* op = P.l2l[l] + (size_t)c * NP * NP;
            T* ul = P.u[l] + vv * P.vq;
            typename M::V* Cl = P.C[l] + vv * P.vQ;
            T pv[PL], acc[PL];
#pragma unroll
            for (int i = 0; i < PL; ++i) {
                pv[i] = npv[i];
                acc[i] = nacc[i];
            }
            if (item + nw < n_box_items) {
                const int64_t v = (item + nw) / nb, bb = (item + nw) - v * nb;
#pragma unroll
                for (int i = 0; i < PL; ++i) {
                    npv[i] = ldcg(P.u[l - 1] + v * P.vq + (size_t)(bb >> 2) * NP + lane + 32 * i);
                    nacc[i] = ldcg(P.u[l] + v * P.vq + (size_t)bb * NP + lane + 32 * i);
                }
            }
#pragma unroll
            for (int i = 0; i < PL; ++i)
#pragma unroll 8
                for (int kk = 0; kk < 32; ++kk) {
                    const T v = shfl(pv[i], kk);
                    const T* row = op + (size_t)(32 * i + kk) * NP;
#pragma unroll
                    for (int o = 0; o < PL; ++o) acc[o] = fma(ldg(row + lane + 32 * o), v, acc[o]);
                }
#pragma unroll
            for (int i = 0; i < PL; ++i) ul[(size_t)b * NP + lane + 32 * i] = acc[i];
            if (lane == 0) Cl[b] = M::add(ldcg(Cl + b), ldcg(P.C[l - 1] + vv * P.vQ + par));
        }
        if (l < l1) grid_barrier(sync, sync + 1, status);
    }
    if (l_sub > l1) return;
    const int warp = threadIdx.x >> 5;
    const int64_t n_roots = ((int64_t)1 << (2 * l_sub)) * P.nvec;  // (charge vector, root box)
    for (int64_t item = blockIdx.x; item < n_roots; item += gridDim.x) {
        const int64_t vv = item >> (2 * l_sub), r = item & (((int64_t)1 << (2 * l_sub)) - 1);
        for (int g = 0; g <= l1 - l_sub; ++g) {
            const int64_t nb = (int64_t)1 << (2 * g);  // the root's descendants on level l_sub + g
            for (int64_t k = warp; k < nb; k += FusedCfg<T, NP>::WARPS)
                l2l_box<T, NP>(P, l_sub + g, vv, (r << (2 * g)) + k, lane);
            __syncthreads();  // the next generation reads this one
        }
    }
}

// ------------------------------------------------------------------------- L2P, final sum
// Far field of every target when the near field runs as a separate pass: one thread per
// sorted target, uf[caller index] = T_ofs(:, J)^T u_hat_leaf + C_leaf in binary64.
// T_ofs^T ([s^2][NP]) is staged in shared memory with row stride NP + 1, so the 32
// targets of a warp, at random local positions, read element p of their rows from 32
// different banks; the leaf's expansion row is shared by its ~N_leaf consecutive targets.
template <typename T, int NP, bool SMEM>
__global__ void __launch_bounds__(256) l2p_kernel(int64_t nt, int side, const int32_t* __restrict__ tleaf,
                                                  const int32_t* __restrict__ tloc, const int32_t* __restrict__ tperm,
                                                  const T* __restrict__ uhat,
                                                  const typename Mono<T>::V* __restrict__ Cleaf,
                                                  const T* __restrict__ tofsT, double* __restrict__ uf, int nvec,
                                                  int64_t vq, int64_t vQ) {
    griddep_wait();
    using M = Mono<T>;
    constexpr int E = (int)(16 / sizeof(T));
    constexpr int RS = NP + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* st = reinterpret_cast<T*>(smem_raw);
    if (SMEM) {
        // 16-byte loads, four in flight per thread, scattered into the padded rows
        constexpr int U = 4;
        const int n16 = side * side * NP / E;
        const uint4* src = reinterpret_cast<const uint4*>(tofsT);
        for (int i0 = threadIdx.x; i0 < n16; i0 += U * blockDim.x) {
            uint4 w[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 + u * (int)blockDim.x;
                if (i < n16) w[u] = __ldg(src + i);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 + u * (int)blockDim.x;
                if (i < n16) {
                    const T* e = reinterpret_cast<const T*>(&w[u]);
#pragma unroll
                    for (int k = 0; k < E; ++k) {
                        const int x = i * E + k;
                        st[(x / NP) * RS + (x % NP)] = e[k];
                    }
                }
            }
        }
        __syncthreads();
    }
    // (charge vector, target): vector v reads uhat + v vq, Cleaf + v vQ, writes uf + v nt.
    // The next item's leaf, position and caller index are loaded before this item's
    // expansion row, so their latency overlaps the arithmetic.
    const int64_t n_items = nt * nvec, stride = (int64_t)gridDim.x * blockDim.x;
    int64_t tv = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int nx_leaf = 0, nx_loc = 0, nx_perm = 0;
    if (tv < n_items) {
        const int64_t t = tv % nt;
        nx_leaf = tleaf[t];
        nx_loc = tloc[t];
        nx_perm = tperm[t];
    }
    for (; tv < n_items; tv += stride) {
        const int64_t v = tv / nt;
        const int leaf = nx_leaf, l = nx_loc, pm = nx_perm;
        if (tv + stride < n_items) {
            const int64_t t2 = (tv + stride) % nt;
            nx_leaf = tleaf[t2];
            nx_loc = tloc[t2];
            nx_perm = tperm[t2];
        }
        const int J = (l & 0xffff) + side * (l >> 16);
        const T* row = SMEM ? st + J * RS : tofsT + (size_t)J * NP;  // (table too large: L1 / L2)
        const uint4* uh = reinterpret_cast<const uint4*>(uhat + v * vq + (size_t)leaf * NP);
        T far = T(0);
#pragma unroll
        for (int c = 0; c < NP / E; ++c) {
            const uint4 ur = __ldg(uh + c);
            const T* v = reinterpret_cast<const T*>(&ur);
#pragma unroll
            for (int e = 0; e < E; ++e) far = fma(row[c * E + e], v[e], far);
        }
        uf[v * nt + pm] = (double)far + M::to_double(Cleaf[v * vQ + leaf]);
    }
}

// u = u_near + u_far (caller order), and the parts where requested
__global__ void combine_kernel(int64_t n, const double* __restrict__ un, const double* __restrict__ uf,
                               double* __restrict__ u, double* __restrict__ u_near, double* __restrict__ u_far) {
    griddep_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double a = un[i], b = uf[i];
        if (u) u[i] = a + b;
        if (u_near) u_near[i] = a;
        if (u_far) u_far[i] = b;
    }
}

}  // namespace

// ------------------------------------------------------------------------- launchers
template <typename T>
cudaError_t launch_p2m(const TreeView& t, const DeviceOps& ops, const double* f, T* f_sorted,
                       T* qhat_leaf, void* Q, cudaStream_t s, int nvec, int64_t vq, int64_t vQ) {
    const int threads = 256;
    int64_t blocks = (t.n_leaves * 8 * nvec + threads - 1) / threads;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) blocks = 1;
    using V = typename Mono<T>::V;
    if (ops.NP == 32)
        return launch_dependent(p2m_kernel<T, 32>, dim3((unsigned)blocks), dim3(threads), 0, s, t.L, t.src_begin,
                                t.src_loc, t.src_perm, f, f_sorted, (const T*)ops.tofsT, t.side, qhat_leaf, (V*)Q,
                                nvec, t.n_src_all, vq, vQ);
    return launch_dependent(p2m_kernel<T, 64>, dim3((unsigned)blocks), dim3(threads), 0, s, t.L, t.src_begin,
                            t.src_loc, t.src_perm, f, f_sorted, (const T*)ops.tofsT, t.side, qhat_leaf, (V*)Q, nvec,
                            t.n_src_all, vq, vQ);
}

template <typename T, int NP, int MODE>
static cudaError_t launch_translate(int level, const T* q, const T* u_par, const T* op, const T* l2l,
                                    const T* mono, const void* Qin, const void* Cpar, T* out, void* Qout,
                                    void* Cout, cudaStream_t s) {
    using C = TrCfg<T, NP>;
    using V = typename Mono<T>::V;
    {
        cudaError_t e = ensure_dynamic_smem((const void*)translate_kernel<T, NP, MODE>, C::SMEM);
        if (e != cudaSuccess) return e;
    }
    const int lg = MODE == kModeM2L ? level - 1 : level;
    const int64_t rows = (int64_t)1 << (2 * lg);
    dim3 grid((unsigned)((rows + C::BB - 1) / C::BB), MODE == kModeM2L ? 4 : 1);
    (void)launch_dependent(translate_kernel<T, NP, MODE>, dim3(grid), dim3(C::THREADS), C::SMEM, s,
        level, q, u_par, op, l2l, mono, (const V*)Qin, (const V*)Cpar, out, (V*)Qout, (V*)Cout);
    return cudaGetLastError();
}

template <typename T, int NP>
static cudaError_t launch_m2m_warp(const DeviceOps& ops, int k, int level, const T* q_child, const void* Q_child,
                                   T* q_parent, void* Q_parent, cudaStream_t s) {
    using V = typename Mono<T>::V;
    const int64_t n_par = (int64_t)1 << (2 * level);
    int64_t blocks = (n_par + 7) / 8;  // 8 warps per block, grid-stride over parents
    if (blocks > 152 * 8) blocks = 152 * 8;
    constexpr size_t op_bytes = (size_t)4 * NP * NP * sizeof(T);
    if constexpr (op_bytes <= 64 * 1024) {
        {
            cudaError_t e = ensure_dynamic_smem((const void*)m2m_warp_kernel<T, NP, true>, op_bytes);
            if (e != cudaSuccess) return e;
        }
        (void)launch_dependent(m2m_warp_kernel<T, NP, true>, dim3((int)blocks), dim3(256), op_bytes, s, level, q_child, (const T*)ops.m2m[k],
                                                                         (const V*)Q_child, q_parent, (V*)Q_parent);
    } else {
        (void)launch_dependent(m2m_warp_kernel<T, NP, false>, dim3((int)blocks), dim3(256), 0, s, level, q_child, (const T*)ops.m2m[k],
                                                                   (const V*)Q_child, q_parent, (V*)Q_parent);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_m2m(const DeviceOps& ops, int k, int level, const T* q_child, const void* Q_child,
                       T* q_parent, void* Q_parent, cudaStream_t s) {
    if (ops.NP == 32) return launch_m2m_warp<T, 32>(ops, k, level, q_child, Q_child, q_parent, Q_parent, s);
    return launch_m2m_warp<T, 64>(ops, k, level, q_child, Q_child, q_parent, Q_parent, s);
}

template <typename T, int NP>
static cudaError_t launch_m2l_splitk(const DeviceOps& ops, int k, int level, const T* q, const void* Qin,
                                     const T* u_par, const void* Cpar, T* out, void* Cout, cudaStream_t s) {
    using V = typename Mono<T>::V;
    const T* l2l = u_par ? (const T*)ops.l2l[k + 1] : nullptr;
    constexpr size_t smem = SkCfg<T, NP>::SMEM;
    static_assert(smem <= 227 * 1024, "split-K M2L block exceeds the shared memory of one SM");
    {
        cudaError_t e = ensure_dynamic_smem((const void*)m2l_splitk_kernel<T, NP>, smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t rows = (int64_t)1 << (2 * (level - 1));
    dim3 grid((unsigned)((rows + 31) / 32), 4);
    (void)launch_dependent(m2l_splitk_kernel<T, NP>, dim3(grid), dim3(SkCfg<T, NP>::WARPS * 32), smem, s, level, q, u_par, (const T*)ops.tifo[k], l2l,
                                                              (const T*)ops.mono[k], (const V*)Qin, (const V*)Cpar,
                                                              out, (V*)Cout);
    return cudaGetLastError();
}

// Levels below this use the split-K kernel, larger ones the tiled SIMT kernel (the
// tensor-core levels of the mixed path are launched by the caller).
constexpr int kM2LSplitKMaxLevel = 7;

template <typename T>
cudaError_t launch_m2l(const DeviceOps& ops, int k, int level, const T* q_level, const void* Q_level,
                       const T* u_parent, const void* C_parent, T* u_level, void* C_level, cudaStream_t s) {
    if (level <= kM2LSplitKMaxLevel) {
        if (ops.NP == 32)
            return launch_m2l_splitk<T, 32>(ops, k, level, q_level, Q_level, u_parent, C_parent, u_level, C_level, s);
        return launch_m2l_splitk<T, 64>(ops, k, level, q_level, Q_level, u_parent, C_parent, u_level, C_level, s);
    }
    const T* l2l = u_parent ? (const T*)ops.l2l[k + 1] : nullptr;
    if (ops.NP == 32)
        return launch_translate<T, 32, kModeM2L>(level, q_level, u_parent, (const T*)ops.tifo[k], l2l,
                                                 (const T*)ops.mono[k], Q_level, C_parent, u_level, nullptr,
                                                 C_level, s);
    return launch_translate<T, 64, kModeM2L>(level, q_level, u_parent, (const T*)ops.tifo[k], l2l,
                                             (const T*)ops.mono[k], Q_level, C_parent, u_level, nullptr, C_level,
                                             s);
}

template <typename T, int NP>
static cudaError_t launch_p2p_np(const TreeView& t, const DeviceOps& ops, const T* f_sorted, const T* uhat,
                                 const void* Cleaf, const void* Qleaf, double* u, double* un, double* uf,
                                 int num_sms, cudaStream_t s) {
    const size_t tab_bytes = (size_t)(2 * ops.tab_H + 1) * ops.tab_W * sizeof(T);
    const size_t smem = ((tab_bytes + 15) & ~(size_t)15) + (size_t)kP2PWarps * kP2PCap * sizeof(SrcEntry<T>) +
                        (size_t)kP2PWarps * NP * sizeof(T);
    {
        cudaError_t e = ensure_dynamic_smem((const void*)p2p_leaf_kernel<T, NP>, smem);
        if (e != cudaSuccess) return e;
    }
    const int per_sm_cached = blocks_per_sm((const void*)p2p_leaf_kernel<T, NP>, kP2PWarps * 32, smem);
    int64_t blocks = (t.n_leaves + kP2PWarps - 1) / kP2PWarps;
    const int64_t cap = (int64_t)num_sms * per_sm_cached;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    using V = typename Mono<T>::V;
    (void)launch_dependent(p2p_leaf_kernel<T, NP>, dim3((int)blocks), dim3(kP2PWarps * 32), smem, s,
        t.L, t.side, t.src_begin, t.src_loc, t.tgt_begin, t.tgt_loc, t.tgt_perm, f_sorted, (const T*)ops.p2p_table,
        ops.tab_H, ops.tab_W, uhat, (const V*)Cleaf, (const V*)Qleaf, (const T*)ops.tofsT, u, un, uf);
    return cudaGetLastError();
}

template <typename T, int NP>
static cudaError_t launch_p2p_strip(const TreeView& t, const DeviceOps& ops, int SW, const T* f_sorted,
                                    const T* uhat, const void* Cleaf, const void* Qleaf, double* u, double* un,
                                    double* uf, int num_sms, cudaStream_t s) {
    using Cfg = StripCfg<T>;
    using V = typename Mono<T>::V;
    const size_t tab_bytes = (size_t)(2 * ops.tab_H + 1) * ops.tab_W * sizeof(T);
    const size_t smem = tab_bytes + (size_t)Cfg::CAPS * sizeof(SrcEntry<T>) +
                        (size_t)(3 * (Cfg::MAXSW + 2) + Cfg::MAXSW) * sizeof(V) + (size_t)2 * Cfg::CAPT * sizeof(int) +
                        (size_t)(3 * (Cfg::MAXSW + 3) + Cfg::MAXSW + 1) * sizeof(int);
    {
        cudaError_t e = ensure_dynamic_smem((const void*)p2p_strip_kernel<T, NP>, smem);
        if (e != cudaSuccess) return e;
    }
    const int per_sm_cached = blocks_per_sm((const void*)p2p_strip_kernel<T, NP>, Cfg::WARPS * 32, smem);
    const int n = 1 << t.L;
    const int64_t strips = (int64_t)n * ((n + SW - 1) / SW);
    int64_t blocks = std::min<int64_t>(strips, (int64_t)num_sms * per_sm_cached);
    if (blocks < 1) blocks = 1;
    p2p_strip_kernel<T, NP><<<(int)blocks, Cfg::WARPS * 32, smem, s>>>(
        t.L, t.side, SW, t.src_begin, t.src_loc, t.tgt_begin, t.tgt_loc, t.tgt_perm, f_sorted,
        (const T*)ops.p2p_table, ops.tab_H, ops.tab_W, (const V*)Cleaf, (const V*)Qleaf, u, un, uf);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_p2p_l2p(const TreeView& t, const DeviceOps& ops, const T* f_sorted, const T* uhat,
                           const void* Cleaf, const void* Qleaf, double* u, double* un, double* uf, int num_sms,
                           cudaStream_t s) {
    using Cfg = StripCfg<T>;
    const int n = 1 << t.L;
    const int ms = std::max(1, t.max_leaf_src), mt = std::max(1, t.max_leaf_tgt);
    int SW = std::min({Cfg::MAXSW, Cfg::CAPS / (3 * ms) - 2, Cfg::CAPT / mt, n});
    if (SW >= 1 && uhat == nullptr) {  // the strip form is the near field alone
        if (ops.NP == 32) return launch_p2p_strip<T, 32>(t, ops, SW, f_sorted, uhat, Cleaf, Qleaf, u, un, uf, num_sms, s);
        return launch_p2p_strip<T, 64>(t, ops, SW, f_sorted, uhat, Cleaf, Qleaf, u, un, uf, num_sms, s);
    }
    if (ops.NP == 32) return launch_p2p_np<T, 32>(t, ops, f_sorted, uhat, Cleaf, Qleaf, u, un, uf, num_sms, s);
    return launch_p2p_np<T, 64>(t, ops, f_sorted, uhat, Cleaf, Qleaf, u, un, uf, num_sms, s);
}

template <typename T, int KR>
static cudaError_t launch_p2p_multi_kr(const TreeView& t, const DeviceOps& ops, int SW, int nr, const T* f_sorted,
                                       int64_t f_stride, const void* Qleaf, int64_t q_stride, double* un,
                                       int64_t u_stride, int num_sms, cudaStream_t s) {
    using Cfg = StripMultiCfg<T, KR>;
    using V = typename Mono<T>::V;
    const size_t tab_bytes = (((size_t)(2 * ops.tab_H + 1) * ops.tab_W * sizeof(T)) + 15) & ~(size_t)15;
    const size_t smem = tab_bytes + (size_t)Cfg::CAPS * (sizeof(VecT<T, KR>) + sizeof(int)) +
                        (size_t)KR * 3 * (Cfg::MAXSW + 2) * sizeof(V) + (size_t)2 * Cfg::CAPT * sizeof(int) +
                        (size_t)(3 * (Cfg::MAXSW + 3) + Cfg::MAXSW + 1) * sizeof(int);
    const void* fn = (const void*)p2p_strip_multi_kernel<T, KR>;
    {
        cudaError_t e = ensure_dynamic_smem(fn, smem);
        if (e != cudaSuccess) return e;
    }
    const int n = 1 << t.L;
    const int64_t strips = (int64_t)n * ((n + SW - 1) / SW);
    int64_t blocks = std::min<int64_t>(strips, (int64_t)num_sms * blocks_per_sm(fn, Cfg::WARPS * 32, smem));
    if (blocks < 1) blocks = 1;
    (void)launch_dependent(p2p_strip_multi_kernel<T, KR>, dim3((int)blocks), dim3(Cfg::WARPS * 32), smem, s,
        t.L, t.side, SW, nr, t.src_begin, t.src_loc, t.tgt_begin, t.tgt_loc, t.tgt_perm, f_sorted, f_stride,
        (const T*)ops.p2p_table, ops.tab_H, ops.tab_W, (const V*)Qleaf, q_stride, un, u_stride);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_p2p_multi(const TreeView& t, const DeviceOps& ops, int k, const T* f_sorted, int64_t f_stride,
                             const void* Qleaf, int64_t q_stride, double* un, int64_t u_stride, int num_sms,
                             cudaStream_t s) {
    using V = typename Mono<T>::V;
    constexpr int KR = 4;
    const int n = 1 << t.L;
    const int ms = std::max(1, t.max_leaf_src), mt = std::max(1, t.max_leaf_tgt);
    const int SW = std::min({StripMultiCfg<T, KR>::MAXSW, StripMultiCfg<T, KR>::CAPS / (3 * ms) - 2,
                             StripMultiCfg<T, KR>::CAPT / mt, n});
    for (int r0 = 0; r0 < k; r0 += KR) {
        const int nr = std::min(KR, k - r0);
        const T* f = f_sorted + (size_t)r0 * f_stride;
        const V* q = (const V*)Qleaf + (size_t)r0 * q_stride;
        double* u = un + (size_t)r0 * u_stride;
        cudaError_t e;
        if (SW >= 1)
            e = launch_p2p_multi_kr<T, KR>(t, ops, SW, nr, f, f_stride, q, q_stride, u, u_stride, num_sms, s);
        else  // leaves too full for the staging: one vector at a time through the leaf kernel
            for (int r = 0; r < nr; ++r)
                if ((e = launch_p2p_l2p<T>(t, ops, f + (size_t)r * f_stride, nullptr, nullptr, q + (size_t)r * q_stride,
                                           nullptr, u + (size_t)r * u_stride, nullptr, num_sms, s)) != cudaSuccess)
                    break;
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}


// ---- fused small levels (cooperative launches)
template <typename T>
static void fill_levels(LevelPtrs<T>& P, const DeviceOps& ops, int L, const LevelBufs& b) {
    using V = typename Mono<T>::V;
    std::memset(&P, 0, sizeof(P));
    for (int l = 0; l <= L && l < kMaxLevels; ++l) {
        P.q[l] = (T*)b.q[l];
        P.u[l] = (T*)b.u[l];
        P.Q[l] = (V*)b.Q[l];
        P.C[l] = (V*)b.C[l];
        const int k = L - l;
        if (l >= 2 && k >= 0 && k < (int)ops.tifo.size()) {
            P.tifo[l] = (const T*)ops.tifo[k];
            P.mono[l] = (const T*)ops.mono[k];
            if (k + 1 < (int)ops.l2l.size()) P.l2l[l] = (const T*)ops.l2l[k + 1];
            if (k >= 1) P.m2m[l] = (const T*)ops.m2m[k];
        }
    }
    P.nvec = b.nvec;
    P.vq = b.vq;
    P.vQ = b.vQ;
}

// Cooperative launch (all blocks co-resident, as the grid barrier needs) through the
// extensible launch API, whose cooperative attribute is also valid for kernels captured
// into a CUDA graph.
static cudaError_t launch_cooperative(const void* fn, int grid, int threads, size_t smem, void** args,
                                      cudaStream_t s) {
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
    return cudaLaunchKernelExC(&cfg, fn, args);
}

template <typename T>
cudaError_t launch_m2m_fused(const DeviceOps& ops, int L, const LevelBufs& b, unsigned* sync, int* status,
                             int num_sms, cudaStream_t s) {
    if (L < 3 || L >= kMaxLevels) return cudaErrorNotSupported;
    LevelPtrs<T> P;
    fill_levels<T>(P, ops, L, b);
    int l_top = L - 1, l_bot = 2;
    auto go = [&](const void* fn, size_t smem) -> cudaError_t {
        cudaError_t e = ensure_dynamic_smem(fn, smem);
        if (e != cudaSuccess) return e;
        // one block per SM: 8 warps per SM cover the largest level (one parent per warp
        // and pass), and every extra block costs each grid barrier an arrival
        const int grid = num_sms;
        void* args[] = {&P, &l_top, &l_bot, &sync, &status};
        e = launch_cooperative(fn, grid, 256, smem, args, s);
        return e == cudaSuccess ? cudaSuccess : clear_and_return(e);
    };
    if (ops.NP == 32) {
        constexpr size_t ob = (size_t)4 * 32 * 32 * sizeof(T);
        // binary32: the operator and one tile of staged children (m2m_tiles_f32)
        if constexpr (std::is_same<T, float>::value) return go((const void*)m2m_up_kernel<T, 32, true>, ob + kM2MTileSmem);
        else if constexpr (ob <= 64 * 1024) return go((const void*)m2m_up_kernel<T, 32, true>, ob);
        else return go((const void*)m2m_up_kernel<T, 32, false>, 0);
    }
    constexpr size_t ob = (size_t)4 * 64 * 64 * sizeof(T);
    if constexpr (ob <= 64 * 1024) return go((const void*)m2m_up_kernel<T, 64, true>, ob);
    else return go((const void*)m2m_up_kernel<T, 64, false>, 0);
}

// K chunks of the fused small-level M2L (up to 9, at least 3 K-steps each).  Binary32
// tiles are short, and only split when they are fewer than half the grid's blocks;
// binary64-width tiles are long enough that balancing the last round pays.  A count n
// costs rounds(n) / n (rounds of work units over the grid, each chunk doing 1/n of a
// tile's work) times 1.1 for the partial sums and their reduction, and replaces the best
// count so far only when it costs less than 0.9 times that count's cost: a split has to
// cut the rounds by about 18 % over one chunk.  The rule is kept as measured (float-float
// uniform_1m evaluation 4.45 -> 4.05 ms with it).
static int fused_split_chunks(int64_t items, int grid, bool wide, int split) {
    if (split > 0) return std::min(split, 9);  // chosen by the caller (opts.m2l_split)
    if (items <= 0 || grid <= 0) return 1;
    if (!wide) return 2 * items >= grid ? 1 : (int)std::min<int64_t>(9, std::max<int64_t>(2, grid / items));
    int best = 1;
    double best_cost = (double)((items + grid - 1) / grid);
    for (int n = 2; n <= 9; ++n) {
        const double cost = (double)((items * n + grid - 1) / grid) / n * 1.1;
        if (cost < best_cost * 0.9 && cost < best_cost) {
            best_cost = cost;
            best = n;
        }
    }
    return best;
}

template <typename T>
int64_t m2l_fused_split_bytes_shape(int NP, bool has_tc, int L, int tc_min_level, int num_sms, int nvec, int split) {
    int Ls = 1;
    for (int l = 2; l <= std::min(L, kM2LSplitKMaxLevel); ++l) {
        if (sizeof(T) == 4 && has_tc && l >= tc_min_level) break;  // m2l_uses_tc
        Ls = l;
    }
    if (Ls < 2 || L >= kMaxLevels) return 0;
    int64_t items = 0, stride = 0;
    for (int l = 2; l <= Ls; ++l) {
        items += 4 * ((((int64_t)1 << (2 * (l - 1))) + 31) / 32);
        stride += (int64_t)1 << (2 * l);
    }
    auto bytes = [&](auto np_tag) -> int64_t {
        constexpr int NPc = decltype(np_tag)::value;
        const void* fn = (const void*)m2l_small_kernel<T, NPc>;
        constexpr size_t smem = FusedCfg<T, NPc>::SMEM;
        if (ensure_dynamic_smem(fn, smem) != cudaSuccess) return 0;
        const int grid = num_sms * blocks_per_sm(fn, FusedCfg<T, NPc>::WARPS * 32, smem);
        const int nch = fused_split_chunks(items, grid, sizeof(T) == 8, split);
        return nch > 1 ? (int64_t)nvec * nch * stride * (NPc * (int64_t)sizeof(T) + 8) : 0;
    };
    return NP == 32 ? bytes(std::integral_constant<int, 32>()) : bytes(std::integral_constant<int, 64>());
}

template <typename T>
int64_t m2l_fused_split_bytes(const DeviceOps& ops, int L, int tc_min_level, int num_sms, int nvec, int split) {
    const bool has_tc = !ops.tc.empty() && ops.tc[0] != nullptr;  // all levels or none
    return m2l_fused_split_bytes_shape<T>(ops.NP, has_tc, L, tc_min_level, num_sms, nvec, split);
}

template <typename T>
cudaError_t launch_m2l_fused(const DeviceOps& ops, int L, const LevelBufs& b, int tc_min_level, unsigned* sync,
                             int* status, int num_sms, int* last_level, cudaStream_t s, int split) {
    *last_level = 1;
    // small levels: 2 .. Ls, the levels the per-level path sends to the split-K kernel
    int Ls = 1;
    for (int l = 2; l <= std::min(L, kM2LSplitKMaxLevel); ++l) {
        if (m2l_uses_tc(ops, L - l, l, tc_min_level, sizeof(T) == 4)) break;
        Ls = l;
    }
    if (Ls < 2 || L >= kMaxLevels) return cudaErrorNotSupported;
    LevelPtrs<T> P;
    fill_levels<T>(P, ops, L, b);
    int l0 = 2, l1 = Ls;
    P.item_off[0] = 0;
    for (int l = l0; l <= l1; ++l)
        P.item_off[l - l0 + 1] = P.item_off[l - l0] + 4 * ((((int64_t)1 << (2 * (l - 1))) + 31) / 32);
    auto go = [&](auto np_tag) -> cudaError_t {
        constexpr int NPc = decltype(np_tag)::value;
        const void* fn = (const void*)m2l_small_kernel<T, NPc>;
        constexpr size_t smem = FusedCfg<T, NPc>::SMEM;
        constexpr int threads = FusedCfg<T, NPc>::WARPS * 32;
        cudaError_t e = ensure_dynamic_smem(fn, smem);
        if (e != cudaSuccess) return e;
        const int grid = num_sms * blocks_per_sm(fn, threads, smem);
        // few tiles for the grid: split the 27 K-steps into chunks (partial sums)
        const int nch = fused_split_chunks(P.item_off[l1 - l0 + 1], grid, sizeof(T) == 8, split);
        P.nch = 1;
        if (nch > 1) {
            int64_t stride = 0;
            for (int l = l0; l <= l1; ++l) stride += (int64_t)1 << (2 * l);
            const int64_t need = (int64_t)P.nvec * nch * stride * (NPc * (int64_t)sizeof(T) + 8);
            if (!b.part || b.part_bytes < need) return cudaErrorInvalidValue;  // the caller sizes it
            P.part = (T*)b.part;
            P.nch = nch;
            P.part_stride = stride;
        }
        void* args[] = {&P, &l0, &l1, &sync, &status};
        e = launch_cooperative(fn, grid, threads, smem, args, s);
        return e == cudaSuccess ? cudaSuccess : clear_and_return(e);
    };
    cudaError_t e = ops.NP == 32 ? go(std::integral_constant<int, 32>()) : go(std::integral_constant<int, 64>());
    if (e == cudaSuccess) *last_level = Ls;
    return e;
}

template <typename T>
cudaError_t launch_l2p(const TreeView& t, const DeviceOps& ops, const T* uhat_leaf, const void* Cleaf, double* uf,
                       cudaStream_t s, int nvec, int64_t vq, int64_t vQ) {
    using V = typename Mono<T>::V;
    if (!t.tgt_leaf) return cudaErrorInvalidValue;
    const size_t table = (size_t)t.side * t.side * (ops.NP + 1) * sizeof(T);
    const bool in_smem = table <= 96 * 1024;
    const size_t smem = in_smem ? table : 0;
    auto go = [&](auto np_tag, auto smem_tag) -> cudaError_t {
        constexpr int NPc = decltype(np_tag)::value;
        constexpr bool SM = decltype(smem_tag)::value;
        const void* fn = (const void*)l2p_kernel<T, NPc, SM>;
        cudaError_t e = ensure_dynamic_smem(fn, smem);
        if (e != cudaSuccess) return e;
        // persistent: each block stages the table once
        int64_t blocks = (t.n_tgt * nvec + 255) / 256;
        const int64_t cap = (int64_t)152 * blocks_per_sm(fn, 256, smem);
        if (blocks > cap) blocks = cap;
        if (blocks < 1) blocks = 1;
        return launch_dependent(l2p_kernel<T, NPc, SM>, dim3((unsigned)blocks), dim3(256), smem, s, t.n_tgt, t.side,
                                t.tgt_leaf, t.tgt_loc, t.tgt_perm, uhat_leaf, (const V*)Cleaf, (const T*)ops.tofsT,
                                uf, nvec, vq, vQ);
    };
    using I32 = std::integral_constant<int, 32>;
    using I64 = std::integral_constant<int, 64>;
    using BT = std::true_type;
    using BF = std::false_type;
    if (ops.NP == 32) return in_smem ? go(I32(), BT()) : go(I32(), BF());
    return in_smem ? go(I64(), BT()) : go(I64(), BF());
}

cudaError_t launch_combine(int64_t n, const double* un, const double* uf, double* u, double* u_near, double* u_far,
                           cudaStream_t s) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    return launch_dependent(combine_kernel, dim3((unsigned)blocks), dim3(256), 0, s, n, un, uf, u, u_near, u_far);
}

#define LFMM_INSTANTIATE(T)                                                                                   \
    template cudaError_t launch_m2m_fused<T>(const DeviceOps&, int, const LevelBufs&, unsigned*, int*, int,      \
                                             cudaStream_t);                                                  \
    template int64_t m2l_fused_split_bytes<T>(const DeviceOps&, int, int, int, int, int);                     \
    template int64_t m2l_fused_split_bytes_shape<T>(int, bool, int, int, int, int, int);                     \
    template cudaError_t launch_m2l_fused<T>(const DeviceOps&, int, const LevelBufs&, int, unsigned*, int*, int, \
                                             int*, cudaStream_t, int);                                       \
    template cudaError_t launch_l2p<T>(const TreeView&, const DeviceOps&, const T*, const void*, double*,          \
                                       cudaStream_t, int, int64_t, int64_t);                                  \
    template cudaError_t launch_p2m<T>(const TreeView&, const DeviceOps&, const double*, T*, T*, void*,       \
                                       cudaStream_t, int, int64_t, int64_t);                                  \
    template cudaError_t launch_m2m<T>(const DeviceOps&, int, int, const T*, const void*, T*, void*,         \
                                       cudaStream_t);                                                         \
    template cudaError_t launch_m2l<T>(const DeviceOps&, int, int, const T*, const void*, const T*,          \
                                       const void*, T*, void*, cudaStream_t);                                \
    template cudaError_t launch_p2p_multi<T>(const TreeView&, const DeviceOps&, int, const T*, int64_t, const void*, \
                                             int64_t, double*, int64_t, int, cudaStream_t);                     \
    template cudaError_t launch_p2p_l2p<T>(const TreeView&, const DeviceOps&, const T*, const T*, const void*, \
                                           const void*, double*, double*, double*, int, cudaStream_t);

LFMM_INSTANTIATE(float)
LFMM_INSTANTIATE(double)
LFMM_INSTANTIATE(DF)

}  // namespace lfmm
