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
// [4^l][NP].  phi near the origin comes from a shared-memory table, so every
// near-field pair costs one table load and one FMA (Sec. 2: "a table look-up").
#include <cstdio>

#include "lfmm_internal.h"

namespace lfmm {

namespace {

constexpr unsigned kFull = 0xffffffffu;

template <typename T>
__device__ __forceinline__ T shfl(T v, int src) {
    return __shfl_sync(kFull, v, src);
}

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
            v[i] = keep + __shfl_xor_sync(kFull, send, off);
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

// ------------------------------------------------------------------------- P2M
template <typename T, int NP>
__global__ void __launch_bounds__(256) p2m_kernel(int64_t n_leaves, const int32_t* __restrict__ begin,
                                                  const int32_t* __restrict__ loc,
                                                  const int32_t* __restrict__ perm,
                                                  const double* __restrict__ f,
                                                  T* __restrict__ f_sorted,
                                                  const T* __restrict__ tofsT, int side,
                                                  T* __restrict__ qhat) {
    constexpr int PL = NP / 32;
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t leaf = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; leaf < n_leaves;
         leaf += nw) {
        const int b = begin[leaf], e = begin[leaf + 1];
        T acc[PL];
#pragma unroll
        for (int i = 0; i < PL; ++i) acc[i] = T(0);
        for (int j0 = b; j0 < e; j0 += 32) {
            const int j = j0 + lane;
            T fj = T(0);
            int J = 0;
            if (j < e) {
                const int l = loc[j];
                J = (l & 0xffff) + side * (l >> 16);
                fj = (T)f[perm[j]];
                f_sorted[j] = fj;
            }
            const int cnt = min(32, e - j0);
            for (int k = 0; k < cnt; ++k) {
                const T fk = shfl(fj, k);
                const T* row = tofsT + (size_t)shfl(J, k) * NP;
#pragma unroll
                for (int i = 0; i < PL; ++i) acc[i] = fma(__ldg(row + lane + 32 * i), fk, acc[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < PL; ++i) qhat[(size_t)leaf * NP + lane + 32 * i] = acc[i];
    }
}

// ------------------------------------------------------------------------- M2M
template <typename T, int NP>
__global__ void __launch_bounds__(256) m2m_kernel(int64_t n_parent, const T* __restrict__ qc,
                                                  const T* __restrict__ m2m, T* __restrict__ qp) {
    constexpr int CL = 4 * NP / 32, PL = NP / 32;
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t par = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; par < n_parent;
         par += nw) {
        T x[CL];
#pragma unroll
        for (int c = 0; c < CL; ++c) x[c] = qc[(size_t)par * 4 * NP + lane + 32 * c];
        T acc[PL];
#pragma unroll
        for (int i = 0; i < PL; ++i) acc[i] = T(0);
#pragma unroll
        for (int c = 0; c < CL; ++c) {
#pragma unroll 8
            for (int l = 0; l < 32; ++l) {
                const T v = shfl(x[c], l);
                const T* row = m2m + (size_t)(32 * c + l) * NP;
#pragma unroll
                for (int i = 0; i < PL; ++i) acc[i] = fma(__ldg(row + lane + 32 * i), v, acc[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < PL; ++i) qp[(size_t)par * NP + lane + 32 * i] = acc[i];
    }
}

// ------------------------------------------------------------------------- M2L (+L2L)
// One block: BB target boxes of one parity class c = (px, py) (boxes (2i+px, 2j+py)),
// all NP outputs.  K loop: the class's 27 interaction offsets (Def. 6.1), then the
// parent's incoming expansion through T_ifi (level >= 3).  Per step the gathered
// source rows (A, [BB][AS]) and the operator (B, [NP][NP], k-major) are staged in
// shared memory with cp.async, double buffered.  Lane tile: MB boxes x MP outputs.
template <typename T, int NP>
struct M2LCfg {
    static constexpr int MB = 4, MP = 8;
    static constexpr int NPG = NP / MP;           // lanes along outputs
    static constexpr int NBG = 32 / NPG;          // lanes along boxes
    static constexpr int WB = MB * NBG;           // boxes per warp
    static constexpr int WARPS = 4;
    static constexpr int BB = WB * WARPS;         // boxes per block
    static constexpr int AS = NP + 16 / (int)sizeof(T);  // A row stride (elements)
    static constexpr int A_ELEMS = BB * AS;
    static constexpr int B_ELEMS = NP * NP;
    static constexpr int STAGE = A_ELEMS + B_ELEMS;
    static constexpr size_t SMEM = 2 * (size_t)STAGE * sizeof(T);
};

template <typename T, int NP>
__global__ void __launch_bounds__(128) m2l_kernel(int level, const T* __restrict__ q,
                                                  const T* __restrict__ u_par,
                                                  const T* __restrict__ tifo,
                                                  const T* __restrict__ l2l,
                                                  T* __restrict__ u) {
    using C = M2LCfg<T, NP>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* smem = reinterpret_cast<T*>(smem_raw);
    const int cls = blockIdx.y;
    const int px = cls & 1, py = cls >> 1;
    const int np_side = 1 << (level - 1);          // parents per axis
    const int64_t n_par = (int64_t)np_side * np_side;
    const int64_t tile0 = (int64_t)blockIdx.x * C::BB;
    const int side = 1 << level;
    const bool has_l2l = (u_par != nullptr);

    // the class's offsets: ox in [-2-px, 3-px], oy in [-2-py, 3-py], not in [-1,1]^2
    const int n_steps = 27 + (has_l2l ? 1 : 0);

    auto stage = [&](int step, int buf) {
        T* As = smem + (size_t)buf * C::STAGE;
        T* Bs = As + C::A_ELEMS;
        const T* op;
        int ox = 0, oy = 0;
        bool l2l_step = step >= 27;
        if (!l2l_step) {
            int cnt = 0, o_idx = 0;
            // enumerate the 6x6 block minus the 3x3 core, row-major
            for (int d = 0; d < 36; ++d) {
                const int dx = (d % 6) - 2 - px, dy = (d / 6) - 2 - py;
                if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
                if (cnt == step) {
                    ox = dx;
                    oy = dy;
                    break;
                }
                ++cnt;
            }
            // index among the 40 offsets: row-major over [-3,3]^2 minus the core
            {
                int idx = 0;
                for (int yy = -3; yy <= 3; ++yy)
                    for (int xx = -3; xx <= 3; ++xx) {
                        if (xx >= -1 && xx <= 1 && yy >= -1 && yy <= 1) continue;
                        if (xx == ox && yy == oy) o_idx = idx;
                        ++idx;
                    }
            }
            op = tifo + (size_t)o_idx * NP * NP;
        } else {
            op = l2l + (size_t)cls * NP * NP;
        }
        // B: NP*NP elements, contiguous
        constexpr int B_CHUNKS = C::B_ELEMS * (int)sizeof(T) / 16;
        for (int c = threadIdx.x; c < B_CHUNKS; c += blockDim.x)
            cp_async16(reinterpret_cast<char*>(Bs) + 16 * c,
                       reinterpret_cast<const char*>(op) + 16 * c, 16);
        // A: BB rows of NP elements, gathered
        constexpr int ROW_CHUNKS = NP * (int)sizeof(T) / 16;
        for (int c = threadIdx.x; c < C::BB * ROW_CHUNKS; c += blockDim.x) {
            const int r = c / ROW_CHUNKS, ch = c % ROW_CHUNKS;
            const int64_t pi = tile0 + r;
            const T* src = q;
            int bytes = 0;
            if (pi < n_par) {
                const int i = (int)(pi % np_side), j = (int)(pi / np_side);
                if (!l2l_step) {
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

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bg = lane % C::NBG, pg = lane / C::NBG;
    const int wbox = warp * C::WB;
    T acc[C::MB][C::MP];
#pragma unroll
    for (int i = 0; i < C::MB; ++i)
#pragma unroll
        for (int j = 0; j < C::MP; ++j) acc[i][j] = T(0);

    stage(0, 0);
    cp_async_commit();
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
        const int64_t pi = tile0 + wbox + bg + C::NBG * i;
        if (pi >= n_par) continue;
        const int ii = (int)(pi % np_side), jj = (int)(pi / np_side);
        T* dst = u + (size_t)morton2(2 * ii + px, 2 * jj + py) * NP + pg * C::MP;
#pragma unroll
        for (int j = 0; j < C::MP; ++j) dst[j] = acc[i][j];
    }
}

// ------------------------------------------------------------------------- P2P + L2P
// One warp per target leaf.  The sources of the leaf and its (up to) 8 neighbours are
// staged in shared memory as (table offset, charge); lanes take sources, loop over up
// to 32 targets held as table offsets, and a reduce-scatter leaves target t's sum in
// lane t.  The table holds phi(dx, dy) for |dx|, |dy| <= 2s-1 at row width W, so
// idx(target) - idx(source) addresses phi(target - source) directly.
constexpr int kP2PWarps = 8;
constexpr int kP2PCap = 9 * 64;  // staged sources per warp per chunk

template <typename T, int NP>
__global__ void __launch_bounds__(kP2PWarps * 32) p2p_l2p_kernel(
    int L, int side, int64_t n_leaves, const int32_t* __restrict__ sbeg,
    const int32_t* __restrict__ sloc, const int32_t* __restrict__ tbeg,
    const int32_t* __restrict__ tloc, const int32_t* __restrict__ tperm,
    const T* __restrict__ f_sorted, const T* __restrict__ table, int tab_H, int tab_W,
    const T* __restrict__ uhat, const T* __restrict__ tofsT, double* __restrict__ u,
    double* __restrict__ u_near, double* __restrict__ u_far) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tab_n = (2 * tab_H + 1) * tab_W;
    T* tab = reinterpret_cast<T*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* s_off = reinterpret_cast<int*>(tab + tab_n) + warp * kP2PCap;
    T* s_f = reinterpret_cast<T*>(reinterpret_cast<int*>(tab + tab_n) + kP2PWarps * kP2PCap) +
             warp * kP2PCap;
    for (int i = threadIdx.x; i < tab_n; i += blockDim.x) tab[i] = table[i];
    __syncthreads();
    const char* tab_c = reinterpret_cast<const char*>(tab) +
                        (size_t)(tab_H + tab_H * tab_W) * sizeof(T);  // centre
    const int nside = 1 << L;
    const int64_t nwarps = (int64_t)gridDim.x * kP2PWarps;
    constexpr int PL = NP / 32;

    for (int64_t leaf = (int64_t)blockIdx.x * kP2PWarps + warp; leaf < n_leaves; leaf += nwarps) {
        const int tb = tbeg[leaf], te = tbeg[leaf + 1];
        if (tb == te) continue;
        uint32_t bx, by;
        unmorton2((uint32_t)leaf, bx, by);
        // neighbour ranges
        int rb[9], rc[9], rbase[9];
        int ns = 0;
#pragma unroll
        for (int d = 0; d < 9; ++d) {
            const int dx = d % 3 - 1, dy = d / 3 - 1;
            const int nx = (int)bx + dx, ny = (int)by + dy;
            rb[d] = 0;
            rc[d] = 0;
            rbase[d] = dx * side + tab_W * (dy * side);
            if (nx >= 0 && nx < nside && ny >= 0 && ny < nside) {
                const uint32_t m = morton2(nx, ny);
                rb[d] = sbeg[m];
                rc[d] = sbeg[m + 1] - rb[d];
            }
            ns += rc[d];
        }
        T uh[PL];
#pragma unroll
        for (int i = 0; i < PL; ++i) uh[i] = uhat ? uhat[(size_t)leaf * NP + lane + 32 * i] : T(0);
        const int n_chunks = (ns + kP2PCap - 1) / kP2PCap;

        auto fill = [&](int c0) {
            const int cn = min(kP2PCap, ns - c0);
            for (int v = lane; v < cn; v += 32) {
                int g = c0 + v, d = 0;
                while (g >= rc[d]) {
                    g -= rc[d];
                    ++d;
                }
                const int j = rb[d] + g;
                const int l = sloc[j];
                s_off[v] = rbase[d] + (l & 0xffff) + tab_W * (l >> 16);
                s_f[v] = f_sorted[j];
            }
            __syncwarp();
            return cn;
        };

        int cn = n_chunks == 1 ? fill(0) : 0;
        for (int t0 = tb; t0 < te; t0 += 32) {
            const int nt = min(32, te - t0);
            int my_toff = 0, my_J = 0;
            if (lane < nt) {
                const int l = tloc[t0 + lane];
                const int tx = l & 0xffff, ty = l >> 16;
                my_toff = tx + tab_W * ty;
                my_J = tx + side * ty;
            }
            int toff[32];
#pragma unroll
            for (int t = 0; t < 32; ++t) toff[t] = shfl(my_toff, t) * (int)sizeof(T);
            T acc[32];
#pragma unroll
            for (int t = 0; t < 32; ++t) acc[t] = T(0);
            for (int ch = 0; ch < n_chunks; ++ch) {
                if (n_chunks > 1) {
                    __syncwarp();
                    cn = fill(ch * kP2PCap);
                }
                for (int r = 0; r < cn; r += 32) {
                    const int v = r + lane;
                    const int so = v < cn ? s_off[v] : s_off[0];
                    const T fj = v < cn ? s_f[v] : T(0);
                    const char* tb_c = tab_c - (ptrdiff_t)so * (ptrdiff_t)sizeof(T);
#pragma unroll
                    for (int tc = 0; tc < 4; ++tc) {
                        if (tc * 8 < nt) {
#pragma unroll
                            for (int q = 0; q < 8; ++q)
                                acc[tc * 8 + q] =
                                    fma(*reinterpret_cast<const T*>(tb_c + toff[tc * 8 + q]), fj,
                                        acc[tc * 8 + q]);
                        }
                    }
                }
            }
            const T near = reduce_scatter32(acc);
            // L2P: u_far(t) = sum_p T_ofs[p][J_t] u_hat[p]
            T far = T(0);
            if (uhat) {
#pragma unroll
                for (int t = 0; t < 32; ++t) acc[t] = T(0);
#pragma unroll
                for (int tc = 0; tc < 4; ++tc) {
                    if (tc * 8 < nt) {
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const T* row = tofsT + (size_t)shfl(my_J, tc * 8 + q) * NP;
                            T s = T(0);
#pragma unroll
                            for (int i = 0; i < PL; ++i) s = fma(__ldg(row + lane + 32 * i), uh[i], s);
                            acc[tc * 8 + q] = s;
                        }
                    }
                }
                far = reduce_scatter32(acc);
            }
            if (lane < nt) {
                const int dst = tperm[t0 + lane];
                const double dn = (double)near, df = (double)far;
                if (u) u[dst] = dn + df;
                if (u_near) u_near[dst] = dn;
                if (u_far) u_far[dst] = df;
            }
        }
        __syncwarp();
    }
}

}  // namespace

// ------------------------------------------------------------------------- launchers
template <typename T>
cudaError_t launch_p2m(const TreeView& t, const DeviceOps& ops, const double* f, T* f_sorted,
                       T* qhat_leaf, cudaStream_t s) {
    const int threads = 256;
    int64_t blocks = (t.n_leaves * 32 + threads - 1) / threads;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) blocks = 1;
    if (ops.NP == 32)
        p2m_kernel<T, 32><<<(int)blocks, threads, 0, s>>>(t.n_leaves, t.src_begin, t.src_loc, t.src_perm, f,
                                                          f_sorted, (const T*)ops.tofsT, t.side, qhat_leaf);
    else
        p2m_kernel<T, 64><<<(int)blocks, threads, 0, s>>>(t.n_leaves, t.src_begin, t.src_loc, t.src_perm, f,
                                                          f_sorted, (const T*)ops.tofsT, t.side, qhat_leaf);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_m2m(const DeviceOps& ops, int k, const T* q_child, T* q_parent, int64_t n_parent,
                       cudaStream_t s) {
    const int threads = 256;
    int64_t blocks = (n_parent * 32 + threads - 1) / threads;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) blocks = 1;
    if (ops.NP == 32)
        m2m_kernel<T, 32><<<(int)blocks, threads, 0, s>>>(n_parent, q_child, (const T*)ops.m2m[k], q_parent);
    else
        m2m_kernel<T, 64><<<(int)blocks, threads, 0, s>>>(n_parent, q_child, (const T*)ops.m2m[k], q_parent);
    return cudaGetLastError();
}

template <typename T, int NP>
static cudaError_t launch_m2l_np(const DeviceOps& ops, int k, int level, const T* q, const T* u_par,
                                 T* u, cudaStream_t s) {
    using C = M2LCfg<T, NP>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(m2l_kernel<T, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)C::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int64_t n_par = (int64_t)1 << (2 * (level - 1));
    dim3 grid((unsigned)((n_par + C::BB - 1) / C::BB), 4);
    m2l_kernel<T, NP><<<grid, 128, C::SMEM, s>>>(level, q, u_par, (const T*)ops.tifo[k],
                                                 u_par ? (const T*)ops.l2l[k + 1] : nullptr, u);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_m2l(const DeviceOps& ops, int k, int level, const T* q_level, const T* u_parent,
                       T* u_level, cudaStream_t s) {
    if (ops.NP == 32) return launch_m2l_np<T, 32>(ops, k, level, q_level, u_parent, u_level, s);
    return launch_m2l_np<T, 64>(ops, k, level, q_level, u_parent, u_level, s);
}

template <typename T, int NP>
static cudaError_t launch_p2p_np(const TreeView& t, const DeviceOps& ops, const T* f_sorted,
                                 const T* uhat, double* u, double* un, double* uf, int num_sms,
                                 cudaStream_t s) {
    const size_t tab_bytes = (size_t)(2 * ops.tab_H + 1) * ops.tab_W * sizeof(T);
    const size_t smem = ((tab_bytes + 15) & ~(size_t)15) +
                        (size_t)kP2PWarps * kP2PCap * (sizeof(int) + sizeof(T));
    static size_t attr_bytes = 0;
    if (smem > attr_bytes) {
        cudaError_t e = cudaFuncSetAttribute(p2p_l2p_kernel<T, NP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_bytes = smem;
    }
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, p2p_l2p_kernel<T, NP>, kP2PWarps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (t.n_leaves + kP2PWarps - 1) / kP2PWarps;
    const int64_t cap = (int64_t)num_sms * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    p2p_l2p_kernel<T, NP><<<(int)blocks, kP2PWarps * 32, smem, s>>>(
        t.L, t.side, t.n_leaves, t.src_begin, t.src_loc, t.tgt_begin, t.tgt_loc, t.tgt_perm, f_sorted,
        (const T*)ops.p2p_table, ops.tab_H, ops.tab_W, uhat, (const T*)ops.tofsT, u, un, uf);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_p2p_l2p(const TreeView& t, const DeviceOps& ops, const T* f_sorted, const T* uhat,
                           double* u, double* un, double* uf, int num_sms, cudaStream_t s) {
    if (ops.NP == 32) return launch_p2p_np<T, 32>(t, ops, f_sorted, uhat, u, un, uf, num_sms, s);
    return launch_p2p_np<T, 64>(t, ops, f_sorted, uhat, u, un, uf, num_sms, s);
}

#define LFMM_INSTANTIATE(T)                                                                         \
    template cudaError_t launch_p2m<T>(const TreeView&, const DeviceOps&, const double*, T*, T*,    \
                                       cudaStream_t);                                               \
    template cudaError_t launch_m2m<T>(const DeviceOps&, int, const T*, T*, int64_t, cudaStream_t); \
    template cudaError_t launch_m2l<T>(const DeviceOps&, int, int, const T*, const T*, T*,          \
                                       cudaStream_t);                                               \
    template cudaError_t launch_p2p_l2p<T>(const TreeView&, const DeviceOps&, const T*, const T*,   \
                                           double*, double*, double*, int, cudaStream_t);

LFMM_INSTANTIATE(float)
LFMM_INSTANTIATE(double)

}  // namespace lfmm
