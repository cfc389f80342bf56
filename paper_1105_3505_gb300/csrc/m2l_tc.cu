// M2L (+ fused L2L) on the 5th-generation tensor cores, mixed path (Sec. 7, Sec. 8.2
// steps 3-4): for the boxes tau of one parity class,
//
//   u_hat^tau = sum_{sigma in int(tau)} (T_ifo^o - c_o 1 1^T) q_hat^sigma + T_ifi^c u_hat^parent
//
// as an implicit GEMM per CTA: M = 128 target boxes (TMEM lanes), N = 32 outputs,
// K = 27 x 32 source expansions (+ 32 for the parent).  Operands are split into TF32
// hi + lo parts (round to nearest) and three products hi*hi + hi*lo + lo*hi are formed
// (the lo*lo term is below 2^-22 relative).  The tensor core's fp32 accumulation rounds
// toward zero, and that bias grows linearly with the number of MMAs feeding one
// accumulator; so every K-step writes fresh TMEM accumulators (hi*hi in one, the small
// hi*lo + lo*hi terms in another), which are read back after the step and added in
// registers with round-to-nearest fp32.
//
// A (source expansions) arrives by tiled TMA loads from parity-plane layouts of the
// split expansions, B (operators) as pre-split, pre-swizzled 4 KB tiles of the device
// image by bulk copies; both land in the 128-byte-swizzled K-major layout that the
// shared-memory matrix descriptors describe.  The pipeline is described at the kernel.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "lfmm_internal.h"

namespace lfmm {

namespace {

constexpr long long kWaitBudget = 4000000000ll;  // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_n(uint64_t* bar, uint32_t n) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(n) : "memory");
}
// one arrival on `bar` once every cp.async this thread issued before has landed (the
// arrival counts against the barrier's expected count)
__device__ __forceinline__ void cp_async_mbar_arrive_noinc(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// non-blocking probe of a phase; the pipeline's role threads poll with it (a suspended
// try_wait can sleep past the phase change, and every K-step waits three times)
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded by kWaitBudget clock cycles and, for the pipeline's waits, by the plan's poll
// budget (max_polls); the teardown's waits for work already issued keep the clock bound
// only, so that no copy or product is in flight when the CTA frees its memory.
__device__ __forceinline__ bool mbar_poll_bounded(uint64_t* bar, uint32_t parity, uint32_t max_polls = 0xffffffffu) {
    if (mbar_test(bar, parity)) return true;
    const long long t0 = clock64();
    uint32_t n = 0;
    while (!mbar_test(bar, parity))
        if (clock64() - t0 > kWaitBudget || ++n > max_polls) return false;
    return true;
}
__device__ __forceinline__ void bulk_g2s_u32(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
          "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// D[tmem] (+)= A[smem descriptor] x B[smem descriptor], kind::tf32, cta_group::1
__device__ __forceinline__ void mma_tf32_ss(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
    d |= (uint64_t)0 << 16;                          // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                          // descriptor version
    d |= (uint64_t)2 << 61;                          // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::tf32: fp32 accumulate, A and B tf32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t tf32_rna_bits(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ int offset_index_tc(int ox, int oy) {
    const int raw = (oy + 3) * 7 + (ox + 3);
    int inner_before;
    if (oy < -1) inner_before = 0;
    else if (oy > 1) inner_before = 9;
    else inner_before = 3 * (oy + 1) + (ox > 1 ? 3 : 0);
    return raw - inner_before;
}

struct DFv {
    float hi, lo;
};
__device__ __forceinline__ DFv tsum(float a, float b) {
    const float s = a + b, bp = s - a, ap = s - bp;
    return {s, (a - ap) + (b - bp)};
}
__device__ __forceinline__ DFv qsum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ DFv dadd(DFv a, DFv b) {
    DFv s = tsum(a.hi, b.hi), t = tsum(a.lo, b.lo);
    s.lo += t.hi;
    s = qsum(s.hi, s.lo);
    s.lo += t.lo;
    return qsum(s.hi, s.lo);
}
__device__ __forceinline__ DFv dmul(DFv a, DFv b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    return qsum(p, e);
}

// ---------------------------------------------------------------------------------
// TMA form.  The level's expansions are split into TF32 hi / lo once and stored by
// parity plane, Q5[hl][py'][px'][y'][x'][NP] with box (x, y) = (2x' + px', 2y' + py'):
// for a target tile of one parity class, the sources at one interaction offset are then
// a rectangle of one plane, so a single tiled TMA load (5-D tensor map, 128-byte
// swizzle, zero fill outside the level) writes the A operand of a K-block directly in
// the layout the tensor core reads.  The parent level's incoming expansions are stored
// row-major (4-D map) and their window is the tile itself.
//
// A K-block is 32 expansion coefficients (one 128-byte swizzled row per box): NP = 32
// takes one K-block per interaction offset, NP = 64 two, accumulated into the same
// fresh accumulator of that offset.
//
// Persistent CTAs (one per SM) walk the tiles with a continuous pipeline:
//   warp 4 (one thread): producer - for every K-block of every offset of every tile,
//     wait until the stage is free, then two TMA loads (A hi, A lo) and one bulk copy
//     (B hi + lo) completing on the stage's "full" mbarrier;
//   warp 5 (one thread): MMA issuer - wait "full" (and, at an offset's first K-block,
//     until the accumulator buffer is folded), issue the block's 8 MMAs, commit to the
//     stage's "empty" barrier (frees the shared memory) and, at the offset's last
//     K-block, to the buffer's "acc_full" barrier;
//   warps 0-3: one target box per thread (TMEM lane) - fold every offset's fresh
//     accumulators into round-to-nearest fp32 registers, arrive on "acc_empty"; at a
//     tile's last offset write the row of u_hat;
//   warp 6: the compensated incoming constant of every box of the CTA's tiles (plain
//     loads and float-pair arithmetic, independent of the pipeline).
// Every wait is bounded; on expiry the CTA records LFMM_ETIMEOUT, every role stops at
// its next iteration, and the teardown waits (bounded) for the copies and MMAs issued.
constexpr int kTmaStagesDefault = 3;  // ring depth unless opts.m2l_stages says otherwise
constexpr int kTmaAcc = 4;
constexpr int kTmaThreads = 224;
constexpr uint32_t kTmaABytes = 128 * 32 * 4;  // one A K-block (hi or lo): 128 rows x 128 B

template <int NP>
struct TmaCfg {
    static constexpr int KB = NP / 32;                          // K-blocks per interaction offset
    static constexpr uint32_t BBytes = 2u * NP * 128u;          // B K-block: [B_hi | B_lo], 2 NP rows x 128 B
    static constexpr uint32_t StageBytes = 2 * kTmaABytes + BBytes;
    static constexpr int AccCols = 2 * NP;                      // buffer: D_big [0, 2NP), D_small [NP, 2NP)
    static constexpr int Cols = kTmaAcc * AccCols;              // TMEM columns (256 or 512)
};

struct TmaGeo {
    int level;            // tree level of the targets
    int lg;               // log2 of np, the side of a parity class (2^(level-1))
    int TX, TY;           // target tile: TX x TY boxes of one class, TX * TY <= 128
    int tiles_x;          // tiles per class row
    int tiles_per_class;
    int n_tiles;          // 4 classes x tiles_per_class
    int has_l2l;
    int nvec;             // charge vectors: vector v's expansions at v vq floats, charges /
    long long vq, vQ;     // constants at v vQ pairs; its split layouts at TMA index 2v + hl
};

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            int c4, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5, %6}], [%7];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

template <int NP, int kTmaStages>
__global__ void __launch_bounds__(kTmaThreads, 1) m2l_tma_kernel(
    const __grid_constant__ CUtensorMap tm_q, const __grid_constant__ CUtensorMap tm_u, const TmaGeo g,
    const float* __restrict__ tiles, const float* __restrict__ mono, const DFv* __restrict__ Qin,
    const DFv* __restrict__ Cpar, float* __restrict__ out, DFv* __restrict__ Cout, int* __restrict__ status) {
    griddep_wait();
    using Cfg = TmaCfg<NP>;
    constexpr int KB = Cfg::KB;
    constexpr uint32_t kStageBytes = Cfg::StageBytes;
    extern __shared__ __align__(1024) unsigned char tma_smem[];
    // stage i: A hi, A lo (128 rows x 128 B each, 128-byte swizzled), B hi + lo (2 NP rows x 128 B)
    const uint32_t base = smem_u32(tma_smem) + ((1024u - (smem_u32(tma_smem) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t full[kTmaStages], empty[kTmaStages], acc_full[kTmaAcc], acc_empty[kTmaAcc];
    __shared__ uint32_t s_tmem;
    __shared__ int s_off[4][27][3];
    __shared__ int s_abort;
    __shared__ int s_issued[2];  // K-blocks issued by the producer and by the MMA thread

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_steps = 27 + g.has_l2l;  // interaction offsets (+ the parent) per tile
    const int np = 1 << g.lg, side = 2 << g.lg;
    const int rows = g.TX * g.TY;
    const uint32_t tx_bytes = 2u * (uint32_t)rows * 128u + Cfg::BBytes;
    const int all_tiles = g.n_tiles * g.nvec;
    const int my_tiles = blockIdx.x < (unsigned)all_tiles ? (all_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int total = my_tiles * n_steps * KB;  // K-blocks of this CTA
    volatile int* vabort = &s_abort;
    // the plan's wait budget in polls (status[3], 0: the clock bound alone)
    const uint32_t wb = ((volatile int*)status)[3] > 0 ? (uint32_t)((volatile int*)status)[3] : 0xffffffffu;

    if (threadIdx.x == 0) {
        for (int c = 0; c < 4; ++c) {
            const int px = c & 1, py = c >> 1;
            int nn = 0;
            for (int d = 0; d < 36; ++d) {
                const int dx = (d % 6) - 2 - px, dy = (d / 6) - 2 - py;
                if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
                s_off[c][nn][0] = dx;
                s_off[c][nn][1] = dy;
                s_off[c][nn][2] = offset_index_tc(dx, dy);
                ++nn;
            }
        }
        for (int i = 0; i < kTmaStages; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < kTmaAcc; ++i) {
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], 4);
        }
        fence_barrier_init();
        s_abort = 0;
        s_issued[0] = s_issued[1] = 0;
    }
    if (warp == 0) {
        tmem_alloc(&s_tmem, Cfg::Cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    auto abort_now = [&]() {
        atomicExch(&s_abort, 1);
        atomicExch(status, LFMM_ETIMEOUT);
    };
    // it-th tile of this CTA: t = blockIdx.x + it * gridDim.x; charge vector t / n_tiles,
    // then class (t mod n_tiles) & 3 (classes interleave for balance) and row-major tiles
    // of the class
    auto tile_of = [&](int it, int& cls, int& ri0, int& rj0, int& v) {
        const int t = (int)blockIdx.x + it * (int)gridDim.x;
        v = t / g.n_tiles;
        const int tt = t - v * g.n_tiles;
        cls = tt & 3;
        const int k = tt >> 2;
        ri0 = (k % g.tiles_x) * g.TX;
        rj0 = (k / g.tiles_x) * g.TY;
    };
    // The roles walk the same sequence of K-blocks gs = (it * n_steps + st) * KB + h with
    // running counters: stage slot gs % kTmaStages and its use count; the accumulator
    // buffer advances once per offset (every KB blocks).

    if (warp == 4) {
        if (lane == 0) {
            int it = 0, st = 0, h = 0, slot = 0, use = 0;
            int cls = 0, ri0 = 0, rj0 = 0, v = 0;
            tile_of(0, cls, ri0, rj0, v);
            for (int gs = 0; gs < total; ++gs) {
                if (*vabort) break;
                if (use > 0 && !mbar_poll_bounded(&empty[slot], (uint32_t)((use - 1) & 1), wb)) {
                    abort_now();
                    break;
                }
                const uint32_t sa = base + (uint32_t)slot * kStageBytes;
                mbar_arrive_expect_tx(&full[slot], tx_bytes);
                const int c0 = 32 * h;
                if (st < 27) {
                    const int sx = (cls & 1) + s_off[cls][st][0], sy = (cls >> 1) + s_off[cls][st][1];
                    const int plane = (sx & 1) + 2 * (sy & 1);
                    tma_load_5d(sa, &tm_q, c0, ri0 + (sx >> 1), rj0 + (sy >> 1), plane, 2 * v, &full[slot]);
                    tma_load_5d(sa + kTmaABytes, &tm_q, c0, ri0 + (sx >> 1), rj0 + (sy >> 1), plane, 2 * v + 1,
                                &full[slot]);
                    bulk_g2s_u32(sa + 2 * kTmaABytes, tiles + ((size_t)s_off[cls][st][2] * KB + h) * (Cfg::BBytes / 4),
                                 Cfg::BBytes, &full[slot]);
                } else {
                    tma_load_4d(sa, &tm_u, c0, ri0, rj0, 2 * v, &full[slot]);
                    tma_load_4d(sa + kTmaABytes, &tm_u, c0, ri0, rj0, 2 * v + 1, &full[slot]);
                    bulk_g2s_u32(sa + 2 * kTmaABytes, tiles + ((size_t)(kNumOffsets + cls) * KB + h) * (Cfg::BBytes / 4),
                                 Cfg::BBytes, &full[slot]);
                }
                s_issued[0] = gs + 1;
                if (++slot == kTmaStages) {
                    slot = 0;
                    ++use;
                }
                if (++h == KB) {
                    h = 0;
                    if (++st == n_steps) {
                        st = 0;
                        if (++it < my_tiles) tile_of(it, cls, ri0, rj0, v);
                    }
                }
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {
            // per K slice kk of the block: D_big[0, 2NP) (+)= A_hi x [B_hi | B_lo] (N = 2 NP:
            // the hi*hi and hi*lo terms side by side), then D_small = D_big + NP += A_lo x B_hi
            // (N = NP)
            constexpr uint32_t kIdescBig = idesc_tf32(128, 2 * NP), kIdescSmall = idesc_tf32(128, NP);
            int slot = 0, use = 0, h = 0, d = 0, du = 0;
            for (int gs = 0; gs < total; ++gs) {
                if (*vabort) break;
                if (!mbar_poll_bounded(&full[slot], (uint32_t)(use & 1), wb) ||
                    (h == 0 && du > 0 && !mbar_poll_bounded(&acc_empty[d], (uint32_t)((du - 1) & 1), wb))) {
                    abort_now();
                    break;
                }
                tc_fence_after();
                const uint32_t a_hi = base + (uint32_t)slot * kStageBytes, a_lo = a_hi + kTmaABytes;
                const uint32_t b_hi = a_hi + 2 * kTmaABytes;
                const uint32_t d_big = tmem + Cfg::AccCols * d, d_small = d_big + NP;
                const uint64_t dah = smem_desc_sw128(a_hi), dal = smem_desc_sw128(a_lo), dbh = smem_desc_sw128(b_hi);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    // +32 bytes along K inside the swizzled rows = +2 in the descriptor's address field
                    mma_tf32_ss(d_big, dah + 2 * kk, dbh + 2 * kk, kIdescBig, (h > 0 || kk > 0) ? 1u : 0u);
                    mma_tf32_ss(d_small, dal + 2 * kk, dbh + 2 * kk, kIdescSmall, 1u);
                }
                mma_commit(&empty[slot]);
                s_issued[1] = gs + 1;
                if (++slot == kTmaStages) {
                    slot = 0;
                    ++use;
                }
                if (++h == KB) {
                    h = 0;
                    mma_commit(&acc_full[d]);
                    if (++d == kTmaAcc) {
                        d = 0;
                        ++du;
                    }
                }
            }
        }
    } else if (warp == 6) {
        for (int it = 0; it < my_tiles; ++it) {
            int cls, ri0, rj0, v;
            tile_of(it, cls, ri0, rj0, v);
            const int px = cls & 1, py = cls >> 1;
            const DFv* Qv = Qin + v * g.vQ;
            for (int r = lane; r < rows; r += 32) {
                const int ri = ri0 + r % g.TX, rj = rj0 + r / g.TX;
                DFv sacc = g.has_l2l ? Cpar[v * g.vQ + (size_t)morton2(ri, rj)] : DFv{0.f, 0.f};
                for (int k0 = 0; k0 < 27; k0 += 9) {  // nine loads in flight at a time
                    DFv qv[9];
#pragma unroll
                    for (int k = 0; k < 9; ++k) {
                        const int sx = 2 * ri + px + s_off[cls][k0 + k][0], sy = 2 * rj + py + s_off[cls][k0 + k][1];
                        qv[k] = (sx >= 0 && sx < side && sy >= 0 && sy < side) ? Qv[morton2(sx, sy)]
                                                                                 : DFv{0.f, 0.f};
                    }
#pragma unroll
                    for (int k = 0; k < 9; ++k) {
                        const int o = s_off[cls][k0 + k][2];
                        sacc = dadd(sacc, dmul(DFv{mono[o], mono[kNumOffsets + o]}, qv[k]));
                    }
                }
                Cout[v * g.vQ + morton2(2 * ri + px, 2 * rj + py)] = sacc;
            }
        }
    } else {
        const int r = threadIdx.x;  // TMEM lane = tile row
        const bool valid = r < rows;
        const int xl = r % g.TX, yl = r / g.TX;
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        float acc[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) acc[j] = 0.f;
        int it = 0, st = 0, d = 0, du = 0;
        int cls = 0, ri = 0, rj = 0, v = 0;
        const int offsets_total = my_tiles * n_steps;
        for (int gs = 0; gs < offsets_total; ++gs) {
            if (st == 0) {
                int ri0, rj0;
                tile_of(it, cls, ri0, rj0, v);
                ri = ri0 + xl;
                rj = rj0 + yl;
            }
            bool ok = *vabort == 0 && mbar_poll_bounded(&acc_full[d], (uint32_t)(du & 1), wb);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) abort_now();
                break;
            }
            tc_fence_after();
#pragma unroll
            for (int c = 0; c < NP / 32; ++c) {
                uint32_t big[32], small[32];
                tmem_ld32(tmem + lane_base + Cfg::AccCols * d + 32 * c, big);
                tmem_ld32(tmem + lane_base + Cfg::AccCols * d + NP + 32 * c, small);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[32 * c + j] += __uint_as_float(small[j]) + __uint_as_float(big[j]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[d]);
            if (st == n_steps - 1) {
                if (valid) {
                    float4* dst = reinterpret_cast<float4*>(
                        out + v * g.vq + (size_t)morton2(2 * ri + (cls & 1), 2 * rj + (cls >> 1)) * NP);
#pragma unroll
                    for (int c = 0; c < NP / 4; ++c)
                        dst[c] = make_float4(acc[4 * c], acc[4 * c + 1], acc[4 * c + 2], acc[4 * c + 3]);
                }
#pragma unroll
                for (int j = 0; j < NP; ++j) acc[j] = 0.f;
            }
            if (++d == kTmaAcc) {
                d = 0;
                ++du;
            }
            if (++st == n_steps) {
                st = 0;
                ++it;
            }
        }
    }
    __syncwarp();
    __syncthreads();
    if (s_abort && threadIdx.x == 0) {
        // copies and MMAs issued before the abort land before the memory is released: the
        // last kTmaStages loads, and the commit of the last issued K-block (a commit
        // tracks every MMA issued before it)
        const int p = s_issued[0], m = s_issued[1];
        for (int gs = p > kTmaStages ? p - kTmaStages : 0; gs < p; ++gs)
            mbar_poll_bounded(&full[gs % kTmaStages], (uint32_t)((gs / kTmaStages) & 1));
        if (m > 0) mbar_poll_bounded(&empty[(m - 1) % kTmaStages], (uint32_t)(((m - 1) / kTmaStages) & 1));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, Cfg::Cols);
    }
}

// ---------------------------------------------------------------------------------
// List form, for pruned storage and forests (P_pad 32 and 64): a level's boxes are compact ids
// grouped by parity class, each with its 27 interaction-list entries (-1: none) and its
// parent.  A tile is 128 consecutive boxes of one class; the A operand of a K-step is
// the gather of the tile's 128 source rows (hi and lo, split beforehand into row-major
// [box][NP] arrays; one 128-byte K-block of each row per ring step), so no tensor map
// applies.  Same pipeline as the TMA form, with the
// copies done by four producer warps, 32 rows each: eight lanes per row and four rows
// per instruction (16-byte cp.async, coalesced 128-byte rows), written straight into the
// 128-byte swizzled layout, missing sources zero-filled.  Every producer lane arrives on
// the stage's "full" barrier through cp.async.mbarrier.arrive.noinc, which fires when
// that lane's copies have landed, so a stage is released to the MMA thread as soon as
// its rows are in, however far ahead the producers have run; the MMA thread makes the
// rows visible to the tensor core with a proxy fence after its wait.  Producer warp 0
// adds the operator tile's bulk copy.  (Measured before: announcing each warp's rows
// two cp.async groups late, the K-steps taken in turn by whole warps, and a deeper ring
// announced later.)
//   warps 0-3: fold (one box per TMEM lane), warps 4-7: gather, warp 8: MMA issuer,
//   warp 9: compensated incoming constants.
constexpr int kLStages = 4;
constexpr int kLThreads = 320;
constexpr int kLSrcInts = 4 * 32 * 28;  // per producer warp: 32 rows x 28 offsets
// P_pad 32: one K-block per offset; P_pad 64: two (each a ring step), accumulated in the
// offset's fresh accumulator, as in the TMA form
template <int NP>
struct ListTcCfg {
    static constexpr int KB = NP / 32;
    static constexpr uint32_t BBytes = 2u * NP * 128u;                 // [B_hi | B_lo] of one K-block
    static constexpr uint32_t StageBytes = 2 * kTmaABytes + BBytes;    // A hi, A lo, B
    static constexpr size_t Smem = 1024 + (size_t)kLStages * StageBytes + (size_t)kLSrcInts * sizeof(int);
    static_assert(Smem <= 227 * 1024, "list ring exceeds shared memory");
};

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <int NP>
__global__ void __launch_bounds__(kLThreads, 1) m2l_tc_list_kernel(
    const int64_t* __restrict__ cls_start, const int32_t* __restrict__ il, const int32_t* __restrict__ par,
    const float* __restrict__ qhi, const float* __restrict__ qlo, const float* __restrict__ uhi,
    const float* __restrict__ ulo, const float* __restrict__ tiles, const float* __restrict__ mono,
    const DFv* __restrict__ Qin, const DFv* __restrict__ Cpar, float* __restrict__ out, DFv* __restrict__ Cout,
    int* __restrict__ status) {
    griddep_wait();
    using Cfg = ListTcCfg<NP>;
    constexpr int KB = Cfg::KB;
    constexpr uint32_t kLStageBytes = Cfg::StageBytes;
    constexpr uint32_t kAccCols = TmaCfg<NP>::AccCols;
    extern __shared__ __align__(1024) unsigned char tl_smem[];
    const uint32_t base = smem_u32(tl_smem) + ((1024u - (smem_u32(tl_smem) & 1023u)) & 1023u);
    int* s_src = reinterpret_cast<int*>(tl_smem + (base - smem_u32(tl_smem)) + (size_t)kLStages * kLStageBytes);
    __shared__ __align__(8) uint64_t full[kLStages], empty[kLStages], acc_full[kTmaAcc], acc_empty[kTmaAcc];
    __shared__ uint32_t s_tmem;
    __shared__ int s_op[4][28];           // operator tile of K-step st for class c
    __shared__ long long s_c[5], s_t[5];  // class starts; first tile of each class
    __shared__ int s_abort;
    __shared__ int s_issued[2];           // K-steps issued by the producers (all four) and by the MMA thread
    __shared__ int s_pissued[4];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool has_l2l = uhi != nullptr;
    const int n_steps = 27 + (has_l2l ? 1 : 0);
    volatile int* vabort = &s_abort;
    const uint32_t wb = ((volatile int*)status)[3] > 0 ? (uint32_t)((volatile int*)status)[3] : 0xffffffffu;
    if (threadIdx.x == 0) {
        for (int c = 0; c < 4; ++c) {
            const int px = c & 1, py = c >> 1;
            int nn = 0;
            for (int d = 0; d < 36; ++d) {
                const int dx = (d % 6) - 2 - px, dy = (d / 6) - 2 - py;
                if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
                s_op[c][nn++] = offset_index_tc(dx, dy);  // interaction-list slot order
            }
            s_op[c][27] = kNumOffsets + c;
        }
        long long t = 0;
        for (int c = 0; c <= 4; ++c) {
            s_c[c] = cls_start[c];
            s_t[c] = t;
            if (c < 4) t += (cls_start[c + 1] - cls_start[c] + 127) / 128;
        }
        for (int i = 0; i < kLStages; ++i) {
            mbar_init(&full[i], 4 * 32 + 1);  // every producer lane's copies + the operator tile (with its bytes)
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < kTmaAcc; ++i) {
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], 4);
        }
        fence_barrier_init();
        s_abort = 0;
        s_issued[0] = s_issued[1] = 0;
        for (int i = 0; i < 4; ++i) s_pissued[i] = 0;
    }
    if (warp == 0) {
        tmem_alloc(&s_tmem, TmaCfg<NP>::Cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const int n_tiles = (int)s_t[4];
    const int my_tiles = (int)blockIdx.x < n_tiles ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int total = my_tiles * n_steps * KB;  // ring steps: K-blocks of every offset of every tile
    auto abort_now = [&]() {
        atomicExch(&s_abort, 1);
        atomicExch(status, LFMM_ETIMEOUT);
    };
    // it-th tile of this CTA: class and first / end box
    auto tile_of = [&](int it, int& cls, long long& b0, long long& b1) {
        const long long t = (long long)blockIdx.x + (long long)it * gridDim.x;
        cls = (t >= s_t[1]) + (t >= s_t[2]) + (t >= s_t[3]);
        b0 = s_c[cls] + (t - s_t[cls]) * 128;
        b1 = min(b0 + 128, s_c[cls + 1]);
    };

    if (warp >= 4 && warp < 8) {
        const int pw = warp - 4;                 // rows 32 pw .. 32 pw + 31 of every tile
        int* my_src = s_src + pw * 32 * 28;      // [row][K-step] source row, -1: none
        const int sub = lane >> 3, ch = lane & 7;  // row within a group of four, 16-byte chunk
        int it = 0, st = 0, h = 0, slot = 0, use = 0, cls = 0;
        long long b0 = 0, b1 = 0;
        int gs = 0;
        for (; gs < total; ++gs) {
            if (__any_sync(0xffffffffu, *vabort != 0)) break;  // warp-uniform
            if (st == 0 && h == 0) {
                // lane r: the 27 list entries and the parent of row r, seven loads in flight
                tile_of(it, cls, b0, b1);
                const long long b = b0 + 32 * pw + lane;
                const bool bv = b < b1;
#pragma unroll
                for (int k0 = 0; k0 < 28; k0 += 7) {
                    int v[7];
#pragma unroll
                    for (int u = 0; u < 7; ++u) {
                        const int k = k0 + u;
                        v[u] = !bv ? -1 : k < 27 ? il[b * 27 + k] : (has_l2l ? par[b] : -1);
                    }
#pragma unroll
                    for (int u = 0; u < 7; ++u) my_src[lane * 28 + k0 + u] = v[u];
                }
                __syncwarp();
            }
            bool ok = true;
            if (use > 0 && lane == 0) ok = mbar_poll_bounded(&empty[slot], (uint32_t)((use - 1) & 1), wb);
            if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) {
                if (lane == 0) abort_now();
                break;
            }
            const uint32_t sa = base + (uint32_t)slot * kLStageBytes;
            if (pw == 0 && lane == 0) {
                mbar_arrive_expect_tx(&full[slot], Cfg::BBytes);
                bulk_g2s_u32(sa + 2 * kTmaABytes, tiles + ((size_t)s_op[cls][st] * KB + h) * (Cfg::BBytes / 4),
                             Cfg::BBytes, &full[slot]);
            }
            const float* hs = st < 27 ? qhi : uhi;
            const float* ls = st < 27 ? qlo : ulo;
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                const int rl = 4 * g + sub;          // row within this warp's 32
                const int r = 32 * pw + rl;          // row of the tile (TMEM lane)
                const int si = my_src[rl * 28 + st];
                const size_t off = si < 0 ? 0 : (size_t)si * NP + 32 * h + 4 * ch;
                const int bytes = si < 0 ? 0 : 16;
                const uint32_t dst = (uint32_t)(r * 128 + ((ch ^ (r & 7)) << 4));
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa + dst), "l"(hs + off),
                             "r"(bytes)
                             : "memory");
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa + kTmaABytes + dst),
                             "l"(ls + off), "r"(bytes)
                             : "memory");
            }
            // the stage's barrier counts this lane once its copies have landed
            cp_async_mbar_arrive_noinc(&full[slot]);
            if (lane == 0) s_pissued[pw] = gs + 1;
            if (++slot == kLStages) {
                slot = 0;
                ++use;
            }
            if (++h == KB) {
                h = 0;
                if (++st == n_steps) {
                    st = 0;
                    ++it;
                }
            }
        }
        // nothing of this lane's in flight when the CTA ends
        asm volatile("cp.async.wait_all;\n" ::: "memory");
    } else if (warp == 8) {
        if (lane == 0) {
            // per K slice: D_big[0, 2 NP) (+)= A_hi x [B_hi | B_lo], D_small = D_big + NP +=
            // A_lo x B_hi
            constexpr uint32_t kIdescBig = idesc_tf32(128, 2 * NP), kIdescSmall = idesc_tf32(128, NP);
            int slot = 0, use = 0, h = 0, d = 0, du = 0;
            for (int gs = 0; gs < total; ++gs) {
                if (*vabort) break;
                if (!mbar_poll_bounded(&full[slot], (uint32_t)(use & 1), wb) ||
                    (h == 0 && du > 0 && !mbar_poll_bounded(&acc_empty[d], (uint32_t)((du - 1) & 1), wb))) {
                    abort_now();
                    break;
                }
                fence_proxy_async_smem();  // the producers' cp.async rows, seen by the tensor core
                tc_fence_after();
                const uint32_t a_hi = base + (uint32_t)slot * kLStageBytes, a_lo = a_hi + kTmaABytes;
                const uint32_t b_hi = a_hi + 2 * kTmaABytes;
                const uint32_t d_big = tmem + kAccCols * d, d_small = d_big + NP;
                const uint64_t dah = smem_desc_sw128(a_hi), dal = smem_desc_sw128(a_lo), dbh = smem_desc_sw128(b_hi);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    mma_tf32_ss(d_big, dah + 2 * kk, dbh + 2 * kk, kIdescBig, (h > 0 || kk > 0) ? 1u : 0u);
                    mma_tf32_ss(d_small, dal + 2 * kk, dbh + 2 * kk, kIdescSmall, 1u);
                }
                mma_commit(&empty[slot]);
                s_issued[1] = gs + 1;
                if (++slot == kLStages) {
                    slot = 0;
                    ++use;
                }
                if (++h == KB) {
                    h = 0;
                    mma_commit(&acc_full[d]);
                    if (++d == kTmaAcc) {
                        d = 0;
                        ++du;
                    }
                }
            }
        }
    } else if (warp == 9) {
        for (int it = 0; it < my_tiles; ++it) {
            int cls;
            long long b0, b1;
            tile_of(it, cls, b0, b1);
            for (long long b = b0 + lane; b < b1; b += 32) {
                const int pb = has_l2l ? par[b] : -1;
                DFv sacc = pb >= 0 ? Cpar[pb] : DFv{0.f, 0.f};
                for (int k0 = 0; k0 < 27; k0 += 9) {
                    int sb[9];
                    DFv qv[9];
#pragma unroll
                    for (int k = 0; k < 9; ++k) sb[k] = il[b * 27 + k0 + k];
#pragma unroll
                    for (int k = 0; k < 9; ++k) qv[k] = sb[k] >= 0 ? Qin[sb[k]] : DFv{0.f, 0.f};
#pragma unroll
                    for (int k = 0; k < 9; ++k) {
                        const int o = s_op[cls][k0 + k];
                        if (sb[k] >= 0) sacc = dadd(sacc, dmul(DFv{mono[o], mono[kNumOffsets + o]}, qv[k]));
                    }
                }
                Cout[b] = sacc;
            }
        }
    } else if (warp < 4) {
        const int r = threadIdx.x;  // TMEM lane = tile row
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        float acc[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) acc[j] = 0.f;
        int it = 0, st = 0, d = 0, du = 0, cls = 0;
        long long b0 = 0, b1 = 0;
        const int offsets_total = total / KB;
        for (int gs = 0; gs < offsets_total; ++gs) {
            if (st == 0) tile_of(it, cls, b0, b1);
            bool ok = *vabort == 0 && mbar_poll_bounded(&acc_full[d], (uint32_t)(du & 1), wb);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) abort_now();
                break;
            }
            tc_fence_after();
#pragma unroll
            for (int c = 0; c < NP / 32; ++c) {
                uint32_t big[32], small[32];
                tmem_ld32(tmem + lane_base + kAccCols * d + 32 * c, big);
                tmem_ld32(tmem + lane_base + kAccCols * d + NP + 32 * c, small);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[32 * c + j] += __uint_as_float(small[j]) + __uint_as_float(big[j]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[d]);
            if (st == n_steps - 1) {
                if (b0 + r < b1) {
                    float4* dst = reinterpret_cast<float4*>(out + (size_t)(b0 + r) * NP);
#pragma unroll
                    for (int c = 0; c < NP / 4; ++c)
                        dst[c] = make_float4(acc[4 * c], acc[4 * c + 1], acc[4 * c + 2], acc[4 * c + 3]);
                }
#pragma unroll
                for (int j = 0; j < NP; ++j) acc[j] = 0.f;
            }
            if (++d == kTmaAcc) {
                d = 0;
                ++du;
            }
            if (++st == n_steps) {
                st = 0;
                ++it;
            }
        }
    }
    __syncwarp();
    __syncthreads();
    if (s_abort && threadIdx.x == 0) {
        // Every producer lane arrived for the steps its warp issued, but the warps stopped
        // at different steps.  A warp issues step g + kLStages only after step g's stage
        // was consumed, so the steps issued by some warps and not by others are fewer than
        // kLStages, each in its own slot and phase: arrive for the 32 lanes of each warp
        // that skipped them (and for warp 0's operator-tile arrival), then wait until the
        // operator copies of the last kLStages issued steps have landed (the lanes waited
        // for their own cp.async) and the MMAs issued have completed (a commit tracks every
        // MMA before it).
        int pmin = s_pissued[0], pmax = s_pissued[0];
        for (int i = 1; i < 4; ++i) {
            pmin = min(pmin, s_pissued[i]);
            pmax = max(pmax, s_pissued[i]);
        }
        for (int g = pmin; g < pmax; ++g) {
            int missing = s_pissued[0] <= g ? 1 : 0;
            for (int i = 0; i < 4; ++i) missing += s_pissued[i] <= g ? 32 : 0;
            if (missing > 0) mbar_arrive_n(&full[g % kLStages], (uint32_t)missing);
        }
        for (int g = pmax > kLStages ? pmax - kLStages : 0; g < pmax; ++g)
            mbar_poll_bounded(&full[g % kLStages], (uint32_t)((g / kLStages) & 1));
        const int m = s_issued[1];
        if (m > 0) mbar_poll_bounded(&empty[(m - 1) % kLStages], (uint32_t)(((m - 1) / kLStages) & 1));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, TmaCfg<NP>::Cols);
    }
}

// hi / lo TF32 split of row-major expansions ([box][32]), float4 items: hi and lo arrays
__global__ void split_tf32_rows_kernel(const float4* __restrict__ x, int64_t n4, float4* __restrict__ hi,
                                       float4* __restrict__ lo) {
    griddep_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = x[i];
        const float a[4] = {v.x, v.y, v.z, v.w};
        float h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            h[e] = __uint_as_float(tf32_rna_bits(a[e]));
            l[e] = __uint_as_float(tf32_rna_bits(a[e] - h[e]));
        }
        hi[i] = make_float4(h[0], h[1], h[2], h[3]);
        lo[i] = make_float4(l[0], l[1], l[2], l[3]);
    }
}

// hi / lo TF32 split of a level's expansions (Morton order in) into the layouts the
// tensor maps describe: planes = 1 -> [hl][plane][y'][x'][NP] (targets' level),
// planes = 0 -> [hl][y][x][NP] (parent level, row-major).  Item iv is one float4 of
// vector iv / n4.
template <int NP>
__device__ __forceinline__ void split_tf32_item(const float4* __restrict__ x0, float4* __restrict__ dst0, int lg,
                                                int planes, int64_t vq4, int64_t n4, int64_t iv) {
    constexpr int Q = NP / 4;  // float4 per box
    const int np = 1 << lg;
    const int64_t vec = iv / n4, i = iv - vec * n4;
    const float4* x = x0 + vec * vq4;
    float4* dst = dst0 + 2 * vec * n4;  // vector vec: hi then lo
    const int64_t b = i / Q;
    const int c = (int)(i - b * Q);
    uint32_t bx, by;
    if (planes) {
        const int plane = (int)(b >> (2 * lg));
        const int64_t rem = b & (((int64_t)1 << (2 * lg)) - 1);
        bx = 2 * (uint32_t)(rem & (np - 1)) + (plane & 1);
        by = 2 * (uint32_t)(rem >> lg) + (plane >> 1);
    } else {
        bx = (uint32_t)(b & (np - 1));
        by = (uint32_t)(b >> lg);
    }
    const float4 v = x[(size_t)morton2(bx, by) * Q + c];
    const float a[4] = {v.x, v.y, v.z, v.w};
    float h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        h[e] = __uint_as_float(tf32_rna_bits(a[e]));
        l[e] = __uint_as_float(tf32_rna_bits(a[e] - h[e]));
    }
    dst[i] = make_float4(h[0], h[1], h[2], h[3]);
    dst[i + n4] = make_float4(l[0], l[1], l[2], l[3]);
}

// The target level's expansions (parity planes) and, when xu is set, the parent level's
// (row-major) in one launch: items [0, nvec nq4) are the former, the rest the latter.
template <int NP>
__global__ void split_tf32_layout_kernel(const float4* __restrict__ xq, float4* __restrict__ dq,
                                         const float4* __restrict__ xu, float4* __restrict__ du, int lg, int nvec,
                                         int64_t vq4) {
    griddep_wait();
    const int64_t nq4 = ((int64_t)4 << (2 * lg)) * (NP / 4), nu4 = ((int64_t)1 << (2 * lg)) * (NP / 4);
    const int64_t nq = nq4 * nvec, n = nq + (xu ? nu4 * nvec : 0);
    for (int64_t iv = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; iv < n; iv += (int64_t)gridDim.x * blockDim.x) {
        if (iv < nq) split_tf32_item<NP>(xq, dq, lg, 1, vq4, nq4, iv);
        else split_tf32_item<NP>(xu, du, lg, 0, vq4, nu4, iv - nq);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

// fp32 tiled map over `rank` dims (dims[0] = NP coefficients, innermost), box
// {32, TX, TY, 1, ...} (one 128-byte K-block), 128-byte swizzle, zero fill outside
bool encode_map(CUtensorMap* m, const float* base, int rank, const uint64_t* dims, int TX, int TY) {
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t gd[5], gs[4];
    cuuint32_t box[5], es[5];
    uint64_t stride = 4;
    for (int i = 0; i < rank; ++i) {
        gd[i] = dims[i];
        if (i > 0) gs[i - 1] = stride;
        stride *= dims[i];
        box[i] = i == 0 ? 32u : i == 1 ? (cuuint32_t)TX : i == 2 ? (cuuint32_t)TY : 1u;
        es[i] = 1;
    }
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<float*>(base), gd, gs, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

cudaError_t launch_m2l_tma(const DeviceOps& ops, int k, int level, const float* q_level, const void* Q_level,
                           const float* u_parent, const void* C_parent, float* u_level, void* C_level, float* split,
                           int* status, int num_sms, cudaStream_t s, int nvec, int64_t vq, int64_t vQ, int tile,
                           int stages) {
    const int NP = ops.NP;
    if (NP != 32 && NP != 64) return cudaErrorInvalidValue;
    const int lg = level - 1;
    const int np = 1 << lg;
    const bool l2l = u_parent != nullptr;
    float* qs = split;                                           // [nvec][2][4][np][np][NP]
    float* us = split + ((size_t)nvec * 2 * 4 * np * np * NP);   // [nvec][2][np][np][NP]
    auto grid_for = [&](int64_t n4) {
        int64_t b = (n4 + 255) / 256;
        return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)num_sms * 16));
    };
    {
        const dim3 sg(grid_for((int64_t)(4 + (l2l ? 1 : 0)) * np * np * (NP / 4) * nvec));
        const cudaError_t e = NP == 32
            ? launch_dependent(split_tf32_layout_kernel<32>, sg, dim3(256), 0, s,
                               reinterpret_cast<const float4*>(q_level), reinterpret_cast<float4*>(qs),
                               l2l ? reinterpret_cast<const float4*>(u_parent) : nullptr, reinterpret_cast<float4*>(us),
                               lg, nvec, vq / 4)
            : launch_dependent(split_tf32_layout_kernel<64>, sg, dim3(256), 0, s,
                               reinterpret_cast<const float4*>(q_level), reinterpret_cast<float4*>(qs),
                               l2l ? reinterpret_cast<const float4*>(u_parent) : nullptr, reinterpret_cast<float4*>(us),
                               lg, nvec, vq / 4);
        if (e != cudaSuccess) return e;
    }
    {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    TmaGeo g;
    g.level = level;
    g.lg = lg;
    // tiles of 128 boxes of one parity class, tile boxes wide (opts.m2l_tile; 0: 128)
    g.TX = std::min(np, tile > 0 ? tile : 128);
    g.TY = std::min(128 / g.TX, np);
    g.tiles_x = np / g.TX;
    g.tiles_per_class = g.tiles_x * (np / g.TY);
    g.n_tiles = 4 * g.tiles_per_class;
    g.has_l2l = l2l ? 1 : 0;
    g.nvec = nvec;
    g.vq = vq;
    g.vQ = vQ;
    CUtensorMap mq, mu;
    const uint64_t dq[5] = {(uint64_t)NP, (uint64_t)np, (uint64_t)np, 4, (uint64_t)(2 * nvec)};
    const uint64_t du[4] = {(uint64_t)NP, (uint64_t)np, (uint64_t)np, (uint64_t)(2 * nvec)};
    if (!encode_map(&mq, qs, 5, dq, g.TX, g.TY)) return cudaErrorInvalidValue;
    if (!encode_map(&mu, l2l ? us : qs, 4, du, g.TX, g.TY)) return cudaErrorInvalidValue;
    const int grid = std::min(g.n_tiles * nvec, num_sms);
    auto go = [&](auto np_tag, auto stages_tag) -> cudaError_t {
        constexpr int NPc = decltype(np_tag)::value;
        constexpr int S = decltype(stages_tag)::value;
        constexpr size_t smem = 1024 + (size_t)S * TmaCfg<NPc>::StageBytes;
        static_assert(smem <= 227 * 1024, "TMA ring exceeds shared memory");
        cudaError_t e = ensure_dynamic_smem((const void*)m2l_tma_kernel<NPc, S>, smem);
        if (e != cudaSuccess) return e;
        return launch_dependent(m2l_tma_kernel<NPc, S>, dim3(grid), dim3(kTmaThreads), smem, s, mq, mu, g,
                                (const float*)ops.tc[k], (const float*)ops.mono[k], (const DFv*)Q_level,
                                (const DFv*)C_parent, u_level, (DFv*)C_level, status);
    };
    auto by_stages = [&](auto np_tag) -> cudaError_t {
        switch (stages > 0 ? stages : kTmaStagesDefault) {
            case 2: return go(np_tag, std::integral_constant<int, 2>());
            case 4: return go(np_tag, std::integral_constant<int, 4>());
            default: return go(np_tag, std::integral_constant<int, 3>());
        }
    };
    return NP == 32 ? by_stages(std::integral_constant<int, 32>()) : by_stages(std::integral_constant<int, 64>());
}

int64_t m2l_tc_list_split_floats(int64_t nb, int64_t nb_parent, int NP) { return 2 * (nb + nb_parent) * NP; }

cudaError_t launch_m2l_tc_list(const DeviceOps& ops, int k, const int64_t* cls_start, const int64_t* cls_host,
                               const int32_t* il, const int32_t* par, const float* q_level, int64_t nb,
                               const void* Q_level, const float* u_parent, int64_t nb_parent, const void* C_parent,
                               float* u_level, void* C_level, float* split, int* status, int num_sms,
                               cudaStream_t s) {
    const int NP = ops.NP;
    if ((NP != 32 && NP != 64) || !ops.tc[k]) return cudaErrorInvalidValue;
    int64_t n_tiles = 0;
    for (int c = 0; c < 4; ++c) n_tiles += (cls_host[c + 1] - cls_host[c] + 127) / 128;
    if (n_tiles <= 0) return cudaSuccess;
    float* qhi = split;
    float* qlo = qhi + (size_t)nb * NP;
    float* uhi = qlo + (size_t)nb * NP;
    float* ulo = uhi + (size_t)nb_parent * NP;
    auto grid_for = [&](int64_t n4) {
        int64_t b = (n4 + 255) / 256;
        return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)num_sms * 16));
    };
    const int64_t q4 = nb * (NP / 4), u4 = nb_parent * (NP / 4);
    cudaError_t e = launch_dependent(split_tf32_rows_kernel, dim3(grid_for(q4)), dim3(256), 0, s,
                                     reinterpret_cast<const float4*>(q_level), q4, reinterpret_cast<float4*>(qhi),
                                     reinterpret_cast<float4*>(qlo));
    if (e != cudaSuccess) return e;
    if (u_parent) {
        e = launch_dependent(split_tf32_rows_kernel, dim3(grid_for(u4)), dim3(256), 0, s,
                             reinterpret_cast<const float4*>(u_parent), u4, reinterpret_cast<float4*>(uhi),
                             reinterpret_cast<float4*>(ulo));
        if (e != cudaSuccess) return e;
    }
    const int grid = (int)std::min<int64_t>(n_tiles, num_sms);
    auto go = [&](auto np_tag) -> cudaError_t {
        constexpr int NPc = decltype(np_tag)::value;
        cudaError_t r = ensure_dynamic_smem((const void*)m2l_tc_list_kernel<NPc>, ListTcCfg<NPc>::Smem);
        if (r != cudaSuccess) return r;
        return launch_dependent(m2l_tc_list_kernel<NPc>, dim3(grid), dim3(kLThreads), ListTcCfg<NPc>::Smem, s,
                                cls_start, il, u_parent ? par : nullptr, (const float*)qhi, (const float*)qlo,
                                u_parent ? (const float*)uhi : nullptr, u_parent ? (const float*)ulo : nullptr,
                                (const float*)ops.tc[k], (const float*)ops.mono[k], (const DFv*)Q_level,
                                (const DFv*)C_parent, u_level, (DFv*)C_level, status);
    };
    return NP == 32 ? go(std::integral_constant<int, 32>()) : go(std::integral_constant<int, 64>());
}

}  // namespace lfmm
