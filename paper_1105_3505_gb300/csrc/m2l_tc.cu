// M2L (+ fused L2L) on the 5th-generation tensor cores, mixed path (Sec. 7, Sec. 8.2
// steps 3-4): for the boxes tau of one parity class,
//
//   u_hat^tau = sum_{sigma in int(tau)} (T_ifo^o - c_o 1 1^T) q_hat^sigma + T_ifi^c u_hat^parent
//
// as an implicit GEMM per CTA: M = 128 target boxes (TMEM lanes), N = 32 outputs,
// K = 27 x 32 gathered source expansions (+ 32 for the parent).  Operands are split
// into TF32 hi + lo parts (round to nearest) and three products hi*hi + hi*lo + lo*hi
// are formed (the lo*lo term is below 2^-22 relative).  The tensor core's fp32
// accumulation rounds toward zero, and that bias grows linearly with the number of
// MMAs feeding one accumulator; so every K-step writes fresh TMEM accumulators (hi*hi
// in one, the small hi*lo + lo*hi terms in another), which the threads read back one
// step later and add in registers with round-to-nearest fp32.
//
//  - A (gathered expansions): the level's expansions, and the parent level's incoming
//    expansions, are split once into TF32 hi and lo arrays (split_tf32_kernel).  Each
//    K-step copies the 128 gathered source rows of hi and of lo with cp.async (16-byte
//    chunks) straight into the 128-byte-swizzled K-major layout that a shared-memory
//    matrix descriptor describes, so the tensor core reads A like B and no thread
//    touches the values between the gather and the MMA.
//  - B (operators): pre-split, pre-swizzled 4 KB tiles in the device image, fetched
//    with cp.async.bulk into a 3-deep ring in shared memory two steps ahead, completion
//    tracked by mbarriers.
//  - TMEM holds only the two accumulator pairs (128 columns).
//  - step s: fold in the partials of step s-1 (waiting for its MMAs, which also frees
//    the A stage they read), start the gather of step s+1 into that stage, wait for the
//    own copies of step s, make them visible to the tensor core, barrier; one elected
//    thread issues the 12 MMAs (K = 8 each) of step s and the B copy of step s+2.
// Every mbarrier wait is bounded (clock64 budget, suspend-time hint); on expiry the CTA
// records LFMM_ETIMEOUT in the plan's status word, all its threads stop issuing work
// together (the abort flag is block-uniform), wait (bounded) for what was issued, free
// the TMEM and return.
#include "lfmm_internal.h"

namespace lfmm {

namespace {

constexpr int kTcThreads = 128;          // 4 warps, one TMEM lane quarter each
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
// try_wait with a suspend-time hint: the thread sleeps until the phase completes or the
// hint (ns) runs out, instead of spinning through issue slots
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitBudget) return false;
    return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
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
// makes this thread's completed cp.async writes to shared memory visible to the tensor core
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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

constexpr int kTc2Cols = 128;  // D_big[b]: [32b, 32b+32), D_small[b]: [64+32b, 96+32b)

__global__ void __launch_bounds__(kTcThreads) m2l_tc_ss_kernel(int level, const float* __restrict__ qhi,
                                                               const float* __restrict__ qlo,
                                                               const float* __restrict__ uhi,
                                                               const float* __restrict__ ulo,
                                                               const float* __restrict__ tiles,
                                                               const float* __restrict__ mono,
                                                               const DFv* __restrict__ Qin, const DFv* __restrict__ Cpar,
                                                               float* __restrict__ out, DFv* __restrict__ Cout,
                                                               int* __restrict__ status) {
    constexpr int NP = 32;
    // dynamic shared memory (1024-byte aligned): B ring [3][hi, lo][32 x 32], then the A
    // stages [2][hi, lo][128 x 32], all 128-byte swizzled
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    float (*sB)[2][1024] = reinterpret_cast<float (*)[2][1024]>(
        tc_smem + ((1024u - (smem_u32(tc_smem) & 1023u)) & 1023u));
    float (*sA)[2][kTcThreads * 32] = reinterpret_cast<float (*)[2][kTcThreads * 32]>(&sB[3][0][0]);
    __shared__ __align__(8) uint64_t bar_b[3], bar_mma[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_off[27][3];
    __shared__ int s_abort;
    __shared__ int s_src[28][kTcThreads];

    const int cls = blockIdx.y;
    const int px = cls & 1, py = cls >> 1;
    const int lg = level - 1;
    const int np_side = 1 << lg;
    const int64_t n_rows = (int64_t)1 << (2 * lg);
    const int64_t row = (int64_t)blockIdx.x * kTcThreads + threadIdx.x;
    const bool valid = row < n_rows;
    const int side = 1 << level;
    const bool has_l2l = uhi != nullptr;
    const int n_steps = 27 + (has_l2l ? 1 : 0);
    const int warp = threadIdx.x >> 5;
    const int ri = valid ? (int)(row & (np_side - 1)) : 0;
    const int rj = valid ? (int)(row >> lg) : 0;

    if (smem_u32(&sB[0][0][0]) & 1023u) {
        if (threadIdx.x == 0) atomicExch(status, LFMM_EINTERNAL);
        return;
    }
    if (threadIdx.x == 0) {
        int nn = 0;
        for (int d = 0; d < 36; ++d) {
            const int dx = (d % 6) - 2 - px, dy = (d / 6) - 2 - py;
            if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
            s_off[nn][0] = dx;
            s_off[nn][1] = dy;
            s_off[nn][2] = offset_index_tc(dx, dy);
            ++nn;
        }
        for (int i = 0; i < 3; ++i) mbar_init(&bar_b[i], 1);
        mbar_init(&bar_mma[0], 1);
        mbar_init(&bar_mma[1], 1);
        fence_barrier_init();
        s_abort = 0;
    }
    if (warp == 0) {
        tmem_alloc(&s_tmem, kTc2Cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    for (int st = 0; st < 27; ++st) {
        int si = -1;
        if (valid) {
            const int sx = 2 * ri + px + s_off[st][0], sy = 2 * rj + py + s_off[st][1];
            if (sx >= 0 && sx < side && sy >= 0 && sy < side) si = (int)morton2(sx, sy);
        }
        s_src[st][threadIdx.x] = si;
    }
    s_src[27][threadIdx.x] = (valid && has_l2l) ? (int)morton2(ri, rj) : -1;
    __syncthreads();
    const uint32_t tmem = s_tmem;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;

    // gather of step `step` into A stage b: thread t copies 16-byte chunk t % 8 of rows
    // t / 8 + 16 j of hi and of lo; chunk c of row r lands at chunk c ^ (r % 8)
    auto gather = [&](int step, int b) {
        const int ch = threadIdx.x & 7;
        const float* hsrc = step < 27 ? qhi : uhi;
        const float* lsrc = step < 27 ? qlo : ulo;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int r = (threadIdx.x >> 3) + 16 * j;
            const int si = s_src[step][r];
            const size_t off = si < 0 ? 0 : (size_t)si * NP + 4 * ch;
            const int bytes = si < 0 ? 0 : 16;
            const int pos = r * 32 + ((ch ^ (r & 7)) << 2);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(&sA[b][0][pos])),
                         "l"(hsrc + off), "r"(bytes)
                         : "memory");
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(&sA[b][1][pos])),
                         "l"(lsrc + off), "r"(bytes)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    auto b_src = [&](int step) -> const float* {
        return step < 27 ? tiles + (size_t)s_off[step][2] * 2048 : tiles + (size_t)(kNumOffsets + cls) * 2048;
    };

    constexpr uint32_t kIdesc = idesc_tf32(128, NP);
    float acc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = 0.f;
    auto flush = [&](int b) {
        uint32_t big[32], small[32];
        tmem_ld32(tmem + lane_base + 32 * b, big);
        tmem_ld32(tmem + lane_base + 64 + 32 * b, small);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] += __uint_as_float(small[j]) + __uint_as_float(big[j]);
    };
    volatile int* vabort = &s_abort;
    int issued_steps = 0, b_issued = 0;
    if (threadIdx.x == 0) {  // B tiles of steps 0 and 1
        for (int st = 0; st < 2 && st < n_steps; ++st) {
            mbar_arrive_expect_tx(&bar_b[st], 8192);
            bulk_g2s(&sB[st][0][0], b_src(st), 8192, &bar_b[st]);
            b_issued = st + 1;
        }
    }
    gather(0, 0);
    // Aborts are block-uniform: a failed wait only records s_abort; every thread tests
    // it right after the step's barrier, so all warps leave the loop at the same step
    // and meet the same barriers afterwards.
    for (int step = 0; step < n_steps; ++step) {
        const int buf = step & 1;
        bool w_ok = true;
        if (step >= 1) {
            // MMAs of step - 1 done: their partials in, their A stage free
            w_ok = *vabort == 0 && mbar_wait_bounded(&bar_mma[buf ^ 1], ((step - 1) >> 1) & 1);
            w_ok = __all_sync(0xffffffffu, w_ok);
            if (w_ok) {
                tc_fence_after();
                flush(buf ^ 1);
            } else {
                atomicExch(&s_abort, 1);
            }
        }
        if (w_ok && step + 1 < n_steps) {
            gather(step + 1, buf ^ 1);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (*vabort != 0) break;
        if (threadIdx.x == 0) {
            const int slot = step % 3;
            const bool good = mbar_wait_bounded(&bar_b[slot], (step / 3) & 1);
            if (!good) {
                atomicExch(&s_abort, 1);  // seen by all after the next barrier
            } else {
                tc_fence_after();
                const uint32_t a_hi = smem_u32(&sA[buf][0][0]), a_lo = smem_u32(&sA[buf][1][0]);
                const uint32_t b_hi = smem_u32(&sB[slot][0][0]), b_lo = smem_u32(&sB[slot][1][0]);
                const uint32_t d_big = tmem + 32 * buf, d_small = tmem + 64 + 32 * buf;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t ah = smem_desc_sw128(a_hi + 32 * kk), al = smem_desc_sw128(a_lo + 32 * kk);
                    const uint64_t bh = smem_desc_sw128(b_hi + 32 * kk), bl = smem_desc_sw128(b_lo + 32 * kk);
                    mma_tf32_ss(d_big, ah, bh, kIdesc, kk > 0 ? 1u : 0u);
                    mma_tf32_ss(d_small, ah, bl, kIdesc, kk > 0 ? 1u : 0u);
                    mma_tf32_ss(d_small, al, bh, kIdesc, 1u);
                }
                mma_commit(&bar_mma[buf]);
                // B tiles of step + 2 into the slot step - 1 used (its MMAs are done)
                if (step + 2 < n_steps) {
                    const int ns = (step + 2) % 3;
                    mbar_arrive_expect_tx(&bar_b[ns], 8192);
                    bulk_g2s(&sB[ns][0][0], b_src(step + 2), 8192, &bar_b[ns]);
                    b_issued = step + 3;
                }
            }
        }
        issued_steps = step + 1;
    }

    // incoming constant (compensated), one box per thread, while the last MMAs run
    if (valid) {
        DFv sacc = has_l2l ? Cpar[(size_t)morton2(ri, rj)] : DFv{0.f, 0.f};
        for (int c0 = 0; c0 < 27; c0 += 9) {
            DFv qv[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const int si = s_src[c0 + k][threadIdx.x];
                qv[k] = si >= 0 ? Qin[si] : DFv{0.f, 0.f};
            }
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const int o = s_off[c0 + k][2];
                sacc = dadd(sacc, dmul(DFv{mono[o], mono[kNumOffsets + o]}, qv[k]));
            }
        }
        Cout[morton2(2 * ri + px, 2 * rj + py)] = sacc;
    }

    // partials of the last step; after an abort, wait (bounded) for what was issued
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    bool ok = s_abort == 0;
    if (ok && n_steps > 0) {
        const int st = n_steps - 1;
        bool w_ok = *vabort == 0 && mbar_wait_bounded(&bar_mma[st & 1], (st >> 1) & 1);
        w_ok = __all_sync(0xffffffffu, w_ok);
        if (!w_ok) {
            atomicExch(&s_abort, 1);
            ok = false;
        } else {
            tc_fence_after();
            flush(st & 1);
        }
    }
    __syncthreads();
    if (s_abort) ok = false;
    if (!ok) {
        for (int st = max(0, issued_steps - 2); st < issued_steps; ++st)
            mbar_wait_bounded(&bar_mma[st & 1], (st >> 1) & 1);
        if (threadIdx.x == 0 && b_issued > 0)
            for (int st = max(0, b_issued - 2); st < b_issued; ++st) mbar_wait_bounded(&bar_b[st % 3], (st / 3) & 1);
    }
    if (ok) {
        if (valid) {
            float4* dst = reinterpret_cast<float4*>(out + (size_t)morton2(2 * ri + px, 2 * rj + py) * NP);
#pragma unroll
            for (int c = 0; c < 8; ++c) dst[c] = make_float4(acc[4 * c], acc[4 * c + 1], acc[4 * c + 2], acc[4 * c + 3]);
        }
    } else if (threadIdx.x == 0) {
        atomicExch(status, LFMM_ETIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kTc2Cols);
    }
}

// hi = TF32 round-to-nearest of x, lo = the same of the remainder (the A operand split
// of the shared-memory form), elementwise over n floats (n a multiple of 4)
__global__ void split_tf32_kernel(const float4* __restrict__ x, float4* __restrict__ hi, float4* __restrict__ lo,
                                  int64_t n4) {
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

}  // namespace

cudaError_t launch_split_tf32(const float* x, float* hi, float* lo, int64_t n, cudaStream_t s) {
    const int64_t n4 = n / 4;
    int64_t blocks = (n4 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    split_tf32_kernel<<<(int)blocks, 256, 0, s>>>(reinterpret_cast<const float4*>(x), reinterpret_cast<float4*>(hi),
                                                   reinterpret_cast<float4*>(lo), n4);
    return cudaGetLastError();
}

cudaError_t launch_m2l_tc_ss(const DeviceOps& ops, int k, int level, const float* qhi, const float* qlo,
                             const void* Q_level, const float* uhi, const float* ulo, const void* C_parent,
                             float* u_level, void* C_level, int* status, cudaStream_t s) {
    constexpr size_t smem = 1024 + sizeof(float) * (3 * 2 * 1024 + 2 * 2 * kTcThreads * 32);
    {
        cudaError_t e = ensure_dynamic_smem((const void*)m2l_tc_ss_kernel, smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t rows = (int64_t)1 << (2 * (level - 1));
    dim3 grid((unsigned)((rows + kTcThreads - 1) / kTcThreads), 4);
    m2l_tc_ss_kernel<<<grid, kTcThreads, smem, s>>>(level, qhi, qlo, uhi, ulo, (const float*)ops.tc[k],
                                                    (const float*)ops.mono[k], (const DFv*)Q_level,
                                                    (const DFv*)C_parent, u_level, (DFv*)C_level, status);
    return cudaGetLastError();
}

}  // namespace lfmm
