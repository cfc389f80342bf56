// Lattice fundamental solution near the origin by two-dimensional quadrature on the
// GPU (Sec. 3.2), for any symmetric lattice operator with constant coefficients:
//
//   (A u)(m) = sum_k w_k (2 u(m) - u(m + d_k) - u(m - d_k)),   w_k > 0,
//   phi(m)   = (2 pi)^-2 int_{[-pi,pi]^2} (cos(m.t) - 1) / sigma(t) dt,
//   sigma(t) = sum_k 4 w_k sin^2(t.d_k / 2),
//
// so that A phi = delta_0 and phi(0) = 0 (eq. 1.8 for the 5-point operator of eq. 1.2:
// d = (1,0), (0,1), w = 1, 1).  Such operators have no closed recurrence in general; the
// quadrature needs only the symbol.  For a table entry m:
//   - the square is cut into n x n boxes, n the odd number >= |m|_inf (about one
//     oscillation of the integrand per box); the rings of boxes around the centre one
//     get a 20 x 20 Gauss-Legendre rule, the boxes from about three box sizes out (see
//     below) 14 x 14;
//   - the centre box [-a, a]^2, a = pi / n, is the sum of the annuli
//     Omega_j = [-a 2^-j, a 2^-j]^2 minus [-a 2^-j-1, a 2^-j-1]^2, j >= 0, each cut
//     into eight rectangles with a 20 x 20 rule; the integrand is bounded at 0 and its
//     expansion there is even in t, so the part left after J annuli is c1 4^-J +
//     c2 16^-J + ..., and Richardson extrapolation in powers of 4 accelerates the
//     partial sums.
// The rule on a piece converges at a rate set by how far the complex zeros of the
// symbol lie from it, relative to its size.  Near the origin those zeros are the zeros of
// the quadratic form t'Qt, Q = sum_k w_k d_k d_k', whose imaginary parts are c |t| with
// c = sqrt(det Q) / max(Q_11, Q_22) (c = 1 for the 5-point operator); along t1 alone the
// distance is set by c_x = sqrt(det Q) / Q_11, along t2 by c_y = sqrt(det Q) / Q_22.
// Every annulus piece is therefore split into ceil(1 / c_x) x ceil(1 / c_y)
// sub-rectangles, and an outer box in ring k around the centre (Chebyshev distance k
// boxes) into ceil(1 / (c_x (2k - 1))) x ceil(1 / (c_y (2k - 1))), which keeps the
// relative distance at least that of the 5-point operator with no splitting.  Operators
// with c < 1/8 (a split above 8, strongly anisotropic) are rejected.
// The numerator is written -2 sin^2(m.t / 2) and the symbol as a sum of squares, so
// neither loses digits near t = 0.  One block per table entry; binary64 throughout.
#include <algorithm>
#include <cmath>
#include <vector>

#include "lfmm_internal.h"

namespace lfmm {

namespace {

constexpr int kQuadMaxTerms = 8;
constexpr int kQuadNodes = 20;
constexpr int kQuadNodesFar = 14;  // boxes two or more rings away from the centre
constexpr int kQuadAnnuli = 16;
constexpr int kQuadThreads = 256;
constexpr int kQuadMaxSplit = 8;
constexpr double kPiQ = 3.1415926535897932384626433832795;
constexpr double kTwoPi = 2.0 * kPiQ;

struct QuadStencil {
    int n_terms;
    int dx[kQuadMaxTerms], dy[kQuadMaxTerms];
    double w[kQuadMaxTerms];
    double gx[kQuadNodes], gw[kQuadNodes];  // Gauss-Legendre on [-1, 1]
    double fx[kQuadNodesFar], fw[kQuadNodesFar];
    double c;                                // sqrt(det Q) / max(Q_11, Q_22)
    double cx, cy;                           // sqrt(det Q) / Q_11, sqrt(det Q) / Q_22
};

// splits per side of a piece whose distance from the origin is `dist` piece sizes
__device__ __forceinline__ int quad_split(double c, int dist) {
    return max(1, (int)ceil(1.0 / (c * dist) - 1e-12));
}

__device__ __forceinline__ double integrand(const QuadStencil& q, int m1, int m2, double t1, double t2) {
    double sig = 0.0;
    for (int k = 0; k < q.n_terms; ++k) {
        const double s = sin(0.5 * (t1 * q.dx[k] + t2 * q.dy[k]));
        sig += 4.0 * q.w[k] * s * s;
    }
    const double h = sin(0.5 * (t1 * m1 + t2 * m2));
    return -2.0 * h * h / sig;
}

// node `idx` of the s x s split of the rectangle [x0, x1] x [y0, y1], a Q-point
// Gauss-Legendre rule (nodes x, weights w) on each sub-rectangle: idx = (sub-rectangle)
// * Q^2 + (node)
template <int Q>
__device__ __forceinline__ double rect_node(const QuadStencil& q, const double* x, const double* w, int m1, int m2,
                                            double x0, double x1, double y0, double y1, int sx, int sy, int idx) {
    constexpr int NN = Q * Q;
    const int sub = idx / NN, node = idx % NN;
    const int si = sub % sx, sj = sub / sx, i = node % Q, j = node / Q;
    const double hx = 0.5 * (x1 - x0) / sx, hy = 0.5 * (y1 - y0) / sy;
    const double xa = x0 + 2.0 * hx * si, ya = y0 + 2.0 * hy * sj;
    const double t1 = xa + hx * (1.0 + x[i]), t2 = ya + hy * (1.0 + x[j]);
    return w[i] * w[j] * hx * hy * integrand(q, m1, m2, t1, t2);
}

__device__ double block_sum(double v, double* red) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kQuadThreads / 32; ++i) t += red[i];
    return t;  // valid in thread 0
}

__global__ void __launch_bounds__(kQuadThreads) phi_quad_kernel(const QuadStencil q, int R, double* __restrict__ out) {
    __shared__ double red[kQuadThreads / 32];
    __shared__ double s_ann[kQuadAnnuli];
    const int side = 2 * R + 1;
    const int e = blockIdx.x;
    const int m1 = e % side - R, m2 = e / side - R;
    if (m1 == 0 && m2 == 0) {
        if (threadIdx.x == 0) out[e] = 0.0;
        return;
    }
    const int mi = max(abs(m1), abs(m2));
    const int n = mi | 1;  // odd, >= |m|_inf
    const double h = kTwoPi / n;
    const int cb = (n - 1) / 2;  // the centre box, and the number of rings around it
    constexpr int NN = kQuadNodes * kQuadNodes;
    // boxes away from the centre: the rings closer than three box sizes (times c) to the
    // origin's complex zeros box by box with the 20-point rule (split as needed), the
    // rest in one flat loop with 14 points per side, which there reach the same accuracy
    // (the integrand is about one oscillation of the numerator wide and far from the
    // zeros).
    double outer = 0.0;
    int k_flat = 2;
    while (k_flat <= cb && q.c * (2 * k_flat - 1) < 3.0 - 1e-12) ++k_flat;
    for (int k = 1; k < k_flat && k <= cb; ++k) {
        const int sx = quad_split(q.cx, 2 * k - 1), sy = quad_split(q.cy, 2 * k - 1);
        for (int bj = cb - k; bj <= cb + k; ++bj)
            for (int bi = cb - k; bi <= cb + k; ++bi) {
                if (max(abs(bi - cb), abs(bj - cb)) != k) continue;
                const double x0 = -kPiQ + bi * h, y0 = -kPiQ + bj * h;
                for (int idx = threadIdx.x; idx < sx * sy * NN; idx += blockDim.x)
                    outer += rect_node<kQuadNodes>(q, q.gx, q.gw, m1, m2, x0, x0 + h, y0, y0 + h, sx, sy, idx);
            }
    }
    constexpr int NF = kQuadNodesFar * kQuadNodesFar;
    const int n_outer = n * n * NF;  // below 2^31: n <= 129
    for (int idx = threadIdx.x; idx < n_outer; idx += blockDim.x) {
        const int box = idx / NF, node = idx - box * NF;
        const int bi = box % n, bj = box / n;
        if (max(abs(bi - cb), abs(bj - cb)) < k_flat) continue;
        const double x0 = -kPiQ + bi * h, y0 = -kPiQ + bj * h;
        outer += rect_node<kQuadNodesFar>(q, q.fx, q.fw, m1, m2, x0, x0 + h, y0, y0 + h, 1, 1, node);
    }
    const double outer_sum = block_sum(outer, red);
    // annuli of the centre box, one partial sum per annulus
    const double a = 0.5 * h;
    const int sx0 = quad_split(q.cx, 1), sy0 = quad_split(q.cy, 1);
    const int per_piece = sx0 * sy0 * NN;
    for (int j = 0; j < kQuadAnnuli; ++j) {
        const double aj = ldexp(a, -j), bj = 0.5 * aj;
        double part = 0.0;
        for (int idx = threadIdx.x; idx < 8 * per_piece; idx += blockDim.x) {
            const int r = idx / per_piece;
            // the 3 x 3 grid of rectangles minus its centre: column r' % 3, row r' / 3
            const int rr = r < 4 ? r : r + 1;
            const double xs[4] = {-aj, -bj, bj, aj};
            const int ci = rr % 3, cj = rr / 3;
            part += rect_node<kQuadNodes>(q, q.gx, q.gw, m1, m2, xs[ci], xs[ci + 1], xs[cj], xs[cj + 1], sx0, sy0,
                                          idx % per_piece);
        }
        const double ps = block_sum(part, red);
        if (threadIdx.x == 0) s_ann[j] = ps;
    }
    if (threadIdx.x == 0) {
        // Richardson extrapolation of the partial sums S_J = sum_{j <= J} I_j, whose
        // errors are c1 4^-J + c2 16^-J + c3 64^-J + ...
        double T[kQuadAnnuli][5];
        double S = 0.0;
        for (int J = 0; J < kQuadAnnuli; ++J) {
            S += s_ann[J];
            T[J][0] = S;
            double p4 = 1.0;
            for (int k = 1; k < 5 && k <= J; ++k) {
                p4 *= 4.0;
                T[J][k] = T[J][k - 1] + (T[J][k - 1] - T[J - 1][k - 1]) / (p4 - 1.0);
            }
        }
        const double centre = T[kQuadAnnuli - 1][4];
        out[e] = (outer_sum + centre) / (kTwoPi * kTwoPi);
    }
}

}  // namespace

}  // namespace lfmm

extern "C" int lfmm_phi_quadrature(const int32_t* d, const double* w, int32_t n_terms, int32_t R, double* out,
                                   void* stream) {
    using namespace lfmm;
    if (!d || !w || !out) return fail(LFMM_EINVAL, "NULL argument");
    if (n_terms < 1 || n_terms > kQuadMaxTerms) return fail(LFMM_EINVAL, "n_terms must be in [1, 8]");
    if (R < 1 || R > 64) return fail(LFMM_EINVAL, "R must be in [1, 64]");
    QuadStencil q{};
    q.n_terms = n_terms;
    for (int k = 0; k < n_terms; ++k) {
        q.dx[k] = d[2 * k];
        q.dy[k] = d[2 * k + 1];
        q.w[k] = w[k];
        if (!(w[k] > 0.0)) return fail(LFMM_EINVAL, "conductivities must be > 0");
        if (q.dx[k] == 0 && q.dy[k] == 0) return fail(LFMM_EINVAL, "zero offset");
        if (std::abs(q.dx[k]) > 64 || std::abs(q.dy[k]) > 64) return fail(LFMM_EINVAL, "offsets must be in [-64, 64]");
    }
    // the symbol may vanish only at t = 0: the offsets must generate Z^2 (determinant
    // of some pair = +-1, a sufficient check for the stencils in use)
    bool spans = false;
    for (int a = 0; a < n_terms && !spans; ++a)
        for (int b = a + 1; b < n_terms && !spans; ++b)
            spans = std::abs(q.dx[a] * q.dy[b] - q.dy[a] * q.dx[b]) == 1;
    if (!spans) return fail(LFMM_EINVAL, "the offsets must include two with determinant +-1");
    double q11 = 0.0, q12 = 0.0, q22 = 0.0;  // Q = sum_k w_k d_k d_k'
    for (int k = 0; k < n_terms; ++k) {
        q11 += q.w[k] * q.dx[k] * q.dx[k];
        q12 += q.w[k] * q.dx[k] * q.dy[k];
        q22 += q.w[k] * q.dy[k] * q.dy[k];
    }
    q.c = std::sqrt(q11 * q22 - q12 * q12) / std::max(q11, q22);
    q.cx = std::sqrt(q11 * q22 - q12 * q12) / q11;
    q.cy = std::sqrt(q11 * q22 - q12 * q12) / q22;
    if (!(q.c * kQuadMaxSplit >= 1.0))
        return fail(LFMM_EINVAL, "operator too anisotropic for the quadrature (sqrt(det Q) / max(Q_11, Q_22) < 1/8)");
    std::vector<double> x, wt;
    gauss_legendre(kQuadNodes, x, wt);
    for (int i = 0; i < kQuadNodes; ++i) {
        q.gx[i] = x[i];
        q.gw[i] = wt[i];
    }
    gauss_legendre(kQuadNodesFar, x, wt);
    for (int i = 0; i < kQuadNodesFar; ++i) {
        q.fx[i] = x[i];
        q.fw[i] = wt[i];
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int side = 2 * R + 1;
    const size_t bytes = (size_t)side * side * sizeof(double);
    const bool dev = [&] {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, out) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
    }();
    double* d_out = out;
    if (!dev) LFMM_CUDA_TRY(dev_malloc((void**)&d_out, bytes, s));
    phi_quad_kernel<<<side * side, kQuadThreads, 0, s>>>(q, R, d_out);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !dev) {
        e = cudaMemcpyAsync(out, d_out, bytes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (!dev) cudaFreeAsync(d_out, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LFMM_ECUDA, std::string("phi quadrature: ") + cudaGetErrorString(e));
    }
    return LFMM_OK;
}
