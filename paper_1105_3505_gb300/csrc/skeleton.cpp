// Skeletons and translation operators of the per-level model boxes (Sec. 5, 7, 8.1).
//
// Leaf level (side s): the candidate skeleton is the set Y of lattice points on the
// boundary of the box [0,s)^2 (Sec. 5).  A pivoted (Businger-Golub) Householder QR of
// A^{F,Y}, F the proxy ring, picks P columns; the dense-leaf operator of Remark 8.2,
// T_ofs (P x s^2), solves the least-squares problem eq. 5.1 for every lattice point of
// the box.  If the box has at most P points, the skeleton is all of them and T_ofs = I.
//
// Level k above the leaf (side 2^k s): candidates are the four children's skeletons,
// shifted into the quadrants of the model box (Sec. 8.1, step 3); the same QR picks P
// of them and the least-squares solution S (P x 4P_child) gives T_ofo = column blocks
// of S and T_ifi = their transposes (Sec. 7).
//
// Proxy ring: lattice points on the boundary of [-s, 2s-1]^2, i.e. the outer edge of
// the 3x3 block of same-level boxes around the model box.  Every box on the
// interaction list lies strictly outside it and the box itself strictly inside, so
// matching potentials there reproduces the far field outward (outgoing expansion)
// and the incoming field inward (Sec. 4.2 well-separatedness, 6a = 3 box sides).
// Per edge, `ppe` evenly spaced points are kept (all of them if the edge is shorter);
// the remark of Sec. 5 reports 40 per edge enough for 1e-10.
//
// M2L (T_ifo) for box offset o (in box sides) is phi sampled between skeletons
// (Sec. 7, Sec. 8.1 step 4): T[p][q] = phi(skel_p - skel_q - o*side).  The 40 offsets
// are all (ox, oy) in [-3,3]^2 outside [-1,1]^2: the distinct relative positions of
// interaction-list boxes under Def. 6.1 (the "42" printed in Sec. 8.1 step 4 counts
// more than Def. 6.1 allows).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <tuple>

#include "lfmm_internal.h"

namespace lfmm {

OffsetTable::OffsetTable() {
    int n = 0;
    for (int i = 0; i < 49; ++i) index[i] = -1;
    for (int oy = -3; oy <= 3; ++oy)
        for (int ox = -3; ox <= 3; ++ox) {
            if (std::abs(ox) <= 1 && std::abs(oy) <= 1) continue;
            this->ox[n] = ox;
            this->oy[n] = oy;
            index[(oy + 3) * 7 + (ox + 3)] = n;
            ++n;
        }
}

const OffsetTable& offsets() {
    static const OffsetTable t;
    return t;
}

namespace {

using Pt = std::array<int, 2>;

struct Mat {  // column-major
    int m = 0, n = 0;
    std::vector<double> a;
    Mat() = default;
    Mat(int m_, int n_) : m(m_), n(n_), a((size_t)m_ * n_, 0.0) {}
    double& operator()(int i, int j) { return a[(size_t)j * m + i]; }
    double operator()(int i, int j) const { return a[(size_t)j * m + i]; }
};

std::vector<Pt> proxy_ring(int side, int ppe) {
    const int a = -side, b = 2 * side - 1, len = b - a;
    const int n = std::min(ppe, len);
    std::vector<Pt> out;
    out.reserve(4 * n);
    for (int e = 0; e < 4; ++e)
        for (int i = 0; i < n; ++i) {
            const int pos = a + (int)std::llround((double)i * len / n);
            const int rev = a + b - pos;
            switch (e) {
                case 0: out.push_back({pos, a}); break;
                case 1: out.push_back({b, pos}); break;
                case 2: out.push_back({rev, b}); break;
                default: out.push_back({a, rev}); break;
            }
        }
    return out;
}

std::vector<Pt> box_boundary(int s) {
    std::vector<Pt> out;
    if (s == 1) return {{0, 0}};
    for (int x = 0; x < s; ++x) out.push_back({x, 0});
    for (int y = 1; y < s; ++y) out.push_back({s - 1, y});
    for (int x = s - 2; x >= 0; --x) out.push_back({x, s - 1});
    for (int y = s - 2; y >= 1; --y) out.push_back({0, y});
    return out;
}

Mat kernel_matrix(const std::vector<Pt>& F, const std::vector<Pt>& Y) {
    Mat A((int)F.size(), (int)Y.size());
    for (int j = 0; j < A.n; ++j)
        for (int i = 0; i < A.m; ++i)
            A(i, j) = phi_host((int64_t)F[i][0] - Y[j][0], (int64_t)F[i][1] - Y[j][1]);
    return A;
}

// Householder QR with column pivoting on A (in place), stopping after kmax steps or
// when the largest remaining column norm drops below rtol times the first one.
struct PivotedQR {
    Mat A;                    // R above the diagonal, Householder vectors below
    std::vector<double> tau;
    std::vector<int> piv;     // column order
    int rank = 0;
};

PivotedQR pivoted_qr(Mat A, int kmax, double rtol) {
    PivotedQR q;
    const int m = A.m, n = A.n;
    q.piv.resize(n);
    std::iota(q.piv.begin(), q.piv.end(), 0);
    const int kend = std::min(kmax, std::min(m, n));
    double norm0 = 0.0;
    int k = 0;
    for (; k < kend; ++k) {
        int best = k;
        double bestv = -1.0;
        for (int j = k; j < n; ++j) {
            double s = 0.0;
            for (int i = k; i < m; ++i) s += A(i, j) * A(i, j);
            if (s > bestv) {
                bestv = s;
                best = j;
            }
        }
        const double bn = std::sqrt(bestv);
        if (k == 0) norm0 = bn;
        if (bn == 0.0 || bn <= rtol * norm0) break;
        if (best != k) {
            for (int i = 0; i < m; ++i) std::swap(A(i, k), A(i, best));
            std::swap(q.piv[k], q.piv[best]);
        }
        const double x0 = A(k, k);
        const double beta = -std::copysign(bn, x0);
        const double v0 = x0 - beta;
        for (int i = k + 1; i < m; ++i) A(i, k) /= v0;
        const double t = (beta - x0) / beta;
        A(k, k) = beta;
        q.tau.push_back(t);
        for (int j = k + 1; j < n; ++j) {
            double d = A(k, j);
            for (int i = k + 1; i < m; ++i) d += A(i, k) * A(i, j);
            d *= t;
            A(k, j) -= d;
            for (int i = k + 1; i < m; ++i) A(i, j) -= d * A(i, k);
        }
    }
    q.rank = k;
    q.A = std::move(A);
    return q;
}

// X (rank x nb) minimising || A[:, piv[:rank]] X - B ||_2  (row-major result)
std::vector<double> least_squares(const PivotedQR& q, Mat B) {
    const int m = q.A.m, r = q.rank;
    for (int k = 0; k < r; ++k)
        for (int j = 0; j < B.n; ++j) {
            double d = B(k, j);
            for (int i = k + 1; i < m; ++i) d += q.A(i, k) * B(i, j);
            d *= q.tau[k];
            B(k, j) -= d;
            for (int i = k + 1; i < m; ++i) B(i, j) -= d * q.A(i, k);
        }
    std::vector<double> X((size_t)r * B.n, 0.0);
    for (int j = 0; j < B.n; ++j)
        for (int i = r - 1; i >= 0; --i) {
            double v = B(i, j);
            for (int l = i + 1; l < r; ++l) v -= q.A(i, l) * X[(size_t)l * B.n + j];
            X[(size_t)i * B.n + j] = v / q.A(i, i);
        }
    return X;
}

constexpr double kRankTol = 1e-14;

void build_leaf(ModelOps& mo) {
    const int s = mo.leaf_side, P = mo.P_target;
    LevelOps lv;
    lv.side = s;
    std::vector<Pt> all;
    for (int y = 0; y < s; ++y)
        for (int x = 0; x < s; ++x) all.push_back({x, y});
    if (s * s <= P) {
        lv.P = s * s;
        for (auto& p : all) {
            lv.skel.push_back(p[0]);
            lv.skel.push_back(p[1]);
        }
        mo.tofs.assign((size_t)lv.P * s * s, 0.0);
        for (int i = 0; i < lv.P; ++i) mo.tofs[(size_t)i * s * s + i] = 1.0;
    } else {
        const std::vector<Pt> Y = box_boundary(s);
        const std::vector<Pt> F = proxy_ring(s, mo.ppe);
        PivotedQR q = pivoted_qr(kernel_matrix(F, Y), P, kRankTol);
        lv.P = q.rank;
        for (int i = 0; i < q.rank; ++i) {
            lv.skel.push_back(Y[q.piv[i]][0]);
            lv.skel.push_back(Y[q.piv[i]][1]);
        }
        mo.tofs = least_squares(q, kernel_matrix(F, all));
    }
    mo.levels.push_back(std::move(lv));
}

void build_level(ModelOps& mo) {
    const LevelOps& ch = mo.levels.back();
    LevelOps lv;
    lv.side = 2 * ch.side;
    std::vector<Pt> Y;
    for (int c = 0; c < 4; ++c) {
        const int dx = (c & 1) * ch.side, dy = (c >> 1) * ch.side;
        for (int q = 0; q < ch.P; ++q) Y.push_back({ch.skel[2 * q] + dx, ch.skel[2 * q + 1] + dy});
    }
    const std::vector<Pt> F = proxy_ring(lv.side, mo.ppe);
    Mat A = kernel_matrix(F, Y);
    PivotedQR q = pivoted_qr(A, mo.P_target, kRankTol);
    lv.P = q.rank;
    for (int i = 0; i < q.rank; ++i) {
        lv.skel.push_back(Y[q.piv[i]][0]);
        lv.skel.push_back(Y[q.piv[i]][1]);
    }
    lv.S = least_squares(q, std::move(A));
    mo.levels.push_back(std::move(lv));
}

std::mutex g_cache_mu;
std::map<std::tuple<int, int, int>, std::unique_ptr<ModelOps>> g_cache;

}  // namespace

void tifo_matrix(const LevelOps& lv, int o, std::vector<double>& out) {
    const OffsetTable& ot = offsets();
    const int64_t ox = (int64_t)ot.ox[o] * lv.side, oy = (int64_t)ot.oy[o] * lv.side;
    out.assign((size_t)lv.P * lv.P, 0.0);
    for (int p = 0; p < lv.P; ++p)
        for (int q = 0; q < lv.P; ++q)
            out[(size_t)p * lv.P + q] =
                phi_host(lv.skel[2 * p] - lv.skel[2 * q] - ox, lv.skel[2 * p + 1] - lv.skel[2 * q + 1] - oy);
}

ModelOps* get_model_ops(int leaf_side, int P, int ppe, int n_levels, std::string* err) {
    if (leaf_side < 1 || leaf_side > kMaxLeafSide || (leaf_side & (leaf_side - 1)) ||
        P < 1 || P > kMaxP || ppe < 8 || n_levels < 1 || n_levels > 31) {
        if (err) *err = "invalid model-box parameters";
        return nullptr;
    }
    ModelOps* mo;
    {
        std::lock_guard<std::mutex> g(g_cache_mu);
        auto& slot = g_cache[{leaf_side, P, ppe}];
        if (!slot) {
            slot.reset(new ModelOps());
            slot->leaf_side = leaf_side;
            slot->P_target = P;
            slot->ppe = ppe;
        }
        mo = slot.get();
    }
    std::lock_guard<std::mutex> g(mo->mu);
    if (mo->levels.empty()) build_leaf(*mo);
    while ((int)mo->levels.size() < n_levels) build_level(*mo);
    return mo;
}

// ------------------------------------------------------------------ device upload

namespace {

// TF32 with round-to-nearest (ties away): keep 10 explicit mantissa bits.
float tf32_rna(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

// Tensor-core B operand of one operator for K-block h (k in [32h, 32h + 32)): the
// operator's value(n, k) (n = output p < NP) split into TF32 hi and lo and stacked as one
// K-major matrix of 2 NP rows (hi rows, then lo rows) x 32 K in fp32, laid out as the
// 128-byte-swizzled shared-memory image (row r at 128 r bytes, 16-byte chunk c of the
// row at chunk c ^ (r mod 8)).  NP / 32 such blocks per operator, block h at
// dst + h * 64 NP floats.
template <typename F>
void write_tc_tile(float* dst, int NP, int rows, int cols, F value) {
    for (int h = 0; h < NP / 32; ++h) {
        float* blk = dst + (size_t)h * 64 * NP;
        for (int n = 0; n < NP; ++n)
            for (int k = 0; k < 32; ++k) {
                const int kg = 32 * h + k;
                const float v = (n < rows && kg < cols) ? (float)value(n, kg) : 0.0f;
                const float hv = tf32_rna(v);
                const float lv = tf32_rna(v - hv);
                const size_t sw = ((size_t)(((k >> 2) ^ (n & 7)) << 2)) + (k & 3);  // (NP + n) & 7 == n & 7
                blk[(size_t)n * 32 + sw] = hv;
                blk[(size_t)(NP + n) * 32 + sw] = lv;
            }
    }
}

template <typename T>
void fill_device_image(const ModelOps& mo, int NP, int n_levels, int H, int W,
                       std::vector<T>& img, size_t& off_tofs, size_t& off_tab,
                       std::vector<size_t>& off_m2m, std::vector<size_t>& off_l2l,
                       std::vector<size_t>& off_tifo, std::vector<size_t>& off_mono,
                       std::vector<size_t>& off_tc) {
    const int s = mo.leaf_side;
    auto align = [](size_t v) { return (v + 31) & ~(size_t)31; };  // 128/256-byte aligned blocks
    size_t n = 0;
    off_tofs = n;
    n = align(n + (size_t)s * s * NP);
    off_tab = n;
    n = align(n + (size_t)(2 * H + 1) * W + 2);
    off_m2m.assign(n_levels, 0);
    off_l2l.assign(n_levels, 0);
    off_tifo.assign(n_levels, 0);
    off_mono.assign(n_levels, 0);
    off_tc.assign(n_levels, 0);
    const bool tc = sizeof(T) == 4 && (NP == 32 || NP == 64);
    for (int k = 0; k < n_levels; ++k) {
        if (tc) {
            n = (n + 255) & ~(size_t)255;  // 1 KB aligned tiles
            off_tc[k] = n;
            n += (size_t)(kNumOffsets + 4) * 2 * NP * NP;  // per operator NP / 32 blocks of 64 NP floats
        }
        off_mono[k] = n;
        n = align(n + (size_t)2 * kNumOffsets);
        if (k >= 1) {
            off_m2m[k] = n;
            n = align(n + (size_t)4 * NP * NP);
            off_l2l[k] = n;
            n = align(n + (size_t)4 * NP * NP);
        }
        off_tifo[k] = n;
        n = align(n + (size_t)kNumOffsets * NP * NP);
    }
    img.assign(n, T(0));
    // leaf T_ofs, transposed: tofsT[J][p]
    const LevelOps& leaf = mo.levels[0];
    for (int p = 0; p < leaf.P; ++p)
        for (int J = 0; J < s * s; ++J)
            img[off_tofs + (size_t)J * NP + p] = (T)mo.tofs[(size_t)p * s * s + J];
    // P2P table: entry (dx, dy), |dx|,|dy| <= H, at (dy + H) * W + (dx + H), deflated by
    // phi0 = phi(s, 0) (about the middle of the near-field range); phi0 times the charge of
    // the 3x3 leaf block is added back in the compensated channel.  phi0 as (hi, lo) after
    // the table.
    const double phi0 = phi_host(s, 0);
    for (int dy = -H; dy <= H; ++dy)
        for (int dx = -H; dx <= H; ++dx)
            img[off_tab + (size_t)(dy + H) * W + (dx + H)] = (T)(phi_host(dx, dy) - phi0);
    {
        const size_t e = off_tab + (size_t)(2 * H + 1) * W;
        const T hi = (T)phi0;
        img[e] = hi;
        img[e + 1] = (T)(phi0 - (double)hi);
    }
    std::vector<double> t;
    for (int k = 0; k < n_levels; ++k) {
        const LevelOps& lv = mo.levels[k];
        if (k >= 1) {
            const LevelOps& ch = mo.levels[k - 1];
            const int cols = 4 * ch.P;
            for (int c = 0; c < 4; ++c)
                for (int q = 0; q < ch.P; ++q)
                    for (int p = 0; p < lv.P; ++p) {
                        const double v = lv.S[(size_t)p * cols + c * ch.P + q];
                        img[off_m2m[k] + (size_t)(c * NP + q) * NP + p] = (T)v;   // [c*NP+q][p]
                        img[off_l2l[k] + ((size_t)c * NP + p) * NP + q] = (T)v;   // [c][p_par][q_child]
                    }
        }
        // Deflated M2L: T_ifo minus its centre-to-centre value c_o = phi(o * side).  The
        // removed rank-one part c_o 1 1^T acts on a box's total charge Q; the kernels
        // carry c_o * Q in a compensated scalar channel (values ~|Q| that cancel across
        // boxes and levels), so rounding of the expansions only meets the small remainder.
        const OffsetTable& ot = offsets();
        for (int o = 0; o < kNumOffsets; ++o) {
            tifo_matrix(lv, o, t);
            const double c = phi_host((int64_t)ot.ox[o] * lv.side, (int64_t)ot.oy[o] * lv.side);
            const T hi = (T)c;
            img[off_mono[k] + o] = hi;
            img[off_mono[k] + kNumOffsets + o] = (T)(c - (double)hi);
            for (int p = 0; p < lv.P; ++p)
                for (int q = 0; q < lv.P; ++q)
                    img[off_tifo[k] + ((size_t)o * NP + q) * NP + p] = (T)(t[(size_t)p * lv.P + q] - c);
            if (tc) {
                float* base = reinterpret_cast<float*>(img.data() + off_tc[k]) + (size_t)o * 2 * NP * NP;
                write_tc_tile(base, NP, lv.P, lv.P, [&](int n_, int k_) { return t[(size_t)n_ * lv.P + k_] - c; });
            }
        }
        // tensor-core L2L tiles for class c: B[n = child p][k = parent q] = S_{k+1}[q][c P_k + p]
        if (tc && k + 1 < (int)mo.levels.size() && k + 1 < n_levels) {
            const LevelOps& par = mo.levels[k + 1];
            for (int c = 0; c < 4; ++c) {
                float* base = reinterpret_cast<float*>(img.data() + off_tc[k]) + (size_t)(kNumOffsets + c) * 2 * NP * NP;
                write_tc_tile(base, NP, lv.P, par.P, [&](int n_, int k_) {
                    return par.S[(size_t)k_ * (4 * lv.P) + c * lv.P + n_];
                });
            }
        }
    }
}

}  // namespace

const DeviceOps* get_device_ops(ModelOps* mo, int precision, int NP, int n_levels,
                                cudaStream_t stream, std::string* err) {
    std::lock_guard<std::mutex> g(mo->mu);
    while ((int)mo->levels.size() < n_levels) build_level(*mo);
    auto& slot = mo->dev[precision == LFMM_MIXED ? 1 : (precision == LFMM_DF ? 2 : 0)][NP == 64 ? 1 : 0];
    if (slot && slot->n_levels >= n_levels) return slot.get();
    const int nl = std::max(n_levels, slot ? slot->n_levels : 0);
    std::unique_ptr<DeviceOps> d(new DeviceOps());
    d->NP = NP;
    d->precision = precision;
    d->n_levels = nl;
    d->leaf_side = mo->leaf_side;
    d->tab_H = 2 * mo->leaf_side - 1;
    // row width: at least 2H+1, and 16 mod 32 so that targets in the same column but in
    // rows of different parity fall in different shared-memory banks
    d->tab_W = 16;
    while (d->tab_W < 2 * d->tab_H + 1) d->tab_W += 32;
    size_t off_tofs, off_tab;
    std::vector<size_t> om, ol, ot, omono, otc;
    std::vector<char> bytes;
    size_t elem;
    if (precision == LFMM_MIXED) {
        std::vector<float> img;
        fill_device_image<float>(*mo, NP, nl, d->tab_H, d->tab_W, img, off_tofs, off_tab, om, ol, ot, omono, otc);
        elem = sizeof(float);
        bytes.assign((const char*)img.data(), (const char*)img.data() + img.size() * elem);
    } else if (precision == LFMM_DF) {
        std::vector<DF> img;
        fill_device_image<DF>(*mo, NP, nl, d->tab_H, d->tab_W, img, off_tofs, off_tab, om, ol, ot, omono, otc);
        elem = sizeof(DF);
        bytes.assign((const char*)img.data(), (const char*)img.data() + img.size() * elem);
    } else {
        std::vector<double> img;
        fill_device_image<double>(*mo, NP, nl, d->tab_H, d->tab_W, img, off_tofs, off_tab, om, ol, ot, omono, otc);
        elem = sizeof(double);
        bytes.assign((const char*)img.data(), (const char*)img.data() + img.size() * elem);
    }
    d->bytes = bytes.size();
    cudaError_t e = cudaMalloc(&d->base, d->bytes);
    if (e != cudaSuccess) {
        if (err) *err = std::string("cudaMalloc(operators): ") + cudaGetErrorString(e);
        return nullptr;
    }
    e = cudaMemcpyAsync(d->base, bytes.data(), d->bytes, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        cudaFree(d->base);
        if (err) *err = std::string("upload(operators): ") + cudaGetErrorString(e);
        return nullptr;
    }
    char* b = (char*)d->base;
    d->tofsT = b + off_tofs * elem;
    d->p2p_table = b + off_tab * elem;
    d->m2m.resize(nl);
    d->l2l.resize(nl);
    d->tifo.resize(nl);
    d->mono.resize(nl);
    d->tc.assign(nl, nullptr);
    for (int k = 0; k < nl; ++k) {
        if (precision == LFMM_MIXED && (NP == 32 || NP == 64)) d->tc[k] = b + otc[k] * elem;
        d->m2m[k] = k >= 1 ? b + om[k] * elem : nullptr;
        d->l2l[k] = k >= 1 ? b + ol[k] * elem : nullptr;
        d->tifo[k] = b + ot[k] * elem;
        d->mono[k] = b + omono[k] * elem;
    }
    if (slot) d->retired.push_back(slot.release());  // plans built earlier may still use it
    slot = std::move(d);
    return slot.get();
}

}  // namespace lfmm
