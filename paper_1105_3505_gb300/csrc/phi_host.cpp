// Host-side lattice fundamental solution phi (Sec. 3), used at plan time.
//
// Near the origin phi comes from Remark 3.1: integrating eq. 1.8 over t1 in closed
// form leaves the one-dimensional integral
//
//   phi(m) = (1/pi) int_0^pi (exp(-|m1| s(t)) cos(m2 t) - 1) / (2 sinh s(t)) dt,
//   cosh s = 2 - cos t   <=>   s = 2 asinh(sin(t/2)),  sinh s = 2 sin(t/2) sqrt(1 + sin^2(t/2)),
//
// whose integrand is analytic on [0, pi] (the numerator vanishes like t at 0).  We
// integrate it with a composite Gauss-Legendre rule, writing the numerator as
// e - 2 sin^2(m2 t / 2) (1 + e), e = expm1(-|m1| s), to avoid cancellation near t = 0, and
// take m1 = max(|m|), m2 = min(|m|) so the oscillatory factor is damped fastest.
// Far from the origin phi is the asymptotic expansion eq. 3.1 with its O(|m|^-6)
// remainder dropped, written in polar form:
//   phi ~ -(log r + gamma + 3/2 log 2)/(2 pi) + cos(4 theta)/(24 pi r^2)
//         + (25 cos(8 theta) + 18 cos(4 theta))/(480 pi r^4).
// (The r^-4 term of eq. 3.1 is this combination of cos 8theta and cos 4theta.)
#include <cmath>
#include <mutex>
#include <thread>

#include "lfmm_internal.h"

namespace lfmm {

namespace {
constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kEulerGamma = 0.577215664901532860606512090082402431;
}  // namespace

// Gauss-Legendre nodes/weights on [-1, 1]: Newton iteration on the three-term
// recurrence of the Legendre polynomials, started from Tricomi's approximation.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double pm1 = 1.0, p = z;  // P_0, P_1
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * z * p - (k - 1.0) * pm1) / k;
                pm1 = p;
                p = pk;
            }
            dp = n * (z * p - pm1) / (z * z - 1.0);
            double dz = p / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        {
            double pm1 = 1.0, p = z;
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * z * p - (k - 1.0) * pm1) / k;
                pm1 = p;
                p = pk;
            }
            dp = n * (z * p - pm1) / (z * z - 1.0);
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

namespace {

struct Neumaier {
    double s = 0.0, c = 0.0;
    void add(double v) {
        double t = s + v;
        if (std::fabs(s) >= std::fabs(v)) c += (s - t) + v;
        else c += (v - t) + s;
        s = t;
    }
    double value() const { return s + c; }
};

}  // namespace

std::vector<double> compute_phi_octant(int R) {
    // Composite rule: panels of width pi/n_panels with 24 nodes each, three panels
    // per period of cos(m2 t) at the largest m2 = R.
    const int n_gl = 24;
    const int n_panels = std::max(32, (3 * R) / 2);
    std::vector<double> gx, gw;
    gauss_legendre(n_gl, gx, gw);
    const int nn = n_gl * n_panels;
    std::vector<double> t(nn), s(nn), wden(nn);
    const double hw = 0.5 * kPi / n_panels;
    for (int p = 0; p < n_panels; ++p) {
        const double mid = (p + 0.5) * (kPi / n_panels);
        for (int i = 0; i < n_gl; ++i) {
            const int k = p * n_gl + i;
            t[k] = mid + hw * gx[i];
            const double h = std::sin(0.5 * t[k]);
            s[k] = 2.0 * std::asinh(h);
            // weight / (2 sinh s) and the leading 1/pi
            wden[k] = (hw * gw[i]) / (4.0 * h * std::sqrt(1.0 + h * h)) / kPi;
        }
    }
    const size_t size = (size_t)(R + 1) * (R + 2) / 2;
    std::vector<double> out(size, 0.0);
    unsigned nthreads = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    auto work = [&](unsigned tid) {
        std::vector<double> em(nn);
        for (int hi = (int)tid; hi <= R; hi += (int)nthreads) {
            for (int k = 0; k < nn; ++k) em[k] = std::expm1(-(double)hi * s[k]);
            for (int lo = 0; lo <= hi; ++lo) {
                if (hi == 0) {
                    out[0] = 0.0;
                    continue;
                }
                // exp(-a) cos(b) - 1 = em - 2 sin^2(b/2) (1 + em),  em = expm1(-a)
                Neumaier acc;
                for (int k = 0; k < nn; ++k) {
                    const double sh = std::sin(0.5 * lo * t[k]);
                    acc.add(wden[k] * (em[k] - 2.0 * sh * sh * (1.0 + em[k])));
                }
                out[(size_t)hi * (hi + 1) / 2 + lo] = acc.value();
            }
        }
    };
    std::vector<std::thread> pool;
    for (unsigned i = 0; i < nthreads; ++i) pool.emplace_back(work, i);
    for (auto& th : pool) th.join();
    return out;
}

const std::vector<double>& phi_host_table() {
    static std::once_flag once;
    static std::vector<double> table;
    std::call_once(once, [] { table = compute_phi_octant(kPhiHostRadius); });
    return table;
}

double phi_asym_host(double m1, double m2) {
    const double r2 = m1 * m1 + m2 * m2;
    const double inv_r2 = 1.0 / r2;
    // cos(4 theta) = Re((m1 + i m2)^4) / r^4
    const double re2 = m1 * m1 - m2 * m2, im2 = 2.0 * m1 * m2;
    const double c4 = (re2 * re2 - im2 * im2) * inv_r2 * inv_r2;
    const double c8 = 2.0 * c4 * c4 - 1.0;
    return -(0.5 * std::log(r2) + kEulerGamma + 1.5 * std::log(2.0)) / (2.0 * kPi)
           + c4 * inv_r2 / (24.0 * kPi)
           + (25.0 * c8 + 18.0 * c4) * inv_r2 * inv_r2 / (480.0 * kPi);
}

double phi_host(int64_t dx, int64_t dy) {
    int64_t a = dx < 0 ? -dx : dx, b = dy < 0 ? -dy : dy;
    int64_t hi = a > b ? a : b, lo = a > b ? b : a;
    if (hi <= kPhiHostRadius) return phi_host_table()[(size_t)hi * (hi + 1) / 2 + lo];
    return phi_asym_host((double)dx, (double)dy);
}

}  // namespace lfmm
