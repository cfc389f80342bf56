/* Brute-force lattice sum in binary64 (oracle; test infrastructure).
 *
 * Test infrastructure only: linked by tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py, never by the CUDA library, with which it shares
 * no code.
 *
 *   u_i = sum_j phi(x_i - y_j) f_j                       (eq. 1.7 / eq. 2.1)
 *
 * phi comes from an exact octant table (|m|_inf <= R, built by
 * oracle/phi_exact.py) and beyond it from the asymptotic expansion eq. 3.1 with
 * the O(|m|^-6) remainder dropped (Sec. 3.1; Euler's constant taken as
 * 0.5772156649015329, the printed 0.577206 being a typo).  phi(0) = 0, so a
 * source coinciding with a target contributes nothing (eq. 1.8).  Each target
 * is summed with Neumaier's compensated summation.
 *
 * The near-field variant restricts the sum to sources whose leaf is the
 * target's leaf or adjacent to it (eq. 2.2-2.4): leaf(x) = floor((x - x0)/s).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

static const double ORC_PI = 3.14159265358979323846264338327950288;
static const double ORC_EULER_GAMMA = 0.57721566490153286060651209008240243;

/* eq. 3.1 without the O(|m|^-6) remainder */
double orc_phi_asym(double m1, double m2) {
    const double a = m1 * m1, b = m2 * m2;
    const double r2 = a + b;
    const double r6 = r2 * r2 * r2;
    const double lead = -(0.5 * log(r2) + ORC_EULER_GAMMA + 0.5 * log(8.0)) / (2.0 * ORC_PI);
    const double t4 = (a * a - 6.0 * a * b + b * b) / (24.0 * ORC_PI * r6);
    const double t8 = (43.0 * a * a * a * a - 772.0 * a * a * a * b + 1570.0 * a * a * b * b
                       - 772.0 * a * b * b * b + 43.0 * b * b * b * b) / (480.0 * ORC_PI * r6 * r6);
    return lead + t4 + t8;
}

static inline double orc_phi(const double* oct, int64_t R, int64_t dx, int64_t dy) {
    int64_t ax = dx < 0 ? -dx : dx;
    int64_t ay = dy < 0 ? -dy : dy;
    int64_t hi = ax > ay ? ax : ay;
    int64_t lo = ax > ay ? ay : ax;
    if (hi <= R) return oct[hi * (hi + 1) / 2 + lo];
    return orc_phi_asym((double)dx, (double)dy);
}

static inline void neumaier_add(double* s, double* c, double x) {
    double t = *s + x;
    if (fabs(*s) >= fabs(x)) *c += (*s - t) + x;
    else *c += (x - t) + *s;
    *s = t;
}

/* phi at n points given as (dx, dy) pairs */
void orc_phi_many(const int64_t* d, int64_t n, const double* oct, int64_t R, double* out) {
    for (int64_t i = 0; i < n; i++) out[i] = orc_phi(oct, R, d[2 * i], d[2 * i + 1]);
}

/* u[i] = sum_j phi(tgt_i - src_j) f_j for i in [0, nt); xy arrays interleaved (x, y). */
void orc_lattice_sum(const int32_t* src, int64_t ns, const double* f,
                     const int32_t* tgt, int64_t nt,
                     const double* oct, int64_t R, double* u) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < nt; i++) {
        const int64_t tx = tgt[2 * i], ty = tgt[2 * i + 1];
        double s = 0.0, c = 0.0;
        for (int64_t j = 0; j < ns; j++) {
            const int64_t dx = tx - (int64_t)src[2 * j];
            const int64_t dy = ty - (int64_t)src[2 * j + 1];
            if (dx == 0 && dy == 0) continue; /* phi(0) = 0 */
            neumaier_add(&s, &c, orc_phi(oct, R, dx, dy) * f[j]);
        }
        u[i] = s + c;
    }
}

static inline int64_t floordiv(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
    return q;
}

/* Near-field part (eq. 2.2-2.4) for a uniform tree with leaf side s and root
 * corner (x0, y0): only pairs whose leaves coincide or are adjacent. */
void orc_near_sum(const int32_t* src, int64_t ns, const double* f,
                  const int32_t* tgt, int64_t nt,
                  int64_t x0, int64_t y0, int64_t s,
                  const double* oct, int64_t R, double* u) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < nt; i++) {
        const int64_t tx = tgt[2 * i], ty = tgt[2 * i + 1];
        const int64_t bx = floordiv(tx - x0, s), by = floordiv(ty - y0, s);
        double sum = 0.0, c = 0.0;
        for (int64_t j = 0; j < ns; j++) {
            const int64_t sx = src[2 * j], sy = src[2 * j + 1];
            const int64_t cx = floordiv(sx - x0, s), cy = floordiv(sy - y0, s);
            if (llabs(cx - bx) > 1 || llabs(cy - by) > 1) continue;
            const int64_t dx = tx - sx, dy = ty - sy;
            if (dx == 0 && dy == 0) continue;
            neumaier_add(&sum, &c, orc_phi(oct, R, dx, dy) * f[j]);
        }
        u[i] = sum + c;
    }
}

int orc_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
