// Host-side set-up: the lattice-crossing quadrature of Sec. 2.2 and the interpolation table
// of the smoothing functions of Eqs. (s1)-(s3).
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "ers_internal.h"

namespace ers {

// ------------------------------------------------------------------------------------------
// Quadrature (Sec. 2.2, Eq. (quadrature)).  For each axis k, the lattice lines parallel to
// e_k through the points (p h, q h) of the other two coordinates meet the ellipsoid in at most
// two points; a point belongs to Gamma_k when |n_k| >= cos(theta), theta = 70 degrees, and
// carries the weight psi_k(n)/|n_k| h^2, psi_k = beta_k / sum_j beta_j,
// beta_j = bump(arccos|n_j| / theta), bump(r) = exp(2 r^2 / (r^2 - 1)) for |r| < 1 else 0.
// Order: k ascending; the lattice index of the lower remaining axis; that of the upper one;
// the root with the smaller coordinate first.
// ------------------------------------------------------------------------------------------
int64_t quadrature(const double c[3], const double a[3], double h, std::vector<double> *xs,
                   std::vector<double> *ns, std::vector<double> *ws) {
    const double theta = 70.0 * M_PI / 180.0;
    const double cth = std::cos(theta);
    auto bump = [](double r) {
        if (!(std::fabs(r) < 1.0)) return 0.0;
        const double r2 = r * r;
        return std::exp(2.0 * r2 / (r2 - 1.0));
    };
    int64_t count = 0;
    for (int k = 0; k < 3; ++k) {
        const int ax[2] = {k == 0 ? 1 : 0, k == 2 ? 1 : 2};
        long lo[2], hi[2];
        for (int e = 0; e < 2; ++e) {
            lo[e] = (long)std::ceil((c[ax[e]] - a[ax[e]]) / h) - 1;
            hi[e] = (long)std::floor((c[ax[e]] + a[ax[e]]) / h) + 1;
        }
        for (long i = lo[0]; i <= hi[0]; ++i) {
            const double xp = (double)i * h;
            const double up = (xp - c[ax[0]]) / a[ax[0]];
            for (long j = lo[1]; j <= hi[1]; ++j) {
                const double xq = (double)j * h;
                const double uq = (xq - c[ax[1]]) / a[ax[1]];
                const double disc = 1.0 - up * up - uq * uq;
                if (!(disc > 0.0)) continue;
                const double half = a[k] * std::sqrt(disc);
                for (int side = -1; side <= 1; side += 2) {
                    double p[3];
                    p[ax[0]] = xp;
                    p[ax[1]] = xq;
                    p[k] = c[k] + side * half;
                    double g[3], gn = 0.0;
                    for (int m = 0; m < 3; ++m) {
                        g[m] = (p[m] - c[m]) / (a[m] * a[m]);
                        gn += g[m] * g[m];
                    }
                    gn = std::sqrt(gn);
                    double nv[3] = {g[0] / gn, g[1] / gn, g[2] / gn};
                    if (std::fabs(nv[k]) < cth) continue;
                    if (xs) {
                        double beta[3], bsum = 0.0;
                        for (int m = 0; m < 3; ++m) {
                            beta[m] = bump(std::acos(std::fabs(nv[m])) / theta);
                            bsum += beta[m];
                        }
                        xs->insert(xs->end(), p, p + 3);
                        ns->insert(ns->end(), nv, nv + 3);
                        ws->push_back(beta[k] / bsum / std::fabs(nv[k]) * h * h);
                    }
                    ++count;
                }
            }
        }
    }
    return count;
}

// ------------------------------------------------------------------------------------------
// sigma_p(tau) = s_p(t) / t^p with tau = t^2, p = 1, 3, 5 for s_1, s_2, s_3 of
// Eqs. (s1)-(s3).  These are entire functions of tau.  Evaluated in long double: by the
// power series in tau of erf(t)/t and of the exponential terms for t < 1/2, otherwise by the
// closed forms; then interpolated on each interval [i/16, (i+1)/16] at the 7 Chebyshev points
// and converted to a degree-6 polynomial in s = 32 tau - (2 i + 1).
// ------------------------------------------------------------------------------------------
namespace {

void sigma_ld(long double tau, long double out[3]) {
    const long double c = 2.0L / std::sqrt((long double)M_PI);
    const long double t = std::sqrt(tau);
    if (t < 0.5L) {
        // Term-by-term from erf(t) = c sum_n (-1)^n t^(2n+1) / (n! (2n+1)) and
        // e^{-t^2} = sum_n (-tau)^n / n!:
        //   s1/t   = c sum_{n>=0} (-tau)^n / (n! (2n+1))
        //   s2/t^3 = c sum_{n>=1} (-1)^(n+1) 2n / (n! (2n+1)) tau^(n-1)
        //   s3/t^5 = c sum_{n>=2} (-1)^n 4n(n-1) / (3 (2n+1) n!) tau^(n-2)
        long double a1 = 0, a2 = 0, a3 = 0;
        long double term = 1.0L;  // (-tau)^n / n!
        for (int n = 0; n < 40; ++n) {
            if (n > 0) term *= -tau / n;
            a1 += term / (2 * n + 1);
        }
        long double pw = 1.0L, fact = 1.0L;
        for (int n = 1; n < 40; ++n) {
            fact *= n;
            if (n > 1) pw *= tau;  // tau^(n-1)
            long double sgn = (n % 2 == 1) ? 1.0L : -1.0L;
            a2 += sgn * (2.0L * n) / (fact * (2 * n + 1)) * pw;
        }
        pw = 1.0L;
        fact = 2.0L;
        for (int n = 2; n < 40; ++n) {
            if (n > 2) {
                fact *= n;
                pw *= tau;  // tau^(n-2)
            }
            long double sgn = (n % 2 == 0) ? 1.0L : -1.0L;
            a3 += sgn * (4.0L * n * (n - 1)) / (3.0L * (2 * n + 1) * fact) * pw;
        }
        out[0] = c * a1;
        out[1] = c * a2;
        out[2] = c * a3;
        return;
    }
    const long double e = std::erf(t), g = std::exp(-tau);
    out[0] = e / t;
    out[1] = (e - c * t * g) / (t * tau);
    out[2] = (e - c * (t + 2.0L / 3.0L * t * tau) * g) / (t * tau * tau);
}

// sigma#_p(tau) = s#_p(t) / t^p for the modified smoothing functions of Sec. 2.1:
//   s#_1 = erf t + c/3 (5t - 2t^3) e^{-t^2},  s#_2 = erf t - c/3 (3t - 14t^3 + 4t^5) e^{-t^2},
//   s#_3 = erf t - c/9 (9t + 6t^3 - 4t^5) e^{-t^2},  c = 2/sqrt(pi).
// For t < 1 the series in tau: collecting the t^(2n+1) terms of erf t and of P(t) e^{-t^2},
//   s#_1/t   = c sum_{n>=0} (-tau)^n [1/(2n+1) + (5 + 2n)/3] / n!
//   s#_2/t^3 = c sum_{n>=1} (-1)^n tau^(n-1) [1/(2n+1) - (4n^2 + 10n + 3)/3] / n!
//   s#_3/t^5 = c sum_{n>=2} (-1)^n tau^(n-2) [1/(2n+1) - (9 - 2n - 4n^2)/9] / n!
void sigma_sharp_ld(long double tau, long double out[3]) {
    const long double c = 2.0L / std::sqrt((long double)M_PI);
    const long double t = std::sqrt(tau);
    if (t < 1.0L) {
        long double a1 = 0, a2 = 0, a3 = 0, fact = 1.0L;
        for (int n = 0; n < 50; ++n) {
            if (n > 0) fact *= n;
            const long double sg = (n % 2 == 0) ? 1.0L : -1.0L;
            const long double e = 1.0L / (2 * n + 1);
            a1 += sg * std::pow(tau, (long double)n) * (e + (5.0L + 2 * n) / 3.0L) / fact;
            if (n >= 1) a2 += sg * std::pow(tau, (long double)(n - 1)) * (e - (4.0L * n * n + 10.0L * n + 3.0L) / 3.0L) / fact;
            if (n >= 2) a3 += sg * std::pow(tau, (long double)(n - 2)) * (e - (9.0L - 2.0L * n - 4.0L * n * n) / 9.0L) / fact;
        }
        out[0] = c * a1;
        out[1] = c * a2;
        out[2] = c * a3;
        return;
    }
    const long double e = std::erf(t), g = std::exp(-tau);
    out[0] = (e + c / 3.0L * (5.0L * t - 2.0L * t * tau) * g) / t;
    out[1] = (e - c / 3.0L * (3.0L * t - 14.0L * t * tau + 4.0L * t * tau * tau) * g) / (t * tau);
    out[2] = (e - c / 9.0L * (9.0L * t + 6.0L * t * tau - 4.0L * t * tau * tau) * g) / (t * tau * tau);
}

std::vector<double> build_table(int nint, int inv_w, void (*fn)(long double, long double[3])) {
    std::vector<double> tab((size_t)nint * 3 * TAB_NC);
    const int D = TAB_DEG;
    long double sk[TAB_NC];
    for (int k = 0; k <= D; ++k) sk[k] = std::cos((2.0L * k + 1.0L) * (long double)M_PI / (2.0L * (D + 1)));
    for (int i = 0; i < nint; ++i) {
        long double f[3][TAB_NC];
        for (int k = 0; k <= D; ++k) {
            long double tau = ((long double)sk[k] + 2.0L * i + 1.0L) / (2.0L * inv_w);
            long double o[3];
            fn(tau, o);
            for (int p = 0; p < 3; ++p) f[p][k] = o[p];
        }
        for (int p = 0; p < 3; ++p) {
            // Chebyshev coefficients
            long double ch[TAB_NC];
            for (int j = 0; j <= D; ++j) {
                long double s = 0;
                for (int k = 0; k <= D; ++k)
                    s += f[p][k] * std::cos(j * (2.0L * k + 1.0L) * (long double)M_PI / (2.0L * (D + 1)));
                ch[j] = s * 2.0L / (D + 1);
            }
            ch[0] *= 0.5L;
            // monomial coefficients: T_0 = 1, T_1 = s, T_{j+1} = 2 s T_j - T_{j-1}
            long double Tm[TAB_NC][TAB_NC];
            std::memset(Tm, 0, sizeof Tm);
            Tm[0][0] = 1;
            Tm[1][1] = 1;
            for (int j = 1; j < D; ++j)
                for (int e = 0; e <= D; ++e)
                    Tm[j + 1][e] = (e > 0 ? 2 * Tm[j][e - 1] : 0) - Tm[j - 1][e];
            long double mono[TAB_NC] = {0};
            for (int j = 0; j <= D; ++j)
                for (int e = 0; e <= D; ++e) mono[e] += ch[j] * Tm[j][e];
            for (int e = 0; e <= D; ++e) tab[((size_t)i * 3 + p) * TAB_NC + e] = (double)mono[D - e];
        }
    }
    return tab;
}

}  // namespace

const double *sigma_table_host() {
    static std::vector<double> tab = build_table(TAB_N, TAB_INV_W, sigma_ld);
    return tab.data();
}

const double *sigma_sharp_table_host() {
    static std::vector<double> tab = build_table(SH_N, SH_INV_W, sigma_sharp_ld);
    return tab.data();
}

namespace {
// Device copy: per interval i and function p three float4:
//   (c6, c5, c4, 2 i + 1), (c3 hi, c3 lo, c2 hi, c2 lo), (c1 hi, c1 lo, c0 hi, c0 lo),
// degrees 6..4 as floats, degrees 3..0 as float pairs (hi = the coefficient rounded to a float,
// lo = the rest rounded to a float: hi + lo carries the coefficient to ~2^-48).
void device_layout(const double *h, int nint, void *dst) {
    float *f = static_cast<float *>(dst);
    for (int i = 0; i < nint; ++i)
        for (int p = 0; p < 3; ++p) {
            const double *c = h + ((size_t)i * 3 + p) * TAB_NC;  // degrees 6..0
            float *q = f + ((size_t)i * 3 + p) * 12;
            q[0] = (float)c[0];
            q[1] = (float)c[1];
            q[2] = (float)c[2];
            q[3] = (float)(2 * i + 1);
            for (int e = 0; e < 4; ++e) {
                const float hi = (float)c[3 + e];
                q[4 + 2 * e] = hi;
                q[5 + 2 * e] = (float)(c[3 + e] - (double)hi);
            }
        }
}
}  // namespace

void sigma_table_device_layout(void *dst) { device_layout(sigma_table_host(), TAB_N, dst); }
void sigma_sharp_table_device_layout(void *dst) { device_layout(sigma_sharp_table_host(), SH_N, dst); }

}  // namespace ers

// Test hook (not in the public header): copy of the host table for inspection.
extern "C" int ers_debug_sigma_table(double *out, int64_t count) {
    const int64_t n = (int64_t)ers::TAB_N * 3 * ers::TAB_NC;
    if (!out || count < n) return ERS_E_INVAL;
    std::memcpy(out, ers::sigma_table_host(), sizeof(double) * n);
    return ERS_OK;
}

// Test hook (not in the public header): the device layout of the table (TAB_DEV_BYTES bytes).
extern "C" int ers_debug_sigma_device(void *out, int64_t bytes) {
    if (!out || bytes < (int64_t)ers::TAB_DEV_BYTES) return ERS_E_INVAL;
    ers::sigma_table_device_layout(out);
    return ERS_OK;
}

// Test hook (not in the public header): the device layout of the on-surface table
// (SH_DEV_BYTES bytes).
extern "C" int ers_debug_sigma_sharp_device(void *out, int64_t bytes) {
    if (!out || bytes < (int64_t)ers::SH_DEV_BYTES) return ERS_E_INVAL;
    ers::sigma_sharp_table_device_layout(out);
    return ERS_OK;
}

// Test hook (not in the public header): the host quadrature without any device work.
// With x == NULL only the count is returned; otherwise up to cap nodes are written.
extern "C" int64_t ers_debug_quadrature(const double c[3], const double a[3], double h, double *x, double *n,
                                        double *w, int64_t cap) {
    std::vector<double> xs, ns, ws;
    const int64_t N = ers::quadrature(c, a, h, x ? &xs : nullptr, x ? &ns : nullptr, x ? &ws : nullptr);
    if (x) {
        const int64_t k = N < cap ? N : cap;
        std::memcpy(x, xs.data(), sizeof(double) * 3 * k);
        std::memcpy(n, ns.data(), sizeof(double) * 3 * k);
        std::memcpy(w, ws.data(), sizeof(double) * k);
    }
    return N;
}
