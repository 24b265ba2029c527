// Closest point / signed distance (Sec. 2: y = x0 + b n0) and density records.
#include "ers_internal.h"

namespace ers {
namespace {

// One thread per target.  Sphere: closed form.  Ellipsoid: the closest point solves
// x_i = a_i^2 p_i / (t + a_i^2), p = y - c, with F(t) = sum_i (a_i p_i / (t + a_i^2))^2 - 1 = 0;
// the closest point belongs to the largest root, which is the only root on
// (-min a_i^2, inf) where F is decreasing and convex.  Newton's method from the side where
// F > 0 converges monotonically; each step is kept inside the current bracket (bisection
// otherwise).  At most 200 iterations.
__global__ void k_closest(double c0, double c1, double c2, double a0, double a1, double a2, int sphere,
                          double on_tol, const double *__restrict__ y, int64_t M, double *__restrict__ x0,
                          double *__restrict__ n0, double *__restrict__ bout) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const double c[3] = {c0, c1, c2}, a[3] = {a0, a1, a2};
    double p[3];
    for (int i = 0; i < 3; ++i) p[i] = y[3 * m + i] - c[i];
    double xr[3], nr[3], b;
    if (sphere) {
        const double rp = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
        double d[3] = {0.0, 0.0, 1.0};
        if (rp > 0.0)
            for (int i = 0; i < 3; ++i) d[i] = p[i] / rp;
        for (int i = 0; i < 3; ++i) {
            xr[i] = c[i] + a[0] * d[i];
            nr[i] = d[i];
        }
        b = rp - a[0];
    } else {
        double a2v[3], ap2[3];
        double amin2 = a[0] * a[0], amax = a[0];
        for (int i = 0; i < 3; ++i) {
            a2v[i] = a[i] * a[i];
            ap2[i] = (a[i] * p[i]) * (a[i] * p[i]);
            amin2 = fmin(amin2, a2v[i]);
            amax = fmax(amax, a[i]);
        }
        double F0 = ap2[0] / (a2v[0] * a2v[0]) + ap2[1] / (a2v[1] * a2v[1]) + ap2[2] / (a2v[2] * a2v[2]) - 1.0;
        const double pn = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
        double lo, hi;
        if (F0 > 0.0) {
            lo = 0.0;
            hi = amax * pn + amax * amax;
        } else {
            lo = -amin2;
            hi = 0.0;
        }
        // start on the F > 0 side: for an inside point, close to the pole of the smallest axis
        double t = (F0 > 0.0) ? 0.0 : -amin2 + (amin2 + 0.0) * 1e-3;
        for (int it = 0; it < 200; ++it) {
            double F = -1.0, dF = 0.0;
            for (int i = 0; i < 3; ++i) {
                if (ap2[i] == 0.0) continue;
                const double inv = 1.0 / (t + a2v[i]);
                const double v = ap2[i] * inv * inv;
                F += v;
                dF -= 2.0 * v * inv;
            }
            if (F > 0.0) lo = fmax(lo, t); else hi = fmin(hi, t);
            double tn = (dF < 0.0) ? t - F / dF : 0.5 * (lo + hi);
            if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
            if (tn == t || hi - lo <= 4.0 * 2.220446049250313e-16 * fmax(1.0, fabs(t))) {
                t = tn;
                break;
            }
            t = tn;
        }
        double s = 0.0;
        for (int i = 0; i < 3; ++i) {
            const double den = t + a2v[i];
            xr[i] = (p[i] == 0.0 || den <= 0.0) ? 0.0 : a2v[i] * p[i] / den;
            s += (xr[i] / a[i]) * (xr[i] / a[i]);
        }
        if (s < 1.0 - 1e-12) {  // medial set: fill the first zero coordinate along a smallest axis
            for (int i = 0; i < 3; ++i) {
                if (p[i] == 0.0 && a2v[i] == amin2) {
                    xr[i] = a[i] * sqrt(1.0 - s);
                    break;
                }
            }
        }
        double g[3], gn = 0.0, d2 = 0.0;
        for (int i = 0; i < 3; ++i) {
            g[i] = xr[i] / a2v[i];
            gn += g[i] * g[i];
        }
        gn = sqrt(gn);
        for (int i = 0; i < 3; ++i) {
            nr[i] = g[i] / gn;
            const double dd = p[i] - xr[i];
            d2 += dd * dd;
            xr[i] += c[i];
        }
        b = sqrt(d2);
        if (F0 < 0.0) b = -b;
    }
    if (fabs(b) <= on_tol) b = 0.0;
    for (int i = 0; i < 3; ++i) {
        x0[3 * m + i] = xr[i];
        n0[3 * m + i] = nr[i];
    }
    bout[m] = b;
}

// rec[j] = (x, w f, w n, q) and rec32[j] = (x - c_tile, w f, w n, q) in floats, for the
// sorted node j of canonical index perm[j].  Only the density parts are written here.
__global__ void k_density(const int *__restrict__ perm, const double *__restrict__ w, const double *__restrict__ f,
                          const double *__restrict__ q, int64_t N, double *__restrict__ rec,
                          float *__restrict__ rec32, float *__restrict__ recp, double *__restrict__ fq) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const int64_t i = perm[j];
    const double wi = w[i];
    // float pair of v in the near-field record: hi = v rounded, lo = the rest rounded
    auto put_pair = [&](int off, double v) {
        const float hi = __double2float_rn(v);
        recp[j * NREC + off] = hi;
        recp[j * NREC + off + 1] = __double2float_rn(v - (double)hi);
    };
    if (f) {
        for (int k = 0; k < 3; ++k) {
            const double v = wi * f[3 * i + k];
            rec[j * REC + R_WF + k] = v;
            rec32[j * REC + R_WF + k] = __double2float_rn(v);
            put_pair(NR_WF + 2 * k, v);
            fq[j * 6 + k] = f[3 * i + k];
        }
    }
    if (q) {
        for (int k = 0; k < 3; ++k) {
            const double v = q[3 * i + k];
            rec[j * REC + R_Q + k] = v;
            rec32[j * REC + R_Q + k] = __double2float_rn(v);
            put_pair(NR_Q + 2 * k, v);
            fq[j * 6 + 3 + k] = v;
        }
    }
}

}  // namespace

cudaError_t launch_closest(const ers_surface *s, const double *y, int64_t M, double *x0, double *n0, double *b,
                           cudaStream_t st) {
    if (M == 0) return cudaSuccess;
    const double amax = fmax(s->a[0], fmax(s->a[1], s->a[2]));
    const int bs = 128;
    const int64_t grid = (M + bs - 1) / bs;
    k_closest<<<(unsigned)grid, bs, 0, st>>>(s->c[0], s->c[1], s->c[2], s->a[0], s->a[1], s->a[2],
                                             s->is_sphere ? 1 : 0, 1e-12 * amax, y, M, x0, n0, b);
    return cudaGetLastError();
}

cudaError_t launch_density(ers_surface *s, const double *f, const double *q, cudaStream_t st) {
    const int bs = 256;
    const int64_t grid = (s->N + bs - 1) / bs;
    k_density<<<(unsigned)grid, bs, 0, st>>>(s->perm, s->w, f, q, s->N, s->rec, s->rec32, s->recp, s->fq);
    return cudaGetLastError();
}

}  // namespace ers
