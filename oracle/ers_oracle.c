/*
 * FP64 CPU oracle for the extrapolated-regularization evaluation of the Stokes single- and
 * double-layer integrals (Siebor & Tlupova, "Localized evaluation and fast summation in the
 * extrapolated regularization method for integrals in Stokes flow").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the GPU library is
 * checked against.  Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  It shares no code, header, table or helper with the GPU library.
 *
 * Every quantity is IEEE double precision; loops are written in the order the paper states
 * the method.  OpenMP splits the outer loop over targets (Sec. 3.1); each target is computed
 * by one thread in a fixed order, so results do not depend on the thread count.
 *
 * Parity status of each function: pinned by tests/test_oracle_*.py (node counts of Table 1,
 * surface areas, sphere closed forms, exact extrapolation weights at b = 0, O(h^5) observed
 * convergence, localized == direct; for the on-surface s# functions of Sec. 2.1: 60-digit
 * values, the limits at 0 and infinity, O(h^5) against the sphere closed form and in
 * self-convergence at shared nodes; for the four-delta variant: I4 against quadrature of its
 * defining integral, I4' = -4 lambda I2, exact weights at b = 0, faster than O(h^5) against the
 * sphere closed form; for the reduced one- and two-delta sums of the learned closure: the exact
 * two-delta weights at b = 0, their defining identities at every b, and the two-delta value with
 * the three-delta solve's c2 reproducing the three-delta value; the treecode far field of Sec. 3.4
 * lives in ers_treecode.c with its own pins).  Nothing here is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_PI 3.14159265358979323846
#define ORA_SQRTPI 1.77245385090551602730

/* ------------------------------------------------------------------------------------ */
/* Quadrature (Sec. 2.2, Eq. (quadrature)): lattice-crossing nodes with partition-of-unity  */
/* weights.  Surface: ellipsoid sum(((x-c)/a)^2) = 1.                                      */
/* ------------------------------------------------------------------------------------ */

/* Bump function b(r) = exp(2 r^2 / (r^2 - 1)) for |r| < 1, else 0 (Sec. 2.2). */
static double ora_bump(double r) {
    if (fabs(r) >= 1.0) return 0.0;
    double r2 = r * r;
    return exp(2.0 * r2 / (r2 - 1.0));
}

/* Outward unit normal of the ellipsoid at x: gradient of the implicit function, normalised. */
static void ora_ellipsoid_normal(const double c[3], const double a[3], const double x[3], double n[3]) {
    double g[3], s = 0.0;
    for (int i = 0; i < 3; ++i) { g[i] = (x[i] - c[i]) / (a[i] * a[i]); s += g[i] * g[i]; }
    s = sqrt(s);
    for (int i = 0; i < 3; ++i) n[i] = g[i] / s;
}

/*
 * Nodes of the sets Gamma_1, Gamma_2, Gamma_3 (Sec. 2.2).  Gamma_k holds the points where a
 * lattice line parallel to e_k, through (i h, j h) in the other two coordinates, crosses the
 * surface, kept when |n_k| >= cos(theta) with theta = 70 degrees.  The weight is
 * w = psi_k(n) / |n_k| * h^2 with beta_j(n) = b(arccos|n_j| / theta) and
 * psi_k = beta_k / sum_j beta_j.
 *
 * Enumeration order (fixed, so that another implementation can reproduce the node array):
 * k = 1, 2, 3; then the lower lattice index p over the first remaining axis, then q over the
 * second remaining axis, both ascending; then the lower root before the upper root.
 *
 * With x == NULL the nodes are only counted.  Returns the number of nodes.
 */
int64_t ora_quadrature(const double c[3], const double a[3], double h,
                       double *x, double *n, double *w) {
    const double theta = 70.0 * ORA_PI / 180.0;
    const double cos_theta = cos(theta);
    int64_t count = 0;
    for (int k = 0; k < 3; ++k) {
        int p = (k == 0) ? 1 : 0;
        int q = (k == 2) ? 1 : 2;
        long ilo = (long)floor((c[p] - a[p]) / h) - 1, ihi = (long)ceil((c[p] + a[p]) / h) + 1;
        long jlo = (long)floor((c[q] - a[q]) / h) - 1, jhi = (long)ceil((c[q] + a[q]) / h) + 1;
        for (long i = ilo; i <= ihi; ++i) {
            for (long j = jlo; j <= jhi; ++j) {
                double xp = (double)i * h, xq = (double)j * h;
                double up = (xp - c[p]) / a[p], uq = (xq - c[q]) / a[q];
                double disc = 1.0 - up * up - uq * uq;
                if (!(disc > 0.0)) continue;
                double half = a[k] * sqrt(disc);
                double roots[2] = {c[k] - half, c[k] + half};
                for (int r = 0; r < 2; ++r) {
                    double xx[3], nn[3];
                    xx[p] = xp; xx[q] = xq; xx[k] = roots[r];
                    ora_ellipsoid_normal(c, a, xx, nn);
                    if (fabs(nn[k]) < cos_theta) continue;
                    if (x) {
                        double beta[3], sb = 0.0;
                        for (int m = 0; m < 3; ++m) { beta[m] = ora_bump(acos(fabs(nn[m])) / theta); sb += beta[m]; }
                        double psi = beta[k] / sb;
                        for (int m = 0; m < 3; ++m) { x[3 * count + m] = xx[m]; n[3 * count + m] = nn[m]; }
                        w[count] = psi / fabs(nn[k]) * h * h;
                    }
                    ++count;
                }
            }
        }
    }
    return count;
}

/* ------------------------------------------------------------------------------------ */
/* Closest point and signed distance (Sec. 2: y = x0 + b n0, n0 outward at x0).            */
/* ------------------------------------------------------------------------------------ */

/*
 * Closest point on the ellipsoid.  Stationary points satisfy x_i = a_i^2 p_i / (t + a_i^2)
 * (p = y - c) with F(t) = sum_i (a_i p_i / (t + a_i^2))^2 - 1 = 0; the closest point is the
 * largest root.  F decreases on (-min a_i^2, inf), so the root is found by plain bisection on
 * that interval.  When a coordinate along a smallest axis is zero and F stays negative
 * there, the closest point lies off the regular branch (the target is on the medial set);
 * then t = -a_min^2 and the free coordinate is filled from the surface equation with a
 * positive sign (one valid choice among several).  A sphere uses its closed form.
 * |b| <= on_tol is treated as on the surface (b = 0).
 */
static void ora_closest_one(const double c[3], const double a[3], const double y[3], double on_tol,
                            double x0[3], double n0[3], double *bout) {
    double p[3] = {y[0] - c[0], y[1] - c[1], y[2] - c[2]};
    if (a[0] == a[1] && a[1] == a[2]) {
        double R = a[0];
        double rp = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
        double d[3];
        if (rp == 0.0) { d[0] = 0.0; d[1] = 0.0; d[2] = 1.0; }
        else for (int i = 0; i < 3; ++i) d[i] = p[i] / rp;
        for (int i = 0; i < 3; ++i) { x0[i] = c[i] + R * d[i]; n0[i] = d[i]; }
        double b = rp - R;
        *bout = (fabs(b) <= on_tol) ? 0.0 : b;
        return;
    }
    double amin2 = a[0] * a[0];
    for (int i = 1; i < 3; ++i) if (a[i] * a[i] < amin2) amin2 = a[i] * a[i];
    double pn = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    double amax = fmax(a[0], fmax(a[1], a[2]));
    /* F(t); terms with p_i == 0 are zero */
#define ORA_F(t, out) do { double s_ = 0.0; for (int i_ = 0; i_ < 3; ++i_) { if (p[i_] != 0.0) { \
        double v_ = a[i_] * p[i_] / ((t) + a[i_] * a[i_]); s_ += v_ * v_; } } (out) = s_ - 1.0; } while (0)
    double F0; ORA_F(0.0, F0);
    double lo, hi;
    if (F0 > 0.0) { lo = 0.0; hi = amax * pn + amax * amax; }
    else { lo = -amin2; hi = 0.0; }
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double Fm; ORA_F(mid, Fm);
        if (Fm > 0.0) lo = mid; else hi = mid;
    }
    double t = 0.5 * (lo + hi);
#undef ORA_F
    double s = 0.0;
    for (int i = 0; i < 3; ++i) {
        double den = t + a[i] * a[i];
        x0[i] = (p[i] == 0.0 || den <= 0.0) ? 0.0 : a[i] * a[i] * p[i] / den;
        s += (x0[i] / a[i]) * (x0[i] / a[i]);
    }
    if (s < 1.0 - 1e-12) {
        /* medial set: the regular branch does not reach the surface; fill the first zero
         * coordinate along a smallest axis from the surface equation */
        for (int i = 0; i < 3; ++i) {
            if (p[i] == 0.0 && a[i] * a[i] == amin2) { x0[i] = a[i] * sqrt(1.0 - s); break; }
        }
    }
    for (int i = 0; i < 3; ++i) x0[i] += c[i];
    ora_ellipsoid_normal(c, a, x0, n0);
    double d2 = 0.0;
    for (int i = 0; i < 3; ++i) d2 += (y[i] - x0[i]) * (y[i] - x0[i]);
    double b = sqrt(d2);
    if (F0 < 0.0) b = -b;
    *bout = (fabs(b) <= on_tol) ? 0.0 : b;
}

void ora_closest_point(const double c[3], const double a[3], const double *y, int64_t M, double on_tol,
                       double *x0, double *n0, double *b) {
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < M; ++m) ora_closest_one(c, a, y + 3 * m, on_tol, x0 + 3 * m, n0 + 3 * m, b + m);
}

/* ------------------------------------------------------------------------------------ */
/* Smoothing functions s1, s2, s3 (Eqs. (s1)-(s3)) as the kernel factors s_p(t)/t^p.       */
/* ------------------------------------------------------------------------------------ */

/*
 * sigma_p(t) = s_p(t) / t^p for p = 1, 3, 5 (s_1, s_2, s_3 of Eqs. (s1)-(s3)).
 * For t < 0.5 the Maclaurin series of erf (2/sqrt(pi)) sum (-1)^n t^(2n+1) / (n! (2n+1))
 * gives, term by term,
 *   s1/t   = (2/sqrt(pi)) sum_{n>=0} (-1)^n t^(2n) / (n! (2n+1))
 *   s2/t^3 = (2/sqrt(pi)) sum_{n>=1} (-1)^(n+1) 2n / (n! (2n+1)) t^(2n-2)
 *   s3/t^5 = (2/sqrt(pi)) sum_{n>=2} (-1)^n 4n(n-1) / (3 (2n+1) n!) t^(2n-4)
 * which avoids the cancellation of the closed forms at small t.  Otherwise the closed forms
 * of Eqs. (s1)-(s3) are used with the C library erf and exp.
 */
void ora_sigma(double t, double sig[3]) {
    const double c = 2.0 / ORA_SQRTPI;
    if (t < 0.5) {
        double t2 = t * t;
        double s1 = 0.0, s2 = 0.0, s3 = 0.0;
        double fact = 1.0;                       /* n! */
        double p1 = 1.0, p2 = 1.0, p3 = 1.0;     /* t^(2n), t^(2n-2), t^(2n-4) */
        for (int nn = 0; nn <= 20; ++nn) {
            if (nn > 0) fact *= nn;
            if (nn > 0) p1 *= t2;
            if (nn > 1) p2 *= t2;
            if (nn > 2) p3 *= t2;
            double sgn = (nn % 2 == 0) ? 1.0 : -1.0;
            s1 += sgn * p1 / (fact * (2.0 * nn + 1.0));
            if (nn >= 1) s2 += -sgn * (2.0 * nn) / (fact * (2.0 * nn + 1.0)) * p2;
            if (nn >= 2) s3 += sgn * (4.0 * nn * (nn - 1.0)) / (3.0 * (2.0 * nn + 1.0) * fact) * p3;
        }
        sig[0] = c * s1; sig[1] = c * s2; sig[2] = c * s3;
        return;
    }
    double e = erf(t), g = exp(-t * t);
    double s1 = e;
    double s2 = e - c * t * g;
    double s3 = e - c * (t + 2.0 / 3.0 * t * t * t) * g;
    sig[0] = s1 / t;
    sig[1] = s2 / (t * t * t);
    sig[2] = s3 / (t * t * t * t * t);
}

/*
 * sigma#_p(t) = s#_p(t) / t^p for the modified smoothing functions of Sec. 2.1 (on-surface
 * evaluation):
 *   s#_1 = erf t + (2/(3 sqrt pi)) (5t - 2t^3) e^{-t^2},
 *   s#_2 = erf t - (2/(3 sqrt pi)) (3t - 14t^3 + 4t^5) e^{-t^2},
 *   s#_3 = erf t - (2/(9 sqrt pi)) (9t + 6t^3 - 4t^5) e^{-t^2}.
 * For t < 1 term by term: with erf t = (2/sqrt pi) sum (-1)^n t^(2n+1) / (n! (2n+1)) and the
 * coefficient of t^(2n+1) in P(t) e^{-t^2} collected for each polynomial P,
 *   s#_1 / t   = (2/sqrt pi) sum_{n>=0} (-1)^n t^(2n)   [1/(2n+1) + (5 + 2n)/3]          / n!
 *   s#_2 / t^3 = (2/sqrt pi) sum_{n>=1} (-1)^n t^(2n-2) [1/(2n+1) - (4n^2 + 10n + 3)/3] / n!
 *   s#_3 / t^5 = (2/sqrt pi) sum_{n>=2} (-1)^n t^(2n-4) [1/(2n+1) - (9 - 2n - 4n^2)/9] / n!
 * (the n = 0 term of s#_2 and the n = 0, 1 terms of s#_3 vanish).  Otherwise the closed forms.
 */
void ora_sigma_sharp(double t, double sig[3]) {
    const double c = 2.0 / ORA_SQRTPI;
    if (t < 1.0) {
        double t2 = t * t;
        double s1 = 0.0, s2 = 0.0, s3 = 0.0;
        double fact = 1.0;                    /* n! */
        double p1 = 1.0, p2 = 1.0, p3 = 1.0;  /* t^(2n), t^(2n-2), t^(2n-4) */
        for (int nn = 0; nn <= 30; ++nn) {
            if (nn > 0) fact *= nn;
            if (nn > 0) p1 *= t2;
            if (nn > 1) p2 *= t2;
            if (nn > 2) p3 *= t2;
            double sgn = (nn % 2 == 0) ? 1.0 : -1.0;
            double e = 1.0 / (2.0 * nn + 1.0);
            s1 += sgn * p1 * (e + (5.0 + 2.0 * nn) / 3.0) / fact;
            if (nn >= 1) s2 += sgn * p2 * (e - (4.0 * nn * nn + 10.0 * nn + 3.0) / 3.0) / fact;
            if (nn >= 2) s3 += sgn * p3 * (e - (9.0 - 2.0 * nn - 4.0 * nn * nn) / 9.0) / fact;
        }
        sig[0] = c * s1; sig[1] = c * s2; sig[2] = c * s3;
        return;
    }
    double e = erf(t), g = exp(-t * t), t2 = t * t;
    double s1 = e + c / 3.0 * (5.0 * t - 2.0 * t * t2) * g;
    double s2 = e - c / 3.0 * (3.0 * t - 14.0 * t * t2 + 4.0 * t * t2 * t2) * g;
    double s3 = e - c / 9.0 * (9.0 * t + 6.0 * t * t2 - 4.0 * t * t2 * t2) * g;
    sig[0] = s1 / t;
    sig[1] = s2 / (t * t2);
    sig[2] = s3 / (t * t2 * t2);
}

/* I0 and I2 of Eqs. (I0), (I2). */
double ora_I0(double lam) {
    double l = fabs(lam);
    return exp(-l * l) / ORA_SQRTPI - l * erfc(l);
}
double ora_I2(double lam) {
    double l = fabs(lam);
    return 2.0 / 3.0 * ((0.5 - l * l) * exp(-l * l) / ORA_SQRTPI + l * l * l * erfc(l));
}

/*
 * I4, the lambda-dependence of the next (delta^5) term of the regularization error, for the
 * four-delta O(delta^7) variant the paper mentions (no formula is printed).  Reading: I0 and I2 are
 * I_2k(lambda) = int_{|lambda|}^inf erfc(r) (r^2 - lambda^2)^k dr for k = 0, 1 (the moments of the
 * regularization error of s1 over a plane at distance lambda, in units of delta; this reproduces
 * Eqs. (I0), (I2) exactly), so for k = 2, integrating r^n erfc(r) by parts,
 *   I4(lambda) = (2/15) ((3 - 2 lambda^2 + 4 lambda^4) e^{-lambda^2}/sqrt(pi) - 4 |lambda|^5 erfc|lambda|).
 */
double ora_I4(double lam) {
    double l = fabs(lam), l2 = l * l;
    return 2.0 / 15.0 * ((3.0 - 2.0 * l2 + 4.0 * l2 * l2) * exp(-l2) / ORA_SQRTPI - 4.0 * l2 * l2 * l * erfc(l));
}

/*
 * Solve the K x K system (K = 3: Eq. (extrap_eqn); K = 4: the same with the term c3 rho^5 I4)
 *   u + c1 rho_k I0(lambda_k) + c2 rho_k^3 I2(lambda_k) [+ c3 rho_k^5 I4(lambda_k)] = U_k,
 * lambda_k = b / delta_k, for `nrhs` right-hand sides (Gaussian elimination with partial
 * pivoting).  Returns 0, or -1 when the matrix is singular / not finite (then U_1).
 */
int ora_extrapolate_k(int K, const double *rho, double b, double h, const double *U /* [K][nrhs] */, int nrhs,
                      double *out) {
    double A[4][4], B[4][8];
    for (int k = 0; k < K; ++k) {
        double lam = b / (rho[k] * h), r = rho[k];
        A[k][0] = 1.0;
        A[k][1] = r * ora_I0(lam);
        A[k][2] = r * r * r * ora_I2(lam);
        if (K == 4) A[k][3] = r * r * r * r * r * ora_I4(lam);
        for (int q = 0; q < nrhs; ++q) B[k][q] = U[k * nrhs + q];
    }
    int ok = 1;
    for (int col = 0; col < K && ok; ++col) {
        int piv = col;
        for (int r = col + 1; r < K; ++r) if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (!(fabs(A[piv][col]) > 0.0) || !isfinite(A[piv][col])) { ok = 0; break; }
        if (piv != col) {
            for (int cc = 0; cc < K; ++cc) { double tmp = A[col][cc]; A[col][cc] = A[piv][cc]; A[piv][cc] = tmp; }
            for (int q = 0; q < nrhs; ++q) { double tmp = B[col][q]; B[col][q] = B[piv][q]; B[piv][q] = tmp; }
        }
        for (int r = col + 1; r < K; ++r) {
            double f = A[r][col] / A[col][col];
            for (int cc = col; cc < K; ++cc) A[r][cc] -= f * A[col][cc];
            for (int q = 0; q < nrhs; ++q) B[r][q] -= f * B[col][q];
        }
    }
    if (ok) {
        for (int q = 0; q < nrhs; ++q) {
            double x[4];
            for (int r = K - 1; r >= 0; --r) {
                double acc = B[r][q];
                for (int cc = r + 1; cc < K; ++cc) acc -= A[r][cc] * x[cc];
                x[r] = acc / A[r][r];
            }
            if (!isfinite(x[0])) ok = 0;
            out[q] = x[0];
        }
    }
    if (!ok) { for (int q = 0; q < nrhs; ++q) out[q] = U[q]; return -1; }
    return 0;
}

/*
 * Solve the 3x3 system of Eq. (extrap_eqn) for the extrapolated value:
 *   u + c1 rho_k I0(lambda_k) + c2 rho_k^3 I2(lambda_k) = U_k,  k = 1, 2, 3,
 * with lambda_k = b / delta_k, for `nrhs` right-hand sides at once (Gaussian elimination with
 * partial pivoting).  Returns 0, or -1 when the matrix is singular / not finite (then the
 * smallest-delta value U_1 is returned).
 */
int ora_extrapolate(const double rho[3], double b, double h, const double *U /* [3][nrhs] */,
                    int nrhs, double *out) {
    double A[3][3], B[3][8];
    for (int k = 0; k < 3; ++k) {
        double lam = b / (rho[k] * h);
        A[k][0] = 1.0;
        A[k][1] = rho[k] * ora_I0(lam);
        A[k][2] = rho[k] * rho[k] * rho[k] * ora_I2(lam);
        for (int r = 0; r < nrhs; ++r) B[k][r] = U[k * nrhs + r];
    }
    int ok = 1;
    for (int col = 0; col < 3 && ok; ++col) {
        int piv = col;
        for (int r = col + 1; r < 3; ++r) if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (!(fabs(A[piv][col]) > 0.0) || !isfinite(A[piv][col])) { ok = 0; break; }
        if (piv != col) {
            for (int cc = 0; cc < 3; ++cc) { double tmp = A[col][cc]; A[col][cc] = A[piv][cc]; A[piv][cc] = tmp; }
            for (int r = 0; r < nrhs; ++r) { double tmp = B[col][r]; B[col][r] = B[piv][r]; B[piv][r] = tmp; }
        }
        for (int r = col + 1; r < 3; ++r) {
            double f = A[r][col] / A[col][col];
            for (int cc = col; cc < 3; ++cc) A[r][cc] -= f * A[col][cc];
            for (int q = 0; q < nrhs; ++q) B[r][q] -= f * B[col][q];
        }
    }
    if (ok) {
        for (int r = 0; r < nrhs; ++r) {
            double x2 = B[2][r] / A[2][2];
            double x1 = (B[1][r] - A[1][2] * x2) / A[1][1];
            double x0 = (B[0][r] - A[0][1] * x1 - A[0][2] * x2) / A[0][0];
            if (!isfinite(x0)) ok = 0;
            out[r] = x0;
        }
    }
    if (!ok) { for (int r = 0; r < nrhs; ++r) out[r] = U[0 * nrhs + r]; return -1; }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Pair terms                                                                              */
/* ------------------------------------------------------------------------------------ */

/*
 * Regularized single-layer pair term, Eq. (Sreg) applied to the subtracted density of
 * Eq. (Stokes_SL2):  S^delta_ij g_j w = (s1/r) g_i w + d_i (d.g) (s2/r^3) w, d = y - x.
 * t = r/delta; s_p := 1 when t > tc (Sec. 3.2).  Adds into acc[3] (without 1/(8 pi)).
 */
void ora_sl_term(const double d[3], double r, double delta, double tc, const double g[3], double w,
                        double acc[3], int sharp) {
    double t = r / delta;
    double k1, k3; /* s1/r and s2/r^3 (s#1, s#2 when sharp) */
    if (t > tc) { k1 = 1.0 / r; k3 = 1.0 / (r * r * r); }
    else {
        double sig[3];
        if (sharp) ora_sigma_sharp(t, sig); else ora_sigma(t, sig);
        k1 = sig[0] / delta;
        k3 = sig[1] / (delta * delta * delta);
    }
    double dg = d[0] * g[0] + d[1] * g[1] + d[2] * g[2];
    for (int i = 0; i < 3; ++i) acc[i] += (k1 * g[i] + k3 * dg * d[i]) * w;
}

/*
 * Regularized double-layer pair term, Eqs. (Tsplit) and (Treg), contracted with the
 * subtracted density Q = q(x) - q(x0) and the source normal n(x) (Eq. (Stokes_DL2)):
 *   T^delta_ijk Q_j n_k w,  T^delta = T^(1) s2 + T^(2) s3,
 *   T^(1) = -6 t1 / r^3,  T^(2) = -6 (t2 - (r^2 - b^2) t1) / r^5,
 *   t1_ijk = b n_i n_j n_k - (xh_i n_j n_k + n_i xh_j n_k + n_i n_j xh_k),
 *   t2_ijk = b (xh_i xh_j n_k + xh_i n_j xh_k + n_i xh_j xh_k) - xh_i xh_j xh_k,
 * with n = n0 (normal at the closest point) and xh = x - x0.  The tensors are formed
 * explicitly and contracted, as written.  s_p := 1 when t > tc.
 */
void ora_dl_term(double r, double delta, double tc, double b, const double nrm0[3], const double xh[3],
                        const double Q[3], const double nx[3], double w, double acc[3], int sharp) {
    double t = r / delta;
    double k3, k5; /* s2/r^3 and s3/r^5 (s#2, s#3 when sharp) */
    if (t > tc) { k3 = 1.0 / (r * r * r); k5 = 1.0 / (r * r * r * r * r); }
    else {
        double sig[3];
        if (sharp) ora_sigma_sharp(t, sig); else ora_sigma(t, sig);
        k3 = sig[1] / (delta * delta * delta);
        k5 = sig[2] / (delta * delta * delta * delta * delta);
    }
    double r2mb2 = r * r - b * b;
    for (int i = 0; i < 3; ++i) {
        double s = 0.0;
        for (int j = 0; j < 3; ++j) {
            for (int k = 0; k < 3; ++k) {
                const double *ni = nrm0, *xi = xh;
                double t1 = b * ni[i] * ni[j] * ni[k] - (xi[i] * ni[j] * ni[k] + ni[i] * xi[j] * ni[k] + ni[i] * ni[j] * xi[k]);
                double t2 = b * (xi[i] * xi[j] * ni[k] + xi[i] * ni[j] * xi[k] + ni[i] * xi[j] * xi[k]) - xi[i] * xi[j] * xi[k];
                double T = -6.0 * (t1 * k3 + (t2 - r2mb2 * t1) * k5);
                s += T * Q[j] * nx[k];
            }
        }
        acc[i] += s * w;
    }
}

/*
 * On-surface regularized double-layer pair term with the modified function s#_3 of Sec. 2.1
 * applied to the stresslet itself, -6 d_i d_j d_k s#_3(r/delta)/r^5 (at b = 0 the split
 * T^(1) s_2 + T^(2) s_3 equals this form plus t1 (s_2 - s_3)/r^3, which for s# is not small);
 * s#_3 := 1 when t > tc.  Adds -6 d (d.Q)(d.n) s#_3/r^5 w into acc.
 */
static void ora_dl_term_sharp(const double d[3], double r, double delta, double tc, const double Q[3],
                              const double nx[3], double w, double acc[3]) {
    double t = r / delta;
    double k5;
    if (t > tc) k5 = 1.0 / (r * r * r * r * r);
    else {
        double sig[3]; ora_sigma_sharp(t, sig);
        k5 = sig[2] / (delta * delta * delta * delta * delta);
    }
    double dq = d[0] * Q[0] + d[1] * Q[1] + d[2] * Q[2];
    double dn = d[0] * nx[0] + d[1] * nx[1] + d[2] * nx[2];
    for (int i = 0; i < 3; ++i) acc[i] += -6.0 * d[i] * dq * dn * k5 * w;
}

/* Plain (unregularized) pair terms, Eqs. (Stokeslet), (Stresslet). */
void ora_sl_plain(const double d[3], double r, const double g[3], double w, double acc[3]) {
    double dg = d[0] * g[0] + d[1] * g[1] + d[2] * g[2];
    for (int i = 0; i < 3; ++i) acc[i] += (g[i] / r + d[i] * dg / (r * r * r)) * w;
}
void ora_dl_plain(const double d[3], double r, const double Q[3], const double nx[3], double w, double acc[3]) {
    double dq = d[0] * Q[0] + d[1] * Q[1] + d[2] * Q[2];
    double dn = d[0] * nx[0] + d[1] * nx[1] + d[2] * nx[2];
    double r5 = r * r * r * r * r;
    for (int i = 0; i < 3; ++i) acc[i] += -6.0 * d[i] * dq * dn / r5 * w;
}

/* ------------------------------------------------------------------------------------ */
/* Evaluation                                                                              */
/* ------------------------------------------------------------------------------------ */

/*
 * Evaluate both layers at M targets.
 *   nodes x (N,3), normals n (N,3), weights w (N), densities f, q at the nodes (N,3);
 *   targets y (M,3) with closest point data x0, n0 (M,3), b (M) and the densities at the
 *   closest point f0, q0 (M,3).
 *   params: h, rho[K] (K = 3 deltas, or 4 for the O(delta^7) variant), tc (regularization
 *   cut-off t = r/delta > tc => s_p = 1, Sec. 3.2).
 *   mode 0 = DIRECT: for each delta_k the full sum over every node (Table 1 procedure);
 *   mode 1 = LOCALIZED: u = u_far + u_near_k (Eq. (near_far)); far = nodes with
 *            r > Rc = tc * delta_K, evaluated once without regularization; near = the rest,
 *            evaluated for each delta_k (Sec. 3.3).
 * Targets with |b| > Rc have no node within Rc: their value is the plain sum of
 * Eqs. (Stokes_SL), (Stokes_DL) without subtraction.  The others use the subtracted forms
 * (Eqs. (Stokes_SL2), (Stokes_DL2)) for the K delta_k and the solve (ora_extrapolate_k).
 * Outputs u, v (M,3).  Returns the number of targets whose solve fell back.
 */
int64_t ora_eval_k(int K, const double *x, const double *nrm, const double *w, const double *f, const double *q,
                   int64_t N, const double *y, const double *x0, const double *n0, const double *b,
                   const double *f0, const double *q0, int64_t M,
                   double h, const double *rho, double tc, int mode, double *u, double *v) {
    const double inv8pi = 1.0 / (8.0 * ORA_PI);
    const double Rc = tc * rho[K - 1] * h;
    int64_t nfail = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : nfail)
    for (int64_t m = 0; m < M; ++m) {
        const double *ym = y + 3 * m;
        double bm = b[m];
        if (fabs(bm) > Rc) {
            double su[3] = {0, 0, 0}, sv[3] = {0, 0, 0};
            for (int64_t j = 0; j < N; ++j) {
                double d[3] = {ym[0] - x[3 * j], ym[1] - x[3 * j + 1], ym[2] - x[3 * j + 2]};
                double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                ora_sl_plain(d, r, f + 3 * j, w[j], su);
                ora_dl_plain(d, r, q + 3 * j, nrm + 3 * j, w[j], sv);
            }
            for (int i = 0; i < 3; ++i) { u[3 * m + i] = su[i] * inv8pi; v[3 * m + i] = sv[i] * inv8pi; }
            continue;
        }
        const double *nm0 = n0 + 3 * m, *xm0 = x0 + 3 * m, *fm0 = f0 + 3 * m, *qm0 = q0 + 3 * m;
        double fn0 = fm0[0] * nm0[0] + fm0[1] * nm0[1] + fm0[2] * nm0[2];
        double chi = (bm < 0.0) ? 1.0 : ((bm > 0.0) ? 0.0 : 0.5);
        double U[4][6];
        double sfar_u[3] = {0, 0, 0}, sfar_v[3] = {0, 0, 0};
        double snear_u[4][3], snear_v[4][3];
        memset(snear_u, 0, sizeof snear_u); memset(snear_v, 0, sizeof snear_v);
        for (int64_t j = 0; j < N; ++j) {
            const double *xj = x + 3 * j, *nj = nrm + 3 * j;
            double d[3] = {ym[0] - xj[0], ym[1] - xj[1], ym[2] - xj[2]};
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            /* subtracted densities: g = f(x) - (f(x0).n0) n(x);  Q = q(x) - q(x0) */
            double g[3], Q[3], xh[3];
            for (int i = 0; i < 3; ++i) {
                g[i] = f[3 * j + i] - fn0 * nj[i];
                Q[i] = q[3 * j + i] - qm0[i];
                xh[i] = xj[i] - xm0[i];
            }
            if (mode == 1 && r > Rc) {
                ora_sl_plain(d, r, g, w[j], sfar_u);
                ora_dl_plain(d, r, Q, nj, w[j], sfar_v);
                continue;
            }
            for (int k = 0; k < K; ++k) {
                double delta = rho[k] * h;
                ora_sl_term(d, r, delta, tc, g, w[j], snear_u[k], 0);
                ora_dl_term(r, delta, tc, bm, nm0, xh, Q, nj, w[j], snear_v[k], 0);
            }
        }
        for (int k = 0; k < K; ++k) {
            for (int i = 0; i < 3; ++i) {
                U[k][i] = (sfar_u[i] + snear_u[k][i]) * inv8pi;
                U[k][3 + i] = (sfar_v[i] + snear_v[k][i]) * inv8pi + chi * qm0[i];
            }
        }
        double out[6];
        if (ora_extrapolate_k(K, rho, bm, h, &U[0][0], 6, out) != 0) nfail += 1;
        for (int i = 0; i < 3; ++i) { u[3 * m + i] = out[i]; v[3 * m + i] = out[3 + i]; }
    }
    return nfail;
}

/* The method with three deltas (Eq. (extrap_eqn)). */
int64_t ora_eval(const double *x, const double *nrm, const double *w, const double *f, const double *q, int64_t N,
                 const double *y, const double *x0, const double *n0, const double *b,
                 const double *f0, const double *q0, int64_t M,
                 double h, const double rho[3], double tc, int mode, double *u, double *v) {
    return ora_eval_k(3, x, nrm, w, f, q, N, y, x0, n0, b, f0, q0, M, h, rho, tc, mode, u, v);
}

/* Regularized sums for one delta at every target (no extrapolation); used to pin the
 * extrapolation model by evaluating u^delta directly.  Same conventions as ora_eval. */
void ora_eval_one_delta(const double *x, const double *nrm, const double *w, const double *f, const double *q,
                        int64_t N, const double *y, const double *x0, const double *n0, const double *b,
                        const double *f0, const double *q0, int64_t M, double delta, double tc,
                        double *u, double *v) {
    const double inv8pi = 1.0 / (8.0 * ORA_PI);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t m = 0; m < M; ++m) {
        const double *ym = y + 3 * m, *nm0 = n0 + 3 * m, *xm0 = x0 + 3 * m, *fm0 = f0 + 3 * m, *qm0 = q0 + 3 * m;
        double bm = b[m];
        double fn0 = fm0[0] * nm0[0] + fm0[1] * nm0[1] + fm0[2] * nm0[2];
        double chi = (bm < 0.0) ? 1.0 : ((bm > 0.0) ? 0.0 : 0.5);
        double su[3] = {0, 0, 0}, sv[3] = {0, 0, 0};
        for (int64_t j = 0; j < N; ++j) {
            const double *xj = x + 3 * j, *nj = nrm + 3 * j;
            double d[3] = {ym[0] - xj[0], ym[1] - xj[1], ym[2] - xj[2]};
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double g[3], Q[3], xh[3];
            for (int i = 0; i < 3; ++i) {
                g[i] = f[3 * j + i] - fn0 * nj[i];
                Q[i] = q[3 * j + i] - qm0[i];
                xh[i] = xj[i] - xm0[i];
            }
            ora_sl_term(d, r, delta, tc, g, w[j], su, 0);
            ora_dl_term(r, delta, tc, bm, nm0, xh, Q, nj, w[j], sv, 0);
        }
        for (int i = 0; i < 3; ++i) { u[3 * m + i] = su[i] * inv8pi; v[3 * m + i] = sv[i] * inv8pi + chi * qm0[i]; }
    }
}

/*
 * The reduced extrapolation of the learned closure (one or two deltas instead of three).
 * Eq. (extrap_eqn) for delta_k = rho_k h reads U_k = u + c1 rho_k I0(lambda_k) + c2 rho_k^3 I2(lambda_k).
 *   K = 1: beta = (1), gamma = 0: the single sum U_0 is returned as it is.
 *   K = 2: the c2 term is kept aside and the two equations for k = 0, 1 are solved for u:
 *          u + gamma c2 = beta_0 U_0 + beta_1 U_1, with beta the weights of the 2 x 2 system
 *          [[1, rho_0 I0(lambda_0)], [1, rho_1 I0(lambda_1)]] (sum beta = 1, sum beta rho I0 = 0)
 *          and gamma = sum beta_k rho_k^3 I2(lambda_k).
 * beta is the first row of the inverse of that matrix: beta = (a1, -a0) / (a1 - a0) with
 * a_k = rho_k I0(lambda_k).  Returns 0, or -1 when a1 - a0 is 0 or not finite (then beta = (1, 0),
 * the single smallest-delta sum, and gamma its I2 term).
 */
int ora_reduced_weights(int K, const double *rho, double b, double h, double beta[2], double *gamma) {
    if (K == 1) {
        beta[0] = 1.0;
        beta[1] = 0.0;
        *gamma = 0.0;
        return 0;
    }
    double a[2], c[2];
    for (int k = 0; k < 2; ++k) {
        double lam = b / (rho[k] * h);
        a[k] = rho[k] * ora_I0(lam);
        c[k] = rho[k] * rho[k] * rho[k] * ora_I2(lam);
    }
    double det = a[1] - a[0];
    int rc = 0;
    if (det != 0.0 && isfinite(det)) {
        beta[0] = a[1] / det;
        beta[1] = -a[0] / det;
    } else {
        beta[0] = 1.0;
        beta[1] = 0.0;
        rc = -1;
    }
    *gamma = beta[0] * c[0] + beta[1] * c[1];
    return rc;
}

/*
 * The one- or two-delta sums of the learned closure at every target, by the definition (every
 * node, s_p := 1 where r/delta_k > tc, Sec. 3.2): for K = 1 the regularized sum for delta_0, for
 * K = 2 the combination sum_k beta_k U_k of ora_reduced_weights (u + gamma c2 of Eq. (extrap_eqn)),
 * with U_k the subtracted sums of Eqs. (Stokes_SL2), (Stokes_DL2) for delta_k.  The near radius is
 * Rc = tc delta_{K-1}; a target with |b| > Rc takes the plain sums of Eqs. (Stokes_SL), (Stokes_DL)
 * without subtraction (as ora_eval_k does beyond its radius) and gamma = 0.  Outputs u, v (M,3) and
 * gamma (M).  Returns the number of targets whose weights fell back.
 */
int64_t ora_eval_reduced(int K, const double *x, const double *nrm, const double *w, const double *f,
                         const double *q, int64_t N, const double *y, const double *x0, const double *n0,
                         const double *b, const double *f0, const double *q0, int64_t M, double h,
                         const double *rho, double tc, double *u, double *v, double *gamma) {
    const double inv8pi = 1.0 / (8.0 * ORA_PI);
    const double Rc = tc * rho[K - 1] * h;
    int64_t nfail = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : nfail)
    for (int64_t m = 0; m < M; ++m) {
        const double *ym = y + 3 * m;
        double bm = b[m];
        if (fabs(bm) > Rc) {
            double su[3] = {0, 0, 0}, sv[3] = {0, 0, 0};
            for (int64_t j = 0; j < N; ++j) {
                double d[3] = {ym[0] - x[3 * j], ym[1] - x[3 * j + 1], ym[2] - x[3 * j + 2]};
                double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                ora_sl_plain(d, r, f + 3 * j, w[j], su);
                ora_dl_plain(d, r, q + 3 * j, nrm + 3 * j, w[j], sv);
            }
            for (int i = 0; i < 3; ++i) { u[3 * m + i] = su[i] * inv8pi; v[3 * m + i] = sv[i] * inv8pi; }
            gamma[m] = 0.0;
            continue;
        }
        const double *nm0 = n0 + 3 * m, *xm0 = x0 + 3 * m, *fm0 = f0 + 3 * m, *qm0 = q0 + 3 * m;
        double fn0 = fm0[0] * nm0[0] + fm0[1] * nm0[1] + fm0[2] * nm0[2];
        double chi = (bm < 0.0) ? 1.0 : ((bm > 0.0) ? 0.0 : 0.5);
        double su[2][3], sv[2][3];
        memset(su, 0, sizeof su); memset(sv, 0, sizeof sv);
        for (int64_t j = 0; j < N; ++j) {
            const double *xj = x + 3 * j, *nj = nrm + 3 * j;
            double d[3] = {ym[0] - xj[0], ym[1] - xj[1], ym[2] - xj[2]};
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double g[3], Q[3], xh[3];
            for (int i = 0; i < 3; ++i) {
                g[i] = f[3 * j + i] - fn0 * nj[i];
                Q[i] = q[3 * j + i] - qm0[i];
                xh[i] = xj[i] - xm0[i];
            }
            for (int k = 0; k < K; ++k) {
                double delta = rho[k] * h;
                ora_sl_term(d, r, delta, tc, g, w[j], su[k], 0);
                ora_dl_term(r, delta, tc, bm, nm0, xh, Q, nj, w[j], sv[k], 0);
            }
        }
        double beta[2], gm;
        if (ora_reduced_weights(K, rho, bm, h, beta, &gm) != 0) nfail += 1;
        for (int i = 0; i < 3; ++i) {
            double uu = 0.0, vv = 0.0;
            for (int k = 0; k < K; ++k) {
                uu += beta[k] * su[k][i] * inv8pi;
                vv += beta[k] * (sv[k][i] * inv8pi + chi * qm0[i]);
            }
            u[3 * m + i] = uu;
            v[3 * m + i] = vv;
        }
        gamma[m] = gm;
    }
    return nfail;
}

/*
 * On-surface evaluation with the modified smoothing functions of Sec. 2.1: for targets on the
 * surface (b == 0 after the snap of ora_closest_point) one regularized sum with s#_p and
 * delta# = rho_sharp h (single layer: Eq. (Sreg) with s#_1, s#_2; double layer: the stresslet
 * with s#_3, ora_dl_term_sharp), localized like Sec. 3.3 with Rc# = tc delta# (far part
 * unregularized, once), no extrapolation; chi = 1/2.  Targets off the surface are evaluated by ora_eval in
 * LOCALIZED mode (three deltas and the solve).  Same conventions and outputs as ora_eval.
 */
int64_t ora_eval_sharp(const double *x, const double *nrm, const double *w, const double *f, const double *q,
                       int64_t N, const double *y, const double *x0, const double *n0, const double *b,
                       const double *f0, const double *q0, int64_t M, double h, const double rho[3], double tc,
                       double rho_sharp, double *u, double *v) {
    const double inv8pi = 1.0 / (8.0 * ORA_PI);
    const double delta = rho_sharp * h, Rc = tc * delta;
    int64_t nfail = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : nfail)
    for (int64_t m = 0; m < M; ++m) {
        if (b[m] != 0.0) {  /* off the surface: the extrapolated method */
            nfail += ora_eval(x, nrm, w, f, q, N, y + 3 * m, x0 + 3 * m, n0 + 3 * m, b + m, f0 + 3 * m, q0 + 3 * m, 1,
                              h, rho, tc, 1, u + 3 * m, v + 3 * m);
            continue;
        }
        const double *ym = y + 3 * m, *nm0 = n0 + 3 * m, *xm0 = x0 + 3 * m, *fm0 = f0 + 3 * m, *qm0 = q0 + 3 * m;
        double fn0 = fm0[0] * nm0[0] + fm0[1] * nm0[1] + fm0[2] * nm0[2];
        double su[3] = {0, 0, 0}, sv[3] = {0, 0, 0};
        for (int64_t j = 0; j < N; ++j) {
            const double *xj = x + 3 * j, *nj = nrm + 3 * j;
            double d[3] = {ym[0] - xj[0], ym[1] - xj[1], ym[2] - xj[2]};
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double g[3], Q[3], xh[3];
            for (int i = 0; i < 3; ++i) {
                g[i] = f[3 * j + i] - fn0 * nj[i];
                Q[i] = q[3 * j + i] - qm0[i];
                xh[i] = xj[i] - xm0[i];
            }
            if (r > Rc) {
                ora_sl_plain(d, r, g, w[j], su);
                ora_dl_plain(d, r, Q, nj, w[j], sv);
            } else {
                ora_sl_term(d, r, delta, tc, g, w[j], su, 1);
                ora_dl_term_sharp(d, r, delta, tc, Q, nj, w[j], sv);
            }
        }
        for (int i = 0; i < 3; ++i) { u[3 * m + i] = su[i] * inv8pi; v[3 * m + i] = sv[i] * inv8pi + 0.5 * qm0[i]; }
    }
    return nfail;
}

/* Plain sums of Eqs. (Stokes_SL), (Stokes_DL) with the given densities and no
 * subtraction or regularization, skipping coincident pairs (r == 0). */
void ora_plain(const double *x, const double *nrm, const double *w, const double *f, const double *q, int64_t N,
               const double *y, int64_t M, double *u, double *v) {
    const double inv8pi = 1.0 / (8.0 * ORA_PI);
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < M; ++m) {
        const double *ym = y + 3 * m;
        double su[3] = {0, 0, 0}, sv[3] = {0, 0, 0};
        for (int64_t j = 0; j < N; ++j) {
            double d[3] = {ym[0] - x[3 * j], ym[1] - x[3 * j + 1], ym[2] - x[3 * j + 2]};
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (r == 0.0) continue;
            ora_sl_plain(d, r, f + 3 * j, w[j], su);
            ora_dl_plain(d, r, q + 3 * j, nrm + 3 * j, w[j], sv);
        }
        for (int i = 0; i < 3; ++i) { u[3 * m + i] = su[i] * inv8pi; v[3 * m + i] = sv[i] * inv8pi; }
    }
}

int ora_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
