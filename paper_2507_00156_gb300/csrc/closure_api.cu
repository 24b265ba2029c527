// The learned closure of the near field: one or two regularized sums instead of three, and what
// they miss of the extrapolated value predicted from local data by a small network.
//
// Eq. (extrap_eqn) says u^{delta_k} = u + c1 rho_k I0(lambda_k) + c2 rho_k^3 I2(lambda_k) + O(delta^5)
// with c1, c2 independent of delta.
//   ndelta = 1 (the single sum u^{delta_0}, near set r <= cutoff_t delta_0): the closure predicts
//     the whole correction u - u^{delta_0}.
//   ndelta = 2 (two deltas, near set r <= cutoff_t delta_1): with the weights beta (sum beta = 1,
//     sum beta rho I0 = 0) the two sums give u + gamma c2, gamma = sum beta rho^3 I2, so
//     u = sum_k beta_k u^{delta_k} - gamma c2, and the closure predicts c2.
// c1 and c2 are fixed by the surface and the density near the closest point x0 and are linear in
// the density.  The single-layer kernel is O(1/r) and its delta^3 term involves the density up to
// second derivatives; the double-layer kernel is O(1/r^2) and involves one derivative more.  So
// the closure is a linear map from the density jets at x0 to the correction whose coefficients
// the network predicts from the local geometry:
//   frame    t1, t2, n0: the principal directions at x0 (where the principal curvatures agree to
//            1e-6, a fixed tangent basis built from n0);
//   geometry lambda_0 = b / delta_0, kappa_1 h, kappa_2 h (principal curvatures, kappa_1 >= kappa_2),
//            rho_0, rho_1;
//   jets     derivatives of the density components along t1, t2, n0 with respect to the
//            tangent-plane coordinates (xi, eta) = ((x - x0).t1, (x - x0).t2) / h, from the
//            least-squares polynomial of total degree <= 4 fitted to the node values within 3.5 h
//            of x0: single layer orders 0..2 (18 values), double layer orders 1..3 (27 values),
//            divided by their largest magnitude S;
//   output   c (3 components in the frame) = sum_j A_ej(geometry) jet_j, the correction divided by
//            S h^p (p = 1 single layer, p = 0 double layer; for ndelta = 2 also by -gamma).
// A validation sample of targets is also given the three-delta method's value (the closure's sums
// plus the difference of the near-field-only sums with three and with nd deltas, the far field
// being the same in both; see k_compare): per layer the
// network's correction is kept only if it brings the sample closer to the method than the sums
// without it, and if either layer still differs by more than a tolerance the whole evaluation
// falls back to the three-delta method.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "ers_internal.h"
#include "mlp.h"

using namespace ers;

struct ers_closure {
    int device = 0;
    uint64_t seed = 0;
    float *p[2] = {nullptr, nullptr};  // FP32 master parameters: [0] single layer, [1] double layer
    float *q[2] = {nullptr, nullptr};  // BF16-rounded copies (reference forward / training)
    float *m[2] = {nullptr, nullptr}, *v[2] = {nullptr, nullptr};  // Adam moments
    int step[2] = {0, 0};
    int *err = nullptr;
    // extent of the training geometry: [layer][0 lo, 1 hi][feature] as order-preserving int keys
    int *range = nullptr;
    int have_range[2] = {0, 0};
    int range_check = 1;     // ers_eval_learned sends targets outside the extent to the method
    int64_t last_out = 0;    // targets of the last ers_eval_learned that were outside it
    // per layer, from the validation of the last ers_eval_learned: network kept (1) or not (0),
    // the sample's error with and without the network's correction
    int last_used[2] = {0, 0};
    double last_err_with[2] = {0.0, 0.0}, last_err_without[2] = {0.0, 0.0};
    Scratch z, a, d4, d, g, idx, loss;
    // evaluation work buffers
    Scratch feat, scale, gamma, outp, sub, valid, oor;
};

namespace ers {
namespace {

using namespace mlp;
constexpr int NFEAT = NGEOM;      // features checked against the training extent (the geometry)
constexpr int NB = 15;            // monomials of total degree <= 4 in two variables
constexpr int NPK = NB * (NB + 1) / 2;
constexpr int NRHS = 6;           // f and q, three components each, in the frame
constexpr double FIT_R = 3.5;     // fit radius in units of h
constexpr int FEAT_THREADS = 64;  // threads per block of the features kernel
constexpr size_t FEAT_SMEM = sizeof(double) * NPK * FEAT_THREADS;  // a Cholesky factor per thread

// t1 = n x a / |n x a| with a = e_x (e_y when |n_x| >= 0.9), t2 = n x t1.
__host__ __device__ __forceinline__ void fallback_frame(const double n[3], double t1[3], double t2[3]) {
    const double a0 = fabs(n[0]) < 0.9 ? 1.0 : 0.0, a1 = 1.0 - a0;
    const double c0 = -n[2] * a1, c1 = n[2] * a0, c2 = n[0] * a1 - n[1] * a0;
    const double inv = 1.0 / sqrt(c0 * c0 + c1 * c1 + c2 * c2);
    t1[0] = c0 * inv;
    t1[1] = c1 * inv;
    t1[2] = c2 * inv;
    t2[0] = n[1] * t1[2] - n[2] * t1[1];
    t2[1] = n[2] * t1[0] - n[0] * t1[2];
    t2[2] = n[0] * t1[1] - n[1] * t1[0];
}

// Principal frame and curvatures of the ellipsoid sum((x - c)/a)^2 = 1 at x0 (p = x0 - c, unit
// normal n): the shape operator on the tangent plane is (Hess F)/|grad F| restricted to it, with
// F the implicit function (Hess F = diag(2/a^2), grad F = 2 p/a^2); in the basis (e1, e2) of
// fallback_frame it is the symmetric 2 x 2 matrix S below.  k1 >= k2 are its eigenvalues; t1 is
// the eigenvector of k1 signed so that its e1 component is >= 0 (its e2 component > 0 when that
// is 0), t2 = n x t1.  Where the eigenvalues agree to 1e-6 of |S00| + |S11| (every point of a
// sphere) the frame is (e1, e2, n).
__device__ __forceinline__ void principal_frame(const double p[3], const double a[3], const double n[3],
                                                double t1[3], double t2[3], double &k1, double &k2) {
    double e1[3], e2[3];
    fallback_frame(n, e1, e2);
    double g2 = 0.0, hd[3];
    for (int i = 0; i < 3; ++i) {
        const double ia2 = 1.0 / (a[i] * a[i]);
        const double gi = 2.0 * p[i] * ia2;
        g2 += gi * gi;
        hd[i] = 2.0 * ia2;
    }
    const double ig = 1.0 / sqrt(g2);
    double S00 = 0.0, S01 = 0.0, S11 = 0.0;
    for (int i = 0; i < 3; ++i) {
        S00 += hd[i] * e1[i] * e1[i];
        S01 += hd[i] * e1[i] * e2[i];
        S11 += hd[i] * e2[i] * e2[i];
    }
    S00 *= ig;
    S01 *= ig;
    S11 *= ig;
    const double mid = 0.5 * (S00 + S11), r = hypot(0.5 * (S00 - S11), S01);
    k1 = mid + r;
    k2 = mid - r;
    if (2.0 * r <= 1e-6 * (fabs(S00) + fabs(S11))) {
        for (int i = 0; i < 3; ++i) {
            t1[i] = e1[i];
            t2[i] = e2[i];
        }
        return;
    }
    // (S - k1 I) v = 0: v = (k1 - S11, S01) or (S01, k1 - S00), the larger one
    double v0 = k1 - S11, v1 = S01;
    const double w0 = S01, w1 = k1 - S00;
    if (w0 * w0 + w1 * w1 > v0 * v0 + v1 * v1) {
        v0 = w0;
        v1 = w1;
    }
    if (v0 < 0.0 || (v0 == 0.0 && v1 < 0.0)) {
        v0 = -v0;
        v1 = -v1;
    }
    double tn = 0.0;
    for (int i = 0; i < 3; ++i) {
        t1[i] = v0 * e1[i] + v1 * e2[i];
        tn += t1[i] * t1[i];
    }
    tn = 1.0 / sqrt(tn);
    for (int i = 0; i < 3; ++i) t1[i] *= tn;
    t2[0] = n[1] * t1[2] - n[2] * t1[1];
    t2[1] = n[2] * t1[0] - n[0] * t1[2];
    t2[2] = n[0] * t1[1] - n[1] * t1[0];
}

// Frame of target m from its closest point (shared by the features, the correction and the
// validation, so that all three use the same frame).
__device__ __forceinline__ void target_frame(const double *x0, const double *n0, int64_t m, const double c[3],
                                             const double a[3], double t1[3], double t2[3], double n[3], double &k1,
                                             double &k2) {
    double p[3];
    for (int i = 0; i < 3; ++i) {
        n[i] = n0[3 * m + i];
        p[i] = x0[3 * m + i] - c[i];
    }
    principal_frame(p, a, n, t1, t2, k1, k2);
}

// The density fit of a target (degree-4 least squares in the scaled tangent-plane coordinates
// (xi, eta) = ((x - x0).t1, (x - x0).t2) / (3.5 h) over the nodes within 3.5 h of x0) in three
// convergent passes (one thread per target each):
//   k_fit_scan   the target's neighbours (an FP32 distance prefilter, the FP64 test |x - x0|^2 <=
//                (3.5 h)^2 where the prefilter is not conclusive) into a list;
//   k_fit_accum  over the list (three passes): the 45 moments sum xi^p eta^q (p + q <= 8), which
//                hold every entry of Phi^T Phi, and Phi^T U for the 6 density components along
//                t1, t2, n0, accumulated in float pairs;
//   k_features   Phi^T Phi from the moments, Cholesky, the coefficients of the monomials of degree
//                <= 3, then the features.
// Separate passes keep the lanes of a warp on the same instructions (one thread per target walking
// its own candidates would run the accumulation whenever any lane found a neighbour).
constexpr int FIT_LMAX = 96;   // neighbours per target at most (about 53 on a lattice surface)
constexpr int NMOM = 45;       // moments of degree <= 8
constexpr int NACC = NMOM + NB * NRHS;  // 135 accumulated values per target

// monomial k of degree <= 4 (ordered by degree, then by falling power of xi) = xi^mi(k) eta^mj(k)
__host__ __device__ constexpr int mono_j(int k) { return k == 0 ? 0 : (k < 3 ? k - 1 : (k < 6 ? k - 3 : (k < 10 ? k - 6 : k - 10))); }
__host__ __device__ constexpr int mono_d(int k) { return k == 0 ? 0 : (k < 3 ? 1 : (k < 6 ? 2 : (k < 10 ? 3 : 4))); }
__host__ __device__ constexpr int mono_i(int k) { return mono_d(k) - mono_j(k); }
// index of the moment xi^p eta^q, p + q = d: d (d + 1) / 2 + q
__host__ __device__ constexpr int mom_idx(int p, int q) { return (p + q) * (p + q + 1) / 2 + q; }

// i! j! / 3.5^(i + j) of monomial k (degrees <= 3): the derivative d^(i+j)/dxi^i deta^j in units
// of h of the fit in the scaled coordinates (xi, eta) / 3.5.
__device__ __forceinline__ double deriv_factor(int k) {
    constexpr double r = 1.0 / FIT_R;
    switch (k) {
        case 0: return 1.0;
        case 1: case 2: return r;
        case 3: case 5: return 2.0 * r * r;
        case 4: return r * r;
        case 6: case 9: return 6.0 * r * r * r;
        default: return 2.0 * r * r * r;  // 7, 8: (2,1), (1,2)
    }
}

struct FitArgs {
    SurfDev sd;
    const double *fq;
    const double *x0, *n0, *b;
    int64_t M;
    double h, Rc, c[3], a[3];
    int *list;    // [FIT_LMAX][M]
    int *cnt;     // [M]: neighbours, or -1 (no fit: beyond Rc, or more than FIT_LMAX)
    double *acc;  // [NACC][M]
};

__device__ __forceinline__ bool fit_target(const FitArgs &A, int64_t m, double x0[3]) {
    for (int i = 0; i < 3; ++i) x0[i] = A.x0[3 * m + i];
    return fabs(A.b[m]) <= A.Rc;
}

__global__ void k_fit_scan(FitArgs A) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= A.M) return;
    double x0[3];
    if (!fit_target(A, m, x0)) {
        A.cnt[m] = -1;
        return;
    }
    const double R = FIT_R * A.h, R2 = R * R;
    const float x0f[3] = {(float)x0[0], (float)x0[1], (float)x0[2]};
    const float R2f = (float)R2;
    // FP32 distances carry an absolute error below 4 (|x0| + R) 2^-23 2R; outside that band the
    // FP32 test decides, inside it the FP64 one
    const double amax = fmax(fabs(x0[0]), fmax(fabs(x0[1]), fabs(x0[2]))) + R;
    const float band = (float)(8.0 * amax * 1.1920928955078125e-7 * 2.0 * R) + 1e-30f;
    const Grid &G = A.sd.grid;
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = max(0, (int)floor((x0[a] - R - G.origin[a]) / G.cw));
        hi[a] = min(G.nc[a] - 1, (int)floor((x0[a] + R - G.origin[a]) / G.cw));
    }
    int cnt = 0;
    for (int iz = lo[2]; iz <= hi[2]; ++iz)
        for (int iy = lo[1]; iy <= hi[1]; ++iy) {
            const int64_t row = ((int64_t)iz * G.nc[1] + iy) * G.nc[0];
            const int js = A.sd.cell_start[row + lo[0]], je = A.sd.cell_start[row + hi[0] + 1];
            for (int j = js; j < je; ++j) {
                const float4 p = __ldg(A.sd.xs32 + j);
                const float dx = p.x - x0f[0], dy = p.y - x0f[1], dz = p.z - x0f[2];
                const float d2 = dx * dx + dy * dy + dz * dz;
                bool in = d2 <= R2f - band;
                if (!in && d2 <= R2f + band) {
                    const double *r = A.sd.rec + (int64_t)j * REC;
                    const double d[3] = {r[0] - x0[0], r[1] - x0[1], r[2] - x0[2]};
                    in = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] <= R2;
                }
                if (in) {
                    if (cnt < FIT_LMAX) A.list[(int64_t)cnt * A.M + m] = j;
                    ++cnt;
                }
            }
        }
    A.cnt[m] = cnt <= FIT_LMAX ? cnt : -1;
}

// The coordinates (xi, eta) and the density components in the frame come from FP64 and are split
// into float pairs once per node; the powers, the 45 moments and Phi^T U accumulate in float-pair
// arithmetic on the FP32 pipe (~1e-14 relative, the FP64 pipe of this part runs 1/64 of its
// rate) and are stored as doubles for the FP64 Cholesky.
__global__ void __launch_bounds__(128) k_fit_accum(FitArgs A) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= A.M) return;
    const int cnt = A.cnt[m];
    if (cnt < NB) return;
    double x0[3], t1[3], t2[3], n[3], k1, k2;
    fit_target(A, m, x0);
    target_frame(A.x0, A.n0, m, A.c, A.a, t1, t2, n, k1, k2);
    const double iR = 1.0 / (FIT_R * A.h);
    // pass 0: the moments; pass 1: Phi^T U of the single-layer density; pass 2: of the double-layer
    // density (three passes over the list keep the float-pair accumulators within the registers)
#pragma unroll
    for (int pass = 0; pass < 3; ++pass) {
        constexpr int NV = NMOM > NB * 3 ? NMOM : NB * 3;
        fpair acc[NV];
#pragma unroll
        for (int e = 0; e < NV; ++e) acc[e] = {0.0f, 0.0f};
        for (int k = 0; k < cnt; ++k) {
            const int j = A.list[(int64_t)k * A.M + m];
            const double *r = A.sd.rec + (int64_t)j * REC;
            const double d[3] = {r[0] - x0[0], r[1] - x0[1], r[2] - x0[2]};
            const fpair xi = fp_split((d[0] * t1[0] + d[1] * t1[1] + d[2] * t1[2]) * iR);
            const fpair eta = fp_split((d[0] * t2[0] + d[1] * t2[1] + d[2] * t2[2]) * iR);
            fpair xp[9], ep[9];
            xp[0] = ep[0] = {1.0f, 0.0f};
#pragma unroll
            for (int i = 1; i < (pass == 0 ? 9 : 5); ++i) {
                xp[i] = fp_mul(xp[i - 1], xi);
                ep[i] = fp_mul(ep[i - 1], eta);
            }
            if (pass == 0) {
#pragma unroll
                for (int dd = 0; dd <= 8; ++dd)
#pragma unroll
                    for (int q = 0; q <= dd; ++q)
                        acc[mom_idx(dd - q, q)] = fp_fma(xp[dd - q], ep[q], acc[mom_idx(dd - q, q)]);
            } else {
                const double *u = A.fq + (int64_t)j * 6 + 3 * (pass - 1);
                const fpair uf[3] = {fp_split(u[0] * t1[0] + u[1] * t1[1] + u[2] * t1[2]),
                                     fp_split(u[0] * t2[0] + u[1] * t2[1] + u[2] * t2[2]),
                                     fp_split(u[0] * n[0] + u[1] * n[1] + u[2] * n[2])};
#pragma unroll
                for (int i = 0; i < NB; ++i) {
                    const fpair phi = fp_mul(xp[mono_i(i)], ep[mono_j(i)]);
#pragma unroll
                    for (int c = 0; c < 3; ++c) acc[3 * i + c] = fp_fma(phi, uf[c], acc[3 * i + c]);
                }
            }
        }
        if (pass == 0) {
#pragma unroll
            for (int e = 0; e < NMOM; ++e) A.acc[(int64_t)e * A.M + m] = fp_to_double(acc[e]);
        } else {
#pragma unroll
            for (int e = 0; e < NB * 3; ++e)
                A.acc[(int64_t)(NMOM + (pass - 1) * NB * 3 + e) * A.M + m] = fp_to_double(acc[e]);
        }
    }
}

// Cholesky of Phi^T Phi (assembled from the moments into this thread's column of shared memory,
// stride FEAT_THREADS) and the coefficients of the monomials of degree <= 3 for the 6 density
// components, as derivatives in units of h: out[k][r].  False with fewer than 15 neighbours or a
// pivot <= 0.
__device__ bool fit_solve(const FitArgs &A, int64_t m, double *L, double out[10][NRHS]) {
    const int S = FEAT_THREADS;
    if (A.cnt[m] < NB) return false;
    for (int i = 0; i < NB; ++i)
        for (int k = 0; k <= i; ++k)
            L[(i * (i + 1) / 2 + k) * S] = A.acc[(int64_t)mom_idx(mono_i(i) + mono_i(k), mono_j(i) + mono_j(k)) * A.M + m];
    // the reciprocals of the diagonal, so that the factorization and the solves multiply (an FP64
    // division costs several FP64-pipe instructions)
    double rd[NB];
    for (int i = 0; i < NB; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = L[(i * (i + 1) / 2 + j) * S];
            for (int q = 0; q < j; ++q) s -= L[(i * (i + 1) / 2 + q) * S] * L[(j * (j + 1) / 2 + q) * S];
            if (i == j) {
                if (!(s > 0.0)) return false;
                const double l = sqrt(s);
                L[(i * (i + 1) / 2 + i) * S] = l;
                rd[i] = 1.0 / l;
            } else {
                L[(i * (i + 1) / 2 + j) * S] = s * rd[j];
            }
        }
    for (int rc = 0; rc < NRHS; ++rc) {
        double y[NB];
        for (int i = 0; i < NB; ++i) {  // L y = (Phi^T U)_rc
            double s = A.acc[(int64_t)(NMOM + (rc / 3) * NB * 3 + 3 * i + rc % 3) * A.M + m];
            for (int q = 0; q < i; ++q) s -= L[(i * (i + 1) / 2 + q) * S] * y[q];
            y[i] = s * rd[i];
        }
        for (int i = NB - 1; i >= 0; --i) {  // L^T x = y
            double s = y[i];
            for (int q = i + 1; q < NB; ++q) s -= L[(q * (q + 1) / 2 + i) * S] * y[q];
            y[i] = s * rd[i];
        }
        for (int k = 0; k < 10; ++k) out[k][rc] = y[k] * deriv_factor(k);
    }
    return true;
}

struct FeatArgs {
    FitArgs fit;
    const double *u2, *v2, *gamma, *u3, *v3;  // u3, v3 optional (training targets)
    double rho0, rho1;
    int nd;            // 1 or 2 deltas
    double gamma0;     // |gamma| at b = 0 (nd = 2)
    float *Xs, *Xd, *Ts, *Td;  // sample records (M x XSTR) and targets (M x TSTR) of both layers
    double *scale;             // (M x 2) density scales, 0 = no correction
    int *valid;
};

// One thread per target: frame, geometry, density jets (both layers) from the fit, training
// targets when u3, v3 are given.
__global__ void __launch_bounds__(FEAT_THREADS) k_features(FeatArgs A) {
    extern __shared__ double fsm[];
    const FitArgs &F = A.fit;
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= F.M) return;
    double t1[3], t2[3], n[3], k1, k2;
    target_frame(F.x0, F.n0, m, F.c, F.a, t1, t2, n, k1, k2);
    const double bm = F.b[m];
    const double lam = bm / (A.rho0 * F.h);
    bool ok = fabs(bm) <= F.Rc && fabs(lam) <= 64.0;
    double J[10][NRHS];
    if (ok) ok = fit_solve(F, m, fsm + threadIdx.x, J);
    bool any = false;
    for (int layer = 0; layer < 2; ++layer) {
        const int nj = jets_of_layer(layer);
        float *X = (layer == 0 ? A.Xs : A.Xd) + m * XSTR;
        X[0] = (float)lam;
        X[1] = (float)(k1 * F.h);
        X[2] = (float)(k2 * F.h);
        X[3] = (float)A.rho0;
        X[4] = (float)A.rho1;
        for (int e = NGEOM; e < JET_OFF; ++e) X[e] = 0.0f;
        // jets, component-major: single layer orders 0..2 (monomials 0..5), double layer 1..3 (1..9)
        double jl[NJ_DL];
        const int k0 = layer == 0 ? 0 : 1, nk = layer == 0 ? 6 : 9;
        double S = 0.0;
        for (int e = 0; e < 3; ++e)
            for (int k = 0; k < nk; ++k) {
                const double v = ok ? J[k0 + k][3 * layer + e] : 0.0;
                jl[e * nk + k] = v;
                S = fmax(S, fabs(v));
            }
        const bool lok = ok && S > 0.0 && isfinite(S);
        for (int j = 0; j < NJ_MAX; ++j) X[JET_OFF + j] = (lok && j < nj) ? (float)(jl[j] / S) : 0.0f;
        A.scale[2 * m + layer] = lok ? S : 0.0;
        float *T = layer == 0 ? A.Ts : A.Td;
        const double *u3 = layer == 0 ? A.u3 : A.v3;
        if (T && u3) {
            const double *ur = (layer == 0 ? A.u2 : A.v2) + 3 * m;
            const double g = A.gamma[m];
            const double hp = layer == 0 ? F.h : 1.0;
            double cv[3] = {0.0, 0.0, 0.0}, w = 0.0;
            if (lok && A.nd == 2 && fabs(g) >= 0.01 * A.gamma0) {
                for (int i = 0; i < 3; ++i) cv[i] = (ur[i] - u3[3 * m + i]) / g;
                w = (g / A.gamma0) * (g / A.gamma0);
            } else if (lok && A.nd == 1) {
                for (int i = 0; i < 3; ++i) cv[i] = u3[3 * m + i] - ur[i];
                w = 1.0;
            }
            const double den = w > 0.0 ? S * hp : 1.0;
            T[m * TSTR + 0] = (float)((cv[0] * t1[0] + cv[1] * t1[1] + cv[2] * t1[2]) / den);
            T[m * TSTR + 1] = (float)((cv[0] * t2[0] + cv[1] * t2[1] + cv[2] * t2[2]) / den);
            T[m * TSTR + 2] = (float)((cv[0] * n[0] + cv[1] * n[1] + cv[2] * n[2]) / den);
            T[m * TSTR + 3] = (float)w;
            any = any || w > 0.0;
        }
    }
    if (A.valid) A.valid[m] = any ? 1 : 0;
}

// The network's correction of layer l where mask bit l is set and the density scale S > 0, added
// with sign `sign` (1 to apply it, -1 to take it back): ndelta = 2: u -= gamma S h^p (R c);
// ndelta = 1: u += S h^p (R c); R = [t1 t2 n0], p = 1 single layer, 0 double layer.
struct ApplyArgs {
    const double *x0, *n0, *gamma, *scale;
    const float *Ys, *Yd;
    int64_t M;
    double h;
    int nd, mask;
    double sign;
    double c[3], a[3];
    double *u, *v;
};

__device__ __forceinline__ void correction(const ApplyArgs &A, int64_t m, int layer, const double t1[3],
                                           const double t2[3], const double n[3], double corr[3]) {
    const double S = A.scale[2 * m + layer];
    const float *Y = (layer == 0 ? A.Ys : A.Yd) + m * OUT_STRIDE;
    const double hp = layer == 0 ? A.h : 1.0;
    const double f = A.nd == 2 ? -A.gamma[m] * S * hp : S * hp;
    for (int i = 0; i < 3; ++i) corr[i] = f * ((double)Y[0] * t1[i] + (double)Y[1] * t2[i] + (double)Y[2] * n[i]);
}

__global__ void k_apply(ApplyArgs A) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= A.M) return;
    if (!(A.scale[2 * m] > 0.0 || A.scale[2 * m + 1] > 0.0)) return;
    double t1[3], t2[3], n[3], k1, k2;
    target_frame(A.x0, A.n0, m, A.c, A.a, t1, t2, n, k1, k2);
    for (int layer = 0; layer < 2; ++layer) {
        double *out = layer == 0 ? A.u : A.v;
        if (!(A.mask & (1 << layer)) || !out || !(A.scale[2 * m + layer] > 0.0)) continue;
        double corr[3];
        correction(A, m, layer, t1, t2, n, corr);
        for (int i = 0; i < 3; ++i) out[3 * m + i] += A.sign * corr[i];
    }
}

// Gather every `stride`-th target (and its closest-point data and densities) into a compact set.
__global__ void k_gather(const double *__restrict__ y, const double *__restrict__ x0, const double *__restrict__ n0,
                         const double *__restrict__ b, const double *__restrict__ f0, const double *__restrict__ q0,
                         int64_t Ms, int stride, double *__restrict__ out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Ms) return;
    const int64_t m = k * stride;
    double *o = out;
    for (int i = 0; i < 3; ++i) {
        o[3 * k + i] = y[3 * m + i];
        o[3 * Ms + 3 * k + i] = x0[3 * m + i];
        o[6 * Ms + 3 * k + i] = n0[3 * m + i];
        o[10 * Ms + 3 * k + i] = f0 ? f0[3 * m + i] : 0.0;
        o[13 * Ms + 3 * k + i] = q0 ? q0[3 * m + i] : 0.0;
    }
    o[9 * Ms + k] = b[m];
}

// Over the validation sample (every stride-th target m = k stride) the three-delta method's value
// is r = (u - corr) + (n3 - nd): the closure's sums without the correction plus the difference of
// the near-field sums with three and with nd deltas (n3u.., ndu.., both over the three-delta near
// radius and without far field, which is then the same in both), or u itself where the method's
// value has replaced the closure's (scale < 0).
// res[0] = max |u - r|, res[1] = max |r| (single layer), res[2], res[3] the same for the double
// layer, and res[4], res[5] = max |u - corr - r| for the two layers: the errors without the
// network's correction (A carries the correction's inputs; A.sign is ignored).
__global__ void k_compare(ApplyArgs A, const double *__restrict__ n3u, const double *__restrict__ n3v,
                          const double *__restrict__ ndu, const double *__restrict__ ndv, int64_t Ms, int stride,
                          double *__restrict__ res) {
    double e[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < Ms; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = k * stride;
        double t1[3], t2[3], n[3], k1, k2;
        target_frame(A.x0, A.n0, m, A.c, A.a, t1, t2, n, k1, k2);
        for (int layer = 0; layer < 2; ++layer) {
            const double *out = layer == 0 ? A.u : A.v;
            const double *n3 = layer == 0 ? n3u : n3v, *nd = layer == 0 ? ndu : ndv;
            const double sc = A.scale[2 * m + layer];
            double corr[3] = {0.0, 0.0, 0.0};
            if (sc > 0.0) correction(A, m, layer, t1, t2, n, corr);
            for (int i = 0; i < 3; ++i) {
                const double o = out[3 * m + i];
                const double r = sc < 0.0 ? o : (o - corr[i]) + (n3[3 * k + i] - nd[3 * k + i]);
                e[2 * layer] = fmax(e[2 * layer], fabs(o - r));
                e[2 * layer + 1] = fmax(e[2 * layer + 1], fabs(r));
                e[4 + layer] = fmax(e[4 + layer], fabs(o - corr[i] - r));
            }
        }
    }
    for (int j = 0; j < 6; ++j) {
        double x = e[j];
        for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
        if ((threadIdx.x & 31) == 0)
            atomicMax(reinterpret_cast<unsigned long long *>(res + j), (unsigned long long)__double_as_longlong(x));
    }
}

__global__ void k_minibatch(int *__restrict__ idx, int n, int64_t total, uint64_t seed, uint64_t step) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (step * 0x100000001B3ull + (uint64_t)i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    idx[i] = (int)(z % (uint64_t)total);
}

// Order-preserving map of a float to an int (and its inverse, the same map): integer order of the
// keys = numeric order of the floats, so that atomicMin / atomicMax on keys track a float extent.
__host__ __device__ __forceinline__ int range_key(int bits) { return bits >= 0 ? bits : bits ^ 0x7fffffff; }

constexpr int RANGE_STRIDE = 2 * IN;  // ints per layer: lo[IN], hi[IN]

// Widen the extent keys[0..NFEAT) (lo), keys[IN..IN+NFEAT) (hi) to cover the finite features of
// the sample records X (n, XSTR).
__global__ void k_range_update(const float *__restrict__ X, int64_t n, int *__restrict__ keys) {
    int lo[NFEAT], hi[NFEAT];
#pragma unroll
    for (int f = 0; f < NFEAT; ++f) {
        lo[f] = 0x7fffffff;
        hi[f] = (int)0x80000000;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int f = 0; f < NFEAT; ++f) {
            const float x = X[i * XSTR + f];
            if (!isfinite(x)) continue;
            const int k = range_key(__float_as_int(x));
            lo[f] = min(lo[f], k);
            hi[f] = max(hi[f], k);
        }
    }
#pragma unroll
    for (int f = 0; f < NFEAT; ++f) {
        const int l = __reduce_min_sync(0xffffffffu, lo[f]), h = __reduce_max_sync(0xffffffffu, hi[f]);
        if ((threadIdx.x & 31) == 0) {
            atomicMin(keys + f, l);
            atomicMax(keys + IN + f, h);
        }
    }
}

// Targets whose features (of a layer with a known extent) lie outside that extent widened by
// 5 % of its width plus 1e-3 of its magnitude plus 1e-6: their indices are appended to idx.
// Only corrected targets (density scale > 0) are checked.
__global__ void k_range_flags(const float *__restrict__ Xs, const float *__restrict__ Xd,
                              const double *__restrict__ scale, int64_t M, const int *__restrict__ keys, int have0,
                              int have1, int64_t *__restrict__ idx, unsigned long long *__restrict__ count) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    bool out = false;
    for (int layer = 0; layer < 2; ++layer) {
        if (!(layer == 0 ? have0 : have1) || !(scale[2 * m + layer] > 0.0)) continue;
        const float *X = (layer == 0 ? Xs : Xd) + m * XSTR;
        const int *K = keys + layer * RANGE_STRIDE;
        for (int f = 0; f < NFEAT; ++f) {
            const float lo = __int_as_float(range_key(K[f])), hi = __int_as_float(range_key(K[IN + f]));
            // explicit roundings (no contraction), so that a host computation can repeat the decision
            const float tol = __fadd_rn(__fadd_rn(__fmul_rn(0.05f, __fsub_rn(hi, lo)),
                                                  __fmul_rn(1e-3f, fmaxf(fabsf(lo), fabsf(hi)))),
                                        1e-6f);
            const float x = X[f];
            if (!(x >= __fsub_rn(lo, tol) && x <= __fadd_rn(hi, tol))) out = true;
        }
    }
    if (out) idx[atomicAdd(count, 1ull)] = m;
}

// Gather the targets idx[0..K) (and their closest-point data and densities) into a compact set
// (the layout of k_gather), and scatter results back.
__global__ void k_gather_idx(const double *__restrict__ y, const double *__restrict__ x0,
                             const double *__restrict__ n0, const double *__restrict__ b,
                             const double *__restrict__ f0, const double *__restrict__ q0,
                             const int64_t *__restrict__ idx, int64_t K, double *__restrict__ out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int64_t m = idx[k];
    for (int i = 0; i < 3; ++i) {
        out[3 * k + i] = y[3 * m + i];
        out[3 * K + 3 * k + i] = x0[3 * m + i];
        out[6 * K + 3 * k + i] = n0[3 * m + i];
        out[10 * K + 3 * k + i] = f0[3 * m + i];
        out[13 * K + 3 * k + i] = q0[3 * m + i];
    }
    out[9 * K + k] = b[m];
}

// ... and give them the method's values: the closure's sums without the correction plus the
// difference of the near-field sums with three and with nd deltas (the far field is the same in
// both); those targets carry no correction any more (scale -1: the method's value).
__global__ void k_replace_idx(ApplyArgs A, const double *__restrict__ n3u, const double *__restrict__ n3v,
                              const double *__restrict__ ndu, const double *__restrict__ ndv,
                              const int64_t *__restrict__ idx, int64_t K, double *__restrict__ scale) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int64_t m = idx[k];
    double t1[3], t2[3], n[3], k1, k2;
    target_frame(A.x0, A.n0, m, A.c, A.a, t1, t2, n, k1, k2);
    for (int layer = 0; layer < 2; ++layer) {
        double *out = layer == 0 ? A.u : A.v;
        const double *n3 = layer == 0 ? n3u : n3v, *nd = layer == 0 ? ndu : ndv;
        double corr[3] = {0.0, 0.0, 0.0};
        if (A.scale[2 * m + layer] > 0.0) correction(A, m, layer, t1, t2, n, corr);
        for (int i = 0; i < 3; ++i) out[3 * m + i] += (n3[3 * k + i] - nd[3 * k + i]) - corr[i];
    }
    scale[2 * m] = -1.0;
    scale[2 * m + 1] = -1.0;
}

int closure_check(const ers_closure *c, int layer) {
    if (!c) return fail(ERS_E_INVAL, "NULL closure");
    if (layer != 0 && layer != 1) return fail(ERS_E_INVAL, "layer must be 0 (single) or 1 (double)");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != c->device) return fail(ERS_E_INVAL, "the current device is not the closure's device");
    return ERS_OK;
}

void free_closure(ers_closure *c) {
    if (!c) return;
    for (int l = 0; l < 2; ++l) {
        if (c->p[l]) cudaFree(c->p[l]);
        if (c->q[l]) cudaFree(c->q[l]);
        if (c->m[l]) cudaFree(c->m[l]);
        if (c->v[l]) cudaFree(c->v[l]);
    }
    if (c->err) cudaFree(c->err);
    if (c->range) cudaFree(c->range);
    Scratch *ss[] = {&c->z, &c->a, &c->d4, &c->d, &c->g, &c->idx, &c->loss, &c->feat, &c->scale, &c->gamma,
                     &c->outp, &c->sub, &c->valid, &c->oor};
    for (Scratch *s : ss)
        if (s->ptr) cudaFree(s->ptr);
    delete c;
}

int infer(ers_closure *c, int layer, const float *X, int64_t n, float *Y, cudaStream_t st) {
    if (n == 0) return ERS_OK;
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    const int64_t tiles = (n + 127) / 128;
    const int grid = (int)std::min<int64_t>(tiles, (int64_t)nsm * 4);
    cudaError_t e = launch_infer_tc(c->p[layer], X, n, Y, jets_of_layer(layer), c->err, grid, st);
    if (e != cudaSuccess) return cuda_fail(e, "closure inference kernel");
    return ERS_OK;
}

}  // namespace
}  // namespace ers

extern "C" {

int ers_closure_create(uint64_t seed, ers_closure **out) {
    clear_error();
    if (!out) return fail(ERS_E_INVAL, "ers_closure_create: NULL output");
    *out = nullptr;
    ers_closure *c = new (std::nothrow) ers_closure();
    if (!c) return fail(ERS_E_NOMEM, "ers_closure_create: host allocation failed");
    cudaGetDevice(&c->device);
    c->seed = seed;
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < 2 && e == cudaSuccess; ++l) {
        e = cudaMalloc(&c->p[l], sizeof(float) * mlp::NPARAM);
        if (e == cudaSuccess) e = cudaMalloc(&c->q[l], sizeof(float) * mlp::NPARAM);
        if (e == cudaSuccess) e = cudaMalloc(&c->m[l], sizeof(float) * mlp::NPARAM);
        if (e == cudaSuccess) e = cudaMalloc(&c->v[l], sizeof(float) * mlp::NPARAM);
    }
    if (e == cudaSuccess) e = cudaMalloc(&c->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->range, sizeof(int) * 2 * RANGE_STRIDE);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_closure(c);
        return fail(ERS_E_NOMEM, "ers_closure_create: device allocation failed");
    }
    // He-uniform hidden weights from a seeded generator, zero biases, and a zero last layer: an
    // untrained network predicts no correction
    std::mt19937_64 rng(seed);
    for (int l = 0; l < 2; ++l) {
        std::vector<float> h(mlp::NPARAM, 0.0f);
        auto fill = [&](int off, int rows, int cols, int used_rows) {
            const double bound = std::sqrt(6.0 / cols);
            std::uniform_real_distribution<double> U(-bound, bound);
            for (int r = 0; r < rows; ++r)
                for (int k = 0; k < cols; ++k) h[off + r * cols + k] = r < used_rows ? (float)U(rng) : 0.0f;
        };
        fill(mlp::OFF_W1, mlp::HID, mlp::IN, mlp::HID);
        fill(mlp::OFF_W2, mlp::HID, mlp::HID, mlp::HID);
        fill(mlp::OFF_W3, mlp::HID, mlp::HID, mlp::HID);
        fill(mlp::OFF_W4, mlp::OUT, mlp::HID, 0);
        e = cudaMemcpy(c->p[l], h.data(), sizeof(float) * mlp::NPARAM, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(c->m[l], 0, sizeof(float) * mlp::NPARAM);
        if (e == cudaSuccess) e = cudaMemset(c->v[l], 0, sizeof(float) * mlp::NPARAM);
        if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = cudaMemset(c->err, 0, sizeof(int));
    if (e == cudaSuccess) {  // empty extents: lo = +inf, hi = -inf
        std::vector<int> k(2 * RANGE_STRIDE);
        for (int l = 0; l < 2; ++l)
            for (int f = 0; f < mlp::IN; ++f) {
                k[l * RANGE_STRIDE + f] = range_key(0x7f800000);
                k[l * RANGE_STRIDE + mlp::IN + f] = range_key((int)0xff800000u);
            }
        e = cudaMemcpy(c->range, k.data(), sizeof(int) * k.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        free_closure(c);
        return cuda_fail(e, "ers_closure_create: initialisation");
    }
    *out = c;
    return ERS_OK;
}

int ers_closure_free(ers_closure *c) {
    clear_error();
    free_closure(c);
    return ERS_OK;
}

int ers_closure_params(ers_closure *c, int layer, float *get, const float *set, int64_t count) {
    clear_error();
    int rc = closure_check(c, layer);
    if (rc != ERS_OK) return rc;
    if (count != mlp::NPARAM) return fail(ERS_E_INVAL, "ers_closure_params: count must be " + std::to_string(mlp::NPARAM));
    cudaError_t e = cudaSuccess;
    if (set) e = cudaMemcpy(c->p[layer], set, sizeof(float) * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && get) e = cudaMemcpy(get, c->p[layer], sizeof(float) * count, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "ers_closure_params");
    return ERS_OK;
}

int ers_closure_infer(ers_closure *c, int layer, const float *X, int64_t n, float *Y, void *stream) {
    clear_error();
    int rc = closure_check(c, layer);
    if (rc != ERS_OK) return rc;
    if (n < 0 || (n > 0 && (!X || !Y))) return fail(ERS_E_INVAL, "ers_closure_infer: bad arrays");
    return infer(c, layer, X, n, Y, (cudaStream_t)stream);
}

int ers_closure_infer_reference(ers_closure *c, int layer, const float *X, int64_t n, float *Y, void *stream) {
    clear_error();
    int rc = closure_check(c, layer);
    if (rc != ERS_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = mlp::launch_quantize(c->p[layer], c->q[layer], st);
    if (e == cudaSuccess) e = mlp::launch_infer_ref(c->q[layer], X, n, Y, mlp::jets_of_layer(layer), st);
    if (e != cudaSuccess) return cuda_fail(e, "ers_closure_infer_reference");
    return ERS_OK;
}

int ers_closure_range(ers_closure *c, int layer, float *get, const float *set, int *have) {
    clear_error();
    int rc = closure_check(c, layer);
    if (rc != ERS_OK) return rc;
    int *dev = c->range + layer * RANGE_STRIDE;
    cudaError_t e = cudaSuccess;
    if (set) {
        int k[RANGE_STRIDE];
        for (int f = 0; f < mlp::IN; ++f) {
            const bool used = f < NFEAT;
            const float lo = used ? set[f] : INFINITY, hi = used ? set[NFEAT + f] : -INFINITY;
            if (used && !(lo <= hi)) return fail(ERS_E_INVAL, "ers_closure_range: need lo <= hi for every feature");
            int bl, bh;
            std::memcpy(&bl, &lo, sizeof bl);
            std::memcpy(&bh, &hi, sizeof bh);
            k[f] = range_key(bl);
            k[mlp::IN + f] = range_key(bh);
        }
        e = cudaMemcpy(dev, k, sizeof k, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) c->have_range[layer] = 1;
    }
    if (e == cudaSuccess && get) {
        int k[RANGE_STRIDE];
        e = cudaMemcpy(k, dev, sizeof k, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            for (int f = 0; f < NFEAT; ++f) {
                const int bl = range_key(k[f]), bh = range_key(k[mlp::IN + f]);
                std::memcpy(get + f, &bl, sizeof bl);
                std::memcpy(get + NFEAT + f, &bh, sizeof bh);
            }
    }
    if (e != cudaSuccess) return cuda_fail(e, "ers_closure_range");
    if (have) *have = c->have_range[layer];
    return ERS_OK;
}

int ers_closure_set_range_check(ers_closure *c, int enabled) {
    clear_error();
    if (!c) return fail(ERS_E_INVAL, "NULL closure");
    c->range_check = enabled ? 1 : 0;
    return ERS_OK;
}

int ers_closure_last_out_of_range(ers_closure *c, int64_t *n) {
    clear_error();
    if (!c || !n) return fail(ERS_E_INVAL, "ers_closure_last_out_of_range: NULL argument");
    *n = c->last_out;
    return ERS_OK;
}

// Test hook (not in the public header): run the bounded-wait probe once on the current device;
// *timed_out = 1 when its wait ran out.  Synchronous.
int ers_debug_wait_timeout(int arrive, int limit, int *timed_out) {
    clear_error();
    if (!timed_out || limit < 1) return fail(ERS_E_INVAL, "ers_debug_wait_timeout: bad arguments");
    int *flag = nullptr;
    cudaError_t e = cudaMalloc(&flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(flag, 0, sizeof(int));
    if (e == cudaSuccess) e = mlp::launch_wait_probe(arrive, (uint32_t)limit, flag, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(timed_out, flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (flag) cudaFree(flag);
    if (e != cudaSuccess) return cuda_fail(e, "ers_debug_wait_timeout");
    return ERS_OK;
}

int ers_closure_status(ers_closure *c, int *timed_out) {
    clear_error();
    if (!c || !timed_out) return fail(ERS_E_INVAL, "ers_closure_status: NULL argument");
    cudaError_t e = cudaMemcpy(timed_out, c->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "ers_closure_status");
    return ERS_OK;
}

static int grad_impl(ers_closure *c, int layer, const float *X, const float *T, const int *idx, int64_t n, float *G,
                     double *loss_dev, cudaStream_t st) {
    int rc = grow(c->z, sizeof(float) * n * 3 * mlp::HID);
    if (rc == ERS_OK) rc = grow(c->a, sizeof(float) * n * mlp::ACT);
    if (rc == ERS_OK) rc = grow(c->d4, sizeof(float) * n * mlp::OUT_USED);
    if (rc == ERS_OK) rc = grow(c->d, sizeof(float) * n * 3 * mlp::HID);
    if (rc != ERS_OK) return rc;
    cudaError_t e = mlp::launch_quantize(c->p[layer], c->q[layer], st);
    if (e == cudaSuccess)
        e = mlp::launch_train_grad(c->q[layer], X, T, idx, n, mlp::jets_of_layer(layer), (float *)c->z.ptr,
                                   (float *)c->a.ptr,
                                   (float *)c->d4.ptr, (float *)c->d.ptr, G, loss_dev, st);
    if (e != cudaSuccess) return cuda_fail(e, "closure training kernels");
    return ERS_OK;
}

int ers_closure_grad(ers_closure *c, int layer, const float *X, const float *T, int64_t n, float *G, double *loss,
                     void *stream) {
    clear_error();
    int rc = closure_check(c, layer);
    if (rc != ERS_OK) return rc;
    if (n <= 0 || !X || !T || !G) return fail(ERS_E_INVAL, "ers_closure_grad: bad arrays");
    if ((rc = grow(c->loss, sizeof(double))) != ERS_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(c->loss.ptr, 0, sizeof(double), st);
    if (e != cudaSuccess) return cuda_fail(e, "ers_closure_grad");
    if ((rc = grad_impl(c, layer, X, T, nullptr, n, G, (double *)c->loss.ptr, st)) != ERS_OK) return rc;
    if (loss) {
        e = cudaMemcpyAsync(loss, c->loss.ptr, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "ers_closure_grad: loss");
    }
    return ERS_OK;
}

int ers_closure_train(ers_closure *c, int layer, const float *X, const float *T, int64_t n, int steps, int batch,
                      float lr, double *final_loss, void *stream) {
    clear_error();
    int rc = closure_check(c, layer);
    if (rc != ERS_OK) return rc;
    if (n <= 0 || !X || !T || steps <= 0 || batch <= 0) return fail(ERS_E_INVAL, "ers_closure_train: bad arguments");
    if (n > INT32_MAX) return fail(ERS_E_UNSUPPORTED, "ers_closure_train: more than 2^31 samples");
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = grow(c->idx, sizeof(int) * batch)) != ERS_OK) return rc;
    if ((rc = grow(c->g, sizeof(float) * mlp::NPARAM)) != ERS_OK) return rc;
    if ((rc = grow(c->loss, sizeof(double))) != ERS_OK) return rc;
    {
        int nsm = 152;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
        const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4 * (int64_t)nsm);
        k_range_update<<<(unsigned)blocks, 256, 0, st>>>(X, n, c->range + layer * RANGE_STRIDE);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "ers_closure_train: feature extent");
        c->have_range[layer] = 1;
    }
    for (int s = 0; s < steps; ++s) {
        const bool last = s == steps - 1;
        k_minibatch<<<(batch + 255) / 256, 256, 0, st>>>((int *)c->idx.ptr, batch, n, c->seed + 7919 * layer,
                                                          (uint64_t)(c->step[layer] + 1));
        if (last) cudaMemsetAsync(c->loss.ptr, 0, sizeof(double), st);
        rc = grad_impl(c, layer, X, T, (const int *)c->idx.ptr, batch, (float *)c->g.ptr,
                       last ? (double *)c->loss.ptr : nullptr, st);
        if (rc != ERS_OK) return rc;
        c->step[layer] += 1;
        // cosine decay of the learning rate over this call
        const float lr_s = lr * 0.5f * (1.0f + cosf(3.14159265f * (float)s / (float)steps));
        cudaError_t e = mlp::launch_adam(c->p[layer], c->m[layer], c->v[layer], (const float *)c->g.ptr, lr_s,
                                         c->step[layer], st);
        if (e != cudaSuccess) return cuda_fail(e, "ers_closure_train: Adam");
    }
    if (final_loss) {
        cudaError_t e = cudaMemcpyAsync(final_loss, c->loss.ptr, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "ers_closure_train: loss");
    }
    return ERS_OK;
}

}  // extern "C"

namespace ers {

// Two-delta evaluation into u, v (+ gamma), far field with the precision of p.
int eval_few_delta(ers_surface *s, const ers_params *p, const double *y, int64_t M, const double *x0,
                   const double *n0, const double *b, const double *f0, const double *q0, double *u, double *v,
                   double *gamma, int ndelta, cudaStream_t st);
// The near-field part alone (ndelta = 1, 2 or 3 deltas; no far-field sums), over the three-delta
// method's near radius for every ndelta: the method's value is then the closure's sums plus the
// difference of two such evaluations.
int eval_near_only(ers_surface *s, const ers_params *p, const double *y, int64_t M, const double *x0,
                   const double *n0, const double *b, const double *f0, const double *q0, double *u, double *v,
                   int ndelta, cudaStream_t st);

}  // namespace ers

namespace {

int features(ers_surface *s, const ers_params *p, int64_t M, const double *x0, const double *n0, const double *b,
             const double *u2, const double *v2, const double *gamma, const double *u3, const double *v3, float *Xs,
             float *Xd, float *Ts, float *Td, double *scale, int *valid, int nd, cudaStream_t st) {
    // fit scratch: neighbour lists [FIT_LMAX][M] ints, counts [M] ints, accumulators [NACC][M] doubles
    const size_t lbytes = sizeof(int) * ((size_t)FIT_LMAX * M + M);
    const size_t off = (lbytes + 255) / 256 * 256;
    int rc = grow(s->fitw, off + sizeof(double) * (size_t)NACC * M);
    if (rc != ERS_OK) return rc;
    FeatArgs A;
    FitArgs &F = A.fit;
    F.sd = surf_dev(s);
    F.fq = s->fq;
    F.x0 = x0;
    F.n0 = n0;
    F.b = b;
    F.M = M;
    F.h = s->h;
    F.Rc = p->cutoff_t * p->rho[nd - 1] * s->h;
    for (int i = 0; i < 3; ++i) {
        F.c[i] = s->c[i];
        F.a[i] = s->a[i];
    }
    F.list = (int *)s->fitw.ptr;
    F.cnt = F.list + (size_t)FIT_LMAX * M;
    F.acc = (double *)((char *)s->fitw.ptr + off);
    A.u2 = u2;
    A.v2 = v2;
    A.gamma = gamma;
    A.u3 = u3;
    A.v3 = v3;
    A.rho0 = p->rho[0];
    A.rho1 = p->rho[1];
    A.nd = nd;
    // |gamma| at b = 0: beta = (rho_1, -rho_0) / (rho_1 - rho_0), I2(0) = 1 / (3 sqrt(pi)), so
    // |gamma(0)| = rho_0 rho_1 (rho_0 + rho_1) / (3 sqrt(pi))
    A.gamma0 = p->rho[0] * p->rho[1] * (p->rho[0] + p->rho[1]) / (3.0 * 1.7724538509055160273);
    A.Xs = Xs;
    A.Xd = Xd;
    A.Ts = Ts;
    A.Td = Td;
    A.scale = scale;
    A.valid = valid;
    const unsigned g128 = (unsigned)((M + 127) / 128);
    k_fit_scan<<<g128, 128, 0, st>>>(F);
    k_fit_accum<<<g128, 128, 0, st>>>(F);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_features, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FEAT_SMEM);
    if (e != cudaSuccess) return cuda_fail(e, "closure density-fit kernels");
    k_features<<<(unsigned)((M + FEAT_THREADS - 1) / FEAT_THREADS), FEAT_THREADS, FEAT_SMEM, st>>>(A);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "closure features kernel");
    return ERS_OK;
}

ApplyArgs apply_args(const ers_surface *s, const double *x0, const double *n0, const double *gamma,
                     const double *scale, const float *Ys, const float *Yd, int64_t M, int nd, double *u, double *v) {
    ApplyArgs A;
    A.x0 = x0;
    A.n0 = n0;
    A.gamma = gamma;
    A.scale = scale;
    A.Ys = Ys;
    A.Yd = Yd;
    A.M = M;
    A.h = s->h;
    A.nd = nd;
    A.mask = 3;
    A.sign = 1.0;
    for (int i = 0; i < 3; ++i) {
        A.c[i] = s->c[i];
        A.a[i] = s->a[i];
    }
    A.u = u;
    A.v = v;
    return A;
}

}  // namespace

extern "C" {

int ers_closure_data(ers_surface *s, const ers_params *p, const double *y, int64_t M, const double *x0,
                     const double *n0, const double *b, const double *f0, const double *q0, const double *u3,
                     const double *v3, int ndelta, float *Xs, float *Xd, float *Ts, float *Td, int *valid,
                     void *stream) {
    clear_error();
    if (ndelta != 1 && ndelta != 2) return fail(ERS_E_INVAL, "ers_closure_data: ndelta must be 1 or 2");
    if (!s || !p || !y || !x0 || !n0 || !b || !f0 || !q0 || !u3 || !v3 || !Xs || !Xd || !Ts || !Td || !valid)
        return fail(ERS_E_INVAL, "ers_closure_data: NULL argument");
    if (p->options & (ERS_OPT_FOUR_DELTA | ERS_OPT_TREECODE | ERS_OPT_SHARP))
        return fail(ERS_E_UNSUPPORTED, "ers_closure_data: ERS_OPT_FOUR_DELTA, ERS_OPT_TREECODE and ERS_OPT_SHARP are not supported");
    if (M <= 0) return fail(ERS_E_INVAL, "ers_closure_data: M <= 0");
    cudaStream_t st = (cudaStream_t)stream;
    Scratch &w = s->host_io;  // reuse the host-io buffer of the surface as scratch: u2 | v2 | gamma | scale
    int rc = grow(w, sizeof(double) * (size_t)M * 9);
    if (rc != ERS_OK) return rc;
    double *u2 = (double *)w.ptr, *v2 = u2 + 3 * M, *gm = v2 + 3 * M, *sc = gm + M;
    ers_params pp = *p;
    pp.layers = ERS_LAYER_SL | ERS_LAYER_DL;
    if ((rc = eval_few_delta(s, &pp, y, M, x0, n0, b, f0, q0, u2, v2, gm, ndelta, st)) < 0) return rc;
    return features(s, &pp, M, x0, n0, b, u2, v2, gm, u3, v3, Xs, Xd, Ts, Td, sc, valid, ndelta, st);
}

int ers_closure_last_gate(ers_closure *c, int used[2], double err_with[2], double err_without[2]) {
    clear_error();
    if (!c) return fail(ERS_E_INVAL, "ers_closure_last_gate: NULL closure");
    for (int l = 0; l < 2; ++l) {
        if (used) used[l] = c->last_used[l];
        if (err_with) err_with[l] = c->last_err_with[l];
        if (err_without) err_without[l] = c->last_err_without[l];
    }
    return ERS_OK;
}

int ers_eval_learned(ers_surface *s, ers_closure *c, const ers_params *p, const double *y, int64_t M,
                     const double *x0, const double *n0, const double *b, const double *f0, const double *q0,
                     int ndelta, double *u, double *v, double tol, int vstride, double *val_err, int *fell_back,
                     void *stream) {
    clear_error();
    if (ndelta != 1 && ndelta != 2) return fail(ERS_E_INVAL, "ers_eval_learned: ndelta must be 1 or 2");
    if (!s || !c || !p || !y || !x0 || !n0 || !b || !f0 || !q0 || !u || !v)
        return fail(ERS_E_INVAL, "ers_eval_learned: NULL argument (both layers and all closest-point data needed)");
    if (p->options & (ERS_OPT_FOUR_DELTA | ERS_OPT_TREECODE | ERS_OPT_SHARP))
        return fail(ERS_E_UNSUPPORTED, "ers_eval_learned: ERS_OPT_FOUR_DELTA, ERS_OPT_TREECODE and ERS_OPT_SHARP are not supported");
    if (M < 0) return fail(ERS_E_INVAL, "ers_eval_learned: M < 0");
    if (vstride < 1) return fail(ERS_E_INVAL, "ers_eval_learned: vstride must be >= 1");
    int rc = closure_check(c, 0);
    if (rc != ERS_OK) return rc;
    if (!s->has_f || !s->has_q)
        return fail(ERS_E_STATE, "ers_eval_learned: both densities must be set (ers_set_density)");
    if (fell_back) *fell_back = 0;
    for (int l = 0; l < 2; ++l) {
        c->last_used[l] = 0;
        c->last_err_with[l] = c->last_err_without[l] = 0.0;
    }
    if (M == 0) return ERS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    ers_params pp = *p;
    pp.layers = ERS_LAYER_SL | ERS_LAYER_DL;
    // work buffers of the closure: sample records (2 x M x XSTR f32), outputs (2 x M x 4 f32),
    // gamma, scale
    if ((rc = grow(c->feat, sizeof(float) * (size_t)M * mlp::XSTR * 2)) != ERS_OK) return rc;
    if ((rc = grow(c->outp, sizeof(float) * (size_t)M * mlp::OUT_STRIDE * 2)) != ERS_OK) return rc;
    if ((rc = grow(c->gamma, sizeof(double) * (size_t)M)) != ERS_OK) return rc;
    if ((rc = grow(c->scale, sizeof(double) * (size_t)M * 2)) != ERS_OK) return rc;
    float *Xs = (float *)c->feat.ptr, *Xd = Xs + M * mlp::XSTR;
    float *Ys = (float *)c->outp.ptr, *Yd = Ys + M * mlp::OUT_STRIDE;
    double *gm = (double *)c->gamma.ptr, *sc = (double *)c->scale.ptr;
    // 1. one- or two-delta sums; 2. features; 3. network (tensor cores); 4. correction
    if ((rc = eval_few_delta(s, &pp, y, M, x0, n0, b, f0, q0, u, v, gm, ndelta, st)) < 0) return rc;
    if ((rc = features(s, &pp, M, x0, n0, b, nullptr, nullptr, gm, nullptr, nullptr, Xs, Xd, nullptr, nullptr, sc,
                       nullptr, ndelta, st)) != ERS_OK)
        return rc;
    if ((rc = infer(c, 0, Xs, M, Ys, st)) != ERS_OK) return rc;
    if ((rc = infer(c, 1, Xd, M, Yd, st)) != ERS_OK) return rc;
    ApplyArgs ap = apply_args(s, x0, n0, gm, sc, Ys, Yd, M, ndelta, u, v);
    k_apply<<<(unsigned)((M + 127) / 128), 128, 0, st>>>(ap);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "closure correction kernel");
    // 4b. targets whose geometry lies outside the training extent: the three-delta method instead
    c->last_out = 0;
    if (c->range_check && (c->have_range[0] || c->have_range[1])) {
        // [count | pad | idx (M) | gathered inputs (16 K) | near sums, three and nd deltas (12 K)], K <= M
        if ((rc = grow(c->oor, sizeof(int64_t) * 2 + sizeof(int64_t) * (size_t)M + sizeof(double) * (size_t)M * 28)) !=
            ERS_OK)
            return rc;
        unsigned long long *cnt = (unsigned long long *)c->oor.ptr;
        int64_t *idx = (int64_t *)c->oor.ptr + 2;
        double *sub = (double *)(idx + M);
        e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return cuda_fail(e, "ers_eval_learned: memset");
        k_range_flags<<<(unsigned)((M + 127) / 128), 128, 0, st>>>(Xs, Xd, sc, M, c->range, c->have_range[0],
                                                                   c->have_range[1], idx, cnt);
        unsigned long long K = 0;
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&K, cnt, sizeof K, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "ers_eval_learned: feature extent check");
        const int64_t Kt = (int64_t)K;
        c->last_out = Kt;
        if (Kt > 0) {
            double *n3u = sub + 16 * Kt, *n3v = n3u + 3 * Kt, *ndu = n3v + 3 * Kt, *ndv = ndu + 3 * Kt;
            k_gather_idx<<<(unsigned)((Kt + 127) / 128), 128, 0, st>>>(y, x0, n0, b, f0, q0, idx, Kt, sub);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "ers_eval_learned: gather");
            if ((rc = eval_near_only(s, &pp, sub, Kt, sub + 3 * Kt, sub + 6 * Kt, sub + 9 * Kt, sub + 10 * Kt,
                                     sub + 13 * Kt, n3u, n3v, 3, st)) < 0)
                return rc;
            if ((rc = eval_near_only(s, &pp, sub, Kt, sub + 3 * Kt, sub + 6 * Kt, sub + 9 * Kt, sub + 10 * Kt,
                                     sub + 13 * Kt, ndu, ndv, ndelta, st)) < 0)
                return rc;
            k_replace_idx<<<(unsigned)((Kt + 127) / 128), 128, 0, st>>>(ap, n3u, n3v, ndu, ndv, idx, Kt, sc);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "ers_eval_learned: replace");
        }
    }
    // 5. validation against the three-delta method on every vstride-th target, with and without
    // the network's correction; per layer the better of the two is kept.  The far field is the
    // same in the closure and in the method, so the method's value comes from the near-field sums
    // alone (three and nd deltas) at the sample (k_compare).
    const int64_t Ms = (M + vstride - 1) / vstride;
    if ((rc = grow(c->sub, sizeof(double) * ((size_t)Ms * 28 + 8))) != ERS_OK) return rc;
    double *sub = (double *)c->sub.ptr;
    double *n3u = sub + 16 * Ms, *n3v = n3u + 3 * Ms, *ndu = n3v + 3 * Ms, *ndv = ndu + 3 * Ms, *res = ndv + 3 * Ms;
    k_gather<<<(unsigned)((Ms + 127) / 128), 128, 0, st>>>(y, x0, n0, b, f0, q0, Ms, vstride, sub);
    e = cudaMemsetAsync(res, 0, sizeof(double) * 6, st);
    if (e != cudaSuccess) return cuda_fail(e, "ers_eval_learned: memset");
    if ((rc = eval_near_only(s, &pp, sub, Ms, sub + 3 * Ms, sub + 6 * Ms, sub + 9 * Ms, sub + 10 * Ms, sub + 13 * Ms,
                             n3u, n3v, 3, st)) < 0)
        return rc;
    if ((rc = eval_near_only(s, &pp, sub, Ms, sub + 3 * Ms, sub + 6 * Ms, sub + 9 * Ms, sub + 10 * Ms, sub + 13 * Ms,
                             ndu, ndv, ndelta, st)) < 0)
        return rc;
    k_compare<<<64, 128, 0, st>>>(ap, n3u, n3v, ndu, ndv, Ms, vstride, res);
    double h[6];
    e = cudaMemcpyAsync(h, res, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "ers_eval_learned: validation");
    int timed_out = 0;
    cudaMemcpy(&timed_out, c->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (timed_out) return fail(ERS_E_TIMEOUT, "ers_eval_learned: a tensor-core wait in the closure kernel expired");
    double err[2];
    int undo = 0;
    for (int l = 0; l < 2; ++l) {
        const double ref = h[2 * l + 1];
        const double ew = ref > 0 ? h[2 * l] / ref : 0.0, eo = ref > 0 ? h[4 + l] / ref : 0.0;
        c->last_err_with[l] = ew;
        c->last_err_without[l] = eo;
        c->last_used[l] = ew <= eo ? 1 : 0;
        if (!c->last_used[l]) undo |= 1 << l;
        err[l] = std::min(ew, eo);
    }
    if (val_err) {
        val_err[0] = err[0];
        val_err[1] = err[1];
    }
    if (!(err[0] <= tol && err[1] <= tol)) {
        if (fell_back) *fell_back = 1;
        return ers_eval(s, &pp, y, M, x0, n0, b, f0, q0, u, v, stream);
    }
    if (undo) {  // take back the correction of a layer whose network did not help on the sample
        ApplyArgs un = ap;
        un.mask = undo;
        un.sign = -1.0;
        k_apply<<<(unsigned)((M + 127) / 128), 128, 0, st>>>(un);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "ers_eval_learned: undo");
    }
    return ERS_OK;
}

}  // extern "C"
