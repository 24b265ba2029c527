// Building blocks of the near field and the extrapolation (Secs. 2, 3.2, 3.3), shared by the
// single-density kernel (k_near.cu) and the batched persistent kernel (k_batch.cu).
//
// Near pair (target y with closest point x0, normal n0, signed distance b; node x):
//   K1 = sum_k alpha_k s1(r/delta_k)/r,  K3 = sum_k alpha_k s2(r/delta_k)/r^3,
//   K5 = sum_k alpha_k s3(r/delta_k)/r^5,  s_p := 1 where r/delta_k > cutoff_t (Sec. 3.2);
//   single layer (Eq. (Sreg)):   K1 g + K3 d (d.g),  g = w f - (f(x0).n0) w n
//   double layer (Eqs. (Tsplit), (Treg)):  -6 [t1 (K3 - (r^2 - b^2) K5) + t2 K5] : Q m,
//     Q = q - q(x0), m = w n; with P = (n0.Q)(n0.m), R = (xh.Q)(xh.m),
//     S = (xh.Q)(n0.m) + (n0.Q)(xh.m), K = K3 - (r^2 - b^2) K5, xh = x - x0:
//       t1 : Q m = n0 (b P - S) - xh P,   t2 : Q m = n0 (b R) + xh (b S - R).
// alpha = first row of the inverse of A_k = [1, rho_k I0(b/delta_k), rho_k^3 I2(b/delta_k)]
// (Eqs. (extrap_eqn), (I0), (I2)), by Cramer's rule.
#pragma once

#include "ers_internal.h"

namespace ers {
namespace nearc {

constexpr unsigned FULL = 0xffffffffu;
constexpr double INV8PI = 0.039788735772973833942;
constexpr double INVSQRTPI = 0.56418958354775628695;

// Density-independent constants of one near target.
struct Geom {
    double y[3], x0[3], n0[3], b;
    double invd2[3], ad1[3], ad3[3], ad5[3], apre[2];
    float yh[3], yl[3];  // y = yh + yl in floats (mixed-mode classification)
    float alf[3];        // extrapolation weights in FP32 (for the small defects 1 - s_p)
    float tcf;           // cutoff_t: s_p := 1 beyond it
};

// Beyond t = r/delta = DEFECT_T the defects 1 - s_p(t) are below 2.1e-8 and are evaluated in
// FP32 instead of from the FP64 table.
constexpr double DEFECT_T = 4.7;

struct ScanParams {
    float rc2f;   // exact FP32 threshold of the mixed far field
    float rpre;   // FP32 prefilter radius (Rc plus a conservative margin)
    float th[2];  // FP32 class thresholds (min(DEFECT_T, cutoff_t) delta_k)^2, k = 0, 1
    float tcf;    // cutoff_t
    double h;
};

// Extrapolation weights for signed distance b; every lane of the warp calls it, lanes 0..2
// evaluate I0, I2 at lambda_k = |b| / (rho_k h).
__device__ __forceinline__ void extrap_weights(int lane, double b, const double rho[3], double h, double al[3]) {
    double i0 = 0.0, i2 = 0.0;
    if (lane < 3) {
        const double rl = lane == 0 ? rho[0] : (lane == 1 ? rho[1] : rho[2]);
        const double lam = fabs(b) / (rl * h);
        const double e = exp(-lam * lam) * INVSQRTPI, ec = erfc(lam);
        i0 = e - lam * ec;
        i2 = (2.0 / 3.0) * ((0.5 - lam * lam) * e + lam * lam * lam * ec);
    }
    double ac[3], bc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double rk = rho[k];
        ac[k] = rk * __shfl_sync(FULL, i0, k);
        bc[k] = rk * rk * rk * __shfl_sync(FULL, i2, k);
    }
    al[0] = ac[1] * bc[2] - ac[2] * bc[1];
    al[1] = ac[2] * bc[0] - ac[0] * bc[2];
    al[2] = ac[0] * bc[1] - ac[1] * bc[0];
    const double det = al[0] + al[1] + al[2];
    if (det != 0.0 && isfinite(det)) {
        for (int k = 0; k < 3; ++k) al[k] /= det;
    } else {
        al[0] = 1.0;
        al[1] = 0.0;
        al[2] = 0.0;
    }
    if (!(isfinite(al[0]) && isfinite(al[1]) && isfinite(al[2]))) {
        al[0] = 1.0;
        al[1] = 0.0;
        al[2] = 0.0;
    }
}

// Two-delta weights: the system of Eq. (extrap_eqn) for delta_0, delta_1 without the c2 column,
// beta_0 + beta_1 = 1, beta_0 rho_0 I0(lambda_0) + beta_1 rho_1 I0(lambda_1) = 0, so that
// sum_k beta_k u^{delta_k} = u + gamma c2 + O(delta^5) with
// gamma = beta_0 rho_0^3 I2(lambda_0) + beta_1 rho_1^3 I2(lambda_1).
__device__ __forceinline__ void two_delta_weights(int lane, double b, const double rho[3], double h, double al[3],
                                                  double &gamma) {
    double i0 = 0.0, i2 = 0.0;
    if (lane < 2) {
        const double rl = lane == 0 ? rho[0] : rho[1];
        const double lam = fabs(b) / (rl * h);
        const double e = exp(-lam * lam) * INVSQRTPI, ec = erfc(lam);
        i0 = e - lam * ec;
        i2 = (2.0 / 3.0) * ((0.5 - lam * lam) * e + lam * lam * lam * ec);
    }
    const double a0 = rho[0] * __shfl_sync(FULL, i0, 0), a1 = rho[1] * __shfl_sync(FULL, i0, 1);
    const double c0 = rho[0] * rho[0] * rho[0] * __shfl_sync(FULL, i2, 0);
    const double c1 = rho[1] * rho[1] * rho[1] * __shfl_sync(FULL, i2, 1);
    const double den = a1 - a0;
    if (den != 0.0 && isfinite(den) && isfinite(a0) && isfinite(a1)) {
        al[0] = a1 / den;
        al[1] = -a0 / den;
    } else {
        al[0] = 1.0;
        al[1] = 0.0;
    }
    al[2] = 0.0;
    gamma = al[0] * c0 + al[1] * c1;
}

// Fill the geometry constants of target m (all lanes; lanes 0..2 also evaluate I0, I2).
// ndelta = 3: the extrapolation weights of Eq. (extrap_eqn); ndelta = 2: the two-delta
// weights above (gamma returned in *gamma).
__device__ __forceinline__ void load_geom(int lane, const double *y, const double *x0, const double *n0, double b,
                                          int64_t m, const double rho[3], double h, Geom &T, int ndelta = 3,
                                          double *gamma = nullptr) {
    for (int i = 0; i < 3; ++i) {
        T.y[i] = y[3 * m + i];
        T.x0[i] = x0[3 * m + i];
        T.n0[i] = n0[3 * m + i];
        T.yh[i] = __double2float_rn(T.y[i]);
        T.yl[i] = __double2float_rn(T.y[i] - (double)T.yh[i]);
    }
    T.b = b;
    double al[3];
    if (ndelta == 2) {
        double g;
        two_delta_weights(lane, b, rho, h, al, g);
        if (gamma) *gamma = g;
    } else if (ndelta == 1) {  // the single regularized sum u^{delta_0} (no extrapolation)
        al[0] = 1.0;
        al[1] = 0.0;
        al[2] = 0.0;
        if (gamma) *gamma = 0.0;
    } else {
        extrap_weights(lane, b, rho, h, al);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double dk = rho[k] * h, id = 1.0 / dk;
        T.invd2[k] = id * id;
        T.ad1[k] = al[k] * id;
        T.ad3[k] = al[k] * id * id * id;
        T.ad5[k] = al[k] * id * id * id * id * id;
    }
    T.apre[0] = al[0];
    T.apre[1] = al[0] + al[1];
    for (int k = 0; k < 3; ++k) T.alf[k] = (float)al[k];
}

// Exact near/far decision of pair (T, j), identical to the far-field mask of the precision
// in use: FP64 r^2 > Rc^2 for the FP64 far field; the FP32 tile-relative r^2 > rc2f for the
// mixed one.  r2 is the FP64 squared distance of the same pair.
template <int PREC>
__device__ __forceinline__ bool is_near(const SurfDev &s, const Geom &T, int64_t j, double r2, double Rc,
                                        float rc2f) {
    if (PREC == ERS_PREC_FP64) return !(__double_as_longlong(r2) > __double_as_longlong(Rc * Rc));
    const float4 cen = __ldg(reinterpret_cast<const float4 *>(s.tilec) + j / TS32);
    const float4 xc = __ldg(reinterpret_cast<const float4 *>(s.rec32 + j * REC));
    float ex, ey, ez;
    const float r2f = dist2_fp32(tile_rel(T.yh[0], cen.x, T.yl[0]), tile_rel(T.yh[1], cen.y, T.yl[1]),
                                 tile_rel(T.yh[2], cen.z, T.yl[2]), xc.x, xc.y, xc.z, &ex, &ey, &ez);
    return !(r2f > rc2f);
}

// alpha-weighted kernel factors of a near pair of class CLS (delta_0..delta_{CLS-1} are not
// regularized at this distance); sigma_p from the interpolation table.
// ND = number of deltas in use (3 for the method; 2 or 1 for the learned closure).
template <int CLS, int ND = 3>
__device__ __forceinline__ void kernel_factors(const Geom &T, const double *__restrict__ tab, double r2, double &K1,
                                               double &K3, double &K5) {
    K1 = 0.0;
    K3 = 0.0;
    K5 = 0.0;
#pragma unroll
    for (int k = CLS; k < ND; ++k) {
        const double tau = r2 * T.invd2[k];
        int idx = (int)(approx_float_pos(tau) * (float)TAB_INV_W);
        idx = min(idx, TAB_N - 1);
        const double *cf = tab + idx * (3 * TAB_NC);
        const double s = fma(tau, 2.0 * TAB_INV_W, -__ldg(tab + TAB_N * 3 * TAB_NC + idx));
        double s1 = __ldg(cf + 0), s2 = __ldg(cf + TAB_NC), s3 = __ldg(cf + 2 * TAB_NC);
#pragma unroll
        for (int e = 1; e < TAB_NC; ++e) {
            s1 = fma(s1, s, __ldg(cf + e));
            s2 = fma(s2, s, __ldg(cf + TAB_NC + e));
            s3 = fma(s3, s, __ldg(cf + 2 * TAB_NC + e));
        }
        K1 = fma(T.ad1[k], s1, K1);
        K3 = fma(T.ad3[k], s2, K3);
        K5 = fma(T.ad5[k], s3, K5);
    }
    if (CLS >= 1) {
        // delta_0..delta_{CLS-1}: r / delta_k > DEFECT_T, where s_p = 1 - eps_p with
        // eps_1 = erfc t, eps_2 = eps_1 + (2/sqrt pi) t e^{-t^2},
        // eps_3 = eps_1 + (2/sqrt pi)(t + 2/3 t^3) e^{-t^2} (Eqs. (s1)-(s3)) below 2.1e-8;
        // eps_p is evaluated in FP32 (its error ~1e-14 relative to the term), and eps_p = 0 where
        // t > cutoff_t (Sec. 3.2).  The term is (sum_k alpha_k - sum_k alpha_k eps_p(t_k)) / r^p.
        float E1 = 0.0f, E3 = 0.0f, E5 = 0.0f;
        const float r2f = approx_float_pos(r2);
#pragma unroll
        for (int k = 0; k < CLS; ++k) {
            const float t = sqrtf(r2f * approx_float_pos(T.invd2[k]));
            if (t <= T.tcf) {
                const float e = erfcf(t), g = 1.12837916709551257f * t * expf(-t * t);
                const float a = (float)T.alf[k];
                E1 = fmaf(a, e, E1);
                E3 = fmaf(a, e + g, E3);
                E5 = fmaf(a, e + g * (1.0f + 0.6666666666666667f * t * t), E5);
            }
        }
        const double Ain = T.apre[CLS - 1];
        const double ri = rsqrt(r2);
        const double ri2 = ri * ri;
        const double ri3 = ri2 * ri;
        K1 = fma(Ain - float_to_double(E1), ri, K1);
        K3 = fma(Ain - float_to_double(E3), ri3, K3);
        K5 = fma(Ain - float_to_double(E5), ri3 * ri2, K5);
    }
}

// Single-layer contraction: accU += K1 g + K3 d (d.g), g = wf - c wn.
__device__ __forceinline__ void sl_accumulate(double dx, double dy, double dz, double K1, double K3, double c,
                                              const double wf[3], const double wn[3], double accU[3]) {
    const double g0 = fma(-c, wn[0], wf[0]);
    const double g1 = fma(-c, wn[1], wf[1]);
    const double g2 = fma(-c, wn[2], wf[2]);
    const double t = K3 * fma(dz, g2, fma(dy, g1, dx * g0));
    accU[0] = fma(t, dx, fma(K1, g0, accU[0]));
    accU[1] = fma(t, dy, fma(K1, g1, accU[1]));
    accU[2] = fma(t, dz, fma(K1, g2, accU[2]));
}

// Double-layer contraction in the basis (n0, xh): accN += cn, accX += cx xh.
// nm = n0.m and xm = xh.m are density independent (shared by several densities).
__device__ __forceinline__ void dl_accumulate(const Geom &T, double r2, double K3, double K5, const double h3[3],
                                              double nm, double xm, const double qs[3], const double q0[3],
                                              double &accN, double accX[3]) {
    const double Q0 = qs[0] - q0[0], Q1 = qs[1] - q0[1], Q2 = qs[2] - q0[2];
    const double nQ = fma(T.n0[2], Q2, fma(T.n0[1], Q1, T.n0[0] * Q0));
    const double xQ = fma(h3[2], Q2, fma(h3[1], Q1, h3[0] * Q0));
    const double P = nQ * nm, R = xQ * xm, S = fma(xQ, nm, nQ * xm);
    const double K = fma(-(r2 - T.b * T.b), K5, K3);
    const double cn = fma(K, fma(T.b, P, -S), K5 * T.b * R);
    const double cx = fma(K5, fma(T.b, S, -R), -K * P);
    accN += cn;
    accX[0] = fma(cx, h3[0], accX[0]);
    accX[1] = fma(cx, h3[1], accX[1]);
    accX[2] = fma(cx, h3[2], accX[2]);
}

// Walk the rows of the surface's cell grid that meet the prefilter ball around the target,
// test candidates in FP32, queue survivors by class in the warp's shared queues sq[3][64],
// and call batch(cls, j, valid) with one node per lane whenever a class has 32 entries, then
// once more per class for the remainder (lanes with valid = false hold no node).
template <class Batch>
__device__ __forceinline__ void scan_near(const SurfDev &s, const Geom &T, const ScanParams &P, int (*sq)[64],
                                          int lane, Batch &&batch) {
    int qn[3] = {0, 0, 0};
    const unsigned lt = (1u << lane) - 1u;
    const Grid &G = s.grid;
    const float yf[3] = {T.yh[0], T.yh[1], T.yh[2]};
    const float of[3] = {(float)G.origin[0], (float)G.origin[1], (float)G.origin[2]};
    const float cw = (float)G.cw, inv_cw = 1.0f / cw;
    const float R = P.rpre, R2 = R * R;
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = max(0, (int)floorf((yf[a] - R - of[a]) * inv_cw));
        hi[a] = min(G.nc[a] - 1, (int)floorf((yf[a] + R - of[a]) * inv_cw));
    }
    const int *__restrict__ cs = s.cell_start;
    const float4 *__restrict__ xs32 = s.xs32;
    for (int iz = lo[2]; iz <= hi[2]; ++iz) {
        const float zl = of[2] + iz * cw;
        const float dzr = fmaxf(0.0f, fmaxf(zl - yf[2], yf[2] - (zl + cw)));
        for (int iy = lo[1]; iy <= hi[1]; ++iy) {
            const float yl0 = of[1] + iy * cw;
            const float dyr = fmaxf(0.0f, fmaxf(yl0 - yf[1], yf[1] - (yl0 + cw)));
            const float rem = R2 - dyr * dyr - dzr * dzr;
            if (rem < 0.0f) continue;
            const float half = sqrtf(rem) * 1.0001f + 1e-6f * cw;
            const int ia = max(lo[0], (int)floorf((yf[0] - half - of[0]) * inv_cw));
            const int ib = min(hi[0], (int)floorf((yf[0] + half - of[0]) * inv_cw));
            if (ia > ib) continue;
            const int64_t rowbase = ((int64_t)iz * G.nc[1] + iy) * G.nc[0];
            const int js = cs[rowbase + ia], je = cs[rowbase + ib + 1];
            for (int jb = js; jb < je; jb += 32) {
                const int j = jb + lane;
                bool pass = false;
                int cls = 0;
                if (j < je) {
                    const float4 p = __ldg(xs32 + j);
                    const float ex = yf[0] - p.x, ey = yf[1] - p.y, ez = yf[2] - p.z;
                    const float r2f = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
                    pass = r2f <= R2;
                    cls = (r2f > P.th[0]) + (r2f > P.th[1]);
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const unsigned mk = __ballot_sync(FULL, pass && cls == c);
                    if (pass && cls == c) sq[c][qn[c] + __popc(mk & lt)] = j;
                    qn[c] += __popc(mk);
                }
                __syncwarp();
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (qn[c] >= 32) {
                        batch(c, sq[c][qn[c] - 32 + lane], true);
                        qn[c] -= 32;
                        __syncwarp();
                    }
                }
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (qn[c] > 0) {
            const bool v = lane < qn[c];
            batch(c, v ? sq[c][lane] : 0, v);
        }
    }
    __syncwarp();
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

inline ScanParams scan_params(const ers_surface *s, double Rc, const double rho[3], double cutoff_t) {
    ScanParams P;
    P.rc2f = (float)(Rc * Rc);
    double L = 0.0;
    for (int i = 0; i < 3; ++i) L = fmax(L, fabs(s->c[i]) + s->a[i]);
    P.rpre = (float)(Rc * (1.0 + 1e-5) + 4e-6 * (L + Rc));
    for (int k = 0; k < 2; ++k) {
        const double t = fmin(DEFECT_T, cutoff_t) * rho[k] * s->h;
        P.th[k] = (float)(t * t);
    }
    P.tcf = (float)cutoff_t;
    P.h = s->h;
    return P;
}

}  // namespace nearc
// One problem of the batched evaluation, as the persistent kernel sees it.
struct BatchProblemDev {
    SurfDev sd;
    const double *dens64;  // [N][NR][6] sorted order: w f (3), q (3)
    const float *dens32;   // [N][NR][6] floats
    const double *y, *x0, *n0, *b, *f0, *q0;  // f0, q0: [NR][M][3]
    double *u, *v;                            // [NR][M][3]
    int64_t M;
    double Rc;
    nearc::ScanParams sp;
};

struct BatchItem {
    int prob;
    int tb;
};

}  // namespace ers
