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
//       t1 : Q m = n0 (b P - S) - xh P,   t2 : Q m = n0 (b R) + xh (b S - R),
//     evaluated in the equivalent form of dl_accumulate_pair (in terms of d = y - x = b n0 - xh).
// alpha = first row of the inverse of A_k = [1, rho_k I0(b/delta_k), rho_k^3 I2(b/delta_k)]
// (Eqs. (extrap_eqn), (I0), (I2)), by Cramer's rule; with four deltas (the O(delta^7) variant of
// Sec. 1) A_k gains the column rho_k^5 I4(b/delta_k).
#pragma once

#include "ers_internal.h"

namespace ers {
namespace nearc {

constexpr unsigned FULL = 0xffffffffu;
constexpr double INV8PI = 0.039788735772973833942;
constexpr double INVSQRTPI = 0.56418958354775628695;

// Most deltas of one evaluation: three for Eq. (extrap_eqn), four for the O(delta^7) variant.
constexpr int MAXD = 4;

// Density-independent constants of one near target (entries k < number of deltas in use).
struct Geom {
    double y[3], x0[3], n0[3], b, b2;  // b2 = 2 b
    double invd2[MAXD], ad1[MAXD], ad3[MAXD], ad5[MAXD];
    double s2w[MAXD];          // 2 TAB_INV_W / delta_k^2: the table's local variable is r^2 s2w - (2 i + 1)
    double apre[MAXD];         // partial sums alpha_0 + ... + alpha_k
    float yh[3], yl[3];        // y = yh + yl in floats (mixed-mode classification)
    float id2h[MAXD], id2l[MAXD]; // 1/delta_k^2 = id2h + id2l in floats
    float alf[MAXD];           // extrapolation weights in FP32 (for the small defects 1 - s_p)
    float adh[3][MAXD], adl[3][MAXD];  // alpha_k / delta_k^p (p = 1, 3, 5) as float pairs
    float aph[MAXD], apl[MAXD];        // apre as float pairs
    fpair n0p[3], b2p;                 // n0 and 2 b as float pairs (the near kernel's contractions)
    float tcf2;             // cutoff_t^2: s_p := 1 beyond t = cutoff_t
    bool cut_small;         // cutoff_t < DEFECT_T: the table path may meet the cutoff
};

// Beyond t = r/delta = DEFECT_T the defects 1 - s_p(t) are below 2.1e-8 and are evaluated in
// FP32 instead of from the FP64 table.
constexpr double DEFECT_T = 4.7;
// Near-pair classes: c = number of delta_k (from delta_0 up) with r > min(DEFECT_T, cutoff_t) delta_k,
// 0..3 with three deltas (NCLS of them), 0..4 with four.
constexpr int NCLS = 4;
constexpr int NCLS_MAX = MAXD + 1;

struct ScanParams {
    float rc2f;     // exact FP32 threshold of the mixed far field
    float rpre;     // FP32 prefilter radius (Rc plus a conservative margin)
    float th[MAXD];    // FP32 class thresholds (min(DEFECT_T, cutoff_t) delta_k)^2 (+inf past the deltas in use)
    float cut2[MAXD - 1];  // (cutoff_t delta_k)^2, k below the largest delta: pair counts by regularized deltas
    float tcf2;       // cutoff_t^2
    double tc2;       // cutoff_t^2 in FP64
    double cut2d[MAXD];  // (cutoff_t delta_k)^2 in FP64, delta_k = rho_k h
    double h;
};

// Relative width of the band around cutoff_t^2 where the FP32 value of t^2 cannot decide
// t > cutoff_t (FP32 t^2 is within 3e-7 of the exact one).  There the decision is r^2 >
// (cutoff_t rho_k h)^2 in FP64, which is exact for the many node pairs of the lattice rule whose
// distance is an exact multiple of h (r = 2 i h, so t = i at delta = 2h): such ties count as
// t = cutoff_t, regularized, as in exact arithmetic.
constexpr float CUT_BAND = 1e-6f;

__device__ __forceinline__ void set_cutoff(Geom &T, const ScanParams &P) {
    T.tcf2 = P.tcf2;
    T.cut_small = P.tc2 < DEFECT_T * DEFECT_T;
}

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

// The O(delta^7) variant with four deltas: A_k = [1, a_k, c_k, e_k] with a_k = rho_k I0(lambda_k),
// c_k = rho_k^3 I2(lambda_k), e_k = rho_k^5 I4(lambda_k), I4(lambda) = (2/15)((3 - 2 lambda^2 +
// 4 lambda^4) e^{-lambda^2}/sqrt(pi) - 4 lambda^5 erfc lambda).  alpha solves A^T alpha = e_0: by
// Cramer's rule alpha_k = C_k / sum_j C_j with C_k = (-1)^k det of the 3x3 matrix of rows a, c, e
// without column k (expanding det A^T along its first row of ones).  Lanes 0..3 evaluate the I's.
__device__ __forceinline__ void extrap_weights4(int lane, double b, const double rho[MAXD], double h,
                                                double al[MAXD]) {
    double i0 = 0.0, i2 = 0.0, i4 = 0.0;
    if (lane < 4) {
        const double rl = lane == 0 ? rho[0] : (lane == 1 ? rho[1] : (lane == 2 ? rho[2] : rho[3]));
        const double lam = fabs(b) / (rl * h), l2 = lam * lam;
        const double e = exp(-l2) * INVSQRTPI, ec = erfc(lam);
        i0 = e - lam * ec;
        i2 = (2.0 / 3.0) * ((0.5 - l2) * e + l2 * lam * ec);
        i4 = (2.0 / 15.0) * (fma(fma(4.0, l2, -2.0), l2, 3.0) * e - 4.0 * l2 * l2 * lam * ec);
    }
    double a[MAXD], c[MAXD], e[MAXD];
#pragma unroll
    for (int k = 0; k < MAXD; ++k) {
        const double rk = rho[k], r3 = rk * rk * rk;
        a[k] = rk * __shfl_sync(FULL, i0, k);
        c[k] = r3 * __shfl_sync(FULL, i2, k);
        e[k] = r3 * rk * rk * __shfl_sync(FULL, i4, k);
    }
    // 2x2 minors of rows c, e: m_ij = c_i e_j - c_j e_i
    const double m01 = c[0] * e[1] - c[1] * e[0], m02 = c[0] * e[2] - c[2] * e[0];
    const double m03 = c[0] * e[3] - c[3] * e[0], m12 = c[1] * e[2] - c[2] * e[1];
    const double m13 = c[1] * e[3] - c[3] * e[1], m23 = c[2] * e[3] - c[3] * e[2];
    al[0] = a[1] * m23 - a[2] * m13 + a[3] * m12;
    al[1] = -(a[0] * m23 - a[2] * m03 + a[3] * m02);
    al[2] = a[0] * m13 - a[1] * m03 + a[3] * m01;
    al[3] = -(a[0] * m12 - a[1] * m02 + a[2] * m01);
    const double det = (al[0] + al[1]) + (al[2] + al[3]);
    bool ok = det != 0.0 && isfinite(det);
    if (ok) {
#pragma unroll
        for (int k = 0; k < MAXD; ++k) al[k] /= det;
        ok = isfinite(al[0]) && isfinite(al[1]) && isfinite(al[2]) && isfinite(al[3]);
    }
    if (!ok) {
        al[0] = 1.0;
        al[1] = 0.0;
        al[2] = 0.0;
        al[3] = 0.0;
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

// Fill the geometry constants of target m (all lanes; lanes 0..ndelta-1 also evaluate the I's).
// ndelta = 3: the extrapolation weights of Eq. (extrap_eqn); 4: the O(delta^7) variant;
// 2: the two-delta weights above (gamma returned in *gamma); 1: alpha = (1, 0, 0).
// rho holds max(ndelta, 3) entries.
__device__ __forceinline__ void load_geom(int lane, const double *y, const double *x0, const double *n0, double b,
                                          int64_t m, const double *rho, double h, Geom &T, int ndelta = 3,
                                          double *gamma = nullptr) {
    for (int i = 0; i < 3; ++i) {
        T.y[i] = y[3 * m + i];
        T.x0[i] = x0[3 * m + i];
        T.n0[i] = n0[3 * m + i];
        T.yh[i] = __double2float_rn(T.y[i]);
        T.yl[i] = __double2float_rn(T.y[i] - (double)T.yh[i]);
    }
    T.b = b;
    T.b2 = 2.0 * b;
    for (int i = 0; i < 3; ++i) T.n0p[i] = fp_split(T.n0[i]);
    T.b2p = fp_split(T.b2);
    double al[MAXD] = {1.0, 0.0, 0.0, 0.0};
    if (ndelta == 4) {
        extrap_weights4(lane, b, rho, h, al);
        if (gamma) *gamma = 0.0;
    } else if (ndelta == 2) {
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
    const int nk = ndelta == 4 ? 4 : 3;
#pragma unroll
    for (int k = 0; k < MAXD; ++k) {
        if (k >= nk) break;
        const double dk = rho[k] * h, id = 1.0 / dk;
        T.invd2[k] = id * id;
        T.s2w[k] = (2.0 * TAB_INV_W) * T.invd2[k];  // a power-of-two multiple: exact
        T.ad1[k] = al[k] * id;
        T.ad3[k] = al[k] * id * id * id;
        T.ad5[k] = al[k] * id * id * id * id * id;
        T.id2h[k] = (float)T.invd2[k];
        T.id2l[k] = (float)(T.invd2[k] - (double)T.id2h[k]);
        const double adp[3] = {T.ad1[k], T.ad3[k], T.ad5[k]};
        for (int p = 0; p < 3; ++p) {
            T.adh[p][k] = (float)adp[p];
            T.adl[p][k] = (float)(adp[p] - (double)T.adh[p][k]);
        }
    }
    T.apre[0] = al[0];
    T.apre[1] = al[0] + al[1];
    T.apre[2] = al[0] + al[1] + al[2];
    T.apre[3] = (al[0] + al[1]) + (al[2] + al[3]);
    for (int k = 0; k < MAXD; ++k) {
        T.aph[k] = (float)T.apre[k];
        T.apl[k] = (float)(T.apre[k] - (double)T.aph[k]);
    }
    for (int k = 0; k < MAXD; ++k) T.alf[k] = (float)al[k];
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

// alpha-weighted kernel factors of a near pair of class CLS: delta_0..delta_{CLS-1} have
// r > min(DEFECT_T, cutoff_t) delta_k and take the defect path below; the others take sigma_p
// from the interpolation table.  ND = number of deltas in use (3 for the method; 2 or 1 for the
// learned closure).
// sigma_p(tau) (or sigma#_p with the on-surface table) from a device table of INV_W intervals per
// unit tau and N intervals, for the local variable s (in [-1, 1] up to the interval-choice bound
// below): degrees 6..4 of the local polynomial in FP32, 3..0 in float pairs (Horner), results
// as float pairs sg[p] = (hi, lo), relative error ~2e-15 (the interpolation) + ~1e-14 (the pairs).
template <int N>
__device__ __forceinline__ void table_pairs(const float4 *__restrict__ ftab, int idx, double s, float sg[3][2]) {
    float sh, sl;
    split_pair(s, sh, sl);
    const float4 *t = ftab + (int64_t)idx * 9;
#pragma unroll 1
    for (int p = 0; p < 3; ++p) {
        const float4 a = __ldg(t + 3 * p), c32 = __ldg(t + 3 * p + 1), c10 = __ldg(t + 3 * p + 2);
        float ph = fmaf(fmaf(a.x, sh, a.y), sh, a.z), pl = 0.0f;
        pair_mad(ph, pl, sh, sl, c32.x, c32.y);
        pair_mad(ph, pl, sh, sl, c32.z, c32.w);
        pair_mad(ph, pl, sh, sl, c10.x, c10.y);
        pair_mad(ph, pl, sh, sl, c10.z, c10.w);
        sg[p][0] = ph;
        sg[p][1] = pl;
    }
}

// sigma_p at tau as float pairs (the on-surface path).
template <int INV_W, int N>
__device__ __forceinline__ void table_sigma(const double *__restrict__ tab, double tau, fpair sg[3]) {
    const float4 *ftab = reinterpret_cast<const float4 *>(tab);
    int idx = (int)(approx_float_pos(tau) * (float)INV_W);
    idx = min(idx, N - 1);
    const double s = fma(tau, 2.0 * INV_W, -float_to_double((float)(2 * idx + 1)));  // local variable in [-1, 1]
    float sp[3][2];
    table_pairs<N>(ftab, idx, s, sp);
#pragma unroll
    for (int p = 0; p < 3; ++p) sg[p] = {sp[p][0], sp[p][1]};
}

// table_pairs at tau = r^2 / delta^2 without forming tau in FP64: the interval from the FP32
// product r2f idf (r2f, idf: r^2 and 1/delta^2 as floats), the local variable as
// r^2 (2 INV_W / delta^2) - (2 i + 1) in one FMA.  The FP32 product carries three roundings
// (r2f, idf and the product: at most ~1.8e-7 of tau), so near an interval end it can pick the
// neighbouring interval; the local variable then lies outside [-1, 1] by at most
// 2 INV_W tau 1.8e-7 (below 1.4e-4 for INV_W = 16 and tau < 24), where each piece is still
// accurate to ~1e-15 (checked on the host at |s| = 1 + 2e-4 for every interval).
template <int INV_W, int N>
__device__ __forceinline__ void table_pairs_r2(const double *__restrict__ tab, double r2, float r2f, float idf,
                                               double s2w, float sg[3][2]) {
    const float4 *ftab = reinterpret_cast<const float4 *>(tab);
    int idx = (int)(r2f * idf * (float)INV_W);
    idx = min(idx, N - 1);
    const double s = fma(r2, s2w, -float_to_double((float)(2 * idx + 1)));
    table_pairs<N>(ftab, idx, s, sg);
}

// K1, K3, K5 as float pairs (~1e-14 relative); r2p = r2 as a float pair.  The class is a
// run-time value, uniform over a batch of pairs: one code path for all of them keeps the kernel
// within the instruction cache, and the loops over deltas stay rolled (the unrolled float-pair
// code of several deltas overflows it); T sits in shared memory, since the loops index its arrays
// at run time.
template <int ND>
__device__ __forceinline__ void kernel_factors_pair(const Geom &T, const ScanParams &P, const double *__restrict__ tab,
                                                    double r2, fpair r2p, int cls, fpair K[3]) {
    float kh[3] = {0.0f, 0.0f, 0.0f}, kl[3] = {0.0f, 0.0f, 0.0f};
    if (cls >= 1) {
        // r / delta_k > DEFECT_T: s_p = 1 - eps_p with eps_1 = erfc t, eps_2 = eps_1 + (2/sqrt pi) t e^{-t^2},
        // eps_3 = eps_1 + (2/sqrt pi)(t + 2/3 t^3) e^{-t^2} (Eqs. (s1)-(s3)), all below 2.1e-8, and
        // eps_p = 0 where t > cutoff_t (Sec. 3.2).  The term is (sum_k alpha_k - sum_k alpha_k eps_p(t_k)) / r^p.
        // eps_p in FP32 with a relative error of a few 1e-7, i.e. below 1e-14 of s_p:
        //  - tau = t^2 = r^2 / delta^2 as a float pair (exact product of the leading floats plus the
        //    cross terms), so that e^{-tau} = e^{-tau_h} (1 - tau_l) loses nothing to the rounding of tau;
        //  - erfc t = e^{-t^2} / (t sqrt pi) (1 - 1/(2t^2) + 3/(4t^4) - 15/(8t^6)), the asymptotic series
        //    (Abramowitz & Stegun 7.1.23), truncation below 3e-5 relative for t >= 4.7.
        const float r2h = r2p.h, r2l = r2p.l;
        float E1 = 0.0f, E3 = 0.0f, E5 = 0.0f;
        auto defect = [&](int k) {
            const float th = r2h * T.id2h[k];
            const float tl = fmaf(r2h, T.id2h[k], -th) + fmaf(r2h, T.id2l[k], r2l * T.id2h[k]);
            bool reg = th <= T.tcf2;  // t <= cutoff_t: s_p < 1
            if (fabsf(th - T.tcf2) <= CUT_BAND * T.tcf2) reg = r2 <= P.cut2d[k];
            if (reg) {
                const float g = expf(-th) * (1.0f - tl);  // e^{-t^2}
                const float it = rsqrt_ftz(th);             // 1/t (th > 20)
                const float t = th * it;
                const float u = it * it;  // 1/t^2
                const float ser = fmaf(fmaf(fmaf(-1.875f, u, 0.75f), u, -0.5f), u, 1.0f);
                const float e = 0.56418958354775628f * g * it * ser;  // erfc t
                const float gt = 1.12837916709551257f * g * t;         // (2/sqrt pi) t e^{-t^2}
                const float a = T.alf[k];
                E1 = fmaf(a, e, E1);
                E3 = fmaf(a, e + gt, E3);
                E5 = fmaf(a, fmaf(gt, 0.6666666666666667f * th, e + gt), E5);
            }
        };
#pragma unroll 1
        for (int k = 0; k < cls; ++k) defect(k);
        // 1/r in float pairs from the FP32 estimate y0: with e = 1 - r^2 y0^2 (|e| < 1e-6, from the
        // exact square of y0 and the pair product with r^2), 1/r = y0 (1 + e/2 + 3 e^2/8) + O(e^3 y0)
        const float y0 = rsqrt_ftz(r2h);  // r2h > 0: r > 4.7 delta_0
        const float qh = __fmul_rn(y0, y0), ql = __fmaf_rn(y0, y0, -qh);
        const float ph = __fmul_rn(r2h, qh);
        const float pe = __fmaf_rn(r2h, ql, __fmaf_rn(r2l, qh, __fmaf_rn(r2h, qh, -ph)));
        const float ee = __fsub_rn(__fsub_rn(1.0f, ph), pe);
        const float cr = __fmul_rn(y0, __fmul_rn(ee, __fmaf_rn(0.375f, ee, 0.5f)));
        const float r1h = __fadd_rn(y0, cr), r1l = __fsub_rn(cr, __fsub_rn(r1h, y0));
        float q2h, q2l, r3h, r3l, r5h, r5l;
        pair_mul(r1h, r1l, r1h, r1l, q2h, q2l);
        pair_mul(q2h, q2l, r1h, r1l, r3h, r3l);
        pair_mul(r3h, r3l, q2h, q2l, r5h, r5l);
        // (sum of the alpha of the defect-path deltas) / r^p, and the defects eps_p / r^p in FP32
        // (relative error ~1e-7 of terms below 2.1e-8 of the result)
        const int ia = cls - 1;
        const float ah = T.aph[ia], al = T.apl[ia];
        pair_mul(ah, al, r1h, r1l, kh[0], kl[0]);  // the factors are still zero here
        pair_mul(ah, al, r3h, r3l, kh[1], kl[1]);
        pair_mul(ah, al, r5h, r5l, kh[2], kl[2]);
        pair_add(kh[0], kl[0], -(E1 * r1h));
        pair_add(kh[1], kl[1], -(E3 * r3h));
        pair_add(kh[2], kl[2], -(E5 * r5h));
    }
    {
        // the table-path deltas: (alpha_k / delta_k^p) sigma_p(tau_k)
        const float r2f = approx_float_pos(r2);
        auto table = [&](int k) {
            float sg[3][2];
            table_pairs_r2<TAB_INV_W, TAB_N>(tab, r2, r2f, T.id2h[k], T.s2w[k], sg);
            if (T.cut_small && r2f * T.id2h[k] >= (1.0f - CUT_BAND) * T.tcf2 && r2 > P.cut2d[k]) {
                // t just beyond a cutoff below DEFECT_T: s_p := 1, sigma_p = 1/t^p (Sec. 3.2)
                const double tau = r2 * T.invd2[k];
                const double s1 = rsqrt(tau), s2 = s1 * s1 * s1, s3 = s2 * s1 * s1;
                split_pair(s1, sg[0][0], sg[0][1]);
                split_pair(s2, sg[1][0], sg[1][1]);
                split_pair(s3, sg[2][0], sg[2][1]);
            }
#pragma unroll
            for (int p = 0; p < 3; ++p) pair_acc(kh[p], kl[p], T.adh[p][k], T.adl[p][k], sg[p][0], sg[p][1]);
        };
#pragma unroll 1
        for (int k = cls; k < ND; ++k) table(k);
    }
#pragma unroll
    for (int p = 0; p < 3; ++p) K[p] = {kh[p], kl[p]};
}

// The near-pair contractions in float pairs (k_near, k_batch): operands from the near-field record
// and the target's pairs, results added into per-lane float-pair accumulators.  Each result
// carries an error ~1e-14 of the magnitudes it is formed from, far below the 1e-11 the FP64 path
// is held to.
// Single layer (Eq. (Sreg)): accU += K1 g + K3 d (d.g), g = w f - c w n.
// Double layer: with d = y - x = b n0 - xh, L = r^2 K5 - K3, U = d.Q, W = d.m, nQ = n0.Q,
// nm = n0.m, the contraction -6 [t1 K + t2 K5] : Q m (K = K3 - (r^2 - b^2) K5; t1, t2 as above)
// equals -6 ( n0 [nQ (2 b nm - W) - nm U] L  -  d [L nm nQ - K5 W U] ): substitute xh = b n0 - d
// into n0 (K (b P - S) + K5 b R) + xh (K5 (b S - R) - K P) and collect (K - b^2 K5 = -L);
// accN += the n0 coefficient, accD += the d coefficient (the result is -6/(8 pi) (accN n0 - accD)).
// Where every delta is on the defect path L is ~1e-7 of K3 or less, and its float-pair error,
// ~1e-14 of K3, is of the size of the other terms' errors.
__device__ __forceinline__ void sl_accumulate_pair(const fpair d[3], fpair K1, fpair K3, fpair nc, const fpair wf[3],
                                                   const fpair wn[3], fpair accU[3]) {
    const fpair g0 = fp_fma(nc, wn[0], wf[0]);  // g = w f - c w n, nc = -c
    const fpair g1 = fp_fma(nc, wn[1], wf[1]);
    const fpair g2 = fp_fma(nc, wn[2], wf[2]);
    const fpair t = fp_mul(K3, fp_dot3(d[0], d[1], d[2], g0, g1, g2));
    accU[0] = fp_acc2(accU[0], t, d[0], K1, g0);
    accU[1] = fp_acc2(accU[1], t, d[1], K1, g1);
    accU[2] = fp_acc2(accU[2], t, d[2], K1, g2);
}

__device__ __forceinline__ void dl_accumulate_pair(const Geom &T, const fpair d[3], fpair r2, fpair K3, fpair K5,
                                                   const fpair wn[3], const fpair qs[3], const fpair q0[3],
                                                   fpair &accN, fpair accD[3]) {
    const fpair W = fp_dot3(d[0], d[1], d[2], wn[0], wn[1], wn[2]);
    const fpair nm = fp_dot3(T.n0p[0], T.n0p[1], T.n0p[2], wn[0], wn[1], wn[2]);
    const fpair L = fp_fma(r2, K5, fp_neg(K3));
    const fpair Z = fp_fma(T.b2p, nm, fp_neg(W));
    const fpair Q0 = fp_add(qs[0], fp_neg(q0[0])), Q1 = fp_add(qs[1], fp_neg(q0[1])), Q2 = fp_add(qs[2], fp_neg(q0[2]));
    const fpair nQ = fp_dot3(T.n0p[0], T.n0p[1], T.n0p[2], Q0, Q1, Q2);
    const fpair U = fp_dot3(d[0], d[1], d[2], Q0, Q1, Q2);
    accN = fp_add(accN, fp_mul(L, fp_fma(nQ, Z, fp_neg(fp_mul(nm, U)))));
    const fpair C = fp_fma(fp_mul(L, nm), nQ, fp_neg(fp_mul(fp_mul(K5, W), U)));
    accD[0] = fp_fma(C, d[0], accD[0]);
    accD[1] = fp_fma(C, d[1], accD[1]);
    accD[2] = fp_fma(C, d[2], accD[2]);
}

// Walk the rows of the surface's cell grid that meet the prefilter ball around the target,
// test candidates in FP32, queue survivors by class in the warp's shared queues sq[NC][64],
// and call batch(cls, j, valid) with one node per lane whenever a class has 32 entries, then
// once per class for the remainder (lanes with valid = false hold no node).  NC = number of
// classes: 4 with three deltas, 5 with four.  batch is called from one place, with the class
// as a run-time value, so that its code (the whole pair evaluation) exists once in the kernel:
// each turn of the loop either hands one batch over or tests the next 32 candidates of the
// current row.
template <int NC = NCLS, class Batch>
__device__ __forceinline__ void scan_near(const SurfDev &s, const Geom &T, const ScanParams &P, int (*sq)[64],
                                          int lane, Batch &&batch) {
    int qn[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) qn[c] = 0;
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
    // row cursor: the next row (iz, iy) that meets the ball, as the node range [jb, je) of the
    // cells ia..ib it spans
    int iz = lo[2], iy = lo[1] - 1, jb = 0, je = 0;
    auto next_row = [&]() -> bool {
        for (;;) {
            if (++iy > hi[1]) {
                iy = lo[1];
                if (++iz > hi[2]) return false;
            }
            const float zl = of[2] + iz * cw;
            const float dzr = fmaxf(0.0f, fmaxf(zl - yf[2], yf[2] - (zl + cw)));
            const float yl0 = of[1] + iy * cw;
            const float dyr = fmaxf(0.0f, fmaxf(yl0 - yf[1], yf[1] - (yl0 + cw)));
            const float rem = R2 - dyr * dyr - dzr * dzr;
            if (rem < 0.0f) continue;
            const float half = sqrtf(rem) * 1.0001f + 1e-6f * cw;
            const int ia = max(lo[0], (int)floorf((yf[0] - half - of[0]) * inv_cw));
            const int ib = min(hi[0], (int)floorf((yf[0] + half - of[0]) * inv_cw));
            if (ia > ib) continue;
            const int64_t rowbase = ((int64_t)iz * G.nc[1] + iy) * G.nc[0];
            jb = cs[rowbase + ia];
            je = cs[rowbase + ib + 1];
            if (jb < je) return true;
        }
    };
    bool more = lo[0] <= hi[0] && lo[1] <= hi[1] && lo[2] <= hi[2] && next_row();
    for (;;) {
        // a class with 32 queued nodes or, once the rows are done, with a remainder
        int c = -1;
#pragma unroll
        for (int cc = NC - 1; cc >= 0; --cc)
            if (qn[cc] >= 32 || (!more && qn[cc] > 0)) c = cc;
        if (c >= 0) {
            int n = 0;
#pragma unroll
            for (int cc = 0; cc < NC; ++cc) n = cc == c ? qn[cc] : n;
            const int take = min(n, 32);
            const bool v = lane < take;
            batch(c, v ? sq[c][n - take + lane] : 0, v);
#pragma unroll
            for (int cc = 0; cc < NC; ++cc)
                if (cc == c) qn[cc] = n - take;
            __syncwarp();
            continue;
        }
        if (!more) break;
        // the next 32 candidates of the row (every queue holds < 32 here, so <= 63 after)
        const int j = jb + lane;
        bool pass = false;
        int cls = 0;
        if (j < je) {
            const float4 p = __ldg(xs32 + j);
            const float ex = yf[0] - p.x, ey = yf[1] - p.y, ez = yf[2] - p.z;
            const float r2f = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
            pass = r2f <= R2;
#pragma unroll
            for (int k = 0; k < NC - 1; ++k) cls += r2f > P.th[k];
        }
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) {
            const unsigned mk = __ballot_sync(FULL, pass && cls == cc);
            if (pass && cls == cc) sq[cc][qn[cc] + __popc(mk & lt)] = j;
            qn[cc] += __popc(mk);
        }
        __syncwarp();
        jb += 32;
        if (jb >= je) more = next_row();
    }
    __syncwarp();
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// nd = number of deltas (3 or 4; rho holds nd entries)
inline ScanParams scan_params(const ers_surface *s, double Rc, const double *rho, double cutoff_t, int nd = 3) {
    ScanParams P{};
    P.rc2f = (float)(Rc * Rc);
    double L = 0.0;
    for (int i = 0; i < 3; ++i) L = fmax(L, fabs(s->c[i]) + s->a[i]);
    P.rpre = (float)(Rc * (1.0 + 1e-5) + 4e-6 * (L + Rc));
    for (int k = nd; k < MAXD; ++k) P.th[k] = HUGE_VALF;
    for (int k = 0; k < nd; ++k) {
        // The prefilter's r^2 comes from float coordinates (|coordinate| <= L + Rc, each rounded
        // to 2^-24 relative): widen the threshold by 4x that error bound so that every pair sent
        // to the defect path has r > min(DEFECT_T, cutoff_t) delta_k in exact arithmetic (the
        // asymptotic series needs t >= 4.5; below a cutoff < DEFECT_T nothing is evaluated there).
        const double t = fmin(DEFECT_T, cutoff_t) * rho[k] * s->h;
        const double margin = fmin(0.04, 1e-6 + 4.0 * 2.0 * 6.0 * (L + Rc) * 0x1p-24 / t);
        P.th[k] = (float)(t * t * (1.0 + margin));
    }
    for (int k = 0; k < MAXD - 1; ++k) P.cut2[k] = HUGE_VALF;
    for (int k = 0; k < nd - 1; ++k) {
        const double t = cutoff_t * rho[k] * s->h;
        P.cut2[k] = (float)(t * t);
    }
    P.tcf2 = (float)(cutoff_t * cutoff_t);
    P.tc2 = cutoff_t * cutoff_t;
    for (int k = 0; k < nd; ++k) {
        const double rk = cutoff_t * rho[k] * s->h;
        P.cut2d[k] = rk * rk;
    }
    P.h = s->h;
    return P;
}

}  // namespace nearc
// One problem of the batched evaluation, as the persistent kernel sees it.
struct BatchProblemDev {
    SurfDev sd;
    const float2 *densp;   // [N][NR][6] sorted order: w f (3), q (3) as float pairs (hi, lo)
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
