// Near field and extrapolation (Secs. 2, 3.2, 3.3).
//
// For a target y with |b| <= Rc the three regularized sums over the near nodes (r <= Rc) are
// combined with the extrapolation weights alpha_k before the contraction: since
// u = u_far + sum_k alpha_k u_near_k (Eq. (near_far) with the solve of Eq. (extrap_eqn) and
// sum_k alpha_k = 1), each near pair needs only the alpha-weighted kernel factors
//   K1 = sum_k alpha_k s1(r/delta_k)/r,  K3 = sum_k alpha_k s2(r/delta_k)/r^3,
//   K5 = sum_k alpha_k s3(r/delta_k)/r^5,
// with s_p := 1 where r/delta_k > cutoff_t (Sec. 3.2).  s_p(t)/r^p = sigma_p(tau) / delta^p with
// tau = (r/delta)^2, and sigma_p comes from a piecewise degree-6 interpolation table.
// Single layer (Eq. (Sreg)):  K1 g + K3 d (d.g).
// Double layer (Eqs. (Tsplit), (Treg)):  -6 [ t1 (K3 - (r^2 - b^2) K5) + t2 K5 ] : Q (w n),
// contracted in closed form: with P = (n0.Q)(n0.m), R = (xh.Q)(xh.m),
// S = (xh.Q)(n0.m) + (n0.Q)(xh.m), K = K3 - (r^2 - b^2) K5, xh = x - x0:
//   t1 : Q m = n0 (b P - S) - xh P,   t2 : Q m = n0 (b R) + xh (b S - R).
// The weights alpha are the first row of the inverse of A_k = [1, rho_k I0(b/delta_k),
// rho_k^3 I2(b/delta_k)] (Eqs. (extrap_eqn), (I0), (I2)), by Cramer's rule.
//
// One warp per target.  The warp walks the rows of the cell grid that meet the ball of radius
// Rc, tests candidates with an FP32 prefilter (conservative margin), and queues survivors by
// class c = number of delta_k with r > cutoff_t delta_k, so that each batch of 32 runs one
// code path.  Each batch then makes the exact FP64 (or, for the mixed far field, the
// identical FP32) near/far test, so that the partition matches the far-field mask exactly.
#include "ers_internal.h"

namespace ers {
namespace {

constexpr int WPB = 4;  // warps per block
constexpr unsigned FULL = 0xffffffffu;
constexpr double INV8PI = 0.039788735772973833942;
constexpr double INVSQRTPI = 0.56418958354775628695;

struct NearConst {
    double y[3], x0[3], n0[3], b, c, q0[3];
    double invd2[3], ad1[3], ad3[3], ad5[3], apre[2];
    float yh[3], yl[3];  // mixed-mode classification
};

template <int CLS, int PREC, bool SL, bool DL>
__device__ __forceinline__ void process(const EvalArgs &A, const NearConst &T, const double *__restrict__ tab,
                                        float rc2f, int64_t j, double accU[3], double &accN, double accX[3],
                                        int npairs[3]) {
    const double2 *r = reinterpret_cast<const double2 *>(A.s->rec + j * REC);
    const double2 r0 = __ldg(r + 0), r1 = __ldg(r + 1), r2v = __ldg(r + 2);
    const double2 r3 = __ldg(r + 3), r4 = __ldg(r + 4), r5 = __ldg(r + 5);
    const double xs[3] = {r0.x, r0.y, r1.x};
    const double wf[3] = {r1.y, r2v.x, r2v.y};
    const double wn[3] = {r3.x, r3.y, r4.x};
    const double qs[3] = {r4.y, r5.x, r5.y};
    const double dx = __dsub_rn(T.y[0], xs[0]);
    const double dy = __dsub_rn(T.y[1], xs[1]);
    const double dz = __dsub_rn(T.y[2], xs[2]);
    const double r2 = dist2_fp64(dx, dy, dz);
    bool near;
    if (PREC == ERS_PREC_FP64) {
        near = !(__double_as_longlong(r2) > __double_as_longlong(A.Rc * A.Rc));
    } else {
        const float4 cen = __ldg(reinterpret_cast<const float4 *>(A.s->tilec) + j / TS32);
        const float4 xc = __ldg(reinterpret_cast<const float4 *>(A.s->rec32 + j * REC));
        float ex, ey, ez;
        const float r2f = dist2_fp32(tile_rel(T.yh[0], cen.x, T.yl[0]), tile_rel(T.yh[1], cen.y, T.yl[1]),
                                     tile_rel(T.yh[2], cen.z, T.yl[2]), xc.x, xc.y, xc.z, &ex, &ey, &ez);
        near = !(r2f > rc2f);
    }
    if (!near) return;
    ++npairs[CLS];
    double K1 = 0.0, K3 = 0.0, K5 = 0.0;
#pragma unroll
    for (int k = CLS; k < 3; ++k) {
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
    if (CLS >= 1) {  // delta_0..delta_{CLS-1} are not regularized at this distance: s_p = 1
        const double Ain = T.apre[CLS - 1];
        const double ri = rsqrt(r2);
        const double ri2 = ri * ri;
        const double ri3 = ri2 * ri;
        K1 = fma(Ain, ri, K1);
        K3 = fma(Ain, ri3, K3);
        K5 = fma(Ain, ri3 * ri2, K5);
    }
    if (SL) {
        const double g0 = fma(-T.c, wn[0], wf[0]);
        const double g1 = fma(-T.c, wn[1], wf[1]);
        const double g2 = fma(-T.c, wn[2], wf[2]);
        const double t = K3 * fma(dz, g2, fma(dy, g1, dx * g0));
        accU[0] = fma(t, dx, fma(K1, g0, accU[0]));
        accU[1] = fma(t, dy, fma(K1, g1, accU[1]));
        accU[2] = fma(t, dz, fma(K1, g2, accU[2]));
    }
    if (DL) {
        const double Q0 = qs[0] - T.q0[0], Q1 = qs[1] - T.q0[1], Q2 = qs[2] - T.q0[2];
        const double h0 = xs[0] - T.x0[0], h1 = xs[1] - T.x0[1], h2 = xs[2] - T.x0[2];
        const double nQ = fma(T.n0[2], Q2, fma(T.n0[1], Q1, T.n0[0] * Q0));
        const double nm = fma(T.n0[2], wn[2], fma(T.n0[1], wn[1], T.n0[0] * wn[0]));
        const double xQ = fma(h2, Q2, fma(h1, Q1, h0 * Q0));
        const double xm = fma(h2, wn[2], fma(h1, wn[1], h0 * wn[0]));
        const double P = nQ * nm, R = xQ * xm, S = fma(xQ, nm, nQ * xm);
        const double K = fma(-(r2 - T.b * T.b), K5, K3);
        const double cn = fma(K, fma(T.b, P, -S), K5 * T.b * R);
        const double cx = fma(K5, fma(T.b, S, -R), -K * P);
        accN += cn;
        accX[0] = fma(cx, h0, accX[0]);
        accX[1] = fma(cx, h1, accX[1]);
        accX[2] = fma(cx, h2, accX[2]);
    }
}

template <int PREC, bool SL, bool DL>
__device__ __forceinline__ void process_cls(int cls, const EvalArgs &A, const NearConst &T,
                                            const double *__restrict__ tab, float rc2f, int64_t j, double accU[3],
                                            double &accN, double accX[3], int npairs[3]) {
    if (cls == 0) process<0, PREC, SL, DL>(A, T, tab, rc2f, j, accU, accN, accX, npairs);
    else if (cls == 1) process<1, PREC, SL, DL>(A, T, tab, rc2f, j, accU, accN, accX, npairs);
    else process<2, PREC, SL, DL>(A, T, tab, rc2f, j, accU, accN, accX, npairs);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

struct NearParams {
    float rc2f;      // exact FP32 threshold of the mixed far field
    float rpre;      // FP32 prefilter radius (Rc plus a conservative margin)
    float th[2];     // FP32 class thresholds (cutoff_t delta_0)^2, (cutoff_t delta_1)^2
    double h;
};

template <int PREC, bool SL, bool DL>
__global__ void __launch_bounds__(WPB * 32) k_near(EvalArgs A, NearParams P, const double *__restrict__ tab) {
    __shared__ int sq[WPB][3][64];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t m = (int64_t)blockIdx.x * WPB + wib;
    if (m >= A.M) return;  // warp-uniform

    // sum of the far-field chunk partials: lane i < 6 holds component i
    double fs = 0.0;
    if (lane < 6)
        for (int c = 0; c < A.chunks; ++c) fs += A.part[((int64_t)c * A.M + m) * 6 + lane];
    const double bm = A.b[m];
    if (!(fabs(bm) <= A.Rc)) {
        if (SL && lane < 3) A.u[3 * m + lane] = fs;
        if (DL && lane >= 3 && lane < 6) A.v[3 * m + lane - 3] = fs;
        return;
    }

    NearConst T;
    for (int i = 0; i < 3; ++i) {
        T.y[i] = A.y[3 * m + i];
        T.x0[i] = A.x0[3 * m + i];
        T.n0[i] = A.n0[3 * m + i];
        T.q0[i] = DL ? A.q0[3 * m + i] : 0.0;
        T.yh[i] = __double2float_rn(T.y[i]);
        T.yl[i] = __double2float_rn(T.y[i] - (double)T.yh[i]);
    }
    T.b = bm;
    T.c = SL ? fma(A.f0[3 * m + 2], T.n0[2], fma(A.f0[3 * m + 1], T.n0[1], A.f0[3 * m] * T.n0[0])) : 0.0;

    // extrapolation weights (lane k < 3 evaluates I0, I2 at lambda_k)
    double i0 = 0.0, i2 = 0.0;
    if (lane < 3) {
        const double rl = lane == 0 ? A.rho[0] : (lane == 1 ? A.rho[1] : A.rho[2]);
        const double lam = fabs(bm) / (rl * P.h);
        const double e = exp(-lam * lam) * INVSQRTPI, ec = erfc(lam);
        i0 = e - lam * ec;
        i2 = (2.0 / 3.0) * ((0.5 - lam * lam) * e + lam * lam * lam * ec);
    }
    double ac[3], bc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double rk = A.rho[k];
        ac[k] = rk * __shfl_sync(FULL, i0, k);
        bc[k] = rk * rk * rk * __shfl_sync(FULL, i2, k);
    }
    double al[3] = {ac[1] * bc[2] - ac[2] * bc[1], ac[2] * bc[0] - ac[0] * bc[2], ac[0] * bc[1] - ac[1] * bc[0]};
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
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double dk = A.rho[k] * P.h, id = 1.0 / dk;
        T.invd2[k] = id * id;
        T.ad1[k] = al[k] * id;
        T.ad3[k] = al[k] * id * id * id;
        T.ad5[k] = al[k] * id * id * id * id * id;
    }
    T.apre[0] = al[0];
    T.apre[1] = al[0] + al[1];

    double accU[3] = {0.0, 0.0, 0.0}, accX[3] = {0.0, 0.0, 0.0}, accN = 0.0;
    int npairs[3] = {0, 0, 0};  // near pairs by class (number of unregularized deltas)
    int qn[3] = {0, 0, 0};
    const unsigned lt = (1u << lane) - 1u;

    // rows of the grid meeting the prefilter ball (FP32, conservative)
    const Grid &G = A.s->grid;
    const float yf[3] = {T.yh[0], T.yh[1], T.yh[2]};
    const float of[3] = {(float)G.origin[0], (float)G.origin[1], (float)G.origin[2]};
    const float cw = (float)G.cw, inv_cw = 1.0f / cw;
    const float R = P.rpre, R2 = R * R;
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = max(0, (int)floorf((yf[a] - R - of[a]) * inv_cw));
        hi[a] = min(G.nc[a] - 1, (int)floorf((yf[a] + R - of[a]) * inv_cw));
    }
    const int *__restrict__ cs = A.s->cell_start;
    const float4 *__restrict__ xs32 = A.s->xs32;
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
                    if (pass && cls == c) sq[wib][c][qn[c] + __popc(mk & lt)] = j;
                    qn[c] += __popc(mk);
                }
                __syncwarp();
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (qn[c] >= 32) {
                        const int jj = sq[wib][c][qn[c] - 32 + lane];
                        process_cls<PREC, SL, DL>(c, A, T, tab, P.rc2f, jj, accU, accN, accX, npairs);
                        qn[c] -= 32;
                        __syncwarp();
                    }
                }
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (qn[c] > 0 && lane < qn[c]) {
            const int jj = sq[wib][c][lane];
            process_cls<PREC, SL, DL>(c, A, T, tab, P.rc2f, jj, accU, accN, accX, npairs);
        }
    }
    __syncwarp();
    for (int i = 0; i < 3; ++i) {
        accU[i] = warp_sum(accU[i]);
        accX[i] = warp_sum(accX[i]);
    }
    accN = warp_sum(accN);
    int np[3] = {npairs[0], npairs[1], npairs[2]};
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) np[c] += __shfl_xor_sync(FULL, np[c], o);
    if (lane == 0 && A.counters) {
        atomicAdd(A.counters + 0, 1ull);
        atomicAdd(A.counters + 1, (unsigned long long)(np[0] + np[1] + np[2]));
        atomicAdd(A.counters + 2, (unsigned long long)np[0]);
        atomicAdd(A.counters + 3, (unsigned long long)np[1]);
        atomicAdd(A.counters + 4, (unsigned long long)np[2]);
    }
    if (SL && lane < 3) {
        const double a = lane == 0 ? accU[0] : (lane == 1 ? accU[1] : accU[2]);
        A.u[3 * m + lane] = fs + a * INV8PI;
    }
    if (DL && lane >= 3 && lane < 6) {
        const int i = lane - 3;
        const double ax = i == 0 ? accX[0] : (i == 1 ? accX[1] : accX[2]);
        const double ni = i == 0 ? T.n0[0] : (i == 1 ? T.n0[1] : T.n0[2]);
        const double qi = i == 0 ? T.q0[0] : (i == 1 ? T.q0[1] : T.q0[2]);
        const double chi = bm < 0.0 ? 1.0 : (bm > 0.0 ? 0.0 : 0.5);
        A.v[3 * m + i] = fs + (-6.0 * INV8PI) * fma(accN, ni, ax) + chi * qi;
    }
}

template <int PREC>
cudaError_t near_dispatch(const EvalArgs &a, NearParams P, const double *tab) {
    const int64_t grid = (a.M + WPB - 1) / WPB;
    const bool sl = a.layers & ERS_LAYER_SL, dl = a.layers & ERS_LAYER_DL;
    if (sl && dl) k_near<PREC, true, true><<<(unsigned)grid, WPB * 32, 0, a.stream>>>(a, P, tab);
    else if (sl) k_near<PREC, true, false><<<(unsigned)grid, WPB * 32, 0, a.stream>>>(a, P, tab);
    else k_near<PREC, false, true><<<(unsigned)grid, WPB * 32, 0, a.stream>>>(a, P, tab);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_near(const EvalArgs &a, const double *tab) {
    if (a.M == 0) return cudaSuccess;
    NearParams P;
    P.rc2f = (float)(a.Rc * a.Rc);
    const ers_surface *s = a.s;
    double L = 0.0;
    for (int i = 0; i < 3; ++i) L = fmax(L, fabs(s->c[i]) + s->a[i]);
    P.rpre = (float)(a.Rc * (1.0 + 1e-5) + 4e-6 * (L + a.Rc));
    for (int k = 0; k < 2; ++k) {
        const double t = a.cutoff_t * a.rho[k] * s->h;
        P.th[k] = (float)(t * t);
    }
    P.h = s->h;
    if (a.precision == ERS_PREC_FP64) return near_dispatch<ERS_PREC_FP64>(a, P, tab);
    return near_dispatch<ERS_PREC_MIXED>(a, P, tab);
}

}  // namespace ers
