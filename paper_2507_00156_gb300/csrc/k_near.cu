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
// contracted in closed form (dl_accumulate_pair in near_common.cuh).  Kernel factors and both
// contractions run in float pairs on the FP32 pipe (~1e-14 relative; the FP64 pipe of this part
// runs at 1/64 of the FP32 rate); d, r^2 and the near/far test stay FP64.
// The weights alpha are the first row of the inverse of A_k = [1, rho_k I0(b/delta_k),
// rho_k^3 I2(b/delta_k)] (Eqs. (extrap_eqn), (I0), (I2)), by Cramer's rule.  The O(delta^7)
// variant (Sec. 1) runs the same kernel with four deltas (ND = 4, A_k with rho_k^5 I4 appended).
//
// One warp per target.  The warp walks the rows of the cell grid that meet the ball of radius
// Rc, tests candidates with an FP32 prefilter (conservative margin), and queues survivors by
// class c = number of delta_k with r > min(4.7, cutoff_t) delta_k (0..ND), so that the lanes of a
// batch of 32 run the same loops over the deltas (the class is a run-time value of one code path).
// Each batch then makes the exact FP64 (or, for the mixed far field, the identical FP32) near/far
// test, so that the partition matches the far-field mask exactly.  Node data come from the
// 96-byte near-field records (x in FP64; w f, w n, q as float pairs).
#include <algorithm>
#include <cmath>

#include "near_common.cuh"

namespace ers {
namespace {

using namespace nearc;
constexpr int WPB = 4;  // warps per block
constexpr int NEAR_MIN_BLOCKS = 4;

// One near pair of class cls, a run-time value (one code path for every class keeps the kernel
// within the instruction cache); cls = ND: every delta on the defect path.  The pair geometry d,
// r^2 and the near/far test in FP64; kernel factors and contractions in float pairs (nc = -c and
// q0 of the target as float pairs), accumulated per lane in float pairs.
template <int PREC, bool SL, bool DL, int ND>
__device__ __forceinline__ void process(const EvalArgs &A, const Geom &T, const ScanParams &P, fpair nc,
                                        const fpair q0[3], const double *__restrict__ tab, int64_t j, int cls,
                                        fpair accU[3], fpair &accN, fpair accD[3], int npairs[NCLS_MAX],
                                        int nunreg[MAXD]) {
    const float4 *r = reinterpret_cast<const float4 *>(A.sd.recp + j * NREC);
    const float4 a0 = __ldg(r + 0), a1 = __ldg(r + 1), a2 = __ldg(r + 2);
    const float4 a3 = __ldg(r + 3), a4 = __ldg(r + 4), a5 = __ldg(r + 5);
    const double xs0 = __hiloint2double(__float_as_int(a0.y), __float_as_int(a0.x));
    const double xs1 = __hiloint2double(__float_as_int(a0.w), __float_as_int(a0.z));
    const double xs2 = __hiloint2double(__float_as_int(a1.y), __float_as_int(a1.x));
    const fpair wf[3] = {{a1.z, a1.w}, {a2.x, a2.y}, {a2.z, a2.w}};
    const fpair wn[3] = {{a3.x, a3.y}, {a3.z, a3.w}, {a4.x, a4.y}};
    const fpair qs[3] = {{a4.z, a4.w}, {a5.x, a5.y}, {a5.z, a5.w}};
    const double dx = __dsub_rn(T.y[0], xs0);
    const double dy = __dsub_rn(T.y[1], xs1);
    const double dz = __dsub_rn(T.y[2], xs2);
    const double r2 = dist2_fp64(dx, dy, dz);
    if (!is_near<PREC>(A.sd, T, j, r2, A.Rc, P.rc2f)) return;
#pragma unroll
    for (int k = 0; k < NCLS_MAX; ++k) npairs[k] += k == cls;
    {  // pairs by number of deltas with r > cutoff_t delta_k (the method's own count of regularized terms)
        const float r2f = approx_float_pos(r2);
        int u = (r2f > P.cut2[0]) + (r2f > P.cut2[1]);
        if (ND == 4) u += r2f > P.cut2[2];
#pragma unroll
        for (int k = 0; k < (ND == 4 ? 4 : 3); ++k) nunreg[k] += u == k;
    }
    const fpair r2p = fp_split(r2);
    fpair K[3];
    kernel_factors_pair<ND>(T, P, tab, r2, r2p, cls, K);
    const fpair d[3] = {fp_split(dx), fp_split(dy), fp_split(dz)};
    if (SL) sl_accumulate_pair(d, K[0], K[1], nc, wf, wn, accU);
    if (DL) dl_accumulate_pair(T, d, r2p, K[1], K[2], wn, qs, q0, accN, accD);
}

// On-surface target with ERS_OPT_SHARP (b = 0): one regularized sum with the modified
// smoothing functions s#_p of Sec. 2.1 at delta# (alpha = 1, no extrapolation) over r <= Rc#.
// Single layer: Eq. (Sreg) with s#_1, s#_2; double layer: the stresslet -6 d (d.Q)(d.m) s#_3/r^5
// (at b = 0 the split form would add t1 (s#_2 - s#_3)/r^3, which is not small for s#).
template <int PREC, bool SL, bool DL>
__device__ __forceinline__ void process_sharp(const EvalArgs &A, const Geom &T, const ScanParams &Ps, fpair nc,
                                              const fpair q0[3], int64_t j, fpair accU[3], fpair accV[3],
                                              int &npairs) {
    const float4 *r = reinterpret_cast<const float4 *>(A.sd.recp + j * NREC);
    const float4 a0 = __ldg(r + 0), a1 = __ldg(r + 1), a2 = __ldg(r + 2);
    const float4 a3 = __ldg(r + 3), a4 = __ldg(r + 4), a5 = __ldg(r + 5);
    const double dx = __dsub_rn(T.y[0], __hiloint2double(__float_as_int(a0.y), __float_as_int(a0.x)));
    const double dy = __dsub_rn(T.y[1], __hiloint2double(__float_as_int(a0.w), __float_as_int(a0.z)));
    const double dz = __dsub_rn(T.y[2], __hiloint2double(__float_as_int(a1.y), __float_as_int(a1.x)));
    const double r2 = dist2_fp64(dx, dy, dz);
    if (!is_near<PREC>(A.sd, T, j, r2, A.Rc_sharp, Ps.rc2f)) return;
    ++npairs;
    const fpair wf[3] = {{a1.z, a1.w}, {a2.x, a2.y}, {a2.z, a2.w}};
    const fpair wn[3] = {{a3.x, a3.y}, {a3.z, a3.w}, {a4.x, a4.y}};
    const fpair qs[3] = {{a4.z, a4.w}, {a5.x, a5.y}, {a5.z, a5.w}};
    fpair sg[3];  // t = r/delta# <= cutoff_t here
    table_sigma<SH_INV_W, SH_N>(A.tab_sharp, r2 * T.invd2[0], sg);
    fpair K[3];  // s#_p(t) / r^p = sigma#_p / delta#^p
#pragma unroll
    for (int p = 0; p < 3; ++p) K[p] = fp_mul({T.adh[p][0], T.adl[p][0]}, sg[p]);
    const fpair d[3] = {fp_split(dx), fp_split(dy), fp_split(dz)};
    if (SL) sl_accumulate_pair(d, K[0], K[1], nc, wf, wn, accU);
    if (DL) {
        const fpair Q0 = fp_add(qs[0], fp_neg(q0[0])), Q1 = fp_add(qs[1], fp_neg(q0[1])), Q2 = fp_add(qs[2], fp_neg(q0[2]));
        const fpair dQ = fp_dot3(d[0], d[1], d[2], Q0, Q1, Q2);
        const fpair W = fp_dot3(d[0], d[1], d[2], wn[0], wn[1], wn[2]);
        const fpair sv = fp_mul(fp_mul(dQ, W), K[2]);
        accV[0] = fp_fma(sv, d[0], accV[0]);
        accV[1] = fp_fma(sv, d[1], accV[1]);
        accV[2] = fp_fma(sv, d[2], accV[2]);
    }
}

template <int PREC, bool SL, bool DL>
__device__ __noinline__ void near_target_sharp(const EvalArgs &A, const ScanParams &Ps, int64_t m, int lane,
                                               int (*sq)[64], Geom &G, double fs) {
    {
        Geom Tl;
        const double rs[3] = {A.rho_sharp, A.rho_sharp, A.rho_sharp};
        load_geom(lane, A.y, A.x0, A.n0, 0.0, m, rs, Ps.h, Tl, 1, nullptr);  // alpha = (1, 0, 0)
        set_cutoff(Tl, Ps);
        __syncwarp();
        if (lane == 0) G = Tl;
        __syncwarp();
    }
    const Geom &T = G;
    double q0[3];
    for (int i = 0; i < 3; ++i) q0[i] = DL ? A.q0[3 * m + i] : 0.0;
    const double c = SL ? fma(A.f0[3 * m + 2], T.n0[2], fma(A.f0[3 * m + 1], T.n0[1], A.f0[3 * m] * T.n0[0])) : 0.0;
    const fpair ncp = fp_split(-c), q0p[3] = {fp_split(q0[0]), fp_split(q0[1]), fp_split(q0[2])};
    fpair pU[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}}, pV[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    int npairs = 0;
    scan_near(A.sd, T, Ps, sq, lane, [&](int, int jj, bool valid) {
        if (valid) process_sharp<PREC, SL, DL>(A, T, Ps, ncp, q0p, jj, pU, pV, npairs);
    });
    double accU[3], accV[3];
    for (int i = 0; i < 3; ++i) {
        accU[i] = warp_sum(fp_to_double(pU[i]));
        accV[i] = warp_sum(fp_to_double(pV[i]));
    }
    if (A.counters) {
        int np = npairs;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) np += __shfl_xor_sync(FULL, np, o);
        if (lane == 0) {
            atomicAdd(A.counters + 0, 1ull);
            atomicAdd(A.counters + 1, (unsigned long long)np);
            atomicAdd(A.counters + 9, (unsigned long long)np);
        }
    }
    if (SL && lane < 3) {
        const double a = lane == 0 ? accU[0] : (lane == 1 ? accU[1] : accU[2]);
        A.u[3 * m + lane] = fs + a * INV8PI;
    }
    if (DL && lane >= 3 && lane < 6) {
        const int i = lane - 3;
        const double av = i == 0 ? accV[0] : (i == 1 ? accV[1] : accV[2]);
        const double qi = i == 0 ? q0[0] : (i == 1 ? q0[1] : q0[2]);
        A.v[3 * m + i] = fs + (-6.0 * INV8PI) * av + 0.5 * qi;  // chi = 1/2 on the surface
    }
}

template <int PREC, bool SL, bool DL, int ND>
__device__ __forceinline__ void near_target(const EvalArgs &A, const ScanParams &P, const double *__restrict__ tab,
                                            int64_t m, int lane, int (*sq)[64], Geom &G, const ScanParams &Ps) {
    // sum of the far-field chunk partials: lane i < 6 holds component i
    double fs = 0.0;
    if (lane < 6 && !A.far_later)
        for (int c = 0; c < A.chunks; ++c) fs += A.part[((int64_t)c * A.M + m) * 6 + lane];
    const double bm = A.b[m];
    if (ND >= 3 && A.sharp && bm == 0.0) {
        near_target_sharp<PREC, SL, DL>(A, Ps, m, lane, sq, G, fs);
        return;
    }
    if (!(fabs(bm) <= A.Rc)) {
        if (A.gamma && lane == 0) A.gamma[m] = 0.0;
        if (SL && lane < 3) A.u[3 * m + lane] = fs;
        if (DL && lane >= 3 && lane < 6) A.v[3 * m + lane - 3] = fs;
        return;
    }

    // The per-target constants live in the warp's shared-memory slot G and are read from there
    // at each use (the pair loop would otherwise hold ~70 of them in registers).
    double gam = 0.0;
    {
        Geom Tl;
        load_geom(lane, A.y, A.x0, A.n0, bm, m, A.rho, P.h, Tl, ND, &gam);
        set_cutoff(Tl, P);
        __syncwarp();  // the previous target's reads of G are done
        if (lane == 0) G = Tl;
        __syncwarp();
    }
    const Geom &T = G;
    if (A.gamma && lane == 0) A.gamma[m] = gam;
    double q0[3];
    for (int i = 0; i < 3; ++i) q0[i] = DL ? A.q0[3 * m + i] : 0.0;
    const double c = SL ? fma(A.f0[3 * m + 2], T.n0[2], fma(A.f0[3 * m + 1], T.n0[1], A.f0[3 * m] * T.n0[0])) : 0.0;
    const fpair ncp = fp_split(-c), q0p[3] = {fp_split(q0[0]), fp_split(q0[1]), fp_split(q0[2])};

    constexpr int NC = ND == 4 ? 5 : NCLS;  // pair classes
    fpair pU[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}}, pD[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    fpair pN = {0.0f, 0.0f};
    int npairs[NCLS_MAX] = {0, 0, 0, 0, 0};  // near pairs by class
    int nunreg[MAXD] = {0, 0, 0, 0};         // near pairs by number of deltas beyond the cutoff
    scan_near<NC>(A.sd, T, P, sq, lane, [&](int cls, int jj, bool valid) {
        if (valid) process<PREC, SL, DL, ND>(A, T, P, ncp, q0p, tab, jj, cls, pU, pN, pD, npairs, nunreg);
    });
    double accU[3], accD[3];
    for (int i = 0; i < 3; ++i) {
        accU[i] = warp_sum(fp_to_double(pU[i]));
        accD[i] = warp_sum(fp_to_double(pD[i]));
    }
    const double accN = warp_sum(fp_to_double(pN));
    if (A.counters) {
        // counters: [2 + c] class c < 4, [6 + u] u < 3 deltas beyond the cutoff, [10] class 4, [11] u = 3
        int np[9] = {npairs[0], npairs[1], npairs[2], npairs[3], nunreg[0], nunreg[1], nunreg[2], npairs[4], nunreg[3]};
#pragma unroll
        for (int cc = 0; cc < 9; ++cc)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) np[cc] += __shfl_xor_sync(FULL, np[cc], o);
        if (lane == 0) {
            atomicAdd(A.counters + 0, 1ull);
            atomicAdd(A.counters + 1, (unsigned long long)(np[0] + np[1] + np[2] + np[3] + np[7]));
#pragma unroll
            for (int cc = 0; cc < 7; ++cc) atomicAdd(A.counters + 2 + cc, (unsigned long long)np[cc]);
            if (ND == 4) {
                atomicAdd(A.counters + 10, (unsigned long long)np[7]);
                atomicAdd(A.counters + 11, (unsigned long long)np[8]);
            }
        }
    }
    if (SL && lane < 3) {
        const double a = lane == 0 ? accU[0] : (lane == 1 ? accU[1] : accU[2]);
        A.u[3 * m + lane] = fs + a * INV8PI;
    }
    if (DL && lane >= 3 && lane < 6) {
        const int i = lane - 3;
        const double ad = i == 0 ? accD[0] : (i == 1 ? accD[1] : accD[2]);
        const double ni = i == 0 ? T.n0[0] : (i == 1 ? T.n0[1] : T.n0[2]);
        const double qi = i == 0 ? q0[0] : (i == 1 ? q0[1] : q0[2]);
        const double chi = bm < 0.0 ? 1.0 : (bm > 0.0 ? 0.0 : 0.5);
        A.v[3 * m + i] = fs + (-6.0 * INV8PI) * fma(accN, ni, -ad) + chi * qi;
    }
}

template <int PREC, bool SL, bool DL, int ND>
__global__ void __launch_bounds__(WPB * 32, NEAR_MIN_BLOCKS) k_near(EvalArgs A, ScanParams P, ScanParams Ps,
                                                                   const double *__restrict__ tab) {
    __shared__ int sq[WPB][ND == 4 ? 5 : NCLS][64];
    __shared__ Geom sG[WPB];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    // one target per warp; a capped grid strides over the targets
    for (int64_t m = (int64_t)blockIdx.x * WPB + wib; m < A.M; m += (int64_t)gridDim.x * WPB)
        near_target<PREC, SL, DL, ND>(A, P, tab, m, lane, sq[wib], sG[wib], Ps);
}

template <int PREC>
cudaError_t near_dispatch(const EvalArgs &a, ScanParams P, ScanParams Ps, const double *tab, int ctas_per_sm,
                          int nsm) {
    int64_t grid = (a.M + WPB - 1) / WPB;
    if (ctas_per_sm > 0) grid = std::min<int64_t>(grid, (int64_t)ctas_per_sm * nsm);
    const unsigned g = (unsigned)grid;
    const bool sl = a.layers & ERS_LAYER_SL, dl = a.layers & ERS_LAYER_DL;
    if (a.ndelta == 1 || a.ndelta == 2) {  // learned closure: both layers
        if (!(sl && dl)) return cudaErrorInvalidValue;
        if (a.ndelta == 1) k_near<PREC, true, true, 1><<<g, WPB * 32, 0, a.stream>>>(a, P, Ps, tab);
        else k_near<PREC, true, true, 2><<<g, WPB * 32, 0, a.stream>>>(a, P, Ps, tab);
    } else if (a.ndelta == 4) {  // the O(delta^7) variant
        if (sl && dl) k_near<PREC, true, true, 4><<<g, WPB * 32, 0, a.stream>>>(a, P, Ps, tab);
        else if (sl) k_near<PREC, true, false, 4><<<g, WPB * 32, 0, a.stream>>>(a, P, Ps, tab);
        else k_near<PREC, false, true, 4><<<g, WPB * 32, 0, a.stream>>>(a, P, Ps, tab);
    } else if (sl && dl) k_near<PREC, true, true, 3><<<g, WPB * 32, 0, a.stream>>>(a, P, Ps, tab);
    else if (sl) k_near<PREC, true, false, 3><<<g, WPB * 32, 0, a.stream>>>(a, P, Ps, tab);
    else k_near<PREC, false, true, 3><<<g, WPB * 32, 0, a.stream>>>(a, P, Ps, tab);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_near(const EvalArgs &a, const double *tab, int ctas_per_sm, int nsm) {
    if (a.M == 0) return cudaSuccess;
    const ScanParams P = scan_params(a.s, a.Rc, a.rho, a.cutoff_t, a.ndelta == 4 ? 4 : 3);
    ScanParams Ps = P;
    if (a.sharp) {  // on-surface targets: one delta#, every near pair on the table
        const double rs[3] = {a.rho_sharp, a.rho_sharp, a.rho_sharp};
        Ps = scan_params(a.s, a.Rc_sharp, rs, a.cutoff_t);
        for (int k = 0; k < MAXD; ++k) Ps.th[k] = HUGE_VALF;
    }
    if (a.precision == ERS_PREC_FP64) return near_dispatch<ERS_PREC_FP64>(a, P, Ps, tab, ctas_per_sm, nsm);
    return near_dispatch<ERS_PREC_MIXED>(a, P, Ps, tab, ctas_per_sm, nsm);
}

}  // namespace ers
