// Batched evaluation: several problems (surface, targets, NR right-hand-side densities) in one
// persistent launch, captured in a CUDA graph.
//
// A work item is (problem, block of 128 targets).  One CTA runs an item to completion:
//   1. far field with FP32 operands (the pair term of Eqs. (Stokeslet), (Stresslet) on the
//      subtracted densities of Eqs. (Stokes_SL1), (Stokes_DL1)), r > Rc only; the geometry of a
//      pair (d, 1/r) is computed once and shared by the NR densities; FP32 sums over 512
//      sources are added into FP64 sums kept in the output arrays u, v themselves;
//   2. near field and extrapolation (Secs. 2, 3.2, 3.3), one warp per target: pair geometry in
//      FP64, kernel factors and contractions in float pairs (as in k_near), with the
//      alpha-weighted kernel factors of a pair shared by the NR densities;
//   3. u = far + near (+ chi q(x0) for the double layer), written for every density.
// Items carry no dependency on each other, so CTAs take them from an atomic counter in any
// order (largest first) and never wait.
#include <algorithm>
#include <vector>

#include "near_common.cuh"

namespace ers {

namespace {

using namespace nearc;
constexpr int BT = 128;     // threads per CTA = targets per item
constexpr int BW = BT / 32; // warps per CTA
constexpr int BTS = 64;     // sources per shared-memory stage
constexpr int BFLUSH = 8;   // stages per FP32 partial sum (512 sources)

// FP32 source record of the batched far field, float4 units (see k_density_multi):
// x - c_tile (3), w n (3), then (w f, q) per density, padded to a multiple of 4 floats.
template <int NR>
constexpr int S4 = (6 + 6 * NR + 3) / 4;

template <int NR>
struct BatchSmem {
    union {
        float4 stage[BTS][S4<NR>];   // far phase: one stage of source records
        float2 near[BW][NR][7][32];  // near phase: per-lane float-pair accumulators (SL without c_r wn; N; D)
    } u;
    double tq[BW][NR][4];  // near phase: c_r = f0_r . n0 and q0_r of each warp's target
    fpair tqp[BW][NR][4];  // the same as float pairs
    Geom g[BW];            // near phase: each warp's target constants (indexed at run time)
    int sq[BW][NCLS][64];
    float4 cen;
    int item;
};

// Offset (floats) of value k (w f 0..2, q 0..2) of density r in the FP32 far-field record:
// after x - c_tile and w n, densities come in pairs with their values interleaved, so that one
// 64-bit word holds the same value of two densities (packed f32x2 operands); NR = 1 is plain.
__host__ __device__ constexpr int rec_off(int nr, int r, int k) {
    return nr == 1 ? 6 + k : 6 + 12 * (r / 2) + 2 * k + (r % 2);
}

template <int NR>
__device__ void far_phase(const BatchProblemDev &P, int tb, int layers, BatchSmem<NR> &S) {
    constexpr int NP = NR / 2 > 0 ? NR / 2 : 1;  // density pairs (NR = 1: one half-used pair)
    const int t = threadIdx.x;
    const int64_t m = (int64_t)tb * BT + t;
    const bool valid = m < P.M;
    const bool sl = layers & ERS_LAYER_SL, dl = layers & ERS_LAYER_DL;
    float yh[3] = {0, 0, 0}, yl[3] = {0, 0, 0}, c[2 * NP], q0[2 * NP][3];
    float rc2 = __int_as_float(0x7f800000);  // +inf: nothing is far (invalid target)
    for (int r = 0; r < 2 * NP; ++r) {
        c[r] = 0.0f;
        q0[r][0] = q0[r][1] = q0[r][2] = 0.0f;
    }
    if (valid) {
        for (int i = 0; i < 3; ++i) {
            const double yy = P.y[3 * m + i];
            yh[i] = __double2float_rn(yy);
            yl[i] = __double2float_rn(yy - (double)yh[i]);
        }
        const bool near = fabs(P.b[m]) <= P.Rc;
        rc2 = near ? P.sp.rc2f : -1.0f;
        if (near) {
            const double n0x = P.n0[3 * m], n0y = P.n0[3 * m + 1], n0z = P.n0[3 * m + 2];
            for (int r = 0; r < NR; ++r) {
                const double *f0 = P.f0 + ((int64_t)r * P.M + m) * 3;
                const double *qq = P.q0 + ((int64_t)r * P.M + m) * 3;
                if (sl) c[r] = __double2float_rn(f0[0] * n0x + f0[1] * n0y + f0[2] * n0z);
                if (dl)
                    for (int i = 0; i < 3; ++i) q0[r][i] = __double2float_rn(qq[i]);
            }
        }
    }
    f2 nc[NP], q0p[NP][3], acc[NP][6];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        nc[p] = pk(-c[2 * p], -c[2 * p + 1]);
        for (int i = 0; i < 3; ++i) q0p[p][i] = pk(q0[2 * p][i], q0[2 * p + 1][i]);
        for (int i = 0; i < 6; ++i) acc[p][i] = 0ull;
    }

    const int64_t N = P.sd.N;
    const float4 *__restrict__ src4 = reinterpret_cast<const float4 *>(P.dens32);
    int since = 0;
    bool first = true;
    for (int64_t base = 0; base < N; base += BTS) {
        const int ns = (int)min((int64_t)BTS, N - base);
        __syncthreads();
        const float4 *g = src4 + base * S4<NR>;
        float4 *st = &S.u.stage[0][0];
        for (int k = t; k < ns * S4<NR>; k += BT) st[k] = g[k];
        if (t == 0) S.cen = reinterpret_cast<const float4 *>(P.sd.tilec)[base / TS32];
        __syncthreads();
        const float4 cen = S.cen;
        const float yc0 = tile_rel(yh[0], cen.x, yl[0]), yc1 = tile_rel(yh[1], cen.y, yl[1]),
                    yc2 = tile_rel(yh[2], cen.z, yl[2]);
        for (int j = 0; j < ns; ++j) {
            const float *sp = reinterpret_cast<const float *>(&S.u.stage[j][0]);
            const float4 a0 = S.u.stage[j][0], a1 = S.u.stage[j][1];  // x - c, w n, then densities
            float dx, dy, dz;
            const float r2 = dist2_fp32(yc0, yc1, yc2, a0.x, a0.y, a0.z, &dx, &dy, &dz);
            const float ri = (r2 > rc2) ? rsqrt_ftz(r2) : 0.0f;  // far pairs have r2 >= Rc^2
            const float ri2 = ri * ri;
            const float dwn = fmaf(dz, a1.y, fmaf(dy, a1.x, dx * a0.w));
            const float w5 = dwn * ((ri2 * ri2) * ri);  // (d.m)/r^5
            const f2 Dx = pk(dx, dx), Dy = pk(dy, dy), Dz = pk(dz, dz), RI = pk(ri, ri), RI2 = pk(ri2, ri2);
            const f2 W0 = pk(a0.w, a0.w), W1 = pk(a1.x, a1.x), W2 = pk(a1.y, a1.y), W5 = pk(w5, w5);
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                f2 v[6];  // w f 0..2, q 0..2 of densities 2p, 2p+1
                if (NR == 1) {
#pragma unroll
                    for (int k = 0; k < 6; ++k) v[k] = pk(sp[6 + k], 0.0f);
                } else {
                    const f2 *pp = reinterpret_cast<const f2 *>(sp + 6 + 12 * p);
#pragma unroll
                    for (int k = 0; k < 6; ++k) v[k] = pp[k];
                }
                if (sl) {
                    const f2 g0 = fma2(nc[p], W0, v[0]);
                    const f2 g1 = fma2(nc[p], W1, v[1]);
                    const f2 g2 = fma2(nc[p], W2, v[2]);
                    const f2 sv = mul2(fma2(Dz, g2, fma2(Dy, g1, mul2(Dx, g0))), RI2);
                    acc[p][0] = fma2(fma2(Dx, sv, g0), RI, acc[p][0]);
                    acc[p][1] = fma2(fma2(Dy, sv, g1), RI, acc[p][1]);
                    acc[p][2] = fma2(fma2(Dz, sv, g2), RI, acc[p][2]);
                }
                if (dl) {
                    const f2 Q0 = sub2(v[3], q0p[p][0]), Q1 = sub2(v[4], q0p[p][1]), Q2 = sub2(v[5], q0p[p][2]);
                    const f2 sv = mul2(fma2(Dz, Q2, fma2(Dy, Q1, mul2(Dx, Q0))), W5);
                    acc[p][3] = fma2(Dx, sv, acc[p][3]);
                    acc[p][4] = fma2(Dy, sv, acc[p][4]);
                    acc[p][5] = fma2(Dz, sv, acc[p][5]);
                }
            }
        }
        if (++since == BFLUSH || base + BTS >= N) {
            // FP64 sums (unscaled) in the outputs of this thread's own target
            since = 0;
            if (valid) {
#pragma unroll
                for (int p = 0; p < NP; ++p)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int r = 2 * p + h;
                        if (r >= NR) break;
                        double *ou = P.u + ((int64_t)r * P.M + m) * 3, *ov = P.v + ((int64_t)r * P.M + m) * 3;
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            float s0, s1, d0, d1;
                            upk(acc[p][i], s0, s1);
                            upk(acc[p][3 + i], d0, d1);
                            if (sl) ou[i] = (first ? 0.0 : ou[i]) + (double)(h ? s1 : s0);
                            if (dl) ov[i] = (first ? 0.0 : ov[i]) + (double)(h ? d1 : d0);
                        }
                    }
            }
            first = false;
#pragma unroll
            for (int p = 0; p < NP; ++p)
#pragma unroll
                for (int i = 0; i < 6; ++i) acc[p][i] = 0ull;
        }
    }
    if (valid && N == 0) {
        for (int r = 0; r < NR; ++r)
            for (int i = 0; i < 3; ++i) {
                if (sl) P.u[((int64_t)r * P.M + m) * 3 + i] = 0.0;
                if (dl) P.v[((int64_t)r * P.M + m) * 3 + i] = 0.0;
            }
    }
    __syncthreads();  // the far sums in u, v are visible to the whole CTA
}

// The near-field terms of one pair (class cls, a run-time value) for the NR densities, in float
// pairs as in k_near: d, w n, the kernel factors and the double-layer pair factors are shared by
// the densities; per density the single-layer K1 w f + K3 (d.w f) d (the c_r w n part,
// K1 w n + K3 (d.w n) d, is summed once per pair into accB and subtracted c_r times at the end)
// and the double-layer contraction (dl_accumulate_pair), into the lane's float-pair
// accumulators in shared memory.
template <int NR>
__device__ __forceinline__ void near_pair(const BatchProblemDev &P, const Geom &T, const double *__restrict__ tab,
                                          int64_t j, int cls, int lane, int warp, int layers, BatchSmem<NR> &S,
                                          fpair accB[3]) {
    const float4 *rp = reinterpret_cast<const float4 *>(P.sd.recp + j * NREC);
    const float4 a0 = __ldg(rp + 0), a1 = __ldg(rp + 1), a3 = __ldg(rp + 3), a4 = __ldg(rp + 4);
    const double dx = __dsub_rn(T.y[0], __hiloint2double(__float_as_int(a0.y), __float_as_int(a0.x)));
    const double dy = __dsub_rn(T.y[1], __hiloint2double(__float_as_int(a0.w), __float_as_int(a0.z)));
    const double dz = __dsub_rn(T.y[2], __hiloint2double(__float_as_int(a1.y), __float_as_int(a1.x)));
    const double r2 = dist2_fp64(dx, dy, dz);
    if (!is_near<ERS_PREC_MIXED>(P.sd, T, j, r2, P.Rc, P.sp.rc2f)) return;
    const fpair wn[3] = {{a3.x, a3.y}, {a3.z, a3.w}, {a4.x, a4.y}};
    const fpair r2p = fp_split(r2);
    fpair K[3];
    kernel_factors_pair<3>(T, P.sp, tab, r2, r2p, cls, K);
    const fpair d[3] = {fp_split(dx), fp_split(dy), fp_split(dz)};
    const fpair W = fp_dot3(d[0], d[1], d[2], wn[0], wn[1], wn[2]);
    const bool sl = layers & ERS_LAYER_SL, dl = layers & ERS_LAYER_DL;
    if (sl) {
        const fpair tb = fp_mul(K[1], W);
#pragma unroll
        for (int i = 0; i < 3; ++i) accB[i] = fp_acc2(accB[i], tb, d[i], K[0], wn[i]);
    }
    // double-layer pair factors: L = r^2 K5 - K3, Z = 2 b nm - W, L nm, K5 W (nm = n0.w n)
    fpair nm = {0.0f, 0.0f}, Z = nm, Lnm = nm, K5W = nm, L = nm;
    if (dl) {
        nm = fp_dot3(T.n0p[0], T.n0p[1], T.n0p[2], wn[0], wn[1], wn[2]);
        L = fp_fma(r2p, K[2], fp_neg(K[1]));
        Z = fp_fma(T.b2p, nm, fp_neg(W));
        Lnm = fp_mul(L, nm);
        K5W = fp_mul(K[2], W);
    }
    const float4 *dj = reinterpret_cast<const float4 *>(P.densp + j * (6 * NR));
#pragma unroll 2
    for (int r = 0; r < NR; ++r) {
        float2(*a)[32] = S.u.near[warp][r];
        // (w f0, w f1), (w f2, q0), (q1, q2), each a float pair
        const float4 d0 = __ldg(dj + 3 * r), d1 = __ldg(dj + 3 * r + 1), d2 = __ldg(dj + 3 * r + 2);
        if (sl) {
            const fpair wf[3] = {{d0.x, d0.y}, {d0.z, d0.w}, {d1.x, d1.y}};
            const fpair t = fp_mul(K[1], fp_dot3(d[0], d[1], d[2], wf[0], wf[1], wf[2]));
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const fpair s = fp_acc2({a[i][lane].x, a[i][lane].y}, t, d[i], K[0], wf[i]);
                a[i][lane] = make_float2(s.h, s.l);
            }
        }
        if (dl) {
            const fpair Q0 = fp_add({d1.z, d1.w}, fp_neg(S.tqp[warp][r][1]));
            const fpair Q1 = fp_add({d2.x, d2.y}, fp_neg(S.tqp[warp][r][2]));
            const fpair Q2 = fp_add({d2.z, d2.w}, fp_neg(S.tqp[warp][r][3]));
            const fpair nQ = fp_dot3(T.n0p[0], T.n0p[1], T.n0p[2], Q0, Q1, Q2);
            const fpair U = fp_dot3(d[0], d[1], d[2], Q0, Q1, Q2);
            const fpair n = fp_add({a[3][lane].x, a[3][lane].y}, fp_mul(L, fp_fma(nQ, Z, fp_neg(fp_mul(nm, U)))));
            a[3][lane] = make_float2(n.h, n.l);
            const fpair C = fp_fma(Lnm, nQ, fp_neg(fp_mul(K5W, U)));
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const fpair s = fp_fma(C, d[i], {a[4 + i][lane].x, a[4 + i][lane].y});
                a[4 + i][lane] = make_float2(s.h, s.l);
            }
        }
    }
}

template <int NR>
__device__ void near_phase(const BatchProblemDev &P, int tb, int layers, const double *__restrict__ tab,
                           const double rho[3], BatchSmem<NR> &S) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool sl = layers & ERS_LAYER_SL, dl = layers & ERS_LAYER_DL;
    for (int tt = warp; tt < BT; tt += BW) {
        const int64_t m = (int64_t)tb * BT + tt;
        if (m >= P.M) break;
        const double bm = P.b[m];
        const bool near = fabs(bm) <= P.Rc;
        if (near) {
            {
                Geom Tl;
                load_geom(lane, P.y, P.x0, P.n0, bm, m, rho, P.sp.h, Tl);
                set_cutoff(Tl, P.sp);
                __syncwarp();  // the previous target's reads of S.g are done
                if (lane == 0) S.g[warp] = Tl;
                __syncwarp();
            }
            const Geom &T = S.g[warp];
            if (lane < 4 * NR) {  // lane = 4 r + k: k = 0 c_r, k = 1..3 q0_r
                const int r = lane >> 2, k = lane & 3;
                double val = 0.0;
                if (k == 0 && sl) {
                    const double *f0 = P.f0 + ((int64_t)r * P.M + m) * 3;
                    val = fma(f0[2], T.n0[2], fma(f0[1], T.n0[1], f0[0] * T.n0[0]));
                }
                if (k > 0 && dl) val = P.q0[((int64_t)r * P.M + m) * 3 + k - 1];
                S.tq[warp][r][k] = val;
                S.tqp[warp][r][k] = fp_split(val);
            }
            for (int r = 0; r < NR; ++r)
                for (int i = 0; i < 7; ++i) S.u.near[warp][r][i][lane] = make_float2(0.0f, 0.0f);
            __syncwarp();
            fpair pB[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
            scan_near(P.sd, T, P.sp, S.sq[warp], lane, [&](int cls, int jj, bool valid) {
                if (valid) near_pair<NR>(P, T, tab, jj, cls, lane, warp, layers, S, pB);
            });
            double accB[3];
            for (int i = 0; i < 3; ++i) accB[i] = warp_sum(fp_to_double(pB[i]));
            const double chi = bm < 0.0 ? 1.0 : (bm > 0.0 ? 0.0 : 0.5);
            for (int r = 0; r < NR; ++r) {
                double tot[7];
                for (int i = 0; i < 7; ++i) {
                    const float2 v = S.u.near[warp][r][i][lane];
                    tot[i] = warp_sum(fp_to_double({v.x, v.y}));
                }
                if (sl && lane < 3) {
                    const double a = lane == 0 ? tot[0] : (lane == 1 ? tot[1] : tot[2]);
                    const double bb = lane == 0 ? accB[0] : (lane == 1 ? accB[1] : accB[2]);
                    double *o = P.u + ((int64_t)r * P.M + m) * 3 + lane;
                    *o = INV8PI * (*o + fma(-S.tq[warp][r][0], bb, a));
                }
                if (dl && lane >= 3 && lane < 6) {
                    const int i = lane - 3;
                    const double ad = i == 0 ? tot[4] : (i == 1 ? tot[5] : tot[6]);
                    const double ni = i == 0 ? T.n0[0] : (i == 1 ? T.n0[1] : T.n0[2]);
                    double *o = P.v + ((int64_t)r * P.M + m) * 3 + i;
                    *o = (-6.0 * INV8PI) * (*o + fma(tot[3], ni, -ad)) + chi * S.tq[warp][r][1 + i];
                }
            }
            __syncwarp();
        } else {
            for (int r = 0; r < NR; ++r) {
                if (sl && lane < 3) P.u[((int64_t)r * P.M + m) * 3 + lane] *= INV8PI;
                if (dl && lane >= 3 && lane < 6) P.v[((int64_t)r * P.M + m) * 3 + lane - 3] *= -6.0 * INV8PI;
            }
        }
    }
}

template <int NR>
__global__ void __launch_bounds__(BT, 3) k_batch(const BatchProblemDev *__restrict__ probs,
                                                 const BatchItem *__restrict__ items, int nitems,
                                                 unsigned *__restrict__ counter, double rho0, double rho1,
                                                 double rho2, int layers, const double *__restrict__ tab) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BatchSmem<NR> &S = *reinterpret_cast<BatchSmem<NR> *>(smem_raw);
    const double rho[3] = {rho0, rho1, rho2};
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) S.item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int it = S.item;
        if (it >= nitems) break;
        const BatchItem item = items[it];
        const BatchProblemDev &P = probs[item.prob];
        far_phase<NR>(P, item.tb, layers, S);
        near_phase<NR>(P, item.tb, layers, tab, rho, S);
    }
}

// Densities of nr right-hand sides in cell-sorted order: float pairs [N][nr][6] (w f, q; hi = the
// value rounded, lo = the rest rounded) for the near field, and the FP32 far-field record [N][S] floats (S = 6 + 6 nr rounded up to a multiple of 4):
// x - c_tile and w n from the surface's FP32 record, then (w f, q) per density in the order of
// rec_off (pairs of densities interleaved), zero padding.
__global__ void k_density_multi(const int *__restrict__ perm, const double *__restrict__ w,
                                const float *__restrict__ rec32, const double *__restrict__ f,
                                const double *__restrict__ q, int64_t N, int nr, float2 *__restrict__ dp,
                                float *__restrict__ d32) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const int64_t i = perm[j];
    const double wi = w[i];
    const int S = (6 + 6 * nr + 3) / 4 * 4;
    float *o32 = d32 + j * S;
    for (int k = 0; k < 3; ++k) {
        o32[k] = rec32[j * REC + R_X + k];
        o32[3 + k] = rec32[j * REC + R_WN + k];
    }
    for (int r = 0; r < nr; ++r) {
        for (int k = 0; k < 3; ++k) {
            const double fv = f ? wi * f[((int64_t)r * N + i) * 3 + k] : 0.0;
            const double qv = q ? q[((int64_t)r * N + i) * 3 + k] : 0.0;
            const int64_t o = (j * nr + r) * 6;
            const float fh = __double2float_rn(fv), qh = __double2float_rn(qv);
            dp[o + k] = make_float2(fh, __double2float_rn(fv - (double)fh));
            dp[o + 3 + k] = make_float2(qh, __double2float_rn(qv - (double)qh));
            o32[rec_off(nr, r, k)] = __double2float_rn(fv);
            o32[rec_off(nr, r, 3 + k)] = __double2float_rn(qv);
        }
    }
    for (int k = 6 + 6 * nr; k < S; ++k) o32[k] = 0.0f;
}

template <int NR>
cudaError_t batch_launch_t(const BatchProblemDev *probs, const BatchItem *items, int nitems, unsigned *counter,
                           const double rho[3], int layers, const double *tab, int grid, cudaStream_t st) {
    const size_t smem = sizeof(BatchSmem<NR>);
    k_batch<NR><<<grid, BT, smem, st>>>(probs, items, nitems, counter, rho[0], rho[1], rho[2], layers, tab);
    return cudaGetLastError();
}

template <int NR>
int batch_grid_t(int nsm) {
    int per = 0;
    const size_t smem = sizeof(BatchSmem<NR>);
    if (cudaFuncSetAttribute(k_batch<NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return nsm;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch<NR>, BT, smem) != cudaSuccess || per < 1) per = 1;
    return nsm * per;
}

}  // namespace

cudaError_t launch_density_multi(const int *perm, const double *w, const float *rec32, const double *f,
                                 const double *q, int64_t N, int nr, float2 *dp, float *d32, cudaStream_t st) {
    const int bs = 256;
    k_density_multi<<<(unsigned)((N + bs - 1) / bs), bs, 0, st>>>(perm, w, rec32, f, q, N, nr, dp, d32);
    return cudaGetLastError();
}

// Sets the kernel's shared-memory attribute (call before any stream capture) and returns the
// persistent grid size: SMs x resident CTAs per SM.
int batch_grid(int nr, int nsm) {
    switch (nr) {
        case 1: return batch_grid_t<1>(nsm);
        case 2: return batch_grid_t<2>(nsm);
        case 4: return batch_grid_t<4>(nsm);
        default: return batch_grid_t<8>(nsm);
    }
}

cudaError_t launch_batch(int nr, const BatchProblemDev *probs, const BatchItem *items, int nitems, unsigned *counter,
                         const double rho[3], int layers, const double *tab, int grid, cudaStream_t st) {
    switch (nr) {
        case 1: return batch_launch_t<1>(probs, items, nitems, counter, rho, layers, tab, grid, st);
        case 2: return batch_launch_t<2>(probs, items, nitems, counter, rho, layers, tab, grid, st);
        case 4: return batch_launch_t<4>(probs, items, nitems, counter, rho, layers, tab, grid, st);
        case 8: return batch_launch_t<8>(probs, items, nitems, counter, rho, layers, tab, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ers
