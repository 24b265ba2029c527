// Batched evaluation: several problems (surface, targets, NR right-hand-side densities) in one
// persistent launch, captured in a CUDA graph.
//
// A work item is (problem, block of 128 targets).  One CTA runs an item to completion:
//   1. far field with FP32 operands (the pair term of Eqs. (Stokeslet), (Stresslet) on the
//      subtracted densities of Eqs. (Stokes_SL1), (Stokes_DL1)), r > Rc only; the geometry of a
//      pair (d, 1/r) is computed once and shared by the NR densities; FP32 sums over 512
//      sources are added into FP64 sums kept in the output arrays u, v themselves;
//   2. near field and extrapolation (Secs. 2, 3.2, 3.3) in FP64, one warp per target, with the
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
        double near[BW][NR][7][32];  // near phase: per-lane accumulators (SL without c_r wn; N; D)
    } u;
    double tq[BW][NR][4];  // near phase: c_r = f0_r . n0 and q0_r of each warp's target
    int sq[BW][NCLS][64];
    float4 cen;
    int item;
};

template <int NR>
__device__ void far_phase(const BatchProblemDev &P, int tb, int layers, BatchSmem<NR> &S) {
    const int t = threadIdx.x;
    const int64_t m = (int64_t)tb * BT + t;
    const bool valid = m < P.M;
    const bool sl = layers & ERS_LAYER_SL, dl = layers & ERS_LAYER_DL;
    float yh[3] = {0, 0, 0}, yl[3] = {0, 0, 0}, c[NR], q0[NR][3];
    float rc2 = __int_as_float(0x7f800000);  // +inf: nothing is far (invalid target)
    for (int r = 0; r < NR; ++r) {
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
    float acc[NR][6];
    for (int r = 0; r < NR; ++r)
        for (int i = 0; i < 6; ++i) acc[r][i] = 0.0f;

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
            float sp[4 * S4<NR>];
#pragma unroll
            for (int k = 0; k < S4<NR>; ++k) {
                const float4 v4 = S.u.stage[j][k];
                sp[4 * k] = v4.x;
                sp[4 * k + 1] = v4.y;
                sp[4 * k + 2] = v4.z;
                sp[4 * k + 3] = v4.w;
            }
            float dx, dy, dz;
            const float r2 = dist2_fp32(yc0, yc1, yc2, sp[0], sp[1], sp[2], &dx, &dy, &dz);
            float ri = rsqrt_ftz(r2);  // far pairs have r2 >= Rc^2; the others are masked
            ri = (r2 > rc2) ? ri : 0.0f;
            const float ri2 = ri * ri;
            const float dwn = fmaf(dz, sp[5], fmaf(dy, sp[4], dx * sp[3]));
            const float w5 = dwn * ((ri2 * ri2) * ri);  // (d.m)/r^5
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const float *dr = sp + 6 + 6 * r;
                if (sl) {
                    const float g0 = fmaf(-c[r], sp[3], dr[0]);
                    const float g1 = fmaf(-c[r], sp[4], dr[1]);
                    const float g2 = fmaf(-c[r], sp[5], dr[2]);
                    const float s = fmaf(dz, g2, fmaf(dy, g1, dx * g0)) * ri2;
                    acc[r][0] = fmaf(fmaf(dx, s, g0), ri, acc[r][0]);
                    acc[r][1] = fmaf(fmaf(dy, s, g1), ri, acc[r][1]);
                    acc[r][2] = fmaf(fmaf(dz, s, g2), ri, acc[r][2]);
                }
                if (dl) {
                    const float Q0 = dr[3] - q0[r][0], Q1 = dr[4] - q0[r][1], Q2 = dr[5] - q0[r][2];
                    const float s = fmaf(dz, Q2, fmaf(dy, Q1, dx * Q0)) * w5;
                    acc[r][3] = fmaf(dx, s, acc[r][3]);
                    acc[r][4] = fmaf(dy, s, acc[r][4]);
                    acc[r][5] = fmaf(dz, s, acc[r][5]);
                }
            }
        }
        if (++since == BFLUSH || base + BTS >= N) {
            // FP64 sums (unscaled) in the outputs of this thread's own target
            since = 0;
            if (valid) {
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    double *ou = P.u + ((int64_t)r * P.M + m) * 3, *ov = P.v + ((int64_t)r * P.M + m) * 3;
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        if (sl) ou[i] = (first ? 0.0 : ou[i]) + (double)acc[r][i];
                        if (dl) ov[i] = (first ? 0.0 : ov[i]) + (double)acc[r][3 + i];
                    }
                }
            }
            first = false;
#pragma unroll
            for (int r = 0; r < NR; ++r)
#pragma unroll
                for (int i = 0; i < 6; ++i) acc[r][i] = 0.0f;
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

// One near pair for the NR densities: the kernel factors, the single-layer terms without the
// c_r w n part (K1 w f + K3 (d.w f) d per density, and K1 w n + K3 (d.w n) d once, into accB,
// subtracted c_r times at the end) and the double-layer terms.
template <int CLS, int NR>
__device__ __forceinline__ void near_pair(const BatchProblemDev &P, const Geom &T, const double *__restrict__ tab,
                                          int64_t j, int lane, int warp, int layers, BatchSmem<NR> &S,
                                          double accB[3]) {
    const double *rec = P.sd.rec + j * REC;
    const double xs[3] = {__ldg(rec + R_X), __ldg(rec + R_X + 1), __ldg(rec + R_X + 2)};
    const double wn[3] = {__ldg(rec + R_WN), __ldg(rec + R_WN + 1), __ldg(rec + R_WN + 2)};
    const double dx = __dsub_rn(T.y[0], xs[0]);
    const double dy = __dsub_rn(T.y[1], xs[1]);
    const double dz = __dsub_rn(T.y[2], xs[2]);
    const double r2 = dist2_fp64(dx, dy, dz);
    if (!is_near<ERS_PREC_MIXED>(P.sd, T, j, r2, P.Rc, P.sp.rc2f)) return;
    double K1, K3, K5;
    kernel_factors<CLS>(T, P.sp, tab, r2, K1, K3, K5);
    const double nm = fma(T.n0[2], wn[2], fma(T.n0[1], wn[1], T.n0[0] * wn[0]));
    const double W = fma(dz, wn[2], fma(dy, wn[1], dx * wn[0]));
    const DLPair D = dl_pair(T, r2, K3, K5, nm, W);  // shared by the NR densities
    const bool sl = layers & ERS_LAYER_SL, dl = layers & ERS_LAYER_DL;
    if (sl) {
        const double tb = K3 * W;
        accB[0] = fma(K1, wn[0], fma(tb, dx, accB[0]));
        accB[1] = fma(K1, wn[1], fma(tb, dy, accB[1]));
        accB[2] = fma(K1, wn[2], fma(tb, dz, accB[2]));
    }
    const double2 *dj = reinterpret_cast<const double2 *>(P.dens64 + j * (6 * NR));
#pragma unroll 2
    for (int r = 0; r < NR; ++r) {
        double(*a)[32] = S.u.near[warp][r];
        const double2 d0 = __ldg(dj + 3 * r), d1 = __ldg(dj + 3 * r + 1), d2 = __ldg(dj + 3 * r + 2);
        if (sl) {  // K1 w f + K3 (d.w f) d
            const double t = K3 * fma(dz, d1.x, fma(dy, d0.y, dx * d0.x));
            a[0][lane] = fma(K1, d0.x, fma(t, dx, a[0][lane]));
            a[1][lane] = fma(K1, d0.y, fma(t, dy, a[1][lane]));
            a[2][lane] = fma(K1, d1.x, fma(t, dz, a[2][lane]));
        }
        if (dl) {
            const double qs[3] = {d1.y, d2.x, d2.y};
            const double q0[3] = {S.tq[warp][r][1], S.tq[warp][r][2], S.tq[warp][r][3]};
            double accN = a[3][lane], accD[3] = {a[4][lane], a[5][lane], a[6][lane]};
            dl_accumulate(D, T, dx, dy, dz, nm, qs, q0, accN, accD);
            a[3][lane] = accN;
            a[4][lane] = accD[0];
            a[5][lane] = accD[1];
            a[6][lane] = accD[2];
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
            Geom T;
            load_geom(lane, P.y, P.x0, P.n0, bm, m, rho, P.sp.h, T);
            set_cutoff(T, P.sp);
            if (lane < 4 * NR) {  // lane = 4 r + k: k = 0 c_r, k = 1..3 q0_r
                const int r = lane >> 2, k = lane & 3;
                double val = 0.0;
                if (k == 0 && sl) {
                    const double *f0 = P.f0 + ((int64_t)r * P.M + m) * 3;
                    val = fma(f0[2], T.n0[2], fma(f0[1], T.n0[1], f0[0] * T.n0[0]));
                }
                if (k > 0 && dl) val = P.q0[((int64_t)r * P.M + m) * 3 + k - 1];
                S.tq[warp][r][k] = val;
            }
            for (int r = 0; r < NR; ++r)
                for (int i = 0; i < 7; ++i) S.u.near[warp][r][i][lane] = 0.0;
            __syncwarp();
            double accB[3] = {0.0, 0.0, 0.0};
            scan_near(P.sd, T, P.sp, S.sq[warp], lane, [&](int cls, int jj, bool valid) {
                if (!valid) return;
                if (cls == 0) near_pair<0, NR>(P, T, tab, jj, lane, warp, layers, S, accB);
                else if (cls == 1) near_pair<1, NR>(P, T, tab, jj, lane, warp, layers, S, accB);
                else if (cls == 2) near_pair<2, NR>(P, T, tab, jj, lane, warp, layers, S, accB);
                else near_pair<3, NR>(P, T, tab, jj, lane, warp, layers, S, accB);
            });
            for (int i = 0; i < 3; ++i) accB[i] = warp_sum(accB[i]);
            const double chi = bm < 0.0 ? 1.0 : (bm > 0.0 ? 0.0 : 0.5);
            for (int r = 0; r < NR; ++r) {
                double tot[7];
                for (int i = 0; i < 7; ++i) tot[i] = warp_sum(S.u.near[warp][r][i][lane]);
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

// Densities of nr right-hand sides in cell-sorted order: FP64 [N][nr][6] (w f, q) for the near
// field, and the FP32 far-field record [N][S] floats (S = 6 + 6 nr rounded up to a multiple of 4):
// x - c_tile and w n from the surface's FP32 record, then (w f, q) per density, zero padding.
__global__ void k_density_multi(const int *__restrict__ perm, const double *__restrict__ w,
                                const float *__restrict__ rec32, const double *__restrict__ f,
                                const double *__restrict__ q, int64_t N, int nr, double *__restrict__ d64,
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
            d64[o + k] = fv;
            d64[o + 3 + k] = qv;
            o32[6 + 6 * r + k] = __double2float_rn(fv);
            o32[6 + 6 * r + 3 + k] = __double2float_rn(qv);
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
                                 const double *q, int64_t N, int nr, double *d64, float *d32, cudaStream_t st) {
    const int bs = 256;
    k_density_multi<<<(unsigned)((N + bs - 1) / bs), bs, 0, st>>>(perm, w, rec32, f, q, N, nr, d64, d32);
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
