// Batched evaluation: several problems (surface, targets, NR right-hand-side densities) in one
// persistent launch, captured in a CUDA graph.
//
// A work item is (problem, block of 128 targets).  One CTA runs an item to completion:
//   1. far field with FP32 operands (the pair term of Eqs. (Stokeslet), (Stresslet) on the
//      subtracted densities of Eqs. (Stokes_SL1), (Stokes_DL1)), r > Rc only; the geometry of a
//      pair (d, 1/r) is computed once and shared by the NR densities; FP32 sums over 512
//      sources are added into FP64 accumulators in shared memory;
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

template <int NR>
struct BatchSmem {
    double far[BT][NR][6];  // FP64 far-field accumulators of the CTA's targets
    union {
        float stage[BTS][6 + 6 * NR];      // far phase: x - c_tile, w n, then (w f, q) per density
        double near[BW][NR][7][32];        // near phase: per-lane accumulators
    } u;
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
    for (int r = 0; r < NR; ++r)
        for (int i = 0; i < 6; ++i) S.far[t][r][i] = 0.0;
    float acc[NR][6];
    for (int r = 0; r < NR; ++r)
        for (int i = 0; i < 6; ++i) acc[r][i] = 0.0f;

    const int64_t N = P.sd.N;
    int since = 0;
    for (int64_t base = 0; base < N; base += BTS) {
        const int ns = (int)min((int64_t)BTS, N - base);
        __syncthreads();
        for (int k = t; k < ns * (6 + 6 * NR); k += BT) {
            const int j = k / (6 + 6 * NR), e = k % (6 + 6 * NR);
            const int64_t jj = base + j;
            float val;
            if (e < 3) val = P.sd.rec32[jj * REC + R_X + e];
            else if (e < 6) val = P.sd.rec32[jj * REC + R_WN + (e - 3)];
            else val = P.dens32[jj * (6 * NR) + (e - 6)];
            S.u.stage[j][e] = val;
        }
        if (t == 0) S.cen = reinterpret_cast<const float4 *>(P.sd.tilec)[base / TS32];
        __syncthreads();
        const float4 cen = S.cen;
        const float yc0 = tile_rel(yh[0], cen.x, yl[0]), yc1 = tile_rel(yh[1], cen.y, yl[1]),
                    yc2 = tile_rel(yh[2], cen.z, yl[2]);
        for (int j = 0; j < ns; ++j) {
            const float *sp = S.u.stage[j];
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
            since = 0;
#pragma unroll
            for (int r = 0; r < NR; ++r)
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    S.far[t][r][i] += (double)acc[r][i];
                    acc[r][i] = 0.0f;
                }
        }
    }
    for (int r = 0; r < NR; ++r) {
        for (int i = 0; i < 3; ++i) S.far[t][r][i] *= INV8PI;
        for (int i = 3; i < 6; ++i) S.far[t][r][i] *= -6.0 * INV8PI;
    }
    __syncthreads();
}

template <int CLS, int NR>
__device__ __forceinline__ void near_pair(const BatchProblemDev &P, const Geom &T, const double *__restrict__ tab,
                                          int64_t j, const double (&c)[NR], int64_t m, int lane, int warp,
                                          int layers, BatchSmem<NR> &S) {
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
    const double *dj = P.dens64 + j * (6 * NR);
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        double(*a)[32] = S.u.near[warp][r];
        if (layers & ERS_LAYER_SL) {
            const double wf[3] = {__ldg(dj + 6 * r), __ldg(dj + 6 * r + 1), __ldg(dj + 6 * r + 2)};
            double accU[3] = {a[0][lane], a[1][lane], a[2][lane]};
            sl_accumulate(dx, dy, dz, K1, K3, c[r], wf, wn, accU);
            a[0][lane] = accU[0];
            a[1][lane] = accU[1];
            a[2][lane] = accU[2];
        }
        if (layers & ERS_LAYER_DL) {
            const double qs[3] = {__ldg(dj + 6 * r + 3), __ldg(dj + 6 * r + 4), __ldg(dj + 6 * r + 5)};
            const double *q0p = P.q0 + ((int64_t)r * P.M + m) * 3;
            const double q0[3] = {q0p[0], q0p[1], q0p[2]};
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
            double c[NR];
            for (int r = 0; r < NR; ++r) {
                const double *f0 = P.f0 + ((int64_t)r * P.M + m) * 3;
                c[r] = sl ? fma(f0[2], T.n0[2], fma(f0[1], T.n0[1], f0[0] * T.n0[0])) : 0.0;
                for (int i = 0; i < 7; ++i) S.u.near[warp][r][i][lane] = 0.0;
            }
            __syncwarp();
            scan_near(P.sd, T, P.sp, S.sq[warp], lane, [&](int cls, int jj, bool valid) {
                if (!valid) return;
                if (cls == 0) near_pair<0, NR>(P, T, tab, jj, c, m, lane, warp, layers, S);
                else if (cls == 1) near_pair<1, NR>(P, T, tab, jj, c, m, lane, warp, layers, S);
                else if (cls == 2) near_pair<2, NR>(P, T, tab, jj, c, m, lane, warp, layers, S);
                else near_pair<3, NR>(P, T, tab, jj, c, m, lane, warp, layers, S);
            });
            const double chi = bm < 0.0 ? 1.0 : (bm > 0.0 ? 0.0 : 0.5);
            for (int r = 0; r < NR; ++r) {
                double tot[7];
                for (int i = 0; i < 7; ++i) tot[i] = warp_sum(S.u.near[warp][r][i][lane]);
                if (sl && lane < 3) {
                    const double a = lane == 0 ? tot[0] : (lane == 1 ? tot[1] : tot[2]);
                    P.u[((int64_t)r * P.M + m) * 3 + lane] = S.far[tt][r][lane] + a * INV8PI;
                }
                if (dl && lane >= 3 && lane < 6) {
                    const int i = lane - 3;
                    const double ad = i == 0 ? tot[4] : (i == 1 ? tot[5] : tot[6]);
                    const double ni = i == 0 ? T.n0[0] : (i == 1 ? T.n0[1] : T.n0[2]);
                    const double qi = P.q0[((int64_t)r * P.M + m) * 3 + i];
                    P.v[((int64_t)r * P.M + m) * 3 + i] =
                        S.far[tt][r][lane] + (-6.0 * INV8PI) * fma(tot[3], ni, -ad) + chi * qi;
                }
            }
            __syncwarp();
        } else {
            for (int r = 0; r < NR; ++r) {
                if (sl && lane < 3) P.u[((int64_t)r * P.M + m) * 3 + lane] = S.far[tt][r][lane];
                if (dl && lane >= 3 && lane < 6) P.v[((int64_t)r * P.M + m) * 3 + lane - 3] = S.far[tt][r][lane];
            }
        }
    }
}

template <int NR>
__global__ void __launch_bounds__(BT) k_batch(const BatchProblemDev *__restrict__ probs,
                                              const BatchItem *__restrict__ items, int nitems,
                                              unsigned *__restrict__ counter, double rho0, double rho1, double rho2,
                                              int layers, const double *__restrict__ tab) {
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

__global__ void k_density_multi(const int *__restrict__ perm, const double *__restrict__ w,
                                const double *__restrict__ f, const double *__restrict__ q, int64_t N, int nr,
                                double *__restrict__ d64, float *__restrict__ d32) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const int64_t i = perm[j];
    const double wi = w[i];
    for (int r = 0; r < nr; ++r) {
        for (int k = 0; k < 3; ++k) {
            const double fv = f ? wi * f[((int64_t)r * N + i) * 3 + k] : 0.0;
            const double qv = q ? q[((int64_t)r * N + i) * 3 + k] : 0.0;
            const int64_t o = (j * nr + r) * 6;
            d64[o + k] = fv;
            d64[o + 3 + k] = qv;
            d32[o + k] = __double2float_rn(fv);
            d32[o + 3 + k] = __double2float_rn(qv);
        }
    }
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

cudaError_t launch_density_multi(const int *perm, const double *w, const double *f, const double *q, int64_t N,
                                 int nr, double *d64, float *d32, cudaStream_t st) {
    const int bs = 256;
    k_density_multi<<<(unsigned)((N + bs - 1) / bs), bs, 0, st>>>(perm, w, f, q, N, nr, d64, d32);
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
