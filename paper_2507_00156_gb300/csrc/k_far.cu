// Far field: the unregularized sums over nodes with r > Rc, evaluated once per target and
// shared by the three delta_k (Eq. (near_far), Sec. 3.3), with the subtracted densities of
// Eqs. (Stokes_SL1), (Stokes_DL1) for targets within Rc of the surface and the plain densities
// for the others:
//   SL: u_i += 1/(8 pi) [ g_i / r + d_i (d.g) / r^3 ],           g = w f - (f(x0).n0) w n
//   DL: v_i += 1/(8 pi) (-6) d_i (d.Q) (d.m) / r^5,               Q = q - q(x0), m = w n
// with d = y - x (Eqs. (Stokeslet), (Stresslet)).
//
// Layout: work items (target block, source chunk).  An item is TPB = 128 * TPT targets (TPT per
// thread, held in registers) and one contiguous chunk of the cell-sorted source records; the CTA
// stages tiles of the chunk in shared memory and every thread reads each staged source as a
// broadcast.  Partial sums go to part[chunk][target][6], added by the near-field kernel or, when
// the two kernels run concurrently, by k_combine.  The FP64 kernel runs one item per CTA; the
// mixed kernel loops over items with a stride of the grid, which may be capped (see
// launch_far32) so that near-field CTAs fit on every SM beside it.
// The mask "r^2 > Rc^2" is evaluated with the same operation order as the near-field
// selection, so every pair lands in exactly one of the two sums.
#include <algorithm>

#include "ers_internal.h"

namespace ers {
namespace {

constexpr int NT = 128;
constexpr double INV8PI = 0.039788735772973833942;  // 1/(8 pi)

struct TargetF64 {
    double y[3], c, q0[3];
    long long rc2bits;  // pair is far iff bits(r^2) > rc2bits (signed compare; -1 = all far)
    float rc2f;         // the near radius squared in FP32 (mixed far field)
};

__device__ __forceinline__ void load_target(const EvalArgs &A, int64_t m, bool sl, bool dl, TargetF64 &T,
                                            bool &valid) {
    valid = m < A.M;
    if (!valid) {
        T.y[0] = T.y[1] = T.y[2] = 0.0;
        T.c = 0.0;
        T.q0[0] = T.q0[1] = T.q0[2] = 0.0;
        T.rc2bits = 0x7fffffffffffffffLL;  // nothing is far
        T.rc2f = 0.0f;
        return;
    }
    for (int i = 0; i < 3; ++i) T.y[i] = A.y[3 * m + i];
    const double bm = A.b[m];
    // near radius of this target: cutoff_t times the largest delta, or cutoff_t delta# on the surface (ERS_OPT_SHARP)
    const double Rt = (A.sharp && bm == 0.0) ? A.Rc_sharp : A.Rc;
    const bool near = fabs(bm) <= Rt;
    T.rc2bits = near ? __double_as_longlong(Rt * Rt) : -1LL;
    T.rc2f = (float)(Rt * Rt);  // same rounding as the near-field copy
    T.c = 0.0;
    T.q0[0] = T.q0[1] = T.q0[2] = 0.0;
    if (near) {
        if (sl) T.c = A.f0[3 * m] * A.n0[3 * m] + A.f0[3 * m + 1] * A.n0[3 * m + 1] + A.f0[3 * m + 2] * A.n0[3 * m + 2];
        if (dl)
            for (int i = 0; i < 3; ++i) T.q0[i] = A.q0[3 * m + i];
    }
}

template <bool SL, bool DL, int TPT, int TS>
__global__ void __launch_bounds__(NT) k_far64(EvalArgs A) {
    __shared__ double2 srec[TS * REC / 2];
    const int64_t j0 = (int64_t)blockIdx.y * A.chunk_len;
    const int64_t j1 = min(A.sd.N, j0 + A.chunk_len);
    const double *__restrict__ rec = A.sd.rec;

    TargetF64 T[TPT];
    bool valid[TPT];
    double acc[TPT][6];
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int64_t m = (int64_t)blockIdx.x * (NT * TPT) + t * NT + threadIdx.x;
        load_target(A, m, SL, DL, T[t], valid[t]);
#pragma unroll
        for (int i = 0; i < 6; ++i) acc[t][i] = 0.0;
    }

    for (int64_t base = j0; base < j1; base += TS) {
        const int ns = (int)min((int64_t)TS, j1 - base);
        __syncthreads();
        const double2 *src = reinterpret_cast<const double2 *>(rec + base * REC);
        for (int k = threadIdx.x; k < ns * REC / 2; k += NT) srec[k] = src[k];
        __syncthreads();
        for (int j = 0; j < ns; ++j) {
            const double2 r0 = srec[j * 6 + 0], r1 = srec[j * 6 + 1], r2v = srec[j * 6 + 2];
            const double2 r3 = srec[j * 6 + 3], r4 = srec[j * 6 + 4], r5 = srec[j * 6 + 5];
            const double xs0 = r0.x, xs1 = r0.y, xs2 = r1.x;
            const double wf0 = r1.y, wf1 = r2v.x, wf2 = r2v.y;
            const double wn0 = r3.x, wn1 = r3.y, wn2 = r4.x;
            const double q0s = r4.y, q1s = r5.x, q2s = r5.y;
#pragma unroll
            for (int t = 0; t < TPT; ++t) {
                const double dx = __dsub_rn(T[t].y[0], xs0);
                const double dy = __dsub_rn(T[t].y[1], xs1);
                const double dz = __dsub_rn(T[t].y[2], xs2);
                const double r2 = dist2_fp64(dx, dy, dz);
                double ri = rsqrt(r2);
                ri = (__double_as_longlong(r2) > T[t].rc2bits) ? ri : 0.0;
                const double ri2 = ri * ri;
                if (SL) {
                    const double g0 = fma(-T[t].c, wn0, wf0);
                    const double g1 = fma(-T[t].c, wn1, wf1);
                    const double g2 = fma(-T[t].c, wn2, wf2);
                    const double s = fma(dz, g2, fma(dy, g1, dx * g0)) * ri2;  // (d.g)/r^2
                    acc[t][0] = fma(fma(dx, s, g0), ri, acc[t][0]);
                    acc[t][1] = fma(fma(dy, s, g1), ri, acc[t][1]);
                    acc[t][2] = fma(fma(dz, s, g2), ri, acc[t][2]);
                }
                if (DL) {
                    const double Q0 = q0s - T[t].q0[0], Q1 = q1s - T[t].q0[1], Q2 = q2s - T[t].q0[2];
                    const double dQ = fma(dz, Q2, fma(dy, Q1, dx * Q0));
                    const double dm = fma(dz, wn2, fma(dy, wn1, dx * wn0));
                    const double s = (dQ * dm) * ((ri2 * ri2) * ri);  // (d.Q)(d.m)/r^5
                    acc[t][3] = fma(dx, s, acc[t][3]);
                    acc[t][4] = fma(dy, s, acc[t][4]);
                    acc[t][5] = fma(dz, s, acc[t][5]);
                }
            }
        }
    }
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        if (!valid[t]) continue;
        const int64_t m = (int64_t)blockIdx.x * (NT * TPT) + t * NT + threadIdx.x;
        double *o = A.part + ((int64_t)blockIdx.y * A.M + m) * 6;
        o[0] = acc[t][0] * INV8PI;
        o[1] = acc[t][1] * INV8PI;
        o[2] = acc[t][2] * INV8PI;
        o[3] = acc[t][3] * (-6.0 * INV8PI);
        o[4] = acc[t][4] * (-6.0 * INV8PI);
        o[5] = acc[t][5] * (-6.0 * INV8PI);
    }
}

// Mixed precision: every pair term in FP32 with the target and source both expressed relative
// to the centre c of the source tile (an exact float), yc = (y_hi - c) + y_lo, so that the
// rounding error of d = yc - (x - c) is relative to |y - c| and |x - c| rather than to |y|;
// FP32 partial sums over FLUSH tiles are added into FP64 accumulators, which live in the
// thread's slot of shared memory (touched once per FLUSH tiles; in registers they would cost 48
// registers and one CTA per SM).
struct TargetF32 {
    float yh[3], yl[3], c, q0[3], rc2;
};

// One work item: TPT = 2 NPK targets per thread, as NPK packed pairs.  Per pair term the same
// operations in the same order as the scalar form: d = yc - x, r^2 = fma(dz,dz,fma(dy,dy,dx dx)),
// 1/r by MUFU (masked to 0 where r^2 <= Rc^2), then the SL and DL terms.
template <bool SL, bool DL, int NPK, int FLUSH>
__device__ __forceinline__ void far32_item(const EvalArgs &A, int64_t tbi, int64_t chunk,
                                           float4 *srec, float4 &scen, double *sacc) {
    constexpr int TPT = 2 * NPK;
    const int64_t j0 = chunk * A.chunk_len;  // multiple of TS32
    const int64_t j1 = min(A.sd.N, j0 + A.chunk_len);
    const float *__restrict__ rec = A.sd.rec32;

    float rc2[TPT];
    bool valid[TPT];
    f2 nc[NPK], q0[NPK][3];  // -c and q0 of the two targets of each pair
    // FP64 accumulators: sacc[(t * 6 + i) * NT + thread]
    auto acc = [&](int t, int i) -> double & { return sacc[(t * 6 + i) * NT + threadIdx.x]; };
    f2 accf[NPK][6];
#pragma unroll
    for (int p = 0; p < NPK; ++p) {
        float c[2], q[2][3];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = 2 * p + h;
            const int64_t m = tbi * (NT * TPT) + t * NT + threadIdx.x;
            TargetF64 D;
            load_target(A, m, SL, DL, D, valid[t]);
            for (int i = 0; i < 3; ++i) q[h][i] = __double2float_rn(D.q0[i]);
            c[h] = __double2float_rn(D.c);
            // far iff r2 > rc2: +inf = nothing far (invalid target), -1 = everything far
            rc2[t] = !valid[t] ? __int_as_float(0x7f800000) : (D.rc2bits < 0 ? -1.0f : D.rc2f);
#pragma unroll
            for (int i = 0; i < 6; ++i) acc(t, i) = 0.0;
        }
        nc[p] = pk(-c[0], -c[1]);
        for (int i = 0; i < 3; ++i) q0[p][i] = pk(q[0][i], q[1][i]);
#pragma unroll
        for (int i = 0; i < 6; ++i) accf[p][i] = 0ull;
    }

    int tiles_since_flush = 0;
    for (int64_t base = j0; base < j1; base += TS32) {
        const int ns = (int)min((int64_t)TS32, j1 - base);
        __syncthreads();
        const float4 *src = reinterpret_cast<const float4 *>(rec + base * REC);
        for (int k = threadIdx.x; k < ns * 3; k += NT) srec[k] = src[k];
        if (threadIdx.x == 0) scen = reinterpret_cast<const float4 *>(A.sd.tilec)[base / TS32];
        __syncthreads();
        const float4 cen = scen;
        // targets relative to the tile centre, from their FP64 coordinates (re-read per tile
        // rather than kept in registers): yc = (y_hi - c) + y_lo
        f2 yc[NPK][3];
#pragma unroll
        for (int p = 0; p < NPK; ++p) {
            float v[2][3];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t m = tbi * (NT * TPT) + (2 * p + h) * NT + threadIdx.x;
                const bool ok = valid[2 * p + h];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const double y = ok ? __ldg(A.y + 3 * m + i) : 0.0;
                    const float yh = __double2float_rn(y), yl = __double2float_rn(y - (double)yh);
                    v[h][i] = tile_rel(yh, i == 0 ? cen.x : (i == 1 ? cen.y : cen.z), yl);
                }
            }
            yc[p][0] = pk(v[0][0], v[1][0]);
            yc[p][1] = pk(v[0][1], v[1][1]);
            yc[p][2] = pk(v[0][2], v[1][2]);
        }
        for (int j = 0; j < ns; ++j) {
            const float4 r0 = srec[j * 3 + 0], r1 = srec[j * 3 + 1], r2v = srec[j * 3 + 2];
            // r0 = (xc0 xc1 xc2 wf0), r1 = (wf1 wf2 wn0 wn1), r2v = (wn2 q0 q1 q2)
            const f2 x0 = pk(r0.x, r0.x), x1 = pk(r0.y, r0.y), x2 = pk(r0.z, r0.z);
            const f2 wn0 = pk(r1.z, r1.z), wn1 = pk(r1.w, r1.w), wn2 = pk(r2v.x, r2v.x);
#pragma unroll
            for (int p = 0; p < NPK; ++p) {
                const f2 dx = sub2(yc[p][0], x0), dy = sub2(yc[p][1], x1), dz = sub2(yc[p][2], x2);
                const f2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
                float ra, rb;
                upk(r2, ra, rb);
                // MUFU approximation, relative error ~1e-7; far pairs have r2 >= Rc^2
                const float ia = (ra > rc2[2 * p]) ? rsqrt_ftz(ra) : 0.0f;
                const float ib = (rb > rc2[2 * p + 1]) ? rsqrt_ftz(rb) : 0.0f;
                const f2 ri = pk(ia, ib);
                const f2 ri2 = mul2(ri, ri);
                if (SL) {
                    const f2 g0 = fma2(nc[p], wn0, pk(r0.w, r0.w));
                    const f2 g1 = fma2(nc[p], wn1, pk(r1.x, r1.x));
                    const f2 g2 = fma2(nc[p], wn2, pk(r1.y, r1.y));
                    const f2 sv = mul2(fma2(dz, g2, fma2(dy, g1, mul2(dx, g0))), ri2);
                    accf[p][0] = fma2(fma2(dx, sv, g0), ri, accf[p][0]);
                    accf[p][1] = fma2(fma2(dy, sv, g1), ri, accf[p][1]);
                    accf[p][2] = fma2(fma2(dz, sv, g2), ri, accf[p][2]);
                }
                if (DL) {
                    const f2 Q0 = sub2(pk(r2v.y, r2v.y), q0[p][0]);
                    const f2 Q1 = sub2(pk(r2v.z, r2v.z), q0[p][1]);
                    const f2 Q2 = sub2(pk(r2v.w, r2v.w), q0[p][2]);
                    const f2 dQ = fma2(dz, Q2, fma2(dy, Q1, mul2(dx, Q0)));
                    const f2 dm = fma2(dz, wn2, fma2(dy, wn1, mul2(dx, wn0)));
                    const f2 sv = mul2(mul2(dQ, dm), mul2(mul2(ri2, ri2), ri));
                    accf[p][3] = fma2(dx, sv, accf[p][3]);
                    accf[p][4] = fma2(dy, sv, accf[p][4]);
                    accf[p][5] = fma2(dz, sv, accf[p][5]);
                }
            }
        }
        if (++tiles_since_flush == FLUSH) {
            tiles_since_flush = 0;
#pragma unroll
            for (int p = 0; p < NPK; ++p)
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    float a, b;
                    upk(accf[p][i], a, b);
                    acc(2 * p, i) += (double)a;
                    acc(2 * p + 1, i) += (double)b;
                    accf[p][i] = 0ull;
                }
        }
    }
#pragma unroll
    for (int p = 0; p < NPK; ++p)
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            float a, b;
            upk(accf[p][i], a, b);
            acc(2 * p, i) += (double)a;
            acc(2 * p + 1, i) += (double)b;
        }
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        if (!valid[t]) continue;
        const int64_t m = tbi * (NT * TPT) + t * NT + threadIdx.x;
        double *o = A.part + (chunk * A.M + m) * 6;
        o[0] = acc(t, 0) * INV8PI;
        o[1] = acc(t, 1) * INV8PI;
        o[2] = acc(t, 2) * INV8PI;
        o[3] = acc(t, 3) * (-6.0 * INV8PI);
        o[4] = acc(t, 4) * (-6.0 * INV8PI);
        o[5] = acc(t, 5) * (-6.0 * INV8PI);
    }
}

template <bool SL, bool DL, int NPK, int FLUSH>
__global__ void __launch_bounds__(NT, 4) k_far32(EvalArgs A, int64_t ntb) {
    __shared__ float4 srec[TS32 * 3];
    __shared__ float4 scen;
    __shared__ double sacc[2 * NPK * 6 * NT];
    const int64_t nitems = ntb * A.chunks;
    for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int64_t tbi = item % ntb, chunk = item / ntb;
        __syncthreads();  // the previous item's last tile is no longer read
        far32_item<SL, DL, NPK, FLUSH>(A, tbi, chunk, srec, scen, sacc);
    }
}

template <int TPT, int TS>
cudaError_t far64_dispatch(const EvalArgs &a) {
    const int64_t tb = (a.M + NT * TPT - 1) / (NT * TPT);
    dim3 grid((unsigned)tb, (unsigned)a.chunks);
    const bool sl = a.layers & ERS_LAYER_SL, dl = a.layers & ERS_LAYER_DL;
    if (sl && dl) k_far64<true, true, TPT, TS><<<grid, NT, 0, a.stream>>>(a);
    else if (sl) k_far64<true, false, TPT, TS><<<grid, NT, 0, a.stream>>>(a);
    else k_far64<false, true, TPT, TS><<<grid, NT, 0, a.stream>>>(a);
    return cudaGetLastError();
}

template <int NPK>
cudaError_t far32_dispatch(const EvalArgs &a, int ctas_per_sm, int nsm) {
    constexpr int TPT = 2 * NPK;
    const int64_t tb = (a.M + NT * TPT - 1) / (NT * TPT);
    const int64_t nitems = tb * a.chunks;
    int64_t grid = nitems;
    size_t pad = 0;
    if (ctas_per_sm > 0) {
        // at most ctas_per_sm CTAs per SM: dynamic shared memory that leaves room for no more
        // (228 KB per SM, 1 KB reserved per CTA), and a grid of that many CTAs per SM
        const size_t per_cta = (228u << 10) / (size_t)(ctas_per_sm + 1) + 1;
        const size_t stat = sizeof(float4) * (TS32 * 3 + 1) + sizeof(double) * 2 * NPK * 6 * NT + 1024;
        pad = per_cta > stat ? per_cta - stat : 0;
        grid = std::min<int64_t>(nitems, (int64_t)ctas_per_sm * nsm);
    }
    const bool sl = a.layers & ERS_LAYER_SL, dl = a.layers & ERS_LAYER_DL;
    auto kern = (sl && dl) ? k_far32<true, true, NPK, 2> : (sl ? k_far32<true, false, NPK, 2> : k_far32<false, true, NPK, 2>);
    if (pad > 0) {
        // static + dynamic shared memory above 48 KB needs the opt-in (not a stream operation)
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pad);
        if (e != cudaSuccess) return e;
    }
    kern<<<(unsigned)grid, NT, pad, a.stream>>>(a, tb);
    return cudaGetLastError();
}

// u += sum_c part[c][m][0..2], v += sum_c part[c][m][3..5] (far field into the near-field result).
__global__ void k_combine(const double *__restrict__ part, int chunks, int64_t M, double *u, double *v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // (target, component)
    if (i >= 6 * M) return;
    const int64_t m = i / 6;
    const int c6 = (int)(i - 6 * m);
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += part[((int64_t)c * M + m) * 6 + c6];
    double *o = c6 < 3 ? u : v;
    if (o) o[3 * m + (c6 < 3 ? c6 : c6 - 3)] += s;
}

}  // namespace

cudaError_t launch_far64(const EvalArgs &a) { return far64_dispatch<2, 64>(a); }
cudaError_t launch_far32(const EvalArgs &a, int ctas_per_sm, int nsm) { return far32_dispatch<2>(a, ctas_per_sm, nsm); }

cudaError_t launch_combine(const EvalArgs &a) {
    if (a.M == 0) return cudaSuccess;
    const int64_t n = 6 * a.M;
    const bool sl = a.layers & ERS_LAYER_SL, dl = a.layers & ERS_LAYER_DL;
    k_combine<<<(unsigned)((n + 255) / 256), 256, 0, a.stream>>>(a.part, a.chunks, a.M, sl ? a.u : nullptr,
                                                                  dl ? a.v : nullptr);
    return cudaGetLastError();
}

}  // namespace ers
