// Treecode far field (Sec. 3.4, Eqs. (MAC), (particle-cluster-KITC), (mod_weights)).
//
// The far sums over nodes with r > Rc (Eqs. (Stokes_SL1), (Stokes_DL1)) are split by a walk of
// the octree per target: a cluster C with r_c / R <= theta (Eq. (MAC)) whose bounding sphere
// lies beyond the near radius (R - r_c > (1 + 1e-4) Rc) is summed by barycentric Lagrange
// interpolation at its (p+1)^3 Chebyshev points,
//   sum_{x in C} K(y, x) g(x) ~ sum_k K(y, s_k) g^_k,   g^_k = sum_{x in C} L_k(x) g(x),
// with the 15 modified weights g^ of w f, w n and q_j w n_k, so that the subtracted densities
// g = w f - (f(x0).n0) w n and Q m = (q - q(x0)) w n follow per target; a cluster that fails
// is opened, and a leaf that fails is summed directly over its nodes beyond Rc, with exactly
// the near/far mask of the near-field kernel.  The result goes to the far partial sums that
// k_near completes with the near sums and the extrapolation, as for the direct far field.
//
// Modified weights: leaves directly by Eq. (mod_weights) (FP64), then every parent from its
// children by the exact transfer g^P_k = sum_C sum_k' L^P_k(s^C_k') g^C_k' (the parent's basis
// is a polynomial of degree p in each coordinate, which the child's interpolation reproduces),
// applied as three one-dimensional contractions, level by level upwards.
//
// Evaluation: one warp per 32 targets that are close in space (a counting sort by the cells of
// the surface grid taken in Morton order), one lane per target.  The warp walks the tree depth first with a stack in
// shared memory; at every cluster each lane takes its own decision (approximate, sum the leaf,
// open, or nothing below an approximated ancestor), so every target gets exactly the
// per-target walk of Sec. 3.4.  The lanes that approximate a cluster read its Chebyshev
// weights, and the lanes that sum a leaf its nodes, as warp-uniform loads (one transaction per
// warp, served from L1/L2); the point coordinates come from per-cluster tables of c_a + hw_a
// cos(k pi/p), with d formed plane by plane.  No block-wide barrier.
#include <algorithm>
#include <climits>
#include <cmath>

#include "tree.h"

namespace ers {
namespace {

constexpr int TCH = 64;      // nodes per staged chunk of the leaf weights
constexpr unsigned FULL_MASK = 0xffffffffu;
constexpr double INV8PI = 0.039788735772973833942;
constexpr double ACC_MARGIN = 1.0 + 1e-4;
constexpr double PI = 3.14159265358979323846;

// Barycentric Lagrange basis of degree p at the Chebyshev points c + hw cos(k pi/p) (second
// kind, weights (-1)^k d_k with d_0 = d_p = 1/2), evaluated at x; L_k = 1 where x equals s_k
// (first such k).  Berrut & Trefethen, SIAM Review 46 (2004).
__device__ __forceinline__ void lagrange_basis(const Cheb &ch, double c, double hw, double x, double *L) {
    const int p = ch.p;
    int hit = -1;
    for (int k = 0; k <= p; ++k) {
        const double sk = __dadd_rn(c, __dmul_rn(hw, ch.cosk[k]));
        if (hit < 0 && x == sk) hit = k;
    }
    if (hit >= 0) {
        for (int k = 0; k <= p; ++k) L[k] = k == hit ? 1.0 : 0.0;
        return;
    }
    double den = 0.0;
    for (int k = 0; k <= p; ++k) {
        const double sk = __dadd_rn(c, __dmul_rn(hw, ch.cosk[k]));
        const double wk = ((k & 1) ? -1.0 : 1.0) * ((k == 0 || k == p) ? 0.5 : 1.0);
        L[k] = __ddiv_rn(wk, __dsub_rn(x, sk));
        den = __dadd_rn(den, L[k]);
    }
    for (int k = 0; k <= p; ++k) L[k] = __ddiv_rn(L[k], den);
}

// The same basis written as T (double or float) without a scratch array: the denominator first,
// then each value (the same operations, so T = double gives lagrange_basis's values).
template <class T>
__device__ __forceinline__ void lagrange_basis_to(const Cheb &ch, double c, double hw, double x, T *L) {
    const int p = ch.p;
    int hit = -1;
    for (int k = 0; k <= p; ++k) {
        const double sk = __dadd_rn(c, __dmul_rn(hw, ch.cosk[k]));
        if (hit < 0 && x == sk) hit = k;
    }
    if (hit >= 0) {
        for (int k = 0; k <= p; ++k) L[k] = k == hit ? (T)1 : (T)0;
        return;
    }
    double den = 0.0;
    for (int k = 0; k <= p; ++k) {
        const double sk = __dadd_rn(c, __dmul_rn(hw, ch.cosk[k]));
        const double wk = ((k & 1) ? -1.0 : 1.0) * ((k == 0 || k == p) ? 0.5 : 1.0);
        den = __dadd_rn(den, __ddiv_rn(wk, __dsub_rn(x, sk)));
    }
    for (int k = 0; k <= p; ++k) {
        const double sk = __dadd_rn(c, __dmul_rn(hw, ch.cosk[k]));
        const double wk = ((k & 1) ? -1.0 : 1.0) * ((k == 0 || k == p) ? 0.5 : 1.0);
        L[k] = (T)__ddiv_rn(__ddiv_rn(wk, __dsub_rn(x, sk)), den);
    }
}

// Tree-ordered records: FP64 copy of the cell-sorted record, FP32 copy relative to the leaf centre.
__global__ void k_tree_gather(int64_t N, const int *__restrict__ tsrt, const int *__restrict__ tleaf,
                              const TreeCluster *__restrict__ cl, const double *__restrict__ rec,
                              double *__restrict__ trec, float *__restrict__ trec32) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double *src = rec + (int64_t)tsrt[i] * REC;
    double v[REC];
#pragma unroll
    for (int k = 0; k < REC; ++k) v[k] = src[k];
#pragma unroll
    for (int k = 0; k < REC; ++k) trec[i * REC + k] = v[k];
    const TreeCluster &L = cl[tleaf[i]];
    float *o = trec32 + i * 12;
#pragma unroll
    for (int a = 0; a < 3; ++a) o[a] = __double2float_rn(__dsub_rn(v[a], L.c[a]));
#pragma unroll
    for (int k = 3; k < 12; ++k) o[k] = __double2float_rn(v[k]);
}

// g_i(x) of Eq. (mod_weights) from a record: w f (0..2), w n (3..5), q_j w n_k (6 + 3 j + k)
__device__ __forceinline__ double rec_density(const double *r, int g) {
    if (g < 3) return r[R_WF + g];
    if (g < 6) return r[R_WN + g - 3];
    const int j = (g - 6) / 3, k = (g - 6) % 3;
    return r[R_Q + j] * r[R_WN + k];
}

// Modified weights of the leaves, Eq. (mod_weights): one CTA per leaf; each thread owns one
// Chebyshev index k per pass and its 15 sums; the nodes' basis values (computed in FP64) and
// densities are staged in shared memory, TCH nodes at a time.  T = double: FP64 products and sums;
// T = float (weights for the mixed evaluation only): FP32 products and FP32 sums over each chunk of
// TCH nodes, added in FP64 (relative error ~1e-7, below the interpolation error of the treecode).
template <class T>
__global__ void __launch_bounds__(256, 2) k_leaf_weights(const TreeCluster *__restrict__ cl, const int *__restrict__ ids,
                                                      const double *__restrict__ trec, Cheb ch, double *__restrict__ W) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sm = reinterpret_cast<T *>(smraw);
    const TreeCluster C = cl[ids[blockIdx.x]];
    const int P1 = ch.p + 1, NK = P1 * P1 * P1, per = 3 * P1 + TREE_NW;
    double *Wc = W + (size_t)ids[blockIdx.x] * NK * TREE_WS;
    for (int k0 = 0; k0 < NK; k0 += blockDim.x) {
        const int k = k0 + threadIdx.x;
        const int k1 = k / (P1 * P1), k2 = (k / P1) % P1, k3 = k % P1;
        double acc[TREE_NW];
#pragma unroll
        for (int g = 0; g < TREE_NW; ++g) acc[g] = 0.0;
        for (int n0 = 0; n0 < C.count; n0 += TCH) {
            const int nn = min(TCH, C.count - n0);
            __syncthreads();
            for (int t = threadIdx.x; t < nn * 3; t += blockDim.x) {
                const int node = t / 3, a = t % 3;
                const double xv = trec[(int64_t)(C.start + n0 + node) * REC + R_X + a];
                lagrange_basis_to<T>(ch, C.c[a], C.hw[a], xv, sm + node * per + a * P1);
            }
            for (int t = threadIdx.x; t < nn * TREE_NW; t += blockDim.x) {
                const int node = t / TREE_NW, g = t % TREE_NW;
                sm[node * per + 3 * P1 + g] = (T)rec_density(trec + (int64_t)(C.start + n0 + node) * REC, g);
            }
            __syncthreads();
            if (k < NK) {
                T part[TREE_NW];
#pragma unroll
                for (int g = 0; g < TREE_NW; ++g) part[g] = (T)0;
                for (int node = 0; node < nn; ++node) {
                    const T *e = sm + node * per;
                    const T Lk = e[k1] * e[P1 + k2] * e[2 * P1 + k3];
#pragma unroll
                    for (int g = 0; g < TREE_NW; ++g) part[g] = fma(Lk, e[3 * P1 + g], part[g]);
                }
#pragma unroll
                for (int g = 0; g < TREE_NW; ++g) acc[g] += (double)part[g];
            }
        }
        if (k < NK) {
#pragma unroll
            for (int g = 0; g < TREE_NW; ++g) Wc[(size_t)k * TREE_WS + g] = acc[g];
            Wc[(size_t)k * TREE_WS + TREE_NW] = 0.0;
        }
    }
}

// Modified weights of the inner clusters of one level from their children (see the header):
// one CTA per cluster, densities in groups of G; shared memory: the three transfer matrices
// T_a[k][k'] = L^P_{a,k}(s^C_{a,k'}), two work arrays and the accumulator, NK x G doubles each.
__global__ void __launch_bounds__(256) k_upward(const TreeCluster *__restrict__ cl, const int *__restrict__ ids, Cheb ch,
                                                double *__restrict__ W, int G) {
    extern __shared__ double sm[];
    const int pid = ids[blockIdx.x];
    const TreeCluster P = cl[pid];
    const int P1 = ch.p + 1, NK = P1 * P1 * P1, n = NK * G;
    double *T = sm, *A = T + 3 * P1 * P1, *B = A + n, *Acc = B + n;
    double Lt[TREE_PMAX + 1];
    for (int g0 = 0; g0 < TREE_NW; g0 += G) {
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) Acc[i] = 0.0;
        for (int c = 0; c < P.nchild; ++c) {
            const int cid = P.first_child + c;
            const TreeCluster C = cl[cid];
            __syncthreads();
            for (int t = threadIdx.x; t < 3 * P1; t += blockDim.x) {
                const int a = t / P1, kk = t % P1;
                const double xs = __dadd_rn(C.c[a], __dmul_rn(C.hw[a], ch.cosk[kk]));
                lagrange_basis(ch, P.c[a], P.hw[a], xs, Lt);
                for (int k = 0; k < P1; ++k) T[(a * P1 + k) * P1 + kk] = Lt[k];
            }
            const double *Wc = W + (size_t)cid * NK * TREE_WS + g0;
            for (int i = threadIdx.x; i < n; i += blockDim.x) A[i] = Wc[(size_t)(i / G) * TREE_WS + i % G];
            __syncthreads();
            // along k3
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int k = i / G, g = i % G, k3 = k % P1, base = k - k3;
                const double *Tr = T + (2 * P1 + k3) * P1;
                double s = 0.0;
                for (int kk = 0; kk < P1; ++kk) s = fma(Tr[kk], A[(base + kk) * G + g], s);
                B[i] = s;
            }
            __syncthreads();
            // along k2
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int k = i / G, g = i % G, k2 = (k / P1) % P1, base = k - k2 * P1;
                const double *Tr = T + (1 * P1 + k2) * P1;
                double s = 0.0;
                for (int kk = 0; kk < P1; ++kk) s = fma(Tr[kk], B[(base + kk * P1) * G + g], s);
                A[i] = s;
            }
            __syncthreads();
            // along k1, accumulated over the children
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int k = i / G, g = i % G, k1 = k / (P1 * P1), base = k - k1 * P1 * P1;
                const double *Tr = T + k1 * P1;
                double s = 0.0;
                for (int kk = 0; kk < P1; ++kk) s = fma(Tr[kk], A[(base + kk * P1 * P1) * G + g], s);
                Acc[i] += s;
            }
        }
        __syncthreads();
        double *Wp = W + (size_t)pid * NK * TREE_WS + g0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            Wp[(size_t)(i / G) * TREE_WS + i % G] = Acc[i];
            if (i % G == 0 && g0 == 0) Wp[(size_t)(i / G) * TREE_WS + TREE_NW] = 0.0;
        }
    }
}

// FP32 weights for the mixed evaluation, 12 per point (three float4): w f (3), w n (3) and the
// symmetric part of q_j w n_k, which is all that d . (q w n)^ . d sees: S00, S11, S22, S01, S02,
// S12 with S_jk = W_jk + W_kj off the diagonal.
constexpr int TREE_WS32 = 12;
__global__ void k_weights32(const double *__restrict__ W, float *__restrict__ W32, int64_t npts) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npts) return;
    const double *w = W + i * TREE_WS;
    float *o = W32 + i * TREE_WS32;
    for (int g = 0; g < 6; ++g) o[g] = __double2float_rn(w[g]);
    o[6] = __double2float_rn(w[6]);            // S00
    o[7] = __double2float_rn(w[10]);           // S11
    o[8] = __double2float_rn(w[14]);           // S22
    o[9] = __double2float_rn(w[7] + w[9]);     // S01
    o[10] = __double2float_rn(w[8] + w[12]);   // S02
    o[11] = __double2float_rn(w[11] + w[13]);  // S12
}

// Target order: counting sort by the Morton rank of the target's cell of the surface grid
// (clamped), so that consecutive targets are close.
__device__ __forceinline__ int64_t target_cell(const Grid &G, const double *y) {
    int64_t idx[3];
    for (int a = 0; a < 3; ++a) {
        const double u = (y[a] - G.origin[a]) / G.cw;
        const double cu = fmin(fmax(u, 0.0), (double)(G.nc[a] - 1));
        idx[a] = (int64_t)cu;
    }
    return (idx[2] * G.nc[1] + idx[1]) * G.nc[0] + idx[0];
}

__global__ void k_tkeys(const double *__restrict__ y, int64_t M, Grid G, const int *__restrict__ cell_rank,
                        int *__restrict__ keys, int *__restrict__ hist) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const int key = cell_rank[target_cell(G, y + 3 * m)];
    keys[m] = key;
    atomicAdd(hist + key, 1);
}

// exclusive scan of hist[0..n) in place, one CTA of 1024 threads
__global__ void __launch_bounds__(1024) k_tscan(int *__restrict__ hist, int64_t n) {
    __shared__ int part[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    for (int64_t base = 0; base < n; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const int v = i < n ? hist[i] : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            const int t = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
            __syncthreads();
            part[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < n) hist[i] = carry + part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += part[1023];
        __syncthreads();
    }
}

__global__ void k_tscatter(const int *__restrict__ keys, int64_t M, int *__restrict__ off, int *__restrict__ order) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const int pos = atomicAdd(off + keys[m], 1);
    order[pos] = (int)m;
}

constexpr int TWPB = 4;        // warps per CTA; each warp walks the tree for its own 32 targets
constexpr int TBT = TWPB * 32;
constexpr int TSTACK = 128;    // walk stack entries per warp (a tree of depth d needs 8 (d + 1) at most)
constexpr int BUFB = 4096;     // bytes of each of a warp's two staging buffers
constexpr uint32_t WAIT_LIMIT = 1u << 22;  // polls of a bounded mbarrier wait (well above a second)

struct TreeEval {
    const TreeCluster *cl;
    const double *W;
    const float *W32;
    const double *trec;
    const float *trec32;
    const int *tsrt;
    const int *order;
    Cheb ch;
    double theta;
    unsigned long long *stats;  // [3]: approximated pairs, direct pairs, error flag (a wait ran out)
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Staging by the bulk-copy engine: one thread arms the buffer's mbarrier with the byte count and
// issues cp.async.bulk (contiguous, 16-byte aligned, size a multiple of 16); every thread waits
// on the barrier's phase with a bounded poll.
__device__ __forceinline__ void stage_issue(void *dst, const void *src, uint32_t bytes, uint64_t *mbar) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(mbar))
                 : "memory");
}

__device__ __forceinline__ bool stage_wait(uint64_t *mbar, uint32_t parity) {
    for (uint32_t i = 0; i < WAIT_LIMIT; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(smem_addr(mbar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (i > 64) __nanosleep(64);
    }
    return false;
}

struct TgtF64 {
    double y[3], c, q0[3], Rt, Racc;
    long long rc2bits;
    float yh[3], yl[3], rc2f;
};

// One Chebyshev point (FP64): the unregularized Stokeslet and stresslet against the modified
// weights w (Eq. (particle-cluster-KITC)), subtracted with the target's c = f(x0).n0, q0.
__device__ __forceinline__ void approx_point64(const TgtF64 &T, double dx, double dy, double dz, const double *w,
                                               bool sl, bool dl, double acc[6]) {
    const double r2 = dist2_fp64(dx, dy, dz);
    const double ri = rsqrt(r2), ri2 = ri * ri;
    if (sl) {
        const double g0 = fma(-T.c, w[3], w[0]), g1 = fma(-T.c, w[4], w[1]), g2 = fma(-T.c, w[5], w[2]);
        const double s = fma(dz, g2, fma(dy, g1, dx * g0)) * ri2;
        acc[0] = fma(fma(dx, s, g0), ri, acc[0]);
        acc[1] = fma(fma(dy, s, g1), ri, acc[1]);
        acc[2] = fma(fma(dz, s, g2), ri, acc[2]);
    }
    if (dl) {
        // d . (q w n)^ . d - (d.q0)(d.(w n)^)
        const double dWn = fma(dz, w[5], fma(dy, w[4], dx * w[3]));
        const double t0 = fma(dz, w[8], fma(dy, w[7], dx * w[6]));
        const double t1 = fma(dz, w[11], fma(dy, w[10], dx * w[9]));
        const double t2 = fma(dz, w[14], fma(dy, w[13], dx * w[12]));
        const double quad = fma(dz, t2, fma(dy, t1, dx * t0));
        const double dq0 = fma(dz, T.q0[2], fma(dy, T.q0[1], dx * T.q0[0]));
        const double s = fma(-dq0, dWn, quad) * (ri2 * ri2 * ri);
        acc[3] = fma(dx, s, acc[3]);
        acc[4] = fma(dy, s, acc[4]);
        acc[5] = fma(dz, s, acc[5]);
    }
}

// One node of a leaf (FP64), masked exactly as the FP64 near field (r^2 > Rc^2 in the same order).
__device__ __forceinline__ bool direct_node64(const TgtF64 &T, const double *r, bool sl, bool dl, double acc[6]) {
    const double dx = __dsub_rn(T.y[0], r[0]), dy = __dsub_rn(T.y[1], r[1]), dz = __dsub_rn(T.y[2], r[2]);
    const double r2 = dist2_fp64(dx, dy, dz);
    if (!(__double_as_longlong(r2) > T.rc2bits)) return false;
    const double ri = rsqrt(r2), ri2 = ri * ri;
    if (sl) {
        const double g0 = fma(-T.c, r[6], r[3]), g1 = fma(-T.c, r[7], r[4]), g2 = fma(-T.c, r[8], r[5]);
        const double s = fma(dz, g2, fma(dy, g1, dx * g0)) * ri2;
        acc[0] = fma(fma(dx, s, g0), ri, acc[0]);
        acc[1] = fma(fma(dy, s, g1), ri, acc[1]);
        acc[2] = fma(fma(dz, s, g2), ri, acc[2]);
    }
    if (dl) {
        const double Q0 = r[9] - T.q0[0], Q1 = r[10] - T.q0[1], Q2 = r[11] - T.q0[2];
        const double dQ = fma(dz, Q2, fma(dy, Q1, dx * Q0));
        const double dm = fma(dz, r[8], fma(dy, r[7], dx * r[6]));
        const double s = (dQ * dm) * ((ri2 * ri2) * ri);
        acc[3] = fma(dx, s, acc[3]);
        acc[4] = fma(dy, s, acc[4]);
        acc[5] = fma(dz, s, acc[5]);
    }
    return true;
}


// Staged pass of one warp over `count` items of `bytes_each` bytes from src, CH items per chunk,
// double buffered in the warp's own buffers: lane 0 copies chunk i + 1 while the warp computes
// chunk i with body(buffer, first, n).  Returns false (on every lane) when a wait ran out; the
// caller then leaves the kernel.
template <int CH, class Body>
__device__ __forceinline__ bool staged(unsigned char (*buf)[BUFB], uint64_t *mbar, uint32_t &phase, const unsigned char *src,
                                       int count, int bytes_each, int lane, Body &&body) {
    const int nch = (count + CH - 1) / CH;
    if (lane == 0) stage_issue(buf[0], src, (uint32_t)(min(CH, count) * bytes_each), &mbar[0]);
    for (int i = 0; i < nch; ++i) {
        const int b = i & 1;
        if (lane == 0 && i + 1 < nch) {
            const int n1 = min(CH, count - (i + 1) * CH);
            stage_issue(buf[b ^ 1], src + (size_t)(i + 1) * CH * bytes_each, (uint32_t)(n1 * bytes_each), &mbar[b ^ 1]);
        }
        bool ok = stage_wait(&mbar[b], (phase >> b) & 1u);
        phase ^= 1u << b;
        ok = __all_sync(FULL_MASK, ok);
        if (!ok) {
            // a copy did not complete in time: wait (bounded) for the one still in flight, then stop
            if (lane == 0 && i + 1 < nch) stage_wait(&mbar[b ^ 1], (phase >> (b ^ 1)) & 1u);
            return false;
        }
        body(buf[b], i * CH, min(CH, count - i * CH));
        __syncwarp();  // buffer b is refilled at step i + 2
    }
    return true;
}

template <int PREC, bool SL, bool DL>
__global__ void __launch_bounds__(TBT, 4) k_tree_walk(EvalArgs A, TreeEval X) {
    __shared__ __align__(128) unsigned char sbuf[TWPB][2][BUFB];
    __shared__ __align__(8) uint64_t smbar[TWPB][2];
    __shared__ int sstk[TWPB][TSTACK];
    __shared__ float shwc[TWPB][3][TREE_PMAX + 1];   // hw_a cos(k pi/p) in FP32 (mixed)
    __shared__ double spts[TWPB][3][TREE_PMAX + 1];  // c_a + hw_a cos(k pi/p) (FP64)
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    unsigned char (*buf)[BUFB] = sbuf[wp];
    uint64_t *mbar = smbar[wp];
    int *stk = sstk[wp];
    float (*hwc)[TREE_PMAX + 1] = shwc[wp];
    double (*pts)[TREE_PMAX + 1] = spts[wp];
    const int64_t pos = (int64_t)blockIdx.x * TBT + threadIdx.x;
    const bool valid = pos < A.M;
    if (__ballot_sync(FULL_MASK, valid) == 0) return;  // no block-wide barrier in this kernel
    const int64_t m = valid ? X.order[pos] : 0;
    const int P1 = X.ch.p + 1, NK = P1 * P1 * P1;

    TgtF64 T;
    {
        for (int i = 0; i < 3; ++i) T.y[i] = valid ? A.y[3 * m + i] : 0.0;
        const double bm = valid ? A.b[m] : 0.0;
        T.Rt = (A.sharp && bm == 0.0) ? A.Rc_sharp : A.Rc;
        const bool near = fabs(bm) <= T.Rt;
        T.rc2bits = near ? __double_as_longlong(T.Rt * T.Rt) : -1LL;
        T.rc2f = (float)(T.Rt * T.Rt);
        T.Racc = __dmul_rn(ACC_MARGIN, T.Rt);
        T.c = 0.0;
        T.q0[0] = T.q0[1] = T.q0[2] = 0.0;
        if (valid && near) {
            if (SL) T.c = A.f0[3 * m] * A.n0[3 * m] + A.f0[3 * m + 1] * A.n0[3 * m + 1] + A.f0[3 * m + 2] * A.n0[3 * m + 2];
            if (DL)
                for (int i = 0; i < 3; ++i) T.q0[i] = A.q0[3 * m + i];
        }
        for (int i = 0; i < 3; ++i) {
            T.yh[i] = __double2float_rn(T.y[i]);
            T.yl[i] = __double2float_rn(T.y[i] - (double)T.yh[i]);
        }
    }
    const float cf = (float)T.c, q0x = (float)T.q0[0], q0y = (float)T.q0[1], q0z = (float)T.q0[2];
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    unsigned long long napprox = 0, ndirect = 0;
    int skip = INT_MAX;  // level of the approximated ancestor on the current path
    uint32_t phase = 0;  // parity of the next completion of each buffer's barrier
    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        stk[0] = 0;
    }
    int sp = 1;
    __syncwarp();
    while (sp > 0) {
        const int cid = stk[--sp];
        const TreeCluster C = X.cl[cid];
        __syncwarp();  // the previous cluster's readers of the tables are done
        for (int t = lane; t < 3 * P1; t += 32) {
            const int a = t / P1, k = t % P1;
            const double hc = __dmul_rn(C.hw[a], X.ch.cosk[k]);
            hwc[a][k] = __double2float_rn(hc);
            pts[a][k] = __dadd_rn(C.c[a], hc);
        }
        __syncwarp();  // the tables are visible to the whole warp
        if (C.level <= skip) skip = INT_MAX;
        const bool active = valid && skip == INT_MAX;
        bool acc_c = false, leafd = false, desc = false;
        double R = 0.0;
        if (active) {
            const double dx = __dsub_rn(T.y[0], C.c[0]), dy = __dsub_rn(T.y[1], C.c[1]), dz = __dsub_rn(T.y[2], C.c[2]);
            R = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
            acc_c = C.rc <= __dmul_rn(X.theta, R) && __dsub_rn(R, C.rc) > T.Racc;
            leafd = !acc_c && C.nchild == 0;
            desc = !acc_c && C.nchild > 0;
        }
        const bool any_acc = __any_sync(FULL_MASK, acc_c);
        const bool any_leaf = __any_sync(FULL_MASK, leafd);
        const bool any_desc = __any_sync(FULL_MASK, desc);
        bool ok = true;

        if (any_acc) {
            if (acc_c) ++napprox;
            if (PREC == ERS_PREC_FP64) {
                const unsigned char *src = reinterpret_cast<const unsigned char *>(X.W + (size_t)cid * NK * TREE_WS);
                ok = staged<BUFB / 128>(buf, mbar, phase, src, NK, 128, lane, [&](const unsigned char *bp, int k0, int n) {
                    if (!acc_c) return;
                    const double *w = reinterpret_cast<const double *>(bp);
                    int k1 = k0 / (P1 * P1), k2 = (k0 / P1) % P1, k3 = k0 % P1;
                    double dx = __dsub_rn(T.y[0], pts[0][k1]), dy = __dsub_rn(T.y[1], pts[1][k2]);
                    for (int j = 0; j < n; ++j) {
                        const double dz = __dsub_rn(T.y[2], pts[2][k3]);
                        approx_point64(T, dx, dy, dz, w + j * TREE_WS, SL, DL, acc);
                        if (++k3 == P1) {
                            k3 = 0;
                            if (++k2 == P1) {
                                k2 = 0;
                                ++k1;
                                dx = __dsub_rn(T.y[0], pts[0][k1 < P1 ? k1 : 0]);
                            }
                            dy = __dsub_rn(T.y[1], pts[1][k2]);
                        }
                    }
                });
            } else {
                // FP32 terms relative to the cluster centre; FP32 sums per chunk added in FP64
                const unsigned char *src = reinterpret_cast<const unsigned char *>(X.W32 + (size_t)cid * NK * TREE_WS32);
                const float ycx = __double2float_rn(__dsub_rn(T.y[0], C.c[0]));
                const float ycy = __double2float_rn(__dsub_rn(T.y[1], C.c[1]));
                const float ycz = __double2float_rn(__dsub_rn(T.y[2], C.c[2]));
                ok = staged<BUFB / 48>(buf, mbar, phase, src, NK, 48, lane, [&](const unsigned char *bp, int k0, int n) {
                    if (!acc_c) return;
                    const float4 *w4 = reinterpret_cast<const float4 *>(bp);
                    int k1 = k0 / (P1 * P1), k2 = (k0 / P1) % P1, k3 = k0 % P1;
                    float dx = ycx - hwc[0][k1], dy = ycy - hwc[1][k2];
                    float dxy2 = fmaf(dy, dy, dx * dx), dq0xy = fmaf(dy, q0y, dx * q0x);
                    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f, a5 = 0.f;
                    for (int j = 0; j < n; ++j) {
                        // w0 = (wf0 wf1 wf2 wn0), w1 = (wn1 wn2 S00 S11), w2 = (S22 S01 S02 S12)
                        const float4 w0 = w4[3 * j], w1 = w4[3 * j + 1], w2 = w4[3 * j + 2];
                        const float dz = ycz - hwc[2][k3];
                        const float r2 = fmaf(dz, dz, dxy2);
                        const float ri = rsqrt_ftz(r2), ri2 = ri * ri;
                        if (SL) {
                            const float g0 = fmaf(-cf, w0.w, w0.x), g1 = fmaf(-cf, w1.x, w0.y), g2 = fmaf(-cf, w1.y, w0.z);
                            const float sg = fmaf(dz, g2, fmaf(dy, g1, dx * g0)) * ri2;
                            a0 = fmaf(fmaf(dx, sg, g0), ri, a0);
                            a1 = fmaf(fmaf(dy, sg, g1), ri, a1);
                            a2 = fmaf(fmaf(dz, sg, g2), ri, a2);
                        }
                        if (DL) {
                            const float dWn = fmaf(dz, w1.y, fmaf(dy, w1.x, dx * w0.w));
                            // d.S.d = dx (S00 dx + S01 dy + S02 dz) + dy (S11 dy + S12 dz) + S22 dz^2
                            const float t0 = fmaf(dz, w2.z, fmaf(dy, w2.y, dx * w1.z));
                            const float t1 = fmaf(dz, w2.w, dy * w1.w);
                            const float quad = fmaf(dx, t0, fmaf(dy, t1, w2.x * dz * dz));
                            const float dq0 = fmaf(dz, q0z, dq0xy);
                            const float sv = fmaf(-dq0, dWn, quad) * (ri2 * ri2 * ri);
                            a3 = fmaf(dx, sv, a3);
                            a4 = fmaf(dy, sv, a4);
                            a5 = fmaf(dz, sv, a5);
                        }
                        if (++k3 == P1) {
                            k3 = 0;
                            if (++k2 == P1) {
                                k2 = 0;
                                ++k1;
                                dx = ycx - hwc[0][k1 < P1 ? k1 : 0];
                            }
                            dy = ycy - hwc[1][k2];
                            dxy2 = fmaf(dy, dy, dx * dx);
                            dq0xy = fmaf(dy, q0y, dx * q0x);
                        }
                    }
                    acc[0] += a0;
                    acc[1] += a1;
                    acc[2] += a2;
                    acc[3] += a3;
                    acc[4] += a4;
                    acc[5] += a5;
                });
            }
        }

        if (ok && any_leaf) {
            if (PREC == ERS_PREC_FP64) {
                const unsigned char *src = reinterpret_cast<const unsigned char *>(X.trec + (int64_t)C.start * REC);
                ok = staged<BUFB / 96>(buf, mbar, phase, src, C.count, 96, lane, [&](const unsigned char *bp, int, int n) {
                    if (!leafd) return;
                    const double *r = reinterpret_cast<const double *>(bp);
                    for (int j = 0; j < n; ++j) ndirect += direct_node64(T, r + j * REC, SL, DL, acc);
                });
            } else {
                const float ylx = __double2float_rn(__dsub_rn(T.y[0], C.c[0]));
                const float yly = __double2float_rn(__dsub_rn(T.y[1], C.c[1]));
                const float ylz = __double2float_rn(__dsub_rn(T.y[2], C.c[2]));
                // r^2 from leaf-relative floats decides the mask except in a band around Rc^2, where the
                // near field's own test (tile-relative floats) is repeated exactly
                float lo2 = 0.0f, hi2 = 0.0f;
                if (leafd) {
                    const double band = 1e-4 + 4e-6 * (R + C.rc) / T.Rt;
                    lo2 = (float)(T.Rt * T.Rt * (1.0 - band));
                    hi2 = (float)(T.Rt * T.Rt * (1.0 + band));
                }
                const bool all_far = T.rc2bits < 0;
                const unsigned char *src = reinterpret_cast<const unsigned char *>(X.trec32 + (int64_t)C.start * 12);
                ok = staged<BUFB / 48>(buf, mbar, phase, src, C.count, 48, lane, [&](const unsigned char *bp, int j0, int n) {
                    if (!leafd) return;
                    const float4 *r4 = reinterpret_cast<const float4 *>(bp);
                    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f, a5 = 0.f;
                    for (int j = 0; j < n; ++j) {
                        const float4 r0 = r4[3 * j], r1 = r4[3 * j + 1], r2v = r4[3 * j + 2];
                        const float dx = ylx - r0.x, dy = yly - r0.y, dz = ylz - r0.z;
                        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                        bool far = all_far || r2 > hi2;
                        if (!far && !(r2 < lo2)) {
                            const int js = X.tsrt[C.start + j0 + j];
                            const float4 cen = __ldg(reinterpret_cast<const float4 *>(A.sd.tilec) + js / TS32);
                            const float4 xc = __ldg(reinterpret_cast<const float4 *>(A.sd.rec32 + (int64_t)js * REC));
                            float ex, ey, ez;
                            const float r2t = dist2_fp32(tile_rel(T.yh[0], cen.x, T.yl[0]), tile_rel(T.yh[1], cen.y, T.yl[1]),
                                                         tile_rel(T.yh[2], cen.z, T.yl[2]), xc.x, xc.y, xc.z, &ex, &ey, &ez);
                            far = r2t > T.rc2f;
                        }
                        if (!far) continue;
                        ++ndirect;
                        const float ri = rsqrt_ftz(r2), ri2 = ri * ri;
                        // r0 = (x - c: 3, wf0), r1 = (wf1 wf2 wn0 wn1), r2v = (wn2 q0 q1 q2)
                        if (SL) {
                            const float g0 = fmaf(-cf, r1.z, r0.w), g1 = fmaf(-cf, r1.w, r1.x), g2 = fmaf(-cf, r2v.x, r1.y);
                            const float s = fmaf(dz, g2, fmaf(dy, g1, dx * g0)) * ri2;
                            a0 = fmaf(fmaf(dx, s, g0), ri, a0);
                            a1 = fmaf(fmaf(dy, s, g1), ri, a1);
                            a2 = fmaf(fmaf(dz, s, g2), ri, a2);
                        }
                        if (DL) {
                            const float Q0 = r2v.y - q0x, Q1 = r2v.z - q0y, Q2 = r2v.w - q0z;
                            const float dQ = fmaf(dz, Q2, fmaf(dy, Q1, dx * Q0));
                            const float dm = fmaf(dz, r2v.x, fmaf(dy, r1.w, dx * r1.z));
                            const float s = (dQ * dm) * (ri2 * ri2 * ri);
                            a3 = fmaf(dx, s, a3);
                            a4 = fmaf(dy, s, a4);
                            a5 = fmaf(dz, s, a5);
                        }
                    }
                    acc[0] += a0;
                    acc[1] += a1;
                    acc[2] += a2;
                    acc[3] += a3;
                    acc[4] += a4;
                    acc[5] += a5;
                });
            }
        }
        if (!ok) {
            if (lane == 0) atomicOr(X.stats + 2, 1ull);
            return;
        }

        if (any_desc) {
            if (lane == 0)
                for (int c = C.nchild - 1; c >= 0; --c) stk[sp + (C.nchild - 1 - c)] = C.first_child + c;
            sp += C.nchild;
            __syncwarp();
        }
        if (acc_c) skip = C.level;
    }

    if (valid) {
        double *o = A.part + m * 6;
        o[0] = acc[0] * INV8PI;
        o[1] = acc[1] * INV8PI;
        o[2] = acc[2] * INV8PI;
        o[3] = acc[3] * (-6.0 * INV8PI);
        o[4] = acc[4] * (-6.0 * INV8PI);
        o[5] = acc[5] * (-6.0 * INV8PI);
    }
    if (X.stats) {
        for (int o = 16; o > 0; o >>= 1) {
            napprox += __shfl_xor_sync(FULL_MASK, napprox, o);
            ndirect += __shfl_xor_sync(FULL_MASK, ndirect, o);
        }
        if (lane == 0) {
            atomicAdd(X.stats, napprox);
            atomicAdd(X.stats + 1, ndirect);
        }
    }
}

}  // namespace

int tree_prepare(ers_surface *s, int n0, int p, bool mixed, cudaStream_t st) {
    int rc = tree_build(s, n0);
    if (rc != ERS_OK) return rc;
    TreeCache *t = s->tree;
    const int64_t N = s->N;
    cudaError_t e = cudaSuccess;
    if (t->rec_version != s->dens_version) {
        k_tree_gather<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, t->tsrt, t->tleaf, t->cl, s->rec, t->trec, t->trec32);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "treecode: record gather");
        t->rec_version = s->dens_version;
        t->w_version = ~0ull;
    }
    if (8 * (t->depth + 1) > TSTACK)
        return fail(ERS_E_UNSUPPORTED, "treecode: the tree is deeper than the walk stack allows (use a larger tree_n0)");
    const int P1 = p + 1, NK = P1 * P1 * P1;
    // weights built for the mixed evaluation (FP32 products) are not good enough for an FP64 one
    if (t->w_version != s->dens_version || t->p != p || (!mixed && !t->w_fp64)) {
        const size_t wbytes = sizeof(double) * (size_t)t->ncl * NK * TREE_WS;
        if (wbytes > t->w_cap) {
            if (t->W) cudaFree(t->W);
            t->W = nullptr;
            t->w_cap = 0;
            if ((e = cudaMalloc(&t->W, wbytes)) != cudaSuccess) {
                cudaGetLastError();
                return fail(ERS_E_NOMEM, "treecode: modified weights do not fit in device memory");
            }
            t->w_cap = wbytes;
        }
        t->p = p;
        t->ch.p = p;
        for (int k = 0; k <= TREE_PMAX; ++k) t->ch.cosk[k] = k <= p ? std::cos(k * PI / p) : 0.0;
        if (t->nleaf > 0) {
            if (mixed) {  // weights for the mixed evaluation only: FP32 products
                const size_t smem_leaf = sizeof(float) * TCH * (3 * P1 + TREE_NW);
                k_leaf_weights<float><<<t->nleaf, 256, smem_leaf, st>>>(t->cl, t->leaf_ids, t->trec, t->ch, t->W);
            } else {
                const size_t smem_leaf = sizeof(double) * TCH * (3 * P1 + TREE_NW);
                k_leaf_weights<double><<<t->nleaf, 256, smem_leaf, st>>>(t->cl, t->leaf_ids, t->trec, t->ch, t->W);
            }
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "treecode: leaf weights");
        // densities per pass of the upward transfer: the most that fits in 160 KB
        int G = 1;
        for (int g : {15, 5, 3, 1})
            if (sizeof(double) * (3 * (size_t)P1 * P1 + 3 * (size_t)NK * g) <= 160 * 1024) {
                G = g;
                break;
            }
        const size_t smem_up = sizeof(double) * (3 * (size_t)P1 * P1 + 3 * (size_t)NK * G);
        cudaFuncSetAttribute(k_upward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_up);
        for (int l = t->depth; l >= 0; --l) {
            const int a = t->inner_off[l], b = t->inner_off[l + 1];
            if (b > a) k_upward<<<b - a, 256, smem_up, st>>>(t->cl, t->inner_ids + a, t->ch, t->W, G);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "treecode: upward transfer");
        t->w_version = s->dens_version;
        t->w_fp64 = !mixed;
        t->have_w32 = false;
    }
    if (mixed && !t->have_w32) {
        const size_t bytes = sizeof(float) * (size_t)t->ncl * NK * TREE_WS32;
        if (bytes > t->w32_cap) {
            if (t->W32) cudaFree(t->W32);
            t->W32 = nullptr;
            t->w32_cap = 0;
            if ((e = cudaMalloc(&t->W32, bytes)) != cudaSuccess) {
                cudaGetLastError();
                return fail(ERS_E_NOMEM, "treecode: FP32 modified weights do not fit in device memory");
            }
            t->w32_cap = bytes;
        }
        const int64_t npts = (int64_t)t->ncl * NK;
        k_weights32<<<(unsigned)((npts + 255) / 256), 256, 0, st>>>(t->W, t->W32, npts);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "treecode: FP32 weights");
        t->have_w32 = true;
    }
    return ERS_OK;
}

cudaError_t launch_target_order(ers_surface *s, const double *y, int64_t M, cudaStream_t st, const int **order) {
    *order = nullptr;
    if (M == 0) return cudaSuccess;
    const Grid &G = s->grid;
    int err = grow(s->okeys, sizeof(int) * (size_t)M);
    if (err == ERS_OK) err = grow(s->oorder, sizeof(int) * (size_t)M);
    if (err == ERS_OK) err = grow(s->ohist, sizeof(int) * (size_t)(G.ncell + 1));
    if (err != ERS_OK) return cudaErrorMemoryAllocation;
    int *keys = (int *)s->okeys.ptr, *ord = (int *)s->oorder.ptr, *hist = (int *)s->ohist.ptr;
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int) * (size_t)(G.ncell + 1), st);
    if (e != cudaSuccess) return e;
    const unsigned gb = (unsigned)((M + 255) / 256);
    k_tkeys<<<gb, 256, 0, st>>>(y, M, G, s->cell_rank, keys, hist);
    k_tscan<<<1, 1024, 0, st>>>(hist, G.ncell + 1);
    k_tscatter<<<gb, 256, 0, st>>>(keys, M, hist, ord);
    e = cudaGetLastError();
    if (e == cudaSuccess) *order = ord;
    return e;
}

cudaError_t launch_tree_far(const EvalArgs &a, const TreeParams &tp) {
    if (a.M == 0) return cudaSuccess;
    ers_surface *s = const_cast<ers_surface *>(a.s);
    TreeCache *t = s->tree;
    const int64_t M = a.M;
    const int *order = a.order;
    cudaError_t e = cudaMemsetAsync(t->stats, 0, sizeof(unsigned long long) * 3, a.stream);
    if (e != cudaSuccess) return e;
    if (!order && (e = launch_target_order(s, a.y, M, a.stream, &order)) != cudaSuccess) return e;
    TreeEval X;
    X.cl = t->cl;
    X.W = t->W;
    X.W32 = t->W32;
    X.trec = t->trec;
    X.trec32 = t->trec32;
    X.tsrt = t->tsrt;
    X.order = order;
    X.ch = t->ch;
    X.theta = tp.theta;
    X.stats = t->stats;
    const unsigned grid = (unsigned)((M + TBT - 1) / TBT);
    const bool sl = a.layers & ERS_LAYER_SL, dl = a.layers & ERS_LAYER_DL;
    if (a.precision == ERS_PREC_FP64) {
        if (sl && dl) k_tree_walk<ERS_PREC_FP64, true, true><<<grid, TBT, 0, a.stream>>>(a, X);
        else if (sl) k_tree_walk<ERS_PREC_FP64, true, false><<<grid, TBT, 0, a.stream>>>(a, X);
        else k_tree_walk<ERS_PREC_FP64, false, true><<<grid, TBT, 0, a.stream>>>(a, X);
    } else {
        if (sl && dl) k_tree_walk<ERS_PREC_MIXED, true, true><<<grid, TBT, 0, a.stream>>>(a, X);
        else if (sl) k_tree_walk<ERS_PREC_MIXED, true, false><<<grid, TBT, 0, a.stream>>>(a, X);
        else k_tree_walk<ERS_PREC_MIXED, false, true><<<grid, TBT, 0, a.stream>>>(a, X);
    }
    t->stats_valid = true;
    return cudaGetLastError();
}

}  // namespace ers
