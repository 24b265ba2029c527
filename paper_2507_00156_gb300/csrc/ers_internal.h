// Internal declarations of the GB300 extrapolated-regularization library.
// Not part of the public ABI (include/ers.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "ers.h"

namespace ers {

// ------------------------------------------------------------------------------------------
// Layouts
// ------------------------------------------------------------------------------------------

// FP64 source record, one per node in cell-sorted order (96 B):
//   [x0 x1 x2 | w f0 w f1 w f2 | w n0 w n1 w n2 | q0 q1 q2]
// w f and w n feed the single layer (g w = w f - (f(x0).n0) w n, Eq. (Stokes_SL1)); q and w n
// feed the double layer (Q = q - q(x0), m = w n, Eq. (Stokes_DL1)).
constexpr int REC = 12;
constexpr int NCOUNTERS = 12;  // near-field counters of one evaluation (EvalArgs::counters)
constexpr int R_X = 0, R_WF = 3, R_WN = 6, R_Q = 9;

// FP32 record for the mixed-precision far field (48 B): x - c_tile, w f, w n, q.
constexpr int TS32 = 256;  // sources per FP32 tile (one centre c_tile per tile)

// Interpolation table of sigma_p(tau) = s_p(t)/t^p, tau = t^2 (Eqs. (s1)-(s3)):
// intervals of width 1/16 on tau in [0, 24), degree 6 in the local variable
// s = 32 tau - (2 i + 1) in [-1, 1].  The near field uses it only for t <= 4.7 (tau <= 22.09);
// beyond that the defects 1 - s_p are evaluated directly.
// Host copy: [interval][p][7] monomial coefficients, highest degree first.
// Device copy (TAB_DEV_BYTES): per interval and function three float4: degrees 6, 5, 4 as floats
// with the interval offset 2 i + 1, then degrees 3..0 as float pairs (hi, lo).  Degrees 4..6
// carry less than 2e-8 of the value on every interval, so their FP32 evaluation costs at most
// ~2e-15 relative; degrees 3..0 are evaluated in float-pair arithmetic (~1e-14 relative) on the
// FP32 pipe, which on this part runs 64 times the FP64 rate.
constexpr int TAB_INV_W = 16;     // intervals per unit tau
constexpr int TAB_N = 384;        // tau in [0, 24)
constexpr int TAB_DEG = 6;
constexpr int TAB_NC = TAB_DEG + 1;
constexpr double TAB_TAU_MAX = 24.0;
constexpr size_t TAB_DEV_BYTES = (size_t)TAB_N * 3 * 48;
// Table of sigma#_p(tau) = s#_p(t)/t^p for the on-surface functions of Sec. 2.1, the same layout
// with intervals of width 1/32 on tau in [0, 64) (cutoff_t up to 8; no direct-defect path): their
// polynomial-times-Gaussian parts vary faster than sigma_p, and at width 1/32 degrees 4..6 still
// carry less than 2e-8 of the value.
constexpr int SH_INV_W = 32;
constexpr int SH_N = 2048;
constexpr size_t SH_DEV_BYTES = (size_t)SH_N * 3 * 48;

struct Grid {
    double origin[3];
    double cw;      // cell width
    int nc[3];      // cells per axis
    int64_t ncell;  // nc0 * nc1 * nc2
};

struct Scratch {
    void *ptr = nullptr;
    size_t bytes = 0;
};

// ------------------------------------------------------------------------------------------
// Treecode far field (Sec. 3.4)
// ------------------------------------------------------------------------------------------
constexpr int TREE_NW = 15;    // modified-weight densities per Chebyshev point: w f (3), w n (3), q_j w n_k (9)
constexpr int TREE_WS = 16;    // stride of a Chebyshev point's weights (FP64 and FP32 copies; entry 15 is 0)
constexpr int TREE_PMAX = 16;  // largest interpolation degree p

// One cluster: the bounding box of its nodes (centre c, half-widths hw), r_c = half its diagonal;
// nodes [start, start + count) of the tree order; children [first_child, first_child + nchild)
// (clusters are numbered level by level, so siblings are contiguous).
struct TreeCluster {
    double c[3], hw[3], rc;
    int start, count, first_child, nchild, level, pad;
};

struct TreeCache;  // per surface, built on first use (tree_host.cpp)

}  // namespace ers

struct ers_surface {
    int device = 0;
    double c[3], a[3];
    double h = 0.0;
    int64_t N = 0;
    bool is_sphere = false;
    // canonical order (dev)
    double *x = nullptr, *n = nullptr, *w = nullptr;
    // cell-sorted order (dev)
    int *perm = nullptr;          // sorted index -> canonical index
    double *rec = nullptr;        // N * REC
    float *rec32 = nullptr;       // N * REC floats
    float *tilec = nullptr;       // ntile32 * 4 floats (centre of each FP32 tile, exact floats)
    float4 *xs32 = nullptr;       // N float coordinates for the near-field prefilter
    double *fq = nullptr;         // N * 6: the node densities f, q as given (for the closure's jets)
    float *recp = nullptr;        // N * NREC floats: the near-field record (cell-sorted)
    int *cell_start = nullptr;    // ncell + 1
    ers::Grid grid{};
    int64_t ntile32 = 0;
    bool has_f = false, has_q = false;
    // work buffers (grow-only)
    ers::Scratch part, cp, host_io, counts;
    ers::Scratch fitw;  // the learned closure's density fits: neighbour lists and normal equations
    // densities of several right-hand sides (ers_set_density_multi), cell-sorted: float pairs
    // [N][nrhs][6] (w f, q) for the near field and the FP32 far-field record
    // [N][batch_rec32_floats(nrhs)]
    ers::Scratch densp, dens32;
    int nrhs_multi = 0;
    int64_t last_counts[3] = {0, 0, 0};
    int64_t last_class[4] = {0, 0, 0, 0};     // near pairs by number of deltas with r > cutoff_t delta
    int64_t last_dclass[5] = {0, 0, 0, 0, 0};  // near pairs by number of deltas on the direct-defect path
    int64_t last_sharp = 0;                 // near pairs of on-surface targets (ERS_OPT_SHARP)
    cudaStream_t last_stream = nullptr;
    // optional per-kernel timing
    bool profile = false;
    bool profiled = false;
    bool prof_closest = false;
    bool prof_overlap = false;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    // second stream for the far field when it runs concurrently with the near field
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // treecode: octree, tree-ordered records and modified weights (ERS_OPT_TREECODE)
    ers::TreeCache *tree = nullptr;
    uint64_t dens_version = 0;  // bumped by every ers_set_density
    // target order of an evaluation: the grid cells' Morton ranks and the counting-sort buffers
    int *cell_rank = nullptr;  // [ncell]
    ers::Scratch okeys, oorder, ohist;
};

namespace ers {

// Host-side pieces (C++)
int64_t quadrature(const double c[3], const double a[3], double h, std::vector<double> *x, std::vector<double> *n,
                   std::vector<double> *w);
const double *sigma_table_host();  // TAB_N * 3 * TAB_NC doubles
void sigma_table_device_layout(void *dst);  // TAB_DEV_BYTES bytes, the device copy
const double *sigma_sharp_table_host();  // SH_N * 3 * TAB_NC doubles
void sigma_sharp_table_device_layout(void *dst);  // SH_DEV_BYTES bytes

// Error reporting (thread-local message)
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);
void clear_error();

// Validation of ers_params shared by the evaluation entry points (ERS_OK or an error code;
// *warn receives ERS_W_CUTOFF for cutoff_t < 6).
int check_params(const ers_surface *s, const ers_params *p, int *warn);

// Device table pointer for the current device (uploads once per device).
const double *sigma_table_dev(int *err);
const double *sigma_sharp_table_dev(int *err);  // the on-surface (s#) table

// Device-side view of a surface, passed by value in kernel parameters (the ers_surface
// struct itself lives in host memory).
// Near-field record of a node, 96 bytes in cell-sorted order: x as three doubles (the pair
// geometry and the near/far partition stay FP64), then w f, w n and q as float pairs (hi, lo),
// hi + lo within 2^-48 of the FP64 value.  Float offsets:
constexpr int NREC = 24;
constexpr int NR_WF = 6, NR_WN = 12, NR_Q = 18;

struct SurfDev {
    const double *rec;
    const float *recp;
    const float *rec32;
    const float *tilec;
    const float4 *xs32;
    const int *cell_start;
    Grid grid;
    int64_t N;
    double h;
};

inline SurfDev surf_dev(const ers_surface *s) {
    SurfDev d;
    d.rec = s->rec;
    d.recp = s->recp;
    d.rec32 = s->rec32;
    d.tilec = s->tilec;
    d.xs32 = s->xs32;
    d.cell_start = s->cell_start;
    d.grid = s->grid;
    d.N = s->N;
    d.h = s->h;
    return d;
}

// Kernel launchers (k_*.cu)
struct EvalArgs {
    const ers_surface *s;  // host struct: launchers only, never dereferenced on the device
    SurfDev sd;
    const double *y, *x0, *n0, *b, *f0, *q0;
    int64_t M;
    double rho[4], cutoff_t, Rc;  // rho[3]: the fourth delta of the O(delta^7) variant (ndelta = 4)
    int precision, layers;
    int ndelta;      // 3: extrapolation of Eq. (extrap_eqn); 4: the O(delta^7) variant of Sec. 1;
                     // 2: two-delta weights (learned closure); 1: the single sum with delta_0
    bool far_later;  // the near-field kernel leaves the far partial sums to k_combine
    // ERS_OPT_SHARP: targets with b == 0 use the s#_p of Sec. 2.1 with delta# = dsharp, near
    // radius Rc_sharp = cutoff_t delta#, table tab_sharp (far kernels: per-target radius)
    bool sharp;
    double rho_sharp, dsharp, Rc_sharp;  // rho#, delta# = rho# h, cutoff_t delta#
    const double *tab_sharp;
    double *gamma;   // ndelta == 2: per-target gamma (may be NULL)
    const int *order;  // treecode walk: targets in a spatially coherent order (NULL: computed there)
    double *u, *v;
    double *part;    // [chunks][M][6]
    int chunks;
    int64_t chunk_len;
    // [near_targets, near_pairs, near pairs of class 0..3 (deltas on the defect path),
    //  near pairs with 0, 1, 2 deltas beyond cutoff_t, near pairs of on-surface (s#) targets,
    //  near pairs of class 4, near pairs with 3 deltas beyond cutoff_t (both four deltas only)]
    unsigned long long *counters;
    cudaStream_t stream;
};

cudaError_t launch_closest(const ers_surface *s, const double *y, int64_t M, double *x0, double *n0, double *b,
                           cudaStream_t st);
cudaError_t launch_far64(const EvalArgs &a);
// ctas_per_sm > 0: persistent grid of at most ctas_per_sm CTAs per SM (room left for near-field CTAs)
cudaError_t launch_far32(const EvalArgs &a, int ctas_per_sm = 0, int nsm = 0);
cudaError_t launch_combine(const EvalArgs &a);
// ctas_per_sm > 0: a grid of at most ctas_per_sm CTAs per SM striding over the targets
cudaError_t launch_near(const EvalArgs &a, const double *table, int ctas_per_sm = 0, int nsm = 0);
cudaError_t launch_density(ers_surface *s, const double *f, const double *q, cudaStream_t st);

struct BatchProblemDev;
struct BatchItem;
cudaError_t launch_density_multi(const int *perm, const double *w, const float *rec32, const double *f,
                                 const double *q, int64_t N, int nr, float2 *dp, float *d32, cudaStream_t st);
// floats per node of the batched FP32 far-field record for nr densities (multiple of 4)
inline int batch_rec32_floats(int nr) { return (6 + 6 * nr + 3) / 4 * 4; }
int batch_grid(int nr, int nsm);
cudaError_t launch_batch(int nr, const BatchProblemDev *probs, const BatchItem *items, int nitems, unsigned *counter,
                         const double rho[3], int layers, const double *tab, int grid, cudaStream_t st);
int grow(Scratch &s, size_t bytes);

// Treecode (tree_host.cpp, k_tree.cu)
struct TreeParams {
    double theta;
    int n0, p;
};
void treecode_defaults(double h, double *theta, int *n0, int *p);
// Rank of every cell of the grid in Morton (Z) order (row-major for grids above 2^26 cells).
std::vector<int> morton_cell_rank(const Grid &G);
// order[0..M) = the targets sorted by the Morton rank of their cell (counting sort on `st`).
cudaError_t launch_target_order(ers_surface *s, const double *y, int64_t M, cudaStream_t st, const int **order);
// Build (or reuse) the octree for leaf size n0 and the modified weights of degree p for the
// current densities; ERS_OK or an error code.
int tree_prepare(ers_surface *s, int n0, int p, bool mixed, cudaStream_t st);
void tree_free(ers_surface *s);
// Far sums by the treecode into a.part (one chunk), for the near-field kernel to complete.
cudaError_t launch_tree_far(const EvalArgs &a, const TreeParams &tp);
// clusters, leaves, depth, then (after the last treecode eval) approximated (target, cluster)
// pairs and far pairs summed directly
int tree_stats(ers_surface *s, int64_t out[5]);

}  // namespace ers

// ------------------------------------------------------------------------------------------
// Device helpers shared by the kernels
// ------------------------------------------------------------------------------------------
#ifdef __CUDACC__
namespace ers {

// Squared distance in FP64 with a fixed operation order, so that the far-field mask and the
// near-field selection classify every pair identically.
__device__ __forceinline__ double dist2_fp64(double dx, double dy, double dz) {
    return __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
}

// FP32 squared distance of the mixed far field: target and source are both expressed
// relative to the tile centre c; yc = (y_hi - c) + y_lo.  Fixed operation order (same reason).
__device__ __forceinline__ float dist2_fp32(float ycx, float ycy, float ycz, float xcx, float xcy, float xcz,
                                            float *dx, float *dy, float *dz) {
    *dx = __fsub_rn(ycx, xcx);
    *dy = __fsub_rn(ycy, xcy);
    *dz = __fsub_rn(ycz, xcz);
    return __fmaf_rn(*dz, *dz, __fmaf_rn(*dy, *dy, __fmul_rn(*dx, *dx)));
}

__device__ __forceinline__ float tile_rel(float yhi, float c, float ylo) { return __fadd_rn(__fsub_rn(yhi, c), ylo); }

// Truncating double -> float by bit manipulation (integer pipe only, no FP64 instruction).
// For 0 <= x < 2^127: returns a float <= x with relative error < 2^-23, and 0 for x below
// the float normal range.  The 11-bit exponent is rebased modulo 2^9 inside the 32-bit word,
// which is exact for biased exponents 897..1150 (float exponents 1..254).
__device__ __forceinline__ float approx_float_pos(double x) {
    long long bits = __double_as_longlong(x);
    unsigned hi = (unsigned)(bits >> 32), lo = (unsigned)bits;
    unsigned fb = __funnelshift_l(lo, hi, 3) - (unsigned)((1023 - 127) << 23);
    return (hi < (897u << 20)) ? 0.0f : __int_as_float((int)fb);
}

// MUFU reciprocal square root with denormal inputs flushed to zero (rsqrt(0) = +inf): one
// instruction, relative error ~1e-7.  Callers only use it where the argument is a normal float
// or where the result is discarded (masked pairs).
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Two FP32 lanes in one 64-bit register: Blackwell's packed f32x2 arithmetic issues one
// instruction for two IEEE FP32 operations (each lane rounded as its scalar counterpart).
typedef unsigned long long f2;
__device__ __forceinline__ f2 pk(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Signed form of approx_float_pos: |result| <= |x| with relative error < 2^-23 for
// 2^-126 <= |x| < 2^127, zero below (the shifted-out top bits of the high word hold the sign).
__device__ __forceinline__ float approx_float(double x) {
    long long bits = __double_as_longlong(x);
    const unsigned hi = (unsigned)(bits >> 32), lo = (unsigned)bits;
    const unsigned fb = __funnelshift_l(lo, hi, 3) - (unsigned)((1023 - 127) << 23);
    return ((hi & 0x7fffffffu) < (897u << 20)) ? 0.0f : __int_as_float((int)((fb & 0x7fffffffu) | (hi & 0x80000000u)));
}

// float -> double by bit manipulation (integer pipe only); zero for zero and subnormal input.
__device__ __forceinline__ double float_to_double(float f) {
    const unsigned b = (unsigned)__float_as_int(f);
    if ((b & 0x7f800000u) == 0u) return 0.0;
    const unsigned hi = (b & 0x80000000u) | (((b & 0x7fffffffu) >> 3) + ((1023u - 127u) << 20));
    const unsigned lo = b << 29;
    return __longlong_as_double(((long long)hi << 32) | lo);
}

// ------------------------------------------------------------------------------------------
// Float pairs: x = h + l with two floats carries ~47 significant bits.  The operations below run
// on the FP32 and integer pipes (the FP64 pipe of this part is 1/64 of the FP32 rate); every
// product and sum is written with explicit rounding intrinsics so that no contraction changes
// the error-free transformations.
// ------------------------------------------------------------------------------------------

// x (|x| >= 2^-126 or 0) -> h = x truncated to 24 significant bits, l = the next 29 bits of x's
// significand rounded to a float: |x - h - l| <= 2^-47 |x|.  Integer and int-to-float conversion
// instructions only.
__device__ __forceinline__ void split_pair(double x, float &h, float &l) {
    h = approx_float(x);
    const long long bits = __double_as_longlong(x);
    const int low = (int)(bits & ((1LL << 29) - 1));              // significand bits below the float's
    const int ex = (int)((bits >> 52) & 0x7ff) - 1075 + 127;       // biased float exponent of 2^(e - 52)
    float r = (h != 0.0f && ex > 0) ? __fmul_rn(__int2float_rn(low), __int_as_float(ex << 23)) : 0.0f;
    l = bits < 0 ? -r : r;
}

// p = p s + c in float pairs (products by FMA, the sum by Knuth's two-sum, then renormalized).
__device__ __forceinline__ void pair_mad(float &ph, float &pl, float sh, float sl, float ch, float cl) {
    const float th = __fmul_rn(ph, sh);
    const float te = __fmaf_rn(ph, sl, __fmaf_rn(pl, sh, __fmaf_rn(ph, sh, -th)));
    const float u = __fadd_rn(th, ch);
    const float v = __fsub_rn(u, th);
    const float e = __fadd_rn(__fsub_rn(th, __fsub_rn(u, v)), __fsub_rn(ch, v));
    const float w = __fadd_rn(__fadd_rn(e, te), cl);
    ph = __fadd_rn(u, w);
    pl = __fsub_rn(w, __fsub_rn(ph, u));
}

// k = k + a b in float pairs.
__device__ __forceinline__ void pair_acc(float &kh, float &kl, float ah, float al, float bh, float bl) {
    const float th = __fmul_rn(ah, bh);
    const float te = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, __fmaf_rn(ah, bh, -th)));
    const float u = __fadd_rn(kh, th);
    const float v = __fsub_rn(u, kh);
    const float e = __fadd_rn(__fsub_rn(kh, __fsub_rn(u, v)), __fsub_rn(th, v));
    const float w = __fadd_rn(__fadd_rn(e, te), kl);
    kh = __fadd_rn(u, w);
    kl = __fsub_rn(w, __fsub_rn(kh, u));
}

// (h, l) = a b in float pairs (the product of the leading floats exactly, the cross terms added).
__device__ __forceinline__ void pair_mul(float ah, float al, float bh, float bl, float &h, float &l) {
    const float p = __fmul_rn(ah, bh);
    const float e = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, __fmaf_rn(ah, bh, -p)));
    h = __fadd_rn(p, e);
    l = __fsub_rn(e, __fsub_rn(h, p));
}

// k = k + f (a float) in float pairs.
__device__ __forceinline__ void pair_add(float &kh, float &kl, float f) {
    const float u = __fadd_rn(kh, f);
    const float v = __fsub_rn(u, kh);
    const float e = __fadd_rn(__fsub_rn(kh, __fsub_rn(u, v)), __fsub_rn(f, v));
    const float w = __fadd_rn(e, kl);
    kh = __fadd_rn(u, w);
    kl = __fsub_rn(w, __fsub_rn(kh, u));
}

// h + l as a double (one FP64 add).
__device__ __forceinline__ double pair_to_double(float h, float l) { return float_to_double(h) + float_to_double(l); }

// The same arithmetic on a value type, for the near-field contractions.  Error bounds (u = 2^-24,
// operands with |l| <= 2u |h| as split_pair gives them): fp_mul returns the exact product of the
// leading floats plus the cross terms, unnormalized (|l| <= 5u |h|), with error <= 12 u^2 |a b|
// (the product of the trailing floats, which it leaves out, and two roundings of the cross
// terms); fp_add is Knuth's two-sum of the leading floats with the trailing ones added, then
// renormalized, with error <= 6 u^2 (|a| + |b|); fp_fma, an unnormalized product added,
// <= 24 u^2 (|a b| + |c|).  u^2 = 3.6e-15.
struct fpair {
    float h, l;
};

__device__ __forceinline__ fpair fp_split(double x) {
    fpair r;
    split_pair(x, r.h, r.l);
    return r;
}
__device__ __forceinline__ fpair fp_neg(fpair a) { return {-a.h, -a.l}; }
__device__ __forceinline__ fpair fp_mul(fpair a, fpair b) {
    const float p = __fmul_rn(a.h, b.h);
    return {p, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, __fmaf_rn(a.h, b.h, -p)))};
}
__device__ __forceinline__ fpair fp_add(fpair a, fpair b) {
    const float s = __fadd_rn(a.h, b.h);
    const float v = __fsub_rn(s, a.h);
    const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, v)), __fsub_rn(b.h, v));
    const float w = __fadd_rn(e, __fadd_rn(a.l, b.l));
    const float h = __fadd_rn(s, w);
    return {h, __fsub_rn(w, __fsub_rn(h, s))};
}
__device__ __forceinline__ fpair fp_fma(fpair a, fpair b, fpair c) { return fp_add(fp_mul(a, b), c); }
// x + y + z: the three leading floats summed by two two-sums, everything else (the trailing
// floats, the two-sums' errors) added in FP32, then renormalized: 19 FP32 operations against 22
// for two fp_add; error <= ~6 u^2 (|x| + |y| + |z|) for operands with |l| <= 5u |h|.
__device__ __forceinline__ fpair fp_sum3(fpair x, fpair y, fpair z) {
    const float s = __fadd_rn(x.h, y.h);
    float v = __fsub_rn(s, x.h);
    const float e1 = __fadd_rn(__fsub_rn(x.h, __fsub_rn(s, v)), __fsub_rn(y.h, v));
    const float t = __fadd_rn(s, z.h);
    v = __fsub_rn(t, s);
    const float e2 = __fadd_rn(__fsub_rn(s, __fsub_rn(t, v)), __fsub_rn(z.h, v));
    const float w = __fadd_rn(__fadd_rn(__fadd_rn(x.l, y.l), z.l), __fadd_rn(e1, e2));
    const float h = __fadd_rn(t, w);
    return {h, __fsub_rn(w, __fsub_rn(h, t))};
}
// a0 b0 + a1 b1 + a2 b2; error <= ~20 u^2 (|a0 b0| + |a1 b1| + |a2 b2|).
__device__ __forceinline__ fpair fp_dot3(fpair a0, fpair a1, fpair a2, fpair b0, fpair b1, fpair b2) {
    return fp_sum3(fp_mul(a0, b0), fp_mul(a1, b1), fp_mul(a2, b2));
}
// acc + a b + c d; error <= ~20 u^2 (|acc| + |a b| + |c d|).
__device__ __forceinline__ fpair fp_acc2(fpair acc, fpair a, fpair b, fpair c, fpair d) {
    return fp_sum3(acc, fp_mul(a, b), fp_mul(c, d));
}
__device__ __forceinline__ double fp_to_double(fpair a) { return pair_to_double(a.h, a.l); }

}  // namespace ers
#endif
