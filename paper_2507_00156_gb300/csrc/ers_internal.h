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
constexpr int R_X = 0, R_WF = 3, R_WN = 6, R_Q = 9;

// FP32 record for the mixed-precision far field (48 B): x - c_tile, w f, w n, q.
constexpr int TS32 = 256;  // sources per FP32 tile (one centre c_tile per tile)

// Interpolation table of sigma_p(tau) = s_p(t)/t^p, tau = t^2 (Eqs. (s1)-(s3)):
// intervals of width 1/8 on tau in [0, 64), degree 6 in the local variable
// s = 16 tau - (2 i + 1) in [-1, 1]; coefficients stored [interval][p][7], highest first.
constexpr int TAB_INV_W = 8;      // intervals per unit tau
constexpr int TAB_N = 512;        // tau in [0, 64)
constexpr int TAB_DEG = 6;
constexpr int TAB_NC = TAB_DEG + 1;
constexpr double TAB_TAU_MAX = 64.0;

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
    int *cell_start = nullptr;    // ncell + 1
    ers::Grid grid{};
    int64_t ntile32 = 0;
    bool has_f = false, has_q = false;
    // work buffers (grow-only)
    ers::Scratch part, cp, host_io, counts;
    // densities of several right-hand sides (ers_set_density_multi), cell-sorted:
    // [N][nrhs][6] (w f, q) in FP64 and FP32
    ers::Scratch dens64, dens32;
    int nrhs_multi = 0;
    int64_t last_counts[3] = {0, 0, 0};
    int64_t last_class[3] = {0, 0, 0};
    cudaStream_t last_stream = nullptr;
    // optional per-kernel timing
    bool profile = false;
    bool profiled = false;
    bool prof_closest = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace ers {

// Host-side pieces (C++)
int64_t quadrature(const double c[3], const double a[3], double h, std::vector<double> *x, std::vector<double> *n,
                   std::vector<double> *w);
const double *sigma_table_host();  // TAB_N * 3 * TAB_NC doubles

// Error reporting (thread-local message)
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);
void clear_error();

// Validation of ers_params shared by the evaluation entry points (ERS_OK or an error code;
// *warn receives ERS_W_CUTOFF for cutoff_t < 6).
int check_params(const ers_surface *s, const ers_params *p, int *warn);

// Device table pointer for the current device (uploads once per device).
const double *sigma_table_dev(int *err);

// Device-side view of a surface, passed by value in kernel parameters (the ers_surface
// struct itself lives in host memory).
struct SurfDev {
    const double *rec;
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
    double rho[3], cutoff_t, Rc;
    int precision, layers;
    int ndelta;      // 3: extrapolation of Eq. (extrap_eqn); 2: two-delta weights (learned closure)
    double *gamma;   // ndelta == 2: per-target gamma (may be NULL)
    double *u, *v;
    double *part;    // [chunks][M][6]
    int chunks;
    int64_t chunk_len;
    unsigned long long *counters;  // [near_targets, near_pairs, near pairs of class 0, 1, 2]
    cudaStream_t stream;
};

cudaError_t launch_closest(const ers_surface *s, const double *y, int64_t M, double *x0, double *n0, double *b,
                           cudaStream_t st);
cudaError_t launch_far64(const EvalArgs &a);
cudaError_t launch_far32(const EvalArgs &a);
cudaError_t launch_near(const EvalArgs &a, const double *table);
cudaError_t launch_density(ers_surface *s, const double *f, const double *q, cudaStream_t st);

struct BatchProblemDev;
struct BatchItem;
cudaError_t launch_density_multi(const int *perm, const double *w, const double *f, const double *q, int64_t N,
                                 int nr, double *d64, float *d32, cudaStream_t st);
int batch_grid(int nr, int nsm);
cudaError_t launch_batch(int nr, const BatchProblemDev *probs, const BatchItem *items, int nitems, unsigned *counter,
                         const double rho[3], int layers, const double *tab, int grid, cudaStream_t st);
int grow(Scratch &s, size_t bytes);

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

// float -> double by bit manipulation (integer pipe only); zero for zero and subnormal input.
__device__ __forceinline__ double float_to_double(float f) {
    const unsigned b = (unsigned)__float_as_int(f);
    if ((b & 0x7f800000u) == 0u) return 0.0;
    const unsigned hi = (b & 0x80000000u) | (((b & 0x7fffffffu) >> 3) + ((1023u - 127u) << 20));
    const unsigned lo = b << 29;
    return __longlong_as_double(((long long)hi << 32) | lo);
}

}  // namespace ers
#endif
