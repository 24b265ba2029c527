// The learned closure of the near field: one or two regularized sums instead of three, and what
// they miss of the extrapolated value predicted by a small network.
//
// ndelta = 1 (the single sum u^{delta_0}, near set r <= cutoff_t delta_0): the network predicts
// the whole correction u - u^{delta_0} = -(c1 rho_0 I0 + c2 rho_0^3 I2) + O(delta^5).
// ndelta = 2 (the two smaller deltas):
//
// Eq. (extrap_eqn) says u^{delta_k} = u + c1 rho_k I0(lambda_k) + c2 rho_k^3 I2(lambda_k) + O(delta^5)
// with c1, c2 independent of delta.  With the two-delta weights beta (sum beta = 1,
// sum beta rho I0 = 0) the two sums give u + gamma c2 with gamma = sum beta rho^3 I2, so
//   u = sum_k beta_k u^{delta_k} - gamma c2.
// The network predicts c2 (in the local frame at x0, divided by h^3 and by a density scale) from
// local features: lambda_0, the principal curvatures, the density and its tangential derivatives
// at x0, and rho_0.  The near set shrinks from r <= 6 delta_2 to r <= 6 delta_1 and each pair
// needs at most two smoothing-function evaluations.  A validation sample of targets is also
// evaluated with the three-delta method; if the learned values differ from it by more than a
// tolerance, the whole evaluation falls back to the three-delta method.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "ers_internal.h"
#include "mlp.h"

using namespace ers;

struct ers_closure {
    int device = 0;
    uint64_t seed = 0;
    float *p[2] = {nullptr, nullptr};  // FP32 master parameters: [0] single layer, [1] double layer
    float *q[2] = {nullptr, nullptr};  // BF16-rounded copies (reference forward / training)
    float *m[2] = {nullptr, nullptr}, *v[2] = {nullptr, nullptr};  // Adam moments
    int step[2] = {0, 0};
    int *err = nullptr;
    // extent of the training features: [layer][0 lo, 1 hi][feature] as order-preserving int keys
    int *range = nullptr;
    int have_range[2] = {0, 0};
    int range_check = 1;     // ers_eval_learned sends targets outside the extent to the method
    int64_t last_out = 0;    // targets of the last ers_eval_learned that were outside it
    Scratch z, a, d4, d, g, idx, loss;
    // evaluation work buffers
    Scratch feat, scale, gamma, outp, sub, valid, oor;
};

namespace ers {
namespace {

using namespace mlp;
constexpr int NFEAT = 13;

__device__ __forceinline__ void local_frame(const double n[3], double t1[3], double t2[3]) {
    const double a0 = fabs(n[0]) < 0.9 ? 1.0 : 0.0, a1 = 1.0 - a0;  // e_x, or e_y when n is close to e_x
    // t1 = n x a, normalised; t2 = n x t1
    double c0 = n[1] * 0.0 - n[2] * a1, c1 = n[2] * a0 - n[0] * 0.0, c2 = n[0] * a1 - n[1] * a0;
    const double inv = 1.0 / sqrt(c0 * c0 + c1 * c1 + c2 * c2);
    t1[0] = c0 * inv;
    t1[1] = c1 * inv;
    t1[2] = c2 * inv;
    t2[0] = n[1] * t1[2] - n[2] * t1[1];
    t2[1] = n[2] * t1[0] - n[0] * t1[2];
    t2[2] = n[0] * t1[1] - n[1] * t1[0];
}

// Principal curvatures of the ellipsoid at x0 (p = x0 - c): with g = p / a^2,
// K = 1 / (a^2 b^2 c^2 |g|^4) and the mean curvature H = (a^2 + b^2 + c^2 - |p|^2) / (2 a^2 b^2 c^2 |g|^3).
__device__ __forceinline__ void curvatures(const double p[3], const double a[3], double &k1, double &k2) {
    double g2 = 0.0, p2 = 0.0, s2 = 0.0, abc2 = 1.0;
    for (int i = 0; i < 3; ++i) {
        const double a2 = a[i] * a[i];
        const double gi = p[i] / a2;
        g2 += gi * gi;
        p2 += p[i] * p[i];
        s2 += a2;
        abc2 *= a2;
    }
    const double gn = sqrt(g2);
    const double K = 1.0 / (abc2 * g2 * g2);
    const double H = (s2 - p2) / (2.0 * abc2 * g2 * gn);
    const double disc = sqrt(fmax(H * H - K, 0.0));
    k1 = H + disc;
    k2 = H - disc;
}

struct FeatArgs {
    const double *y, *x0, *n0, *b, *f0, *q0, *gf0, *gq0;
    const double *u2, *v2, *gamma, *u3, *v3;  // u3, v3 optional (training targets)
    int64_t M;
    double h, rho0, Rc;
    int nd;  // 1: target c = (u3 - u1) / (h S); 2: target c2 = (u2 - u3) / (gamma h^3 S)
    double gamma_min;  // nd = 2: samples need |gamma| >= gamma_min
    double c[3], a[3];
    float *Xs, *Xd, *Ts, *Td;  // features (M x 16) and targets (M x 4)
    double *scale;             // (M x 2) density scales, 0 = no correction
    int *valid;
};

// One thread per target: features of both layers; targets when u3, v3 are given.
__global__ void k_features(FeatArgs A) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= A.M) return;
    const bool near = fabs(A.b[m]) <= A.Rc;
    double n[3], t1[3], t2[3], p[3];
    for (int i = 0; i < 3; ++i) {
        n[i] = A.n0[3 * m + i];
        p[i] = A.x0[3 * m + i] - A.c[i];
    }
    local_frame(n, t1, t2);
    double k1, k2;
    curvatures(p, A.a, k1, k2);
    const double lam = A.b[m] / (A.rho0 * A.h);
    for (int layer = 0; layer < 2; ++layer) {
        const double *d0 = (layer == 0 ? A.f0 : A.q0) + 3 * m;
        const double *J = (layer == 0 ? A.gf0 : A.gq0) + 9 * m;  // J[i][j] = d f_i / d x_j
        double loc[12];
        // density value in the local frame
        for (int e = 0; e < 3; ++e) {
            const double *ax = e == 0 ? t1 : (e == 1 ? t2 : n);
            loc[e] = d0[0] * ax[0] + d0[1] * ax[1] + d0[2] * ax[2];
        }
        // tangential derivatives along t1, t2, in the local frame, times h
        for (int dir = 0; dir < 2; ++dir) {
            const double *t = dir == 0 ? t1 : t2;
            double dv[3];
            for (int i = 0; i < 3; ++i) dv[i] = J[3 * i] * t[0] + J[3 * i + 1] * t[1] + J[3 * i + 2] * t[2];
            for (int e = 0; e < 3; ++e) {
                const double *ax = e == 0 ? t1 : (e == 1 ? t2 : n);
                loc[3 + 3 * dir + e] = (dv[0] * ax[0] + dv[1] * ax[1] + dv[2] * ax[2]) * A.h;
            }
        }
        double S = 0.0;
        for (int e = 0; e < 9; ++e) S = fmax(S, fabs(loc[e]));
        const bool ok = near && S > 0.0 && isfinite(S) && fabs(lam) <= 64.0;
        float *X = (layer == 0 ? A.Xs : A.Xd) + m * IN;
        X[0] = (float)lam;
        X[1] = (float)(k1 * A.h);
        X[2] = (float)(k2 * A.h);
        for (int e = 0; e < 9; ++e) X[3 + e] = ok ? (float)(loc[e] / S) : 0.0f;
        X[12] = (float)A.rho0;
        for (int e = NFEAT; e < IN; ++e) X[e] = 0.0f;
        A.scale[2 * m + layer] = ok ? S : 0.0;
        float *T = layer == 0 ? A.Ts : A.Td;
        const double *u3 = layer == 0 ? A.u3 : A.v3;
        if (T && u3) {
            const double *u2 = (layer == 0 ? A.u2 : A.v2) + 3 * m;
            const double g = A.gamma[m];
            double c2[3];
            double den;
            if (A.nd == 2) {
                for (int i = 0; i < 3; ++i) c2[i] = (ok && fabs(g) >= A.gamma_min) ? (u2[i] - u3[3 * m + i]) / g : 0.0;
                den = A.h * A.h * A.h * S;
            } else {
                for (int i = 0; i < 3; ++i) c2[i] = ok ? (u3[3 * m + i] - u2[i]) : 0.0;
                den = A.h * S;
            }
            for (int e = 0; e < 3; ++e) {
                const double *ax = e == 0 ? t1 : (e == 1 ? t2 : n);
                T[m * OUT_STRIDE + e] = ok ? (float)((c2[0] * ax[0] + c2[1] * ax[1] + c2[2] * ax[2]) / den) : 0.0f;
            }
            T[m * OUT_STRIDE + 3] = 0.0f;
        }
    }
    A.valid[m] = (near && (A.nd == 1 || fabs(A.gamma[m]) >= A.gamma_min)) ? 1 : 0;
}

// nd = 2: u = u2 - gamma h^3 S (R c2_local); nd = 1: u = u1 + h S (R c_local); R = [t1 t2 n0].
// Only targets with a density scale S > 0 are corrected.
__global__ void k_apply(const double *__restrict__ n0, const double *__restrict__ gamma,
                        const double *__restrict__ scale, const float *__restrict__ Ys, const float *__restrict__ Yd,
                        int64_t M, double h, int nd, double *__restrict__ u, double *__restrict__ v) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double n[3], t1[3], t2[3];
    for (int i = 0; i < 3; ++i) n[i] = n0[3 * m + i];
    local_frame(n, t1, t2);
    const double h3 = h * h * h;
    for (int layer = 0; layer < 2; ++layer) {
        const double S = scale[2 * m + layer];
        double *out = layer == 0 ? u : v;
        if (!out || S == 0.0) continue;
        const float *Y = (layer == 0 ? Ys : Yd) + m * OUT_STRIDE;
        const double f = nd == 2 ? gamma[m] * h3 * S : -h * S;
        for (int i = 0; i < 3; ++i) out[3 * m + i] -= f * (Y[0] * t1[i] + Y[1] * t2[i] + Y[2] * n[i]);
    }
}

// Gather every `stride`-th target (and its closest-point data and densities) into a compact set.
__global__ void k_gather(const double *__restrict__ y, const double *__restrict__ x0, const double *__restrict__ n0,
                         const double *__restrict__ b, const double *__restrict__ f0, const double *__restrict__ q0,
                         int64_t Ms, int stride, double *__restrict__ out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Ms) return;
    const int64_t m = k * stride;
    double *o = out;
    for (int i = 0; i < 3; ++i) {
        o[3 * k + i] = y[3 * m + i];
        o[3 * Ms + 3 * k + i] = x0[3 * m + i];
        o[6 * Ms + 3 * k + i] = n0[3 * m + i];
        o[10 * Ms + 3 * k + i] = f0 ? f0[3 * m + i] : 0.0;
        o[13 * Ms + 3 * k + i] = q0 ? q0[3 * m + i] : 0.0;
    }
    o[9 * Ms + k] = b[m];
}

// max |learned - plain| and max |plain| over the validation sample, per layer (4 doubles).
__global__ void k_compare(const double *__restrict__ u, const double *__restrict__ v, const double *__restrict__ up,
                          const double *__restrict__ vp, int64_t Ms, int stride, double *__restrict__ res) {
    double e[4] = {0, 0, 0, 0};
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < Ms; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = k * stride;
        for (int i = 0; i < 3; ++i) {
            if (u) {
                e[0] = fmax(e[0], fabs(u[3 * m + i] - up[3 * k + i]));
                e[1] = fmax(e[1], fabs(up[3 * k + i]));
            }
            if (v) {
                e[2] = fmax(e[2], fabs(v[3 * m + i] - vp[3 * k + i]));
                e[3] = fmax(e[3], fabs(vp[3 * k + i]));
            }
        }
    }
    for (int j = 0; j < 4; ++j) {
        double x = e[j];
        for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
        if ((threadIdx.x & 31) == 0)
            atomicMax(reinterpret_cast<unsigned long long *>(res + j), (unsigned long long)__double_as_longlong(x));
    }
}

__global__ void k_minibatch(int *__restrict__ idx, int n, int64_t total, uint64_t seed, uint64_t step) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (step * 0x100000001B3ull + (uint64_t)i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    idx[i] = (int)(z % (uint64_t)total);
}

// Order-preserving map of a float to an int (and its inverse, the same map): integer order of the
// keys = numeric order of the floats, so that atomicMin / atomicMax on keys track a float extent.
__host__ __device__ __forceinline__ int range_key(int bits) { return bits >= 0 ? bits : bits ^ 0x7fffffff; }

constexpr int RANGE_STRIDE = 2 * IN;  // ints per layer: lo[IN], hi[IN]

// Widen the extent keys[0..NFEAT) (lo), keys[IN..IN+NFEAT) (hi) to cover the finite features of
// samples X (n, IN).
__global__ void k_range_update(const float *__restrict__ X, int64_t n, int *__restrict__ keys) {
    int lo[NFEAT], hi[NFEAT];
#pragma unroll
    for (int f = 0; f < NFEAT; ++f) {
        lo[f] = 0x7fffffff;
        hi[f] = (int)0x80000000;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int f = 0; f < NFEAT; ++f) {
            const float x = X[i * IN + f];
            if (!isfinite(x)) continue;
            const int k = range_key(__float_as_int(x));
            lo[f] = min(lo[f], k);
            hi[f] = max(hi[f], k);
        }
    }
#pragma unroll
    for (int f = 0; f < NFEAT; ++f) {
        const int l = __reduce_min_sync(0xffffffffu, lo[f]), h = __reduce_max_sync(0xffffffffu, hi[f]);
        if ((threadIdx.x & 31) == 0) {
            atomicMin(keys + f, l);
            atomicMax(keys + IN + f, h);
        }
    }
}

// Targets whose features (of a layer with a known extent) lie outside that extent widened by
// 5 % of its width plus 1e-3 of its magnitude plus 1e-6: their indices are appended to idx.
// Only corrected targets (density scale > 0) are checked.
__global__ void k_range_flags(const float *__restrict__ Xs, const float *__restrict__ Xd,
                              const double *__restrict__ scale, int64_t M, const int *__restrict__ keys, int have0,
                              int have1, int64_t *__restrict__ idx, unsigned long long *__restrict__ count) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    bool out = false;
    for (int layer = 0; layer < 2; ++layer) {
        if (!(layer == 0 ? have0 : have1) || !(scale[2 * m + layer] > 0.0)) continue;
        const float *X = (layer == 0 ? Xs : Xd) + m * IN;
        const int *K = keys + layer * RANGE_STRIDE;
        for (int f = 0; f < NFEAT; ++f) {
            const float lo = __int_as_float(range_key(K[f])), hi = __int_as_float(range_key(K[IN + f]));
            // explicit roundings (no contraction), so that a host computation can repeat the decision
            const float tol = __fadd_rn(__fadd_rn(__fmul_rn(0.05f, __fsub_rn(hi, lo)),
                                                  __fmul_rn(1e-3f, fmaxf(fabsf(lo), fabsf(hi)))),
                                        1e-6f);
            const float x = X[f];
            if (!(x >= __fsub_rn(lo, tol) && x <= __fadd_rn(hi, tol))) out = true;
        }
    }
    if (out) idx[atomicAdd(count, 1ull)] = m;
}

// Gather the targets idx[0..K) (and their closest-point data and densities) into a compact set
// (the layout of k_gather), and scatter results back.
__global__ void k_gather_idx(const double *__restrict__ y, const double *__restrict__ x0,
                             const double *__restrict__ n0, const double *__restrict__ b,
                             const double *__restrict__ f0, const double *__restrict__ q0,
                             const int64_t *__restrict__ idx, int64_t K, double *__restrict__ out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int64_t m = idx[k];
    for (int i = 0; i < 3; ++i) {
        out[3 * k + i] = y[3 * m + i];
        out[3 * K + 3 * k + i] = x0[3 * m + i];
        out[6 * K + 3 * k + i] = n0[3 * m + i];
        out[10 * K + 3 * k + i] = f0[3 * m + i];
        out[13 * K + 3 * k + i] = q0[3 * m + i];
    }
    out[9 * K + k] = b[m];
}

__global__ void k_scatter_idx(const double *__restrict__ up, const double *__restrict__ vp,
                              const int64_t *__restrict__ idx, int64_t K, double *__restrict__ u,
                              double *__restrict__ v) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int64_t m = idx[k];
    for (int i = 0; i < 3; ++i) {
        u[3 * m + i] = up[3 * k + i];
        v[3 * m + i] = vp[3 * k + i];
    }
}

int closure_check(const ers_closure *c, int layer) {
    if (!c) return fail(ERS_E_INVAL, "NULL closure");
    if (layer != 0 && layer != 1) return fail(ERS_E_INVAL, "layer must be 0 (single) or 1 (double)");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != c->device) return fail(ERS_E_INVAL, "the current device is not the closure's device");
    return ERS_OK;
}

void free_closure(ers_closure *c) {
    if (!c) return;
    for (int l = 0; l < 2; ++l) {
        if (c->p[l]) cudaFree(c->p[l]);
        if (c->q[l]) cudaFree(c->q[l]);
        if (c->m[l]) cudaFree(c->m[l]);
        if (c->v[l]) cudaFree(c->v[l]);
    }
    if (c->err) cudaFree(c->err);
    if (c->range) cudaFree(c->range);
    Scratch *ss[] = {&c->z, &c->a, &c->d4, &c->d, &c->g, &c->idx, &c->loss, &c->feat, &c->scale, &c->gamma,
                     &c->outp, &c->sub, &c->valid, &c->oor};
    for (Scratch *s : ss)
        if (s->ptr) cudaFree(s->ptr);
    delete c;
}

int infer(ers_closure *c, int layer, const float *X, int64_t n, float *Y, cudaStream_t st) {
    if (n == 0) return ERS_OK;
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    const int64_t tiles = (n + 127) / 128;
    const int grid = (int)std::min<int64_t>(tiles, (int64_t)nsm * 4);
    cudaError_t e = launch_infer_tc(c->p[layer], X, n, Y, c->err, grid, st);
    if (e != cudaSuccess) return cuda_fail(e, "closure inference kernel");
    return ERS_OK;
}

}  // namespace
}  // namespace ers

extern "C" {

int ers_closure_create(uint64_t seed, ers_closure **out) {
    clear_error();
    if (!out) return fail(ERS_E_INVAL, "ers_closure_create: NULL output");
    *out = nullptr;
    ers_closure *c = new (std::nothrow) ers_closure();
    if (!c) return fail(ERS_E_NOMEM, "ers_closure_create: host allocation failed");
    cudaGetDevice(&c->device);
    c->seed = seed;
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < 2 && e == cudaSuccess; ++l) {
        e = cudaMalloc(&c->p[l], sizeof(float) * mlp::NPARAM);
        if (e == cudaSuccess) e = cudaMalloc(&c->q[l], sizeof(float) * mlp::NPARAM);
        if (e == cudaSuccess) e = cudaMalloc(&c->m[l], sizeof(float) * mlp::NPARAM);
        if (e == cudaSuccess) e = cudaMalloc(&c->v[l], sizeof(float) * mlp::NPARAM);
    }
    if (e == cudaSuccess) e = cudaMalloc(&c->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->range, sizeof(int) * 2 * RANGE_STRIDE);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_closure(c);
        return fail(ERS_E_NOMEM, "ers_closure_create: device allocation failed");
    }
    // He-uniform initial weights from a seeded generator, zero biases; unused output rows zero
    std::mt19937_64 rng(seed);
    for (int l = 0; l < 2; ++l) {
        std::vector<float> h(mlp::NPARAM, 0.0f);
        auto fill = [&](int off, int rows, int cols, int used_rows) {
            const double bound = std::sqrt(6.0 / cols);
            std::uniform_real_distribution<double> U(-bound, bound);
            for (int r = 0; r < rows; ++r)
                for (int k = 0; k < cols; ++k) h[off + r * cols + k] = r < used_rows ? (float)U(rng) : 0.0f;
        };
        fill(mlp::OFF_W1, mlp::HID, mlp::IN, mlp::HID);
        fill(mlp::OFF_W2, mlp::HID, mlp::HID, mlp::HID);
        fill(mlp::OFF_W3, mlp::HID, mlp::HID, mlp::HID);
        fill(mlp::OFF_W4, mlp::OUT, mlp::HID, mlp::OUT_USED);
        e = cudaMemcpy(c->p[l], h.data(), sizeof(float) * mlp::NPARAM, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(c->m[l], 0, sizeof(float) * mlp::NPARAM);
        if (e == cudaSuccess) e = cudaMemset(c->v[l], 0, sizeof(float) * mlp::NPARAM);
        if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = cudaMemset(c->err, 0, sizeof(int));
    if (e == cudaSuccess) {  // empty extents: lo = +inf, hi = -inf
        std::vector<int> k(2 * RANGE_STRIDE);
        for (int l = 0; l < 2; ++l)
            for (int f = 0; f < mlp::IN; ++f) {
                k[l * RANGE_STRIDE + f] = range_key(0x7f800000);
                k[l * RANGE_STRIDE + mlp::IN + f] = range_key((int)0xff800000u);
            }
        e = cudaMemcpy(c->range, k.data(), sizeof(int) * k.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        free_closure(c);
        return cuda_fail(e, "ers_closure_create: initialisation");
    }
    *out = c;
    return ERS_OK;
}

int ers_closure_free(ers_closure *c) {
    clear_error();
    free_closure(c);
    return ERS_OK;
}

int ers_closure_params(ers_closure *c, int layer, float *get, const float *set, int64_t count) {
    clear_error();
    int rc = closure_check(c, layer);
    if (rc != ERS_OK) return rc;
    if (count != mlp::NPARAM) return fail(ERS_E_INVAL, "ers_closure_params: count must be " + std::to_string(mlp::NPARAM));
    cudaError_t e = cudaSuccess;
    if (set) e = cudaMemcpy(c->p[layer], set, sizeof(float) * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && get) e = cudaMemcpy(get, c->p[layer], sizeof(float) * count, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "ers_closure_params");
    return ERS_OK;
}

int ers_closure_infer(ers_closure *c, int layer, const float *X, int64_t n, float *Y, void *stream) {
    clear_error();
    int rc = closure_check(c, layer);
    if (rc != ERS_OK) return rc;
    if (n < 0 || (n > 0 && (!X || !Y))) return fail(ERS_E_INVAL, "ers_closure_infer: bad arrays");
    return infer(c, layer, X, n, Y, (cudaStream_t)stream);
}

int ers_closure_infer_reference(ers_closure *c, int layer, const float *X, int64_t n, float *Y, void *stream) {
    clear_error();
    int rc = closure_check(c, layer);
    if (rc != ERS_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = mlp::launch_quantize(c->p[layer], c->q[layer], st);
    if (e == cudaSuccess) e = mlp::launch_infer_ref(c->q[layer], X, n, Y, st);
    if (e != cudaSuccess) return cuda_fail(e, "ers_closure_infer_reference");
    return ERS_OK;
}

int ers_closure_range(ers_closure *c, int layer, float *get, const float *set, int *have) {
    clear_error();
    int rc = closure_check(c, layer);
    if (rc != ERS_OK) return rc;
    int *dev = c->range + layer * RANGE_STRIDE;
    cudaError_t e = cudaSuccess;
    if (set) {
        int k[RANGE_STRIDE];
        for (int f = 0; f < mlp::IN; ++f) {
            const bool used = f < NFEAT;
            const float lo = used ? set[f] : INFINITY, hi = used ? set[NFEAT + f] : -INFINITY;
            if (used && !(lo <= hi)) return fail(ERS_E_INVAL, "ers_closure_range: need lo <= hi for every feature");
            int bl, bh;
            std::memcpy(&bl, &lo, sizeof bl);
            std::memcpy(&bh, &hi, sizeof bh);
            k[f] = range_key(bl);
            k[mlp::IN + f] = range_key(bh);
        }
        e = cudaMemcpy(dev, k, sizeof k, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) c->have_range[layer] = 1;
    }
    if (e == cudaSuccess && get) {
        int k[RANGE_STRIDE];
        e = cudaMemcpy(k, dev, sizeof k, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            for (int f = 0; f < NFEAT; ++f) {
                const int bl = range_key(k[f]), bh = range_key(k[mlp::IN + f]);
                std::memcpy(get + f, &bl, sizeof bl);
                std::memcpy(get + NFEAT + f, &bh, sizeof bh);
            }
    }
    if (e != cudaSuccess) return cuda_fail(e, "ers_closure_range");
    if (have) *have = c->have_range[layer];
    return ERS_OK;
}

int ers_closure_set_range_check(ers_closure *c, int enabled) {
    clear_error();
    if (!c) return fail(ERS_E_INVAL, "NULL closure");
    c->range_check = enabled ? 1 : 0;
    return ERS_OK;
}

int ers_closure_last_out_of_range(ers_closure *c, int64_t *n) {
    clear_error();
    if (!c || !n) return fail(ERS_E_INVAL, "ers_closure_last_out_of_range: NULL argument");
    *n = c->last_out;
    return ERS_OK;
}

// Test hook (not in the public header): run the bounded-wait probe once on the current device;
// *timed_out = 1 when its wait ran out.  Synchronous.
int ers_debug_wait_timeout(int arrive, int limit, int *timed_out) {
    clear_error();
    if (!timed_out || limit < 1) return fail(ERS_E_INVAL, "ers_debug_wait_timeout: bad arguments");
    int *flag = nullptr;
    cudaError_t e = cudaMalloc(&flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(flag, 0, sizeof(int));
    if (e == cudaSuccess) e = mlp::launch_wait_probe(arrive, (uint32_t)limit, flag, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(timed_out, flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (flag) cudaFree(flag);
    if (e != cudaSuccess) return cuda_fail(e, "ers_debug_wait_timeout");
    return ERS_OK;
}

int ers_closure_status(ers_closure *c, int *timed_out) {
    clear_error();
    if (!c || !timed_out) return fail(ERS_E_INVAL, "ers_closure_status: NULL argument");
    cudaError_t e = cudaMemcpy(timed_out, c->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "ers_closure_status");
    return ERS_OK;
}

static int grad_impl(ers_closure *c, int layer, const float *X, const float *T, const int *idx, int64_t n, float *G,
                     double *loss_dev, cudaStream_t st) {
    int rc = grow(c->z, sizeof(float) * n * 3 * mlp::HID);
    if (rc == ERS_OK) rc = grow(c->a, sizeof(float) * n * mlp::ACT);
    if (rc == ERS_OK) rc = grow(c->d4, sizeof(float) * n * mlp::OUT_USED);
    if (rc == ERS_OK) rc = grow(c->d, sizeof(float) * n * 3 * mlp::HID);
    if (rc != ERS_OK) return rc;
    cudaError_t e = mlp::launch_quantize(c->p[layer], c->q[layer], st);
    if (e == cudaSuccess)
        e = mlp::launch_train_grad(c->q[layer], X, T, idx, n, (float *)c->z.ptr, (float *)c->a.ptr,
                                   (float *)c->d4.ptr, (float *)c->d.ptr, G, loss_dev, st);
    if (e != cudaSuccess) return cuda_fail(e, "closure training kernels");
    return ERS_OK;
}

int ers_closure_grad(ers_closure *c, int layer, const float *X, const float *T, int64_t n, float *G, double *loss,
                     void *stream) {
    clear_error();
    int rc = closure_check(c, layer);
    if (rc != ERS_OK) return rc;
    if (n <= 0 || !X || !T || !G) return fail(ERS_E_INVAL, "ers_closure_grad: bad arrays");
    if ((rc = grow(c->loss, sizeof(double))) != ERS_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(c->loss.ptr, 0, sizeof(double), st);
    if (e != cudaSuccess) return cuda_fail(e, "ers_closure_grad");
    if ((rc = grad_impl(c, layer, X, T, nullptr, n, G, (double *)c->loss.ptr, st)) != ERS_OK) return rc;
    if (loss) {
        e = cudaMemcpyAsync(loss, c->loss.ptr, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "ers_closure_grad: loss");
    }
    return ERS_OK;
}

int ers_closure_train(ers_closure *c, int layer, const float *X, const float *T, int64_t n, int steps, int batch,
                      float lr, double *final_loss, void *stream) {
    clear_error();
    int rc = closure_check(c, layer);
    if (rc != ERS_OK) return rc;
    if (n <= 0 || !X || !T || steps <= 0 || batch <= 0) return fail(ERS_E_INVAL, "ers_closure_train: bad arguments");
    if (n > INT32_MAX) return fail(ERS_E_UNSUPPORTED, "ers_closure_train: more than 2^31 samples");
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = grow(c->idx, sizeof(int) * batch)) != ERS_OK) return rc;
    if ((rc = grow(c->g, sizeof(float) * mlp::NPARAM)) != ERS_OK) return rc;
    if ((rc = grow(c->loss, sizeof(double))) != ERS_OK) return rc;
    {
        int nsm = 152;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
        const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4 * (int64_t)nsm);
        k_range_update<<<(unsigned)blocks, 256, 0, st>>>(X, n, c->range + layer * RANGE_STRIDE);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "ers_closure_train: feature extent");
        c->have_range[layer] = 1;
    }
    for (int s = 0; s < steps; ++s) {
        const bool last = s == steps - 1;
        k_minibatch<<<(batch + 255) / 256, 256, 0, st>>>((int *)c->idx.ptr, batch, n, c->seed + 7919 * layer,
                                                          (uint64_t)(c->step[layer] + 1));
        if (last) cudaMemsetAsync(c->loss.ptr, 0, sizeof(double), st);
        rc = grad_impl(c, layer, X, T, (const int *)c->idx.ptr, batch, (float *)c->g.ptr,
                       last ? (double *)c->loss.ptr : nullptr, st);
        if (rc != ERS_OK) return rc;
        c->step[layer] += 1;
        // cosine decay of the learning rate over this call
        const float lr_s = lr * 0.5f * (1.0f + cosf(3.14159265f * (float)s / (float)steps));
        cudaError_t e = mlp::launch_adam(c->p[layer], c->m[layer], c->v[layer], (const float *)c->g.ptr, lr_s,
                                         c->step[layer], st);
        if (e != cudaSuccess) return cuda_fail(e, "ers_closure_train: Adam");
    }
    if (final_loss) {
        cudaError_t e = cudaMemcpyAsync(final_loss, c->loss.ptr, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "ers_closure_train: loss");
    }
    return ERS_OK;
}

}  // extern "C"

namespace ers {

// Two-delta evaluation into u, v (+ gamma), far field with the precision of p.
int eval_few_delta(ers_surface *s, const ers_params *p, const double *y, int64_t M, const double *x0,
                   const double *n0, const double *b, const double *f0, const double *q0, double *u, double *v,
                   double *gamma, int ndelta, cudaStream_t st);

}  // namespace ers

namespace {

int features(ers_surface *s, ers_closure *c, const ers_params *p, const double *y, int64_t M, const double *x0,
             const double *n0, const double *b, const double *f0, const double *q0, const double *gf0,
             const double *gq0, const double *u2, const double *v2, const double *gamma, const double *u3,
             const double *v3, float *Xs, float *Xd, float *Ts, float *Td, double *scale, int *valid, int nd,
             cudaStream_t st) {
    FeatArgs A;
    A.y = y;
    A.x0 = x0;
    A.n0 = n0;
    A.b = b;
    A.f0 = f0;
    A.q0 = q0;
    A.gf0 = gf0;
    A.gq0 = gq0;
    A.u2 = u2;
    A.v2 = v2;
    A.gamma = gamma;
    A.u3 = u3;
    A.v3 = v3;
    A.M = M;
    A.h = s->h;
    A.rho0 = p->rho[0];
    A.Rc = p->cutoff_t * p->rho[nd - 1] * s->h;
    A.nd = nd;
    // |gamma| at b = 0: beta = (rho_1, -rho_0) / (rho_1 - rho_0), I2(0) = 1 / (3 sqrt(pi)), so
    // |gamma(0)| = rho_0 rho_1 (rho_0 + rho_1) / (3 sqrt(pi))
    A.gamma_min = 0.01 * p->rho[0] * p->rho[1] * (p->rho[0] + p->rho[1]) / (3.0 * 1.7724538509055160273);
    for (int i = 0; i < 3; ++i) {
        A.c[i] = s->c[i];
        A.a[i] = s->a[i];
    }
    A.Xs = Xs;
    A.Xd = Xd;
    A.Ts = Ts;
    A.Td = Td;
    A.scale = scale;
    A.valid = valid;
    (void)c;
    k_features<<<(unsigned)((M + 127) / 128), 128, 0, st>>>(A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "closure features kernel");
    return ERS_OK;
}

}  // namespace

extern "C" {

int ers_closure_data(ers_surface *s, const ers_params *p, const double *y, int64_t M, const double *x0,
                     const double *n0, const double *b, const double *f0, const double *q0, const double *gf0,
                     const double *gq0, const double *u3, const double *v3, int ndelta, float *Xs, float *Xd,
                     float *Ts, float *Td, int *valid, void *stream) {
    clear_error();
    if (ndelta != 1 && ndelta != 2) return fail(ERS_E_INVAL, "ers_closure_data: ndelta must be 1 or 2");
    if (!s || !p || !y || !x0 || !n0 || !b || !f0 || !q0 || !gf0 || !gq0 || !u3 || !v3 || !Xs || !Xd || !Ts || !Td ||
        !valid)
        return fail(ERS_E_INVAL, "ers_closure_data: NULL argument");
    if (p->options & (ERS_OPT_FOUR_DELTA | ERS_OPT_TREECODE))
        return fail(ERS_E_UNSUPPORTED, "ers_closure_data: ERS_OPT_FOUR_DELTA and ERS_OPT_TREECODE are not supported");
    if (M <= 0) return fail(ERS_E_INVAL, "ers_closure_data: M <= 0");
    cudaStream_t st = (cudaStream_t)stream;
    Scratch &w = s->host_io;  // reuse the host-io buffer of the surface as scratch: u2 | v2 | gamma | scale
    int rc = grow(w, sizeof(double) * (size_t)M * 9);
    if (rc != ERS_OK) return rc;
    double *u2 = (double *)w.ptr, *v2 = u2 + 3 * M, *gm = v2 + 3 * M, *sc = gm + M;
    ers_params pp = *p;
    pp.layers = ERS_LAYER_SL | ERS_LAYER_DL;
    if ((rc = eval_few_delta(s, &pp, y, M, x0, n0, b, f0, q0, u2, v2, gm, ndelta, st)) < 0) return rc;
    return features(s, nullptr, &pp, y, M, x0, n0, b, f0, q0, gf0, gq0, u2, v2, gm, u3, v3, Xs, Xd, Ts, Td, sc,
                    valid, ndelta, st);
}

int ers_eval_learned(ers_surface *s, ers_closure *c, const ers_params *p, const double *y, int64_t M,
                     const double *x0, const double *n0, const double *b, const double *f0, const double *q0,
                     const double *gf0, const double *gq0, int ndelta, double *u, double *v, double tol, int vstride,
                     double *val_err, int *fell_back, void *stream) {
    clear_error();
    if (ndelta != 1 && ndelta != 2) return fail(ERS_E_INVAL, "ers_eval_learned: ndelta must be 1 or 2");
    if (!s || !c || !p || !y || !x0 || !n0 || !b || !f0 || !q0 || !gf0 || !gq0 || !u || !v)
        return fail(ERS_E_INVAL, "ers_eval_learned: NULL argument (both layers and all closest-point data needed)");
    if (p->options & (ERS_OPT_FOUR_DELTA | ERS_OPT_TREECODE))
        return fail(ERS_E_UNSUPPORTED, "ers_eval_learned: ERS_OPT_FOUR_DELTA and ERS_OPT_TREECODE are not supported");
    if (M < 0) return fail(ERS_E_INVAL, "ers_eval_learned: M < 0");
    if (vstride < 1) return fail(ERS_E_INVAL, "ers_eval_learned: vstride must be >= 1");
    int rc = closure_check(c, 0);
    if (rc != ERS_OK) return rc;
    if (fell_back) *fell_back = 0;
    if (M == 0) return ERS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    ers_params pp = *p;
    pp.layers = ERS_LAYER_SL | ERS_LAYER_DL;
    // work buffers of the closure: features (2 x M x 16 f32), outputs (2 x M x 4 f32), gamma, scale
    if ((rc = grow(c->feat, sizeof(float) * (size_t)M * mlp::IN * 2)) != ERS_OK) return rc;
    if ((rc = grow(c->outp, sizeof(float) * (size_t)M * mlp::OUT_STRIDE * 2)) != ERS_OK) return rc;
    if ((rc = grow(c->gamma, sizeof(double) * (size_t)M)) != ERS_OK) return rc;
    if ((rc = grow(c->scale, sizeof(double) * (size_t)M * 2)) != ERS_OK) return rc;
    if ((rc = grow(c->valid, sizeof(int) * (size_t)M)) != ERS_OK) return rc;
    float *Xs = (float *)c->feat.ptr, *Xd = Xs + M * mlp::IN;
    float *Ys = (float *)c->outp.ptr, *Yd = Ys + M * mlp::OUT_STRIDE;
    double *gm = (double *)c->gamma.ptr, *sc = (double *)c->scale.ptr;
    // 1. one- or two-delta sums; 2. features; 3. network (tensor cores); 4. correction
    if ((rc = eval_few_delta(s, &pp, y, M, x0, n0, b, f0, q0, u, v, gm, ndelta, st)) < 0) return rc;
    if ((rc = features(s, c, &pp, y, M, x0, n0, b, f0, q0, gf0, gq0, nullptr, nullptr, gm, nullptr, nullptr, Xs, Xd,
                       nullptr, nullptr, sc, (int *)c->valid.ptr, ndelta, st)) != ERS_OK)
        return rc;
    if ((rc = infer(c, 0, Xs, M, Ys, st)) != ERS_OK) return rc;
    if ((rc = infer(c, 1, Xd, M, Yd, st)) != ERS_OK) return rc;
    k_apply<<<(unsigned)((M + 127) / 128), 128, 0, st>>>(n0, gm, sc, Ys, Yd, M, s->h, ndelta, u, v);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "closure correction kernel");
    // 4b. targets whose features lie outside the training extent: the three-delta method instead
    c->last_out = 0;
    if (c->range_check && (c->have_range[0] || c->have_range[1])) {
        // [count | pad | idx (M) | gathered inputs (16 K) | u, v (6 K)], K <= M
        if ((rc = grow(c->oor, sizeof(int64_t) * 2 + sizeof(int64_t) * (size_t)M + sizeof(double) * (size_t)M * 22)) !=
            ERS_OK)
            return rc;
        unsigned long long *cnt = (unsigned long long *)c->oor.ptr;
        int64_t *idx = (int64_t *)c->oor.ptr + 2;
        double *sub = (double *)(idx + M);
        e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return cuda_fail(e, "ers_eval_learned: memset");
        k_range_flags<<<(unsigned)((M + 127) / 128), 128, 0, st>>>(Xs, Xd, sc, M, c->range, c->have_range[0],
                                                                   c->have_range[1], idx, cnt);
        unsigned long long K = 0;
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&K, cnt, sizeof K, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "ers_eval_learned: feature extent check");
        const int64_t Kt = (int64_t)K;
        c->last_out = Kt;
        if (Kt > 0) {
            double *up = sub + 16 * Kt, *vp = up + 3 * Kt;
            k_gather_idx<<<(unsigned)((Kt + 127) / 128), 128, 0, st>>>(y, x0, n0, b, f0, q0, idx, Kt, sub);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "ers_eval_learned: gather");
            if ((rc = ers_eval(s, &pp, sub, Kt, sub + 3 * Kt, sub + 6 * Kt, sub + 9 * Kt, sub + 10 * Kt,
                               sub + 13 * Kt, up, vp, stream)) < 0)
                return rc;
            k_scatter_idx<<<(unsigned)((Kt + 127) / 128), 128, 0, st>>>(up, vp, idx, Kt, u, v);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "ers_eval_learned: scatter");
        }
    }
    // 5. validation against the three-delta method on every vstride-th target
    const int64_t Ms = (M + vstride - 1) / vstride;
    if ((rc = grow(c->sub, sizeof(double) * ((size_t)Ms * 22 + 8))) != ERS_OK) return rc;
    double *sub = (double *)c->sub.ptr;
    double *up = sub + 16 * Ms, *vp = up + 3 * Ms, *res = vp + 3 * Ms;
    k_gather<<<(unsigned)((Ms + 127) / 128), 128, 0, st>>>(y, x0, n0, b, f0, q0, Ms, vstride, sub);
    e = cudaMemsetAsync(res, 0, sizeof(double) * 4, st);
    if (e != cudaSuccess) return cuda_fail(e, "ers_eval_learned: memset");
    if ((rc = ers_eval(s, &pp, sub, Ms, sub + 3 * Ms, sub + 6 * Ms, sub + 9 * Ms, sub + 10 * Ms, sub + 13 * Ms, up, vp,
                       stream)) < 0)
        return rc;
    k_compare<<<64, 128, 0, st>>>(u, v, up, vp, Ms, vstride, res);
    double h[4];
    e = cudaMemcpyAsync(h, res, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "ers_eval_learned: validation");
    int timed_out = 0;
    cudaMemcpy(&timed_out, c->err, sizeof(int), cudaMemcpyDeviceToHost);
    const double es = h[1] > 0 ? h[0] / h[1] : 0.0, ed = h[3] > 0 ? h[2] / h[3] : 0.0;
    if (val_err) {
        val_err[0] = es;
        val_err[1] = ed;
    }
    if (timed_out) return fail(ERS_E_TIMEOUT, "ers_eval_learned: a tensor-core wait in the closure kernel expired");
    if (!(es <= tol && ed <= tol)) {
        if (fell_back) *fell_back = 1;
        return ers_eval(s, &pp, y, M, x0, n0, b, f0, q0, u, v, stream);
    }
    return ERS_OK;
}

}  // extern "C"
