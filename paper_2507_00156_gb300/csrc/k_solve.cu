// Pieces for solving integral equations with the evaluation (the two-drop problem of Sec. 4.3,
// Eq. (IE-2Surf)): values of a node density at arbitrary surface points, GMRES over device
// vectors, and a vector update.
//
// ers_node_interp: the value at a surface point x0 (unit normal n0) of the least-squares
// polynomial of total degree <= 4 in the tangent-plane coordinates (xi, eta) = ((x - x0).t1,
// (x - x0).t2) / (3.5 h), fitted to the node values within 3.5 h of x0 (t1 from the coordinate
// axis least aligned with n0, t2 = n0 x t1; the fit does not depend on that choice).  The
// subtraction of Eq. (Stokes_DL1) needs the density at the closest point, which for a density
// known only at the nodes is this O(h^5) approximation.  One thread per point: the 15 x 15
// normal equations from the neighbours found through the surface's cell grid, a Cholesky solve
// for z = (Phi^T Phi)^{-1} e_0, then the value sum_j (phi_j . z) u_j.
//
// ers_gmres: GMRES (Saad & Schultz 1986) without restart from x = 0: Arnoldi with modified
// Gram-Schmidt, the small least-squares problem by Givens rotations on the host; inner products
// by a two-stage reduction in a fixed order (deterministic).
#include <cmath>
#include <vector>

#include "ers_internal.h"

namespace ers {
namespace {

constexpr double INTERP_R = 3.5;  // fit radius in units of h
constexpr int NB = 15;            // monomials of total degree <= 4 in two variables

__device__ __forceinline__ void monomials4(double xi, double eta, double *phi) {
    // order: degree 0..4, within a degree xi^(d-b) eta^b for b = 0..d
    int c = 0;
    double xp[5], ep[5];
    xp[0] = ep[0] = 1.0;
    for (int i = 1; i < 5; ++i) {
        xp[i] = xp[i - 1] * xi;
        ep[i] = ep[i - 1] * eta;
    }
    for (int d = 0; d <= 4; ++d)
        for (int b = 0; b <= d; ++b) phi[c++] = xp[d - b] * ep[b];
}

__global__ void k_node_interp(SurfDev sd, const int *__restrict__ perm, double R, const double *__restrict__ vals,
                              const double *__restrict__ x0, const double *__restrict__ n0, int64_t M,
                              double *__restrict__ out) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const double p[3] = {x0[3 * m], x0[3 * m + 1], x0[3 * m + 2]};
    const double nn[3] = {n0[3 * m], n0[3 * m + 1], n0[3 * m + 2]};
    // tangent basis
    int k = 0;
    if (fabs(nn[1]) < fabs(nn[k])) k = 1;
    if (fabs(nn[2]) < fabs(nn[k])) k = 2;
    double t1[3] = {0.0, 0.0, 0.0};
    t1[k] = 1.0;
    const double an = nn[k];
    for (int a = 0; a < 3; ++a) t1[a] -= an * nn[a];
    const double tl = sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
    for (int a = 0; a < 3; ++a) t1[a] /= tl;
    const double t2[3] = {nn[1] * t1[2] - nn[2] * t1[1], nn[2] * t1[0] - nn[0] * t1[2], nn[0] * t1[1] - nn[1] * t1[0]};
    const double R2 = R * R, iR = 1.0 / R;
    const Grid &G = sd.grid;
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = max(0, (int)floor((p[a] - R - G.origin[a]) / G.cw));
        hi[a] = min(G.nc[a] - 1, (int)floor((p[a] + R - G.origin[a]) / G.cw));
    }
    double A[NB * (NB + 1) / 2];  // packed lower triangle of Phi^T Phi
    for (int i = 0; i < NB * (NB + 1) / 2; ++i) A[i] = 0.0;
    int cnt = 0;
    double phi[NB];
    for (int pass = 0; pass < 2; ++pass) {
        double z[NB];
        double val[3] = {0.0, 0.0, 0.0};
        if (pass == 1) {
            // Cholesky A = L L^T in place (packed rows), then z = A^{-1} e_0
            bool ok = cnt >= NB;
            for (int i = 0; i < NB && ok; ++i) {
                for (int j = 0; j <= i; ++j) {
                    double s = A[i * (i + 1) / 2 + j];
                    for (int q = 0; q < j; ++q) s -= A[i * (i + 1) / 2 + q] * A[j * (j + 1) / 2 + q];
                    if (i == j) {
                        if (!(s > 0.0)) ok = false;
                        A[i * (i + 1) / 2 + i] = sqrt(fmax(s, 1e-300));
                    } else {
                        A[i * (i + 1) / 2 + j] = s / A[j * (j + 1) / 2 + j];
                    }
                }
            }
            if (!ok) {
                for (int a = 0; a < 3; ++a) out[3 * m + a] = __longlong_as_double(0x7ff8000000000000LL);  // NaN: no fit
                return;
            }
            double yv[NB];
            for (int i = 0; i < NB; ++i) {  // L y = e_0
                double s = i == 0 ? 1.0 : 0.0;
                for (int q = 0; q < i; ++q) s -= A[i * (i + 1) / 2 + q] * yv[q];
                yv[i] = s / A[i * (i + 1) / 2 + i];
            }
            for (int i = NB - 1; i >= 0; --i) {  // L^T z = y
                double s = yv[i];
                for (int q = i + 1; q < NB; ++q) s -= A[q * (q + 1) / 2 + i] * z[q];
                z[i] = s / A[i * (i + 1) / 2 + i];
            }
        }
        for (int iz = lo[2]; iz <= hi[2]; ++iz)
            for (int iy = lo[1]; iy <= hi[1]; ++iy) {
                const int64_t row = ((int64_t)iz * G.nc[1] + iy) * G.nc[0];
                const int js = sd.cell_start[row + lo[0]], je = sd.cell_start[row + hi[0] + 1];
                for (int j = js; j < je; ++j) {
                    const double *r = sd.rec + (int64_t)j * REC;
                    const double d[3] = {__dsub_rn(r[0], p[0]), __dsub_rn(r[1], p[1]), __dsub_rn(r[2], p[2])};
                    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
                    if (!(r2 <= R2)) continue;
                    const double xi = (d[0] * t1[0] + d[1] * t1[1] + d[2] * t1[2]) * iR;
                    const double eta = (d[0] * t2[0] + d[1] * t2[1] + d[2] * t2[2]) * iR;
                    monomials4(xi, eta, phi);
                    if (pass == 0) {
                        ++cnt;
                        for (int i = 0; i < NB; ++i)
                            for (int q = 0; q <= i; ++q) A[i * (i + 1) / 2 + q] = fma(phi[i], phi[q], A[i * (i + 1) / 2 + q]);
                    } else {
                        double wj = 0.0;
                        for (int i = 0; i < NB; ++i) wj = fma(phi[i], z[i], wj);
                        const int64_t c = perm[j];
                        for (int a = 0; a < 3; ++a) val[a] = fma(wj, vals[3 * c + a], val[a]);
                    }
                }
            }
        if (pass == 1)
            for (int a = 0; a < 3; ++a) out[3 * m + a] = val[a];
    }
}

__global__ void k_axpby(int64_t n, double a, const double *__restrict__ x, double b, double *__restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = fma(a, x[i], b * y[i]);
}

constexpr int DOT_BLOCKS = 304;  // 2 per SM of a 152-SM part
constexpr int DOT_THREADS = 256;

__global__ void __launch_bounds__(DOT_THREADS) k_dot_partial(int64_t n, const double *__restrict__ x,
                                                             const double *__restrict__ y, double *__restrict__ part) {
    __shared__ double s[DOT_THREADS];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * DOT_THREADS + threadIdx.x; i < n; i += (int64_t)DOT_BLOCKS * DOT_THREADS)
        acc = fma(x[i], y[i], acc);
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = DOT_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void __launch_bounds__(DOT_THREADS) k_dot_final(const double *__restrict__ part, double *__restrict__ out) {
    __shared__ double s[DOT_THREADS];
    double acc = 0.0;
    for (int i = threadIdx.x; i < DOT_BLOCKS; i += DOT_THREADS) acc += part[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = DOT_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

struct Dot {
    double *part = nullptr, *res = nullptr;
    cudaStream_t st;
    cudaError_t e = cudaSuccess;
    double operator()(int64_t n, const double *x, const double *y) {
        if (e != cudaSuccess) return 0.0;
        k_dot_partial<<<DOT_BLOCKS, DOT_THREADS, 0, st>>>(n, x, y, part);
        k_dot_final<<<1, DOT_THREADS, 0, st>>>(part, res);
        double h = 0.0;
        e = cudaMemcpyAsync(&h, res, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        return h;
    }
};

}  // namespace
}  // namespace ers

using namespace ers;

extern "C" {

int ers_node_interp(const ers_surface *s, const double *vals, const double *x0, const double *n0, int64_t M,
                    double *out, void *stream) {
    clear_error();
    if (!s) return fail(ERS_E_INVAL, "ers_node_interp: NULL surface");
    if (M < 0) return fail(ERS_E_INVAL, "ers_node_interp: M < 0");
    if (M == 0) return ERS_OK;
    if (!vals || !x0 || !n0 || !out) return fail(ERS_E_INVAL, "ers_node_interp: NULL array");
    const unsigned g = (unsigned)((M + 127) / 128);
    k_node_interp<<<g, 128, 0, (cudaStream_t)stream>>>(surf_dev(s), s->perm, INTERP_R * s->h, vals, x0, n0, M, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "ers_node_interp");
    return ERS_OK;
}

int ers_vec_axpby(int64_t n, double a, const double *x, double b, double *y, void *stream) {
    clear_error();
    if (n < 0 || (n > 0 && (!x || !y))) return fail(ERS_E_INVAL, "ers_vec_axpby: bad argument");
    if (n == 0) return ERS_OK;
    k_axpby<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, a, x, b, y);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "ers_vec_axpby");
    return ERS_OK;
}

int ers_gmres(int64_t n, ers_matvec_fn A, void *ctx, const double *b, double *x, double tol, int maxit, int *iters,
              double *relres, void *stream) {
    clear_error();
    if (n <= 0 || !A || !b || !x || maxit < 1 || !(tol > 0.0)) return fail(ERS_E_INVAL, "ers_gmres: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    double *V = nullptr, *w = nullptr, *part = nullptr, *res = nullptr;
    cudaError_t e = cudaMalloc(&V, sizeof(double) * (size_t)n * (maxit + 1));
    if (e == cudaSuccess) e = cudaMalloc(&w, sizeof(double) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&part, sizeof(double) * DOT_BLOCKS);
    if (e == cudaSuccess) e = cudaMalloc(&res, sizeof(double));
    auto cleanup = [&]() {
        for (void *p : {(void *)V, (void *)w, (void *)part, (void *)res})
            if (p) cudaFree(p);
    };
    if (e != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return fail(ERS_E_NOMEM, "ers_gmres: workspace");
    }
    Dot dot{part, res, st};
    const unsigned g = (unsigned)((n + 255) / 256);
    auto vec = [&](int k) { return V + (size_t)k * n; };
    std::vector<double> H((size_t)(maxit + 1) * maxit, 0.0), cs(maxit), sn(maxit), gv(maxit + 1, 0.0);
    auto Hk = [&](int i, int k) -> double & { return H[(size_t)i * maxit + k]; };
    const double beta = std::sqrt(dot(n, b, b));
    int m = 0, rc = ERS_OK;
    double rel = 1.0;
    if (dot.e == cudaSuccess && beta == 0.0) {
        e = cudaMemsetAsync(x, 0, sizeof(double) * n, st);
        rel = 0.0;
    } else if (dot.e == cudaSuccess) {
        gv[0] = beta;
        e = cudaMemsetAsync(vec(0), 0, sizeof(double) * n, st);
        k_axpby<<<g, 256, 0, st>>>(n, 1.0 / beta, b, 0.0, vec(0));
        for (int k = 0; k < maxit && e == cudaSuccess; ++k) {
            if ((rc = A(ctx, vec(k), w, stream)) != 0) {
                rc = rc < 0 ? rc : ERS_E_STATE;
                break;
            }
            for (int i = 0; i <= k; ++i) {  // modified Gram-Schmidt
                Hk(i, k) = dot(n, w, vec(i));
                k_axpby<<<g, 256, 0, st>>>(n, -Hk(i, k), vec(i), 1.0, w);
            }
            Hk(k + 1, k) = std::sqrt(dot(n, w, w));
            if (dot.e != cudaSuccess) break;
            e = cudaMemsetAsync(vec(k + 1), 0, sizeof(double) * n, st);
            if (Hk(k + 1, k) > 0.0) k_axpby<<<g, 256, 0, st>>>(n, 1.0 / Hk(k + 1, k), w, 0.0, vec(k + 1));
            for (int i = 0; i < k; ++i) {  // apply the previous rotations
                const double t = cs[i] * Hk(i, k) + sn[i] * Hk(i + 1, k);
                Hk(i + 1, k) = -sn[i] * Hk(i, k) + cs[i] * Hk(i + 1, k);
                Hk(i, k) = t;
            }
            const double den = std::hypot(Hk(k, k), Hk(k + 1, k));
            cs[k] = Hk(k, k) / den;
            sn[k] = Hk(k + 1, k) / den;
            Hk(k, k) = den;
            Hk(k + 1, k) = 0.0;
            gv[k + 1] = -sn[k] * gv[k];
            gv[k] = cs[k] * gv[k];
            rel = std::fabs(gv[k + 1]) / beta;
            m = k + 1;
            if (rel <= tol) break;
        }
        if (rc == ERS_OK && e == cudaSuccess && dot.e == cudaSuccess && m > 0) {
            std::vector<double> y(m);
            for (int i = m - 1; i >= 0; --i) {  // back substitution
                double s2 = gv[i];
                for (int q = i + 1; q < m; ++q) s2 -= Hk(i, q) * y[q];
                y[i] = s2 / Hk(i, i);
            }
            e = cudaMemsetAsync(x, 0, sizeof(double) * n, st);
            for (int i = 0; i < m && e == cudaSuccess; ++i) k_axpby<<<g, 256, 0, st>>>(n, y[i], vec(i), 1.0, x);
        }
    }
    if (e == cudaSuccess) e = dot.e;
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (rc != ERS_OK) return rc == ERS_E_STATE ? fail(ERS_E_STATE, "ers_gmres: the matvec callback failed") : rc;
    if (e != cudaSuccess) return cuda_fail(e, "ers_gmres");
    if (iters) *iters = m;
    if (relres) *relres = rel;
    return rel <= tol ? ERS_OK : ERS_W_NOT_CONVERGED;
}

}  // extern "C"
