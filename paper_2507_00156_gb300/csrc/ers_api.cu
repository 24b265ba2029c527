// C ABI of the library (include/ers.h): argument checking, surface set-up, work buffers and
// the launch sequence closest point -> far field -> near field + extrapolation.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "ers_internal.h"

namespace ers {

namespace {
thread_local std::string g_err;
constexpr int CELL_H = 6;  // cell width of the sorting grid, in units of h

template <class T>
cudaError_t dmalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, sizeof(T) * count);
}

bool finite3(const double *v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

}  // namespace

int grow(Scratch &s, size_t bytes) {
    if (s.bytes >= bytes) return ERS_OK;
    if (s.ptr) cudaFree(s.ptr);
    s.ptr = nullptr;
    s.bytes = 0;
    cudaError_t e = cudaMalloc(&s.ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ERS_E_NOMEM, std::string("device allocation of work buffer failed: ") + cudaGetErrorString(e));
    }
    s.bytes = bytes;
    return ERS_OK;
}

namespace {

void free_surface(ers_surface *s) {
    if (!s) return;
    void *ptrs[] = {s->x, s->n, s->w, s->perm, s->rec, s->rec32, s->recp, s->tilec, s->xs32, s->fq, s->cell_start, s->cell_rank,
                    s->okeys.ptr, s->oorder.ptr, s->ohist.ptr,
                    s->part.ptr, s->cp.ptr, s->host_io.ptr, s->counts.ptr, s->densp.ptr, s->dens32.ptr,
                    s->fitw.ptr};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    tree_free(s);
    for (cudaEvent_t e : s->ev)
        if (e) cudaEventDestroy(e);
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->ev_join) cudaEventDestroy(s->ev_join);
    if (s->side) cudaStreamDestroy(s->side);
    delete s;
}

std::mutex g_tab_mu;
const double *g_tab_dev[64] = {nullptr};
const double *g_tabs_dev[64] = {nullptr};  // sigma# (on-surface) table per device
}  // namespace

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}
int cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return ERS_E_CUDA;
}
void clear_error() { g_err.clear(); }

const double *sigma_table_dev(int *err) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        *err = cuda_fail(e == cudaSuccess ? cudaErrorInvalidDevice : e, "cudaGetDevice");
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_tab_mu);
    if (!g_tab_dev[dev]) {
        std::vector<double> host(TAB_DEV_BYTES / sizeof(double));
        sigma_table_device_layout(host.data());
        double *d = nullptr;
        e = cudaMalloc(&d, TAB_DEV_BYTES);
        if (e == cudaSuccess) e = cudaMemcpy(d, host.data(), TAB_DEV_BYTES, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            if (d) cudaFree(d);
            *err = cuda_fail(e, "uploading the smoothing-function table");
            return nullptr;
        }
        g_tab_dev[dev] = d;
    }
    *err = ERS_OK;
    return g_tab_dev[dev];
}

const double *sigma_sharp_table_dev(int *err) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        *err = cuda_fail(e == cudaSuccess ? cudaErrorInvalidDevice : e, "cudaGetDevice");
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_tab_mu);
    if (!g_tabs_dev[dev]) {
        std::vector<double> host(SH_DEV_BYTES / sizeof(double));
        sigma_sharp_table_device_layout(host.data());
        double *d = nullptr;
        e = cudaMalloc(&d, SH_DEV_BYTES);
        if (e == cudaSuccess) e = cudaMemcpy(d, host.data(), SH_DEV_BYTES, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            if (d) cudaFree(d);
            *err = cuda_fail(e, "uploading the on-surface smoothing-function table");
            return nullptr;
        }
        g_tabs_dev[dev] = d;
    }
    *err = ERS_OK;
    return g_tabs_dev[dev];
}

int build_surface(const ers_shape *shape, double h, ers_surface **out) {
    if (!shape || !out) return fail(ERS_E_INVAL, "ers_build_surface: NULL argument");
    *out = nullptr;
    if (!(h > 0.0) || !std::isfinite(h)) return fail(ERS_E_INVAL, "ers_build_surface: h must be finite and > 0");
    if (!finite3(shape->center) || !finite3(shape->axes))
        return fail(ERS_E_INVAL, "ers_build_surface: non-finite shape");
    for (int i = 0; i < 3; ++i)
        if (!(shape->axes[i] > 0.0)) return fail(ERS_E_INVAL, "ers_build_surface: axes must be > 0");
    double amax = std::max(shape->axes[0], std::max(shape->axes[1], shape->axes[2]));
    if (amax / h > 1e5) return fail(ERS_E_UNSUPPORTED, "ers_build_surface: more than 1e5 lattice lines per axis");

    std::vector<double> xs, ns, ws;
    const int64_t N = quadrature(shape->center, shape->axes, h, &xs, &ns, &ws);
    if (N <= 0) return fail(ERS_E_INVAL, "ers_build_surface: the rule produced no node");
    if (N > (int64_t)1 << 30) return fail(ERS_E_UNSUPPORTED, "ers_build_surface: more than 2^30 nodes");

    ers_surface *s = new (std::nothrow) ers_surface();
    if (!s) return fail(ERS_E_NOMEM, "ers_build_surface: host allocation failed");
    cudaGetDevice(&s->device);
    {
        cudaError_t e = cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            free_surface(s);
            return cuda_fail(e, "ers_build_surface: stream/event creation");
        }
    }
    for (int i = 0; i < 3; ++i) {
        s->c[i] = shape->center[i];
        s->a[i] = shape->axes[i];
    }
    s->h = h;
    s->N = N;
    s->is_sphere = shape->axes[0] == shape->axes[1] && shape->axes[1] == shape->axes[2];

    // sorting grid
    Grid &G = s->grid;
    G.cw = CELL_H * h;
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = hi[a] = xs[a];
        for (int64_t i = 1; i < N; ++i) {
            lo[a] = std::min(lo[a], xs[3 * i + a]);
            hi[a] = std::max(hi[a], xs[3 * i + a]);
        }
        G.origin[a] = lo[a] - 0.5 * G.cw;
        G.nc[a] = (int)std::floor((hi[a] - G.origin[a]) / G.cw) + 2;
    }
    G.ncell = (int64_t)G.nc[0] * G.nc[1] * G.nc[2];
    if (G.ncell > ((int64_t)1 << 31) - 2) {
        free_surface(s);
        return fail(ERS_E_UNSUPPORTED, "ers_build_surface: sorting grid too large");
    }
    std::vector<int64_t> cell(N);
    for (int64_t i = 0; i < N; ++i) {
        int64_t id = 0;
        for (int a = 2; a >= 0; --a) {
            int ia = (int)std::floor((xs[3 * i + a] - G.origin[a]) / G.cw);
            ia = std::min(std::max(ia, 0), G.nc[a] - 1);
            id = id * G.nc[a] + ia;
        }
        cell[i] = id;
    }
    std::vector<int> perm(N);
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int p, int q) { return cell[p] < cell[q]; });
    std::vector<int> cstart(G.ncell + 1, 0);
    for (int64_t i = 0; i < N; ++i) cstart[cell[i] + 1]++;
    for (int64_t c = 0; c < G.ncell; ++c) cstart[c + 1] += cstart[c];

    std::vector<double> rec((size_t)N * REC, 0.0);
    std::vector<float> rec32((size_t)N * REC, 0.0f);
    std::vector<float> recp((size_t)N * NREC, 0.0f);
    std::vector<float4> xs32(N);
    s->ntile32 = (N + TS32 - 1) / TS32;
    std::vector<float> tilec((size_t)s->ntile32 * 4, 0.0f);
    for (int64_t t = 0; t < s->ntile32; ++t) {
        const int64_t j0 = t * TS32, j1 = std::min(N, j0 + TS32);
        double cm[3] = {0, 0, 0};
        for (int64_t j = j0; j < j1; ++j)
            for (int a = 0; a < 3; ++a) cm[a] += xs[3 * (int64_t)perm[j] + a];
        for (int a = 0; a < 3; ++a) tilec[4 * t + a] = (float)(cm[a] / (double)(j1 - j0));
        for (int64_t j = j0; j < j1; ++j) {
            const int64_t i = perm[j];
            for (int a = 0; a < 3; ++a) {
                const double xv = xs[3 * i + a];
                const double wn = ws[i] * ns[3 * i + a];
                rec[j * REC + R_X + a] = xv;
                rec[j * REC + R_WN + a] = wn;
                rec32[j * REC + R_X + a] = (float)(xv - (double)tilec[4 * t + a]);
                rec32[j * REC + R_WN + a] = (float)wn;
                std::memcpy(&recp[j * NREC + 2 * a], &xv, sizeof(double));
                const float wh = (float)wn;
                recp[j * NREC + NR_WN + 2 * a] = wh;
                recp[j * NREC + NR_WN + 2 * a + 1] = (float)(wn - (double)wh);
            }
            xs32[j] = make_float4((float)xs[3 * i], (float)xs[3 * i + 1], (float)xs[3 * i + 2], 0.0f);
        }
    }

    cudaError_t e = cudaSuccess;
#define ERS_TRY(call)                 \
    do {                              \
        if (e == cudaSuccess) e = (call); \
    } while (0)
    ERS_TRY(dmalloc(&s->x, 3 * N));
    ERS_TRY(dmalloc(&s->n, 3 * N));
    ERS_TRY(dmalloc(&s->w, N));
    ERS_TRY(dmalloc(&s->perm, N));
    ERS_TRY(dmalloc(&s->rec, (size_t)N * REC));
    ERS_TRY(dmalloc(&s->rec32, (size_t)N * REC));
    ERS_TRY(dmalloc(&s->recp, (size_t)N * NREC));
    ERS_TRY(dmalloc(&s->tilec, (size_t)s->ntile32 * 4));
    ERS_TRY(dmalloc(&s->xs32, N));
    ERS_TRY(dmalloc(&s->fq, (size_t)N * 6));
    ERS_TRY(dmalloc(&s->cell_start, G.ncell + 1));
    ERS_TRY(dmalloc(&s->cell_rank, G.ncell));
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_surface(s);
        return fail(ERS_E_NOMEM, std::string("ers_build_surface: device allocation failed: ") + cudaGetErrorString(e));
    }
    ERS_TRY(cudaMemcpy(s->x, xs.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice));
    ERS_TRY(cudaMemcpy(s->n, ns.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice));
    ERS_TRY(cudaMemcpy(s->w, ws.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
    ERS_TRY(cudaMemcpy(s->perm, perm.data(), sizeof(int) * N, cudaMemcpyHostToDevice));
    ERS_TRY(cudaMemcpy(s->rec, rec.data(), sizeof(double) * N * REC, cudaMemcpyHostToDevice));
    ERS_TRY(cudaMemcpy(s->rec32, rec32.data(), sizeof(float) * N * REC, cudaMemcpyHostToDevice));
    ERS_TRY(cudaMemcpy(s->recp, recp.data(), sizeof(float) * N * NREC, cudaMemcpyHostToDevice));
    ERS_TRY(cudaMemcpy(s->tilec, tilec.data(), sizeof(float) * s->ntile32 * 4, cudaMemcpyHostToDevice));
    ERS_TRY(cudaMemcpy(s->xs32, xs32.data(), sizeof(float4) * N, cudaMemcpyHostToDevice));
    ERS_TRY(cudaMemcpy(s->cell_start, cstart.data(), sizeof(int) * (G.ncell + 1), cudaMemcpyHostToDevice));
    {
        const std::vector<int> rank = morton_cell_rank(G);
        ERS_TRY(cudaMemcpy(s->cell_rank, rank.data(), sizeof(int) * G.ncell, cudaMemcpyHostToDevice));
    }
#undef ERS_TRY
    if (e != cudaSuccess) {
        free_surface(s);
        return cuda_fail(e, "ers_build_surface: upload");
    }
    *out = s;
    return ERS_OK;
}

// The fourth rho of ERS_OPT_FOUR_DELTA: rho4, or 2 rho[2] - rho[1] (the next of an evenly spaced set).
double rho4_of(const ers_params *p) { return p->rho4 > 0.0 ? p->rho4 : 2.0 * p->rho[2] - p->rho[1]; }

int check_params(const ers_surface *s, const ers_params *p, int *warn) {
    *warn = ERS_OK;
    if (!p) return fail(ERS_E_INVAL, "NULL params");
    for (int k = 0; k < 3; ++k)
        if (!(p->rho[k] > 0.0) || !std::isfinite(p->rho[k])) return fail(ERS_E_INVAL, "rho must be finite and > 0");
    if (!(p->rho[0] < p->rho[1] && p->rho[1] < p->rho[2])) return fail(ERS_E_INVAL, "rho must be strictly increasing");
    if (p->options & ERS_OPT_FOUR_DELTA) {
        if (!std::isfinite(p->rho4) || p->rho4 < 0.0 || (p->rho4 > 0.0 && !(p->rho4 > p->rho[2])))
            return fail(ERS_E_INVAL, "rho4 must be 0 or finite and > rho[2]");
    }
    if (!(p->cutoff_t > 0.0) || !std::isfinite(p->cutoff_t)) return fail(ERS_E_INVAL, "cutoff_t must be finite and > 0");
    if (p->cutoff_t > 8.0) return fail(ERS_E_UNSUPPORTED, "cutoff_t above 8 is outside the interpolation table");
    if (p->precision != ERS_PREC_FP64 && p->precision != ERS_PREC_MIXED)
        return fail(ERS_E_INVAL, "precision must be ERS_PREC_FP64 or ERS_PREC_MIXED");
    if (p->layers < 1 || p->layers > 3) return fail(ERS_E_INVAL, "layers must be a non-empty mask of SL/DL");
    if (p->options & ~(ERS_OPT_CONCURRENT | ERS_OPT_SHARP | ERS_OPT_FOUR_DELTA | ERS_OPT_TREECODE))
        return fail(ERS_E_INVAL, "unknown bit in options");
    if (p->options & ERS_OPT_TREECODE) {
        if (!(p->tree_theta >= 0.0 && p->tree_theta < 1.0))
            return fail(ERS_E_INVAL, "tree_theta must be in (0, 1), or 0 for the default");
        if (p->tree_n0 < 0) return fail(ERS_E_INVAL, "tree_n0 must be >= 1, or 0 for the default");
        if (p->tree_p < 0 || p->tree_p > TREE_PMAX) return fail(ERS_E_INVAL, "tree_p must be in 1..16, or 0 for the default");
    }
    if (!(p->rho_sharp >= 0.0) || !std::isfinite(p->rho_sharp)) return fail(ERS_E_INVAL, "rho_sharp must be finite and >= 0");
    if (p->cutoff_t < 6.0) *warn = ERS_W_CUTOFF;
    (void)s;
    return ERS_OK;
}

// CTAs per SM of the far (mixed) and near kernels: [0], [1] when they run concurrently,
// [2], [3] when serial (0 = uncapped).  Changed only by the tuning hook below.
int g_caps[4] = {1, 1, 0, 0};

// ndelta = 3: the method (Eq. (extrap_eqn)); ndelta = 2: the two-delta sums of the learned closure,
// near radius cutoff_t * delta_1, per-target gamma written to `gamma` (may be NULL); ndelta = 1:
// the single regularized sum with delta_0, near radius cutoff_t * delta_0.
int eval_impl(ers_surface *s, const ers_params *p, const double *y, int64_t M, const double *x0, const double *n0,
              const double *b, const double *f0, const double *q0, double *u, double *v, void *stream, int ndelta,
              double *gamma, bool near_only = false) {
    clear_error();
    if (!s) return fail(ERS_E_INVAL, "ers_eval: NULL surface");
    int warn;
    int rc = check_params(s, p, &warn);
    if (rc != ERS_OK) return rc;
    if (M < 0) return fail(ERS_E_INVAL, "ers_eval: M < 0");
    if (M > ((int64_t)1 << 31) - 64) return fail(ERS_E_UNSUPPORTED, "ers_eval: M above 2^31 - 64");
    const bool sl = p->layers & ERS_LAYER_SL, dl = p->layers & ERS_LAYER_DL;
    if (sl && !s->has_f) return fail(ERS_E_STATE, "ers_eval: single layer requested before a density f was set");
    if (dl && !s->has_q) return fail(ERS_E_STATE, "ers_eval: double layer requested before a density q was set");
    const int ncp = (x0 != nullptr) + (n0 != nullptr) + (b != nullptr);
    if (ncp != 0 && ncp != 3) return fail(ERS_E_INVAL, "ers_eval: give all of x0, n0, b or none");
    if (M == 0) return warn;
    if (!y) return fail(ERS_E_INVAL, "ers_eval: NULL targets");
    if (sl && (!f0 || !u)) return fail(ERS_E_INVAL, "ers_eval: single layer needs f0 and u");
    if (dl && (!q0 || !v)) return fail(ERS_E_INVAL, "ers_eval: double layer needs q0 and v");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != s->device) return fail(ERS_E_INVAL, "ers_eval: the current device is not the surface's device");
    int err;
    const double *tab = sigma_table_dev(&err);
    if (!tab) return err;

    EvalArgs a{};
    a.s = s;
    a.sd = surf_dev(s);
    a.y = y;
    a.M = M;
    a.f0 = f0;
    a.q0 = q0;
    a.u = u;
    a.v = v;
    if (ndelta == 3 && (p->options & ERS_OPT_FOUR_DELTA)) ndelta = 4;
    for (int k = 0; k < 3; ++k) a.rho[k] = p->rho[k];
    a.rho[3] = ndelta == 4 ? rho4_of(p) : 0.0;
    a.cutoff_t = p->cutoff_t;
    // near radius cutoff_t delta_{K-1}; the near-field-only sums of fewer deltas extend to the
    // three-delta radius (beyond cutoff_t delta_{K-1} every s_p is 1 and the weights sum to 1, so
    // the extension is the plain sum there), so that they differ from the three-delta ones by
    // the difference of the two methods, whose far fields then coincide
    a.Rc = p->cutoff_t * a.rho[(near_only ? std::max(ndelta, 3) : ndelta) - 1] * s->h;
    a.ndelta = ndelta;
    a.gamma = gamma;
    if ((p->options & ERS_OPT_SHARP) && ndelta >= 3) {  // on-surface targets: s#_p of Sec. 2.1
        a.sharp = true;
        a.rho_sharp = p->rho_sharp > 0.0 ? p->rho_sharp : p->rho[1];
        a.dsharp = a.rho_sharp * s->h;
        a.Rc_sharp = p->cutoff_t * a.dsharp;
        a.tab_sharp = sigma_sharp_table_dev(&err);
        if (!a.tab_sharp) return err;
    }
    a.precision = p->precision;
    a.layers = p->layers;
    a.stream = st;

    const bool prof = s->profile;
    if (prof) cudaEventRecord(s->ev[0], st);
    if (!x0) {
        if ((rc = grow(s->cp, sizeof(double) * 7 * (size_t)M)) != ERS_OK) return rc;
        double *cp = (double *)s->cp.ptr;
        a.x0 = cp;
        a.n0 = cp + 3 * M;
        a.b = cp + 6 * M;
        cudaError_t e = launch_closest(s, y, M, (double *)a.x0, (double *)a.n0, (double *)a.b, st);
        if (e != cudaSuccess) return cuda_fail(e, "closest-point kernel");
    } else {
        a.x0 = x0;
        a.n0 = n0;
        a.b = b;
    }

    const bool tree = (p->options & ERS_OPT_TREECODE) != 0;
    TreeParams tp{};
    if (tree) {
        treecode_defaults(s->h, &tp.theta, &tp.n0, &tp.p);
        if (p->tree_theta > 0.0) tp.theta = p->tree_theta;
        if (p->tree_n0 > 0) tp.n0 = p->tree_n0;
        if (p->tree_p > 0) tp.p = p->tree_p;
    }

    // far-field work split: target blocks x source chunks (chunks aligned to the FP32 tiles)
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tpc = p->precision == ERS_PREC_MIXED ? 512 : 256;  // targets per far-field CTA
    const int64_t tb = (M + tpc - 1) / tpc;
    int64_t chunks = (16LL * nsm + tb - 1) / tb;
    chunks = std::max<int64_t>(1, std::min<int64_t>(chunks, std::max<int64_t>(1, s->N / (4 * TS32))));
    int64_t clen = (s->N + chunks - 1) / chunks;
    clen = (clen + TS32 - 1) / TS32 * TS32;
    chunks = (s->N + clen - 1) / clen;
    if (tree) chunks = 1;  // the treecode writes one partial sum per target
    a.chunks = (int)chunks;
    a.chunk_len = clen;
    if (near_only) {  // no far-field partial sums: the near kernel adds none
        a.chunks = 0;
        a.part = nullptr;
    } else {
        if ((rc = grow(s->part, sizeof(double) * 6 * (size_t)M * chunks)) != ERS_OK) return rc;
        a.part = (double *)s->part.ptr;
    }
    if ((rc = grow(s->counts, sizeof(unsigned long long) * NCOUNTERS)) != ERS_OK) return rc;
    a.counters = (unsigned long long *)s->counts.ptr;
    cudaError_t e = cudaMemsetAsync(a.counters, 0, sizeof(unsigned long long) * NCOUNTERS, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");

    if (prof) cudaEventRecord(s->ev[1], st);
    // ERS_OPT_CONCURRENT: the far field (FP32 pipe) and the near field (FP64 pipe) run concurrently,
    // the far field on the surface's second stream.  Both grids are capped (FAR_CTAS_PER_SM and
    // NEAR_CTAS_PER_SM CTAs per SM, the far one also by its shared memory) so that both kernels
    // are resident on every SM whichever starts first; k_combine then adds the far partial sums.
    const bool overlap = !tree && p->precision == ERS_PREC_MIXED && (p->options & ERS_OPT_CONCURRENT);
    if (near_only) {  // no far field: its profile interval is empty
        if (prof) cudaEventRecord(s->ev[2], st);
        e = launch_near(a, tab, g_caps[3], nsm);
        if (e != cudaSuccess) return cuda_fail(e, "near-field kernel");
        if (prof) cudaEventRecord(s->ev[3], st);
    } else if (tree) {  // modified weights (when stale) and the walk, both in the far-field slot of the profile
        if ((rc = tree_prepare(s, tp.n0, tp.p, p->precision == ERS_PREC_MIXED, st)) != ERS_OK) return rc;
        e = launch_tree_far(a, tp);
        if (e != cudaSuccess) return cuda_fail(e, "treecode far-field kernel");
        if (prof) cudaEventRecord(s->ev[2], st);
        e = launch_near(a, tab, g_caps[3], nsm);
        if (e != cudaSuccess) return cuda_fail(e, "near-field kernel");
        if (prof) cudaEventRecord(s->ev[3], st);
    } else if (overlap) {
        const int FAR_CTAS_PER_SM = g_caps[0], NEAR_CTAS_PER_SM = g_caps[1];
        a.far_later = true;
        EvalArgs af = a;
        af.stream = s->side;
        if ((e = cudaEventRecord(s->ev_fork, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        if ((e = cudaStreamWaitEvent(s->side, s->ev_fork, 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
        e = launch_far32(af, FAR_CTAS_PER_SM, nsm);
        if (e != cudaSuccess) return cuda_fail(e, "far-field kernel");
        if (prof) cudaEventRecord(s->ev[2], s->side);
        if ((e = cudaEventRecord(s->ev_join, s->side)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        e = launch_near(a, tab, NEAR_CTAS_PER_SM, nsm);
        if (e != cudaSuccess) return cuda_fail(e, "near-field kernel");
        if (prof) cudaEventRecord(s->ev[3], st);
        if ((e = cudaStreamWaitEvent(st, s->ev_join, 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
        e = launch_combine(a);
        if (e != cudaSuccess) return cuda_fail(e, "combine kernel");
    } else {
        e = (p->precision == ERS_PREC_MIXED) ? launch_far32(a, g_caps[2], nsm) : launch_far64(a);
        if (e != cudaSuccess) return cuda_fail(e, "far-field kernel");
        if (prof) cudaEventRecord(s->ev[2], st);
        e = launch_near(a, tab, g_caps[3], nsm);
        if (e != cudaSuccess) return cuda_fail(e, "near-field kernel");
        if (prof) cudaEventRecord(s->ev[3], st);
    }
    if (prof) {
        cudaEventRecord(s->ev[4], st);
        s->profiled = true;
        s->prof_closest = (x0 == nullptr);
        s->prof_overlap = overlap;
    }
    s->last_counts[0] = -1;
    s->last_counts[2] = M * s->N;
    s->last_stream = st;
    return warn;
}

int eval(ers_surface *s, const ers_params *p, const double *y, int64_t M, const double *x0, const double *n0,
         const double *b, const double *f0, const double *q0, double *u, double *v, void *stream) {
    return eval_impl(s, p, y, M, x0, n0, b, f0, q0, u, v, stream, 3, nullptr);
}

int eval_few_delta(ers_surface *s, const ers_params *p, const double *y, int64_t M, const double *x0,
                   const double *n0, const double *b, const double *f0, const double *q0, double *u, double *v,
                   double *gamma, int ndelta, cudaStream_t st) {
    try {
        return eval_impl(s, p, y, M, x0, n0, b, f0, q0, u, v, (void *)st, ndelta, gamma);
    } catch (...) {
        return fail(ERS_E_NOMEM, "two-delta evaluation: host exception");
    }
}

int eval_near_only(ers_surface *s, const ers_params *p, const double *y, int64_t M, const double *x0,
                   const double *n0, const double *b, const double *f0, const double *q0, double *u, double *v,
                   int ndelta, cudaStream_t st) {
    try {
        return eval_impl(s, p, y, M, x0, n0, b, f0, q0, u, v, (void *)st, ndelta, nullptr, true);
    } catch (...) {
        return fail(ERS_E_NOMEM, "near-field evaluation: host exception");
    }
}

}  // namespace ers

using namespace ers;

extern "C" {

int ers_build_surface(const ers_shape *shape, double h, ers_surface **out) {
    clear_error();
    try {
        return build_surface(shape, h, out);
    } catch (...) {
        return fail(ERS_E_NOMEM, "ers_build_surface: host exception");
    }
}

int ers_surface_free(ers_surface *s) {
    clear_error();
    free_surface(s);
    return ERS_OK;
}

int ers_surface_info(const ers_surface *s, int64_t *N, double *h, const double **x, const double **n,
                     const double **w) {
    clear_error();
    if (!s) return fail(ERS_E_INVAL, "ers_surface_info: NULL surface");
    if (N) *N = s->N;
    if (h) *h = s->h;
    if (x) *x = s->x;
    if (n) *n = s->n;
    if (w) *w = s->w;
    return ERS_OK;
}

int ers_set_density(ers_surface *s, const double *f, const double *q, void *stream) {
    clear_error();
    if (!s) return fail(ERS_E_INVAL, "ers_set_density: NULL surface");
    if (!f && !q) return ERS_OK;
    cudaError_t e = launch_density(s, f, q, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "density kernel");
    if (f) s->has_f = true;
    if (q) s->has_q = true;
    ++s->dens_version;
    return ERS_OK;
}

int ers_closest_point(const ers_surface *s, const double *y, int64_t M, double *x0, double *n0, double *b,
                      void *stream) {
    clear_error();
    if (!s) return fail(ERS_E_INVAL, "ers_closest_point: NULL surface");
    if (M < 0) return fail(ERS_E_INVAL, "ers_closest_point: M < 0");
    if (M == 0) return ERS_OK;
    if (!y || !x0 || !n0 || !b) return fail(ERS_E_INVAL, "ers_closest_point: NULL array");
    cudaError_t e = launch_closest(s, y, M, x0, n0, b, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "closest-point kernel");
    return ERS_OK;
}

int ers_eval(ers_surface *s, const ers_params *p, const double *y, int64_t M, const double *x0, const double *n0,
             const double *b, const double *f0, const double *q0, double *u, double *v, void *stream) {
    try {
        return eval(s, p, y, M, x0, n0, b, f0, q0, u, v, stream);
    } catch (...) {
        return fail(ERS_E_NOMEM, "ers_eval: host exception");
    }
}

int ers_eval_SL(ers_surface *s, const ers_params *p, const double *y, int64_t M, const double *x0,
                const double *n0, const double *b, const double *f0, double *u, void *stream) {
    if (!p) return fail(ERS_E_INVAL, "NULL params");
    ers_params q = *p;
    q.layers = ERS_LAYER_SL;
    return ers_eval(s, &q, y, M, x0, n0, b, f0, nullptr, u, nullptr, stream);
}

int ers_eval_DL(ers_surface *s, const ers_params *p, const double *y, int64_t M, const double *x0,
                const double *n0, const double *b, const double *q0, double *v, void *stream) {
    if (!p) return fail(ERS_E_INVAL, "NULL params");
    ers_params q = *p;
    q.layers = ERS_LAYER_DL;
    return ers_eval(s, &q, y, M, x0, n0, b, nullptr, q0, nullptr, v, stream);
}

int ers_eval_host(ers_surface *s, const ers_params *p, const double *y, int64_t M, const double *x0,
                  const double *n0, const double *b, const double *f0, const double *q0, double *u, double *v,
                  void *stream) {
    clear_error();
    if (!s || !p) return fail(ERS_E_INVAL, "ers_eval_host: NULL argument");
    if (M < 0) return fail(ERS_E_INVAL, "ers_eval_host: M < 0");
    if (M == 0) return ERS_OK;
    const bool sl = p->layers & ERS_LAYER_SL, dl = p->layers & ERS_LAYER_DL;
    const bool cp = x0 != nullptr;
    // layout of the staging buffer: y | f0 | q0 | x0 | n0 | b | u | v
    const size_t m3 = 3 * (size_t)M;
    size_t off_f0 = m3, off_q0 = off_f0 + m3, off_x0 = off_q0 + m3, off_n0 = off_x0 + m3, off_b = off_n0 + m3,
           off_u = off_b + M, off_v = off_u + m3, total = off_v + m3;
    int rc = grow(s->host_io, sizeof(double) * total);
    if (rc != ERS_OK) return rc;
    double *d = (double *)s->host_io.ptr;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(d, y, sizeof(double) * m3, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && sl && f0) e = cudaMemcpyAsync(d + off_f0, f0, sizeof(double) * m3, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && dl && q0) e = cudaMemcpyAsync(d + off_q0, q0, sizeof(double) * m3, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && cp) {
        if (!n0 || !b) return fail(ERS_E_INVAL, "ers_eval_host: give all of x0, n0, b or none");
        e = cudaMemcpyAsync(d + off_x0, x0, sizeof(double) * m3, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d + off_n0, n0, sizeof(double) * m3, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d + off_b, b, sizeof(double) * M, cudaMemcpyHostToDevice, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "ers_eval_host: host-to-device copy");
    rc = ers_eval(s, p, d, M, cp ? d + off_x0 : nullptr, cp ? d + off_n0 : nullptr, cp ? d + off_b : nullptr,
                  (sl && f0) ? d + off_f0 : nullptr, (dl && q0) ? d + off_q0 : nullptr, sl ? d + off_u : nullptr,
                  dl ? d + off_v : nullptr, stream);
    if (rc < 0) return rc;
    if (sl && u) e = cudaMemcpyAsync(u, d + off_u, sizeof(double) * m3, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && dl && v) e = cudaMemcpyAsync(v, d + off_v, sizeof(double) * m3, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "ers_eval_host: device-to-host copy");
    return rc;
}

int ers_last_counts(ers_surface *s, int64_t *near_targets, int64_t *near_pairs, int64_t *far_pairs) {
    clear_error();
    if (!s) return fail(ERS_E_INVAL, "ers_last_counts: NULL surface");
    if (s->last_counts[0] == -1 && s->counts.ptr) {
        unsigned long long hc[NCOUNTERS] = {};
        cudaError_t e = cudaStreamSynchronize(s->last_stream);
        if (e == cudaSuccess) e = cudaMemcpy(hc, s->counts.ptr, sizeof hc, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "ers_last_counts");
        s->last_counts[0] = (int64_t)hc[0];
        s->last_counts[1] = (int64_t)hc[1];
        s->last_counts[2] -= (int64_t)hc[1];
        for (int c = 0; c < 4; ++c) s->last_dclass[c] = (int64_t)hc[2 + c];
        for (int c = 0; c < 3; ++c) s->last_class[c] = (int64_t)hc[6 + c];
        s->last_sharp = (int64_t)hc[9];
        s->last_dclass[4] = (int64_t)hc[10];
        s->last_class[3] = (int64_t)hc[11];
    }
    if (near_targets) *near_targets = s->last_counts[0];
    if (near_pairs) *near_pairs = s->last_counts[1];
    if (far_pairs) *far_pairs = s->last_counts[2];
    return ERS_OK;
}

// Tuning hook (not in the public header): CTAs per SM of the mixed far-field and near-field
// kernels, concurrent (far_c, near_c) and serial (far_s, near_s); 0 = uncapped in serial mode.
// Not thread-safe with respect to concurrent ers_eval calls.
extern "C" int ers_debug_set_caps(int far_c, int near_c, int far_s, int near_s) {
    if (far_c < 1 || near_c < 1 || far_c > 16 || near_c > 16 || far_s < 0 || near_s < 0 || far_s > 16 || near_s > 16)
        return ERS_E_INVAL;
    ers::g_caps[0] = far_c;
    ers::g_caps[1] = near_c;
    ers::g_caps[2] = far_s;
    ers::g_caps[3] = near_s;
    return ERS_OK;
}

// Test/benchmark hook (not in the public header): near pairs of the last ers_eval, valid after
// ers_last_counts.  out[0..2]: by the number of deltas with r > cutoff_t delta_k (0, 1, 2);
// out[3..6]: by the number of deltas on the direct-defect path (0..3); out[7]: near pairs of
// on-surface targets evaluated with the s#_p (ERS_OPT_SHARP; not in out[0..6]); with n >= 10,
// out[8]: 3 deltas beyond the cutoff, out[9]: 4 deltas on the defect path (ERS_OPT_FOUR_DELTA
// only).  n >= 8.
extern "C" int ers_debug_class_counts(ers_surface *s, int64_t *out, int n) {
    if (!s || !out || n < 8) return ERS_E_INVAL;
    for (int c = 0; c < 3; ++c) out[c] = s->last_class[c];
    for (int c = 0; c < 4; ++c) out[3 + c] = s->last_dclass[c];
    out[7] = s->last_sharp;
    if (n >= 10) {
        out[8] = s->last_class[3];
        out[9] = s->last_dclass[4];
    }
    return ERS_OK;
}

int ers_profile(ers_surface *s, int enable) {
    clear_error();
    if (!s) return fail(ERS_E_INVAL, "ers_profile: NULL surface");
    if (enable && !s->ev[0]) {
        for (cudaEvent_t &e : s->ev) {
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return cuda_fail(r, "ers_profile: cudaEventCreate");
        }
    }
    s->profile = enable != 0;
    return ERS_OK;
}

int ers_last_profile(ers_surface *s, double *ms_closest, double *ms_far, double *ms_near) {
    clear_error();
    if (!s) return fail(ERS_E_INVAL, "ers_last_profile: NULL surface");
    if (!s->profiled) return fail(ERS_E_STATE, "ers_last_profile: no profiled evaluation yet");
    cudaError_t e = cudaEventSynchronize(s->ev[4]);
    if (e != cudaSuccess) return cuda_fail(e, "ers_last_profile: cudaEventSynchronize");
    // serial: closest ev0-ev1, far ev1-ev2, near ev2-ev3; concurrent: far ev1-ev2 (second
    // stream), near ev1-ev3 (both from the fork); ev4 ends the evaluation
    const int pairs[3][2] = {{0, 1}, {1, 2}, {s->prof_overlap ? 1 : 2, 3}};
    float t[3] = {0, 0, 0};
    for (int i = 0; i < 3; ++i) {
        e = cudaEventElapsedTime(&t[i], s->ev[pairs[i][0]], s->ev[pairs[i][1]]);
        if (e != cudaSuccess) return cuda_fail(e, "ers_last_profile: cudaEventElapsedTime");
    }
    if (ms_closest) *ms_closest = s->prof_closest ? t[0] : 0.0;
    if (ms_far) *ms_far = t[1];
    if (ms_near) *ms_near = t[2];
    return ERS_OK;
}

int ers_treecode_defaults(double h, double *theta, int *n0, int *p) {
    clear_error();
    if (!(h > 0.0) || !std::isfinite(h)) return fail(ERS_E_INVAL, "ers_treecode_defaults: h must be finite and > 0");
    double t;
    int n, q;
    treecode_defaults(h, &t, &n, &q);
    if (theta) *theta = t;
    if (n0) *n0 = n;
    if (p) *p = q;
    return ERS_OK;
}

int ers_tree_stats(ers_surface *s, int64_t *out, int n) {
    clear_error();
    if (!s || !out || n < 5) return fail(ERS_E_INVAL, "ers_tree_stats: NULL argument or n < 5");
    return tree_stats(s, out);
}

const char *ers_last_error(void) { return g_err.c_str(); }

const char *ers_version(void) { return "ers-gb300 0.1 (sm_103a)"; }

}  // extern "C"
