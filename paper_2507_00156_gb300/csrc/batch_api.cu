// C ABI of the batched evaluation: several densities per surface and a persistent launch over
// many problems, captured in a CUDA graph (see k_batch.cu for the device side).
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "near_common.cuh"


struct ers_batch {
    int device = 0;
    int nrhs = 0;
    int nitems = 0;
    int grid = 0;
    ers::BatchProblemDev *probs = nullptr;
    ers::BatchItem *items = nullptr;
    unsigned *counter = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

using namespace ers;

namespace {
constexpr int BATCH_TARGETS = 128;  // targets per work item (one CTA)

void free_batch(ers_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->probs) cudaFree(b->probs);
    if (b->items) cudaFree(b->items);
    if (b->counter) cudaFree(b->counter);
    delete b;
}
}  // namespace

extern "C" {

int ers_set_density_multi(ers_surface *s, const double *f, const double *q, int nrhs, void *stream) {
    clear_error();
    if (!s) return fail(ERS_E_INVAL, "ers_set_density_multi: NULL surface");
    if (nrhs != 1 && nrhs != 2 && nrhs != 4 && nrhs != 8)
        return fail(ERS_E_INVAL, "ers_set_density_multi: nrhs must be 1, 2, 4 or 8");
    if (!f && !q) return fail(ERS_E_INVAL, "ers_set_density_multi: give f, q or both");
    const size_t n = (size_t)s->N * nrhs * 6;
    int rc = grow(s->densp, n * sizeof(float2));
    if (rc == ERS_OK) rc = grow(s->dens32, (size_t)s->N * batch_rec32_floats(nrhs) * sizeof(float));
    if (rc != ERS_OK) return rc;
    cudaError_t e = launch_density_multi(s->perm, s->w, s->rec32, f, q, s->N, nrhs, (float2 *)s->densp.ptr,
                                         (float *)s->dens32.ptr, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ers_set_density_multi: density kernel");
    s->nrhs_multi = nrhs;
    return ERS_OK;
}

int ers_batch_create(const ers_problem *probs, int nprob, const ers_params *p, int nrhs, ers_batch **out) {
    clear_error();
    if (!probs || !p || !out || nprob <= 0) return fail(ERS_E_INVAL, "ers_batch_create: NULL argument or nprob <= 0");
    *out = nullptr;
    int warn;
    int rc = check_params(probs[0].s, p, &warn);
    if (rc == ERS_OK && (p->options & ERS_OPT_TREECODE))
        return fail(ERS_E_UNSUPPORTED, "ers_batch_create: ERS_OPT_TREECODE is not supported (use ers_eval)");
    if (rc == ERS_OK && (p->options & ERS_OPT_FOUR_DELTA))
        return fail(ERS_E_UNSUPPORTED, "ers_batch_create: ERS_OPT_FOUR_DELTA is not supported (use ers_eval)");
    if (rc == ERS_OK && (p->options & ERS_OPT_SHARP))
        return fail(ERS_E_UNSUPPORTED, "ers_batch_create: ERS_OPT_SHARP is not supported (the batched kernel extrapolates)");
    if (rc != ERS_OK) return rc;
    if (p->precision != ERS_PREC_MIXED)
        return fail(ERS_E_UNSUPPORTED, "ers_batch_create: the batched path runs the mixed-precision far field only");
    if (nrhs != 1 && nrhs != 2 && nrhs != 4 && nrhs != 8)
        return fail(ERS_E_INVAL, "ers_batch_create: nrhs must be 1, 2, 4 or 8");
    int dev = -1;
    cudaGetDevice(&dev);
    const bool sl = p->layers & ERS_LAYER_SL, dl = p->layers & ERS_LAYER_DL;
    std::vector<BatchProblemDev> hp(nprob);
    std::vector<BatchItem> items;
    std::vector<int64_t> cost;
    for (int i = 0; i < nprob; ++i) {
        const ers_problem &q = probs[i];
        const std::string at = "ers_batch_create: problem " + std::to_string(i) + ": ";
        if (!q.s) return fail(ERS_E_INVAL, at + "NULL surface");
        if (q.s->device != dev) return fail(ERS_E_INVAL, at + "surface on another device");
        if (q.s->nrhs_multi != nrhs) return fail(ERS_E_STATE, at + "densities not set with ers_set_density_multi(nrhs)");
        if (q.M < 0 || q.M > ((int64_t)1 << 31) - 1024) return fail(ERS_E_INVAL, at + "bad M");
        if (q.M > 0 && (!q.y || !q.x0 || !q.n0 || !q.b)) return fail(ERS_E_INVAL, at + "y, x0, n0, b are required");
        if (q.M > 0 && sl && (!q.f0 || !q.u)) return fail(ERS_E_INVAL, at + "single layer needs f0 and u");
        if (q.M > 0 && dl && (!q.q0 || !q.v)) return fail(ERS_E_INVAL, at + "double layer needs q0 and v");
        BatchProblemDev &d = hp[i];
        d.sd = surf_dev(q.s);
        d.densp = (const float2 *)q.s->densp.ptr;
        d.dens32 = (const float *)q.s->dens32.ptr;
        d.y = q.y;
        d.x0 = q.x0;
        d.n0 = q.n0;
        d.b = q.b;
        d.f0 = q.f0;
        d.q0 = q.q0;
        d.u = q.u;
        d.v = q.v;
        d.M = q.M;
        d.Rc = p->cutoff_t * p->rho[2] * q.s->h;
        d.sp = nearc::scan_params(q.s, d.Rc, p->rho, p->cutoff_t);
        const int64_t nb = (q.M + BATCH_TARGETS - 1) / BATCH_TARGETS;
        for (int64_t t = 0; t < nb; ++t) {
            items.push_back({i, (int)t});
            cost.push_back(q.s->N);
        }
    }
    // largest items first (far-field work grows with the number of nodes)
    std::vector<size_t> order(items.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
    std::vector<BatchItem> sorted(items.size());
    for (size_t k = 0; k < order.size(); ++k) sorted[k] = items[order[k]];

    ers_batch *b = new (std::nothrow) ers_batch();
    if (!b) return fail(ERS_E_NOMEM, "ers_batch_create: host allocation failed");
    b->device = dev;
    b->nrhs = nrhs;
    b->nitems = (int)sorted.size();
    int err;
    const double *tab = sigma_table_dev(&err);
    if (!tab) {
        free_batch(b);
        return err;
    }
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    b->grid = std::max(1, std::min(batch_grid(nrhs, nsm), std::max(1, b->nitems)));
    cudaError_t e = cudaMalloc(&b->probs, sizeof(BatchProblemDev) * hp.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->items, sizeof(BatchItem) * std::max<size_t>(1, sorted.size()));
    if (e == cudaSuccess) e = cudaMalloc(&b->counter, sizeof(unsigned));
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_batch(b);
        return fail(ERS_E_NOMEM, std::string("ers_batch_create: device allocation failed: ") + cudaGetErrorString(e));
    }
    e = cudaMemcpy(b->probs, hp.data(), sizeof(BatchProblemDev) * hp.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !sorted.empty())
        e = cudaMemcpy(b->items, sorted.data(), sizeof(BatchItem) * sorted.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_fail(e, "ers_batch_create: upload");
    }
    // capture: reset the work counter, then one persistent launch
    cudaStream_t cs = nullptr;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e1 = cudaMemsetAsync(b->counter, 0, sizeof(unsigned), cs);
        cudaError_t e2 = e1 == cudaSuccess ? launch_batch(nrhs, b->probs, b->items, b->nitems, b->counter, p->rho,
                                                          p->layers, tab, b->grid, cs)
                                           : e1;
        e = cudaStreamEndCapture(cs, &b->graph);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_fail(e, "ers_batch_create: graph capture");
    }
    *out = b;
    return warn;
}

int ers_batch_launch(ers_batch *b, void *stream) {
    clear_error();
    if (!b) return fail(ERS_E_INVAL, "ers_batch_launch: NULL plan");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != b->device) return fail(ERS_E_INVAL, "ers_batch_launch: the current device is not the plan's device");
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ers_batch_launch: cudaGraphLaunch");
    return ERS_OK;
}

int ers_batch_info(const ers_batch *b, int *nitems, int *grid) {
    clear_error();
    if (!b) return fail(ERS_E_INVAL, "ers_batch_info: NULL plan");
    if (nitems) *nitems = b->nitems;
    if (grid) *grid = b->grid;
    return ERS_OK;
}

int ers_batch_free(ers_batch *b) {
    clear_error();
    free_batch(b);
    return ERS_OK;
}

}  // extern "C"
