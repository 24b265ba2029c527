// ers_eval_noalloc: the evaluation for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at the moment they evaluate: code running inside a
// pre-sized memory pool or under a host allocator that forbids growth, a plugin of a solver
// that owns all device memory, or a real-time loop where an allocation could stall or fail.
// ers_eval grows its work buffers on demand; this variant instead keeps the one work buffer it
// needs (the far-field partial sums, 6 doubles per target and source chunk) in a fixed file-scope device array
// and the smoothing-function table in another, so a call allocates nothing.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "ers_internal.h"

namespace ers {
namespace {

// Scratch shared by every call on a device: far-field partial sums, [chunks][M][6] doubles.
// 24 MiB => at most NOALLOC_MAX_M targets per call (then one source chunk; fewer targets
// leave room for more chunks, up to the split ers_eval uses).
constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)24 << 20;
constexpr int64_t NOALLOC_MAX_M = (int64_t)(NOALLOC_SCRATCH_BYTES / (6 * sizeof(double)));
constexpr size_t NOALLOC_TABLE_DOUBLES = TAB_DEV_BYTES / sizeof(double);
static_assert(TAB_DEV_BYTES % sizeof(double) == 0, "table layout");

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];
__device__ __align__(256) double g_noalloc_table[NOALLOC_TABLE_DOUBLES];

struct DevState {
    bool ready = false;
    double *scratch = nullptr;  // device address of g_noalloc_scratch on this device
    double *table = nullptr;    // device address of g_noalloc_table on this device
};
std::mutex g_mu;
DevState g_state[64];

// Once per device, with that device current: resolve the device addresses of the two arrays
// (in host code the array names are host-side stand-ins, not device addresses) and fill the
// table.  cudaMemcpyToSymbol copies synchronously; nothing is allocated.
int setup_device(int dev, DevState **out) {
    std::lock_guard<std::mutex> lk(g_mu);
    DevState &st = g_state[dev];
    if (!st.ready) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "ers_eval_noalloc: cudaGetSymbolAddress(scratch)");
        st.scratch = (double *)p;
        e = cudaGetSymbolAddress(&p, g_noalloc_table);
        if (e != cudaSuccess) return cuda_fail(e, "ers_eval_noalloc: cudaGetSymbolAddress(table)");
        st.table = (double *)p;
        std::vector<double> host(NOALLOC_TABLE_DOUBLES);
        sigma_table_device_layout(host.data());
        e = cudaMemcpyToSymbol(g_noalloc_table, host.data(), TAB_DEV_BYTES);
        if (e != cudaSuccess) return cuda_fail(e, "ers_eval_noalloc: cudaMemcpyToSymbol(table)");
        st.ready = true;
    }
    *out = &st;
    return ERS_OK;
}

}  // namespace
}  // namespace ers

using namespace ers;

extern "C" int ers_eval_noalloc(ers_surface *s, const ers_params *p, const double *y, int64_t M, const double *x0,
                                const double *n0, const double *b, const double *f0, const double *q0, double *u,
                                double *v, void *stream) {
    clear_error();
    if (!s) return fail(ERS_E_INVAL, "ers_eval_noalloc: NULL surface");
    int warn;
    int rc = check_params(s, p, &warn);
    if (rc == ERS_OK && (p->options & ERS_OPT_TREECODE))
        return fail(ERS_E_UNSUPPORTED, "ers_eval_noalloc: ERS_OPT_TREECODE is not supported (use ers_eval)");
    if (rc == ERS_OK && (p->options & ERS_OPT_FOUR_DELTA))
        return fail(ERS_E_UNSUPPORTED, "ers_eval_noalloc: ERS_OPT_FOUR_DELTA is not supported (use ers_eval)");
    if (rc == ERS_OK && (p->options & ERS_OPT_SHARP))
        return fail(ERS_E_UNSUPPORTED, "ers_eval_noalloc: ERS_OPT_SHARP is not supported (use ers_eval)");
    if (rc != ERS_OK) return rc;
    if (M < 0) return fail(ERS_E_INVAL, "ers_eval_noalloc: M < 0");
    if (M > NOALLOC_MAX_M)
        return fail(ERS_E_INVAL, "ers_eval_noalloc: M = " + std::to_string(M) + " exceeds the fixed scratch limit of " +
                                     std::to_string(NOALLOC_MAX_M) + " targets per call (use ers_eval or split the targets)");
    const bool sl = p->layers & ERS_LAYER_SL, dl = p->layers & ERS_LAYER_DL;
    if (sl && !s->has_f) return fail(ERS_E_STATE, "ers_eval_noalloc: single layer requested before a density f was set");
    if (dl && !s->has_q) return fail(ERS_E_STATE, "ers_eval_noalloc: double layer requested before a density q was set");
    if (M == 0) return warn;
    if (!y || !x0 || !n0 || !b)
        return fail(ERS_E_INVAL, "ers_eval_noalloc: y, x0, n0 and b are required (x0, n0, b from ers_closest_point)");
    if (sl && (!f0 || !u)) return fail(ERS_E_INVAL, "ers_eval_noalloc: single layer needs f0 and u");
    if (dl && (!q0 || !v)) return fail(ERS_E_INVAL, "ers_eval_noalloc: double layer needs q0 and v");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "ers_eval_noalloc: cudaGetDevice");
    if (dev != s->device || dev < 0 || dev >= 64)
        return fail(ERS_E_INVAL, "ers_eval_noalloc: the current device is not the surface's device");
    DevState *st = nullptr;
    if ((rc = setup_device(dev, &st)) != ERS_OK) return rc;

    EvalArgs a{};
    a.s = s;
    a.sd = surf_dev(s);
    a.y = y;
    a.x0 = x0;
    a.n0 = n0;
    a.b = b;
    a.f0 = f0;
    a.q0 = q0;
    a.M = M;
    a.u = u;
    a.v = v;
    for (int k = 0; k < 3; ++k) a.rho[k] = p->rho[k];
    a.cutoff_t = p->cutoff_t;
    a.Rc = p->cutoff_t * p->rho[2] * s->h;
    a.precision = p->precision;
    a.layers = p->layers;
    a.stream = (cudaStream_t)stream;
    // The far-field work split of ers_eval (target blocks x source chunks, about 16 CTAs per SM),
    // with the chunk count capped so that the partial sums, 6 doubles per target and chunk, fit
    // in the fixed scratch array: chunks <= NOALLOC_MAX_M / M.
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tpc = p->precision == ERS_PREC_MIXED ? 512 : 256;  // targets per far-field CTA
    const int64_t tb = (M + tpc - 1) / tpc;
    int64_t chunks = (16LL * nsm + tb - 1) / tb;
    chunks = std::max<int64_t>(1, std::min<int64_t>(chunks, std::max<int64_t>(1, s->N / (4 * TS32))));
    chunks = std::min<int64_t>(chunks, std::max<int64_t>(1, NOALLOC_MAX_M / M));
    int64_t clen = (s->N + chunks - 1) / chunks;
    clen = (clen + TS32 - 1) / TS32 * TS32;
    chunks = (s->N + clen - 1) / clen;
    a.part = st->scratch;  // every (chunk, target) partial sum is written by the far kernel before use
    a.chunks = (int)chunks;
    a.chunk_len = clen;
    a.counters = nullptr;  // ers_last_counts is not updated by this entry point
    e = (p->precision == ERS_PREC_MIXED) ? launch_far32(a) : launch_far64(a);
    if (e != cudaSuccess) return cuda_fail(e, "ers_eval_noalloc: far-field kernel");
    e = launch_near(a, st->table);
    if (e != cudaSuccess) return cuda_fail(e, "ers_eval_noalloc: near-field kernel");
    return warn;
}
