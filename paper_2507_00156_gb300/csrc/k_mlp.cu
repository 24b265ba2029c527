// The closure network: an MLP 16 -> 64 -> 64 -> 64 -> 96 (5 inputs used: the local geometry;
// 3 J outputs used: the coefficients of a linear map from the J density jets of the sample to the
// three components of the correction), GELU after the three hidden layers, BF16 weights and
// activations with FP32 accumulation.  The head contracts the coefficients with the jets in FP32:
// c_e = sum_j A[e J + j] jet_j.
//
// Inference runs on the 5th-generation tensor cores: a CTA holds a tile of 128 samples; the
// activations (A operand) and the weights (B operand) sit in shared memory in the canonical
// K-major layout without swizzle (8 x 16-byte core matrices), one elected thread issues
// tcgen05.mma (M = 128, N = 64 or 96, K = 16 per instruction) into an FP32 accumulator in tensor
// memory, the four warps read it back with tcgen05.ld (warp w owns rows 32w..32w+31), add the
// bias, apply GELU, round to BF16 and write the next layer's A operand; after the last layer each
// thread contracts its row's coefficients with its sample's jets.
//
// Training runs in FP32 on the CUDA cores with the same BF16 rounding of weights, inputs and
// hidden activations in the forward pass (straight-through in the backward pass), so that the
// trained network is the one the tensor-core kernel evaluates.  The loss of a sample is
// w/2 |c - t|^2 with the target t and weight w of its training record.
#include <cuda_bf16.h>

#include "ers_internal.h"
#include "mlp.h"

namespace ers {
namespace mlp {
namespace {

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * __expf(-0.5f * x * x);
}

// ------------------------------------------------------------------------------------------
// tcgen05 / mbarrier wrappers (inline PTX)
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: at most `limit` polls; returns false when the limit was hit.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *mbar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i) {
        if (mbar_try_wait(mbar, parity)) return true;
        if (i > 64) __nanosleep(64);
    }
    return false;
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, no swizzle; lbo = byte distance between core matrices
// adjacent along K, sbo = between core matrices adjacent along M (or N).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, layout type 0 (no swizzle)
}
// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Offset in bytes of element (row, k) of a K-major tile with `rows` rows, no swizzle:
// [k block of 16][row group of 8][k half of 8][row % 8][k % 8], 2 bytes per element.
__device__ __forceinline__ uint32_t kmaj_off(int row, int k, int rows) {
    return (uint32_t)((k >> 4) * (rows * 32) + (row >> 3) * 256 + ((k >> 3) & 1) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

constexpr int TILE = 128;
constexpr uint32_t TMEM_COLS = 128;  // the last layer uses OUT = 96 columns
constexpr uint32_t WAIT_LIMIT = 1u << 22;

struct InferSmem {
    __align__(1024) unsigned char a[TILE * HID * 2];     // activations, K-major, 16 KB
    __align__(1024) unsigned char w1[HID * IN * 2];      // 2 KB
    __align__(1024) unsigned char w2[HID * HID * 2];     // 8 KB
    __align__(1024) unsigned char w3[HID * HID * 2];     // 8 KB
    __align__(1024) unsigned char w4[OUT * HID * 2];     // 2 KB
    float b1[HID], b2[HID], b3[HID], b4[OUT];
    uint64_t mbar;
    uint32_t tmem;
};

__device__ __forceinline__ void store_bf16(unsigned char *base, uint32_t off, float v) {
    *reinterpret_cast<__nv_bfloat16 *>(base + off) = __float2bfloat16_rn(v);
}

// Issue one layer: D[128 x N] = A[128 x K] * W[N x K]^T, K in steps of 16.
__device__ __forceinline__ void issue_layer(uint32_t d_tmem, const unsigned char *a, const unsigned char *w, int K,
                                            int N) {
    const uint32_t ia = smem_u32(a), iw = smem_u32(w);
    const uint32_t idesc = idesc_bf16(TILE, N);
    for (int kb = 0; kb < K / 16; ++kb) {
        const uint64_t ad = smem_desc(ia + kb * (TILE * 32), 128, 256);
        const uint64_t bd = smem_desc(iw + kb * (N * 32), 128, 256);
        mma_bf16(d_tmem, ad, bd, idesc, kb > 0 ? 1u : 0u);
    }
}

template <int NJ>
__global__ void __launch_bounds__(TILE) k_mlp_infer_tc(const float *__restrict__ params, const float *__restrict__ X,
                                                       int64_t n, float *__restrict__ Y, int *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    InferSmem &S = *reinterpret_cast<InferSmem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    // weights -> BF16 K-major tiles, biases FP32
    for (int i = t; i < HID * IN; i += TILE) store_bf16(S.w1, kmaj_off(i / IN, i % IN, HID), params[OFF_W1 + i]);
    for (int i = t; i < HID * HID; i += TILE) {
        store_bf16(S.w2, kmaj_off(i / HID, i % HID, HID), params[OFF_W2 + i]);
        store_bf16(S.w3, kmaj_off(i / HID, i % HID, HID), params[OFF_W3 + i]);
    }
    for (int i = t; i < OUT * HID; i += TILE) store_bf16(S.w4, kmaj_off(i / HID, i % HID, OUT), params[OFF_W4 + i]);
    for (int i = t; i < HID; i += TILE) {
        S.b1[i] = params[OFF_B1 + i];
        S.b2[i] = params[OFF_B2 + i];
        S.b3[i] = params[OFF_B3 + i];
    }
    if (t < OUT) S.b4[t] = params[OFF_B4 + t];
    if (t == 0) {
        mbar_init(&S.mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        tmem_alloc(&S.tmem, TMEM_COLS);
        tmem_relinquish();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = S.tmem;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    uint32_t phase = 0;
    bool ok = true;
    const int64_t ntiles = (n + TILE - 1) / TILE;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int64_t row = tile * TILE + t;
        // inputs of this thread's sample -> A (K = 16)
        for (int k = 0; k < IN; ++k) store_bf16(S.a, kmaj_off(t, k, TILE), row < n ? X[row * XSTR + k] : 0.0f);
        for (int layer = 0; layer < 4 && ok; ++layer) {
            fence_proxy_async();
            fence_before_sync();
            __syncthreads();
            fence_after_sync();
            const int K = layer == 0 ? IN : HID, N = layer == 3 ? OUT : HID;
            if (t == 0) {
                const unsigned char *w = layer == 0 ? S.w1 : (layer == 1 ? S.w2 : (layer == 2 ? S.w3 : S.w4));
                issue_layer(tmem, S.a, w, K, N);
                mma_commit(&S.mbar);
            }
            const int timed_out = !mbar_wait_bounded(&S.mbar, phase, WAIT_LIMIT);
            phase ^= 1u;
            fence_after_sync();
            if (__syncthreads_or(timed_out)) {  // block-uniform decision
                ok = false;
                break;
            }
            if (layer < 3) {
                const float *bias = layer == 0 ? S.b1 : (layer == 1 ? S.b2 : S.b3);
                for (int c0 = 0; c0 < HID; c0 += 16) {
                    float v[16];
                    tmem_ld16(tmem + lane_base + c0, v);
                    tmem_wait_ld();
                    for (int i = 0; i < 16; ++i) store_bf16(S.a, kmaj_off(warp * 32 + lane, c0 + i, TILE),
                                                             gelu(v[i] + bias[c0 + i]));
                }
            } else {
                // head: coefficients A (3 NJ of the OUT columns) contracted with the sample's jets
                float a[OUT];
#pragma unroll
                for (int c0 = 0; c0 < OUT; c0 += 16) {
                    float v[16];
                    tmem_ld16(tmem + lane_base + c0, v);
                    tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < 16; ++i) a[c0 + i] = v[i] + S.b4[c0 + i];
                }
                const int64_t r = tile * TILE + warp * 32 + lane;
                if (r < n) {
                    const float *jet = X + r * XSTR + JET_OFF;
                    float c[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
                    for (int j = 0; j < NJ; ++j) {
                        const float g = jet[j];
#pragma unroll
                        for (int e = 0; e < 3; ++e) c[e] = fmaf(a[e * NJ + j], g, c[e]);
                    }
                    for (int e = 0; e < 3; ++e) Y[r * OUT_STRIDE + e] = c[e];
                    Y[r * OUT_STRIDE + 3] = 0.0f;
                }
            }
        }
    }
    if (!ok && t == 0 && err) atomicExch(err, 1);
    if (!ok) {  // give the MMA in flight a bounded chance to finish before its memory is released
        mbar_wait_bounded(&S.mbar, phase ^ 1u, WAIT_LIMIT);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

// ------------------------------------------------------------------------------------------
// FP32 SIMT kernels: reference forward (same rounding as the tensor-core kernel) and training
// ------------------------------------------------------------------------------------------
// Wq = bf16(W) for the weight matrices; biases stay FP32.
__global__ void k_quantize(const float *__restrict__ p, float *__restrict__ q) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    const bool is_w = (i < OFF_B1) || (i >= OFF_W2 && i < OFF_B2) || (i >= OFF_W3 && i < OFF_B3) ||
                      (i >= OFF_W4 && i < OFF_B4);
    q[i] = is_w ? bf16r(p[i]) : p[i];
}

// Forward of one sample with quantized weights q (shared memory); optionally stores the
// pre-activations z1..z3 and the (rounded) activations a0..a3 for the backward pass.
__device__ __forceinline__ void forward_one(const float *q, const float *x, float *out, float *zs, float *as) {
    float a0[IN], h1[HID], h2[HID];
    for (int k = 0; k < IN; ++k) a0[k] = bf16r(x[k]);
    if (as)
        for (int k = 0; k < IN; ++k) as[k] = a0[k];
    for (int o = 0; o < HID; ++o) {
        float s = q[OFF_B1 + o];
        for (int k = 0; k < IN; ++k) s = fmaf(q[OFF_W1 + o * IN + k], a0[k], s);
        if (zs) zs[o] = s;
        h1[o] = bf16r(gelu(s));
        if (as) as[IN + o] = h1[o];
    }
    for (int o = 0; o < HID; ++o) {
        float s = q[OFF_B2 + o];
        for (int k = 0; k < HID; ++k) s = fmaf(q[OFF_W2 + o * HID + k], h1[k], s);
        if (zs) zs[HID + o] = s;
        h2[o] = bf16r(gelu(s));
        if (as) as[IN + HID + o] = h2[o];
    }
    for (int o = 0; o < HID; ++o) {
        float s = q[OFF_B3 + o];
        for (int k = 0; k < HID; ++k) s = fmaf(q[OFF_W3 + o * HID + k], h2[k], s);
        if (zs) zs[2 * HID + o] = s;
        h1[o] = bf16r(gelu(s));  // reuse h1 as a3
        if (as) as[IN + 2 * HID + o] = h1[o];
    }
    for (int o = 0; o < OUT_USED; ++o) {
        float s = q[OFF_B4 + o];
        for (int k = 0; k < HID; ++k) s = fmaf(q[OFF_W4 + o * HID + k], h1[k], s);
        out[o] = s;
    }
}

// c_e = sum_j A[e nj + j] jet_j (the head).
__device__ __forceinline__ void contract(const float *A, const float *jet, int nj, float c[3]) {
    c[0] = c[1] = c[2] = 0.0f;
    for (int j = 0; j < nj; ++j) {
        const float g = jet[j];
        for (int e = 0; e < 3; ++e) c[e] = fmaf(A[e * nj + j], g, c[e]);
    }
}

constexpr int NT_SIMT = 128;

constexpr size_t SIMT_SMEM = sizeof(float) * NPARAM;  // the quantized parameters (above 48 KB: opt-in)

__global__ void __launch_bounds__(NT_SIMT) k_mlp_infer_ref(const float *__restrict__ q, const float *__restrict__ X,
                                                           int64_t n, int nj, float *__restrict__ Y) {
    extern __shared__ float sq[];
    for (int i = threadIdx.x; i < NPARAM; i += NT_SIMT) sq[i] = q[i];
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * NT_SIMT + threadIdx.x;
    if (s >= n) return;
    float x[IN], out[OUT_USED], c[3];
    for (int k = 0; k < IN; ++k) x[k] = X[s * XSTR + k];
    forward_one(sq, x, out, nullptr, nullptr);
    contract(out, X + s * XSTR + JET_OFF, nj, c);
    for (int e = 0; e < 3; ++e) Y[s * OUT_STRIDE + e] = c[e];
    Y[s * OUT_STRIDE + 3] = 0.0f;
}

// Training forward + output error: stores Z (n x 3*HID), A (n x ACT) and
// D4 = dL/d(coefficients) = w (c - t)_e jet_j / n at coefficient e nj + j (0 beyond 3 nj).
__global__ void __launch_bounds__(NT_SIMT) k_train_fwd(const float *__restrict__ q, const float *__restrict__ X,
                                                       const float *__restrict__ T, const int *__restrict__ idx,
                                                       int64_t n, int nj, float inv_n, float *__restrict__ Z,
                                                       float *__restrict__ A, float *__restrict__ D4,
                                                       double *__restrict__ loss) {
    extern __shared__ float sq[];
    __shared__ double sl[NT_SIMT / 32];
    for (int i = threadIdx.x; i < NPARAM; i += NT_SIMT) sq[i] = q[i];
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * NT_SIMT + threadIdx.x;
    double l = 0.0;
    if (s < n) {
        const int64_t src = idx ? idx[s] : s;
        float x[IN], out[OUT_USED], c[3];
        for (int k = 0; k < IN; ++k) x[k] = X[src * XSTR + k];
        forward_one(sq, x, out, Z + s * (3 * HID), A + s * ACT);
        const float *jet = X + src * XSTR + JET_OFF;
        contract(out, jet, nj, c);
        const float w = T[src * TSTR + 3];
        float err[3];
        for (int e = 0; e < 3; ++e) {
            err[e] = c[e] - T[src * TSTR + e];
            l += 0.5 * (double)w * err[e] * err[e];
        }
        for (int k = 0; k < OUT_USED; ++k) {
            const int e = k / nj, j = k - e * nj;
            D4[s * OUT_USED + k] = e < 3 ? w * err[e] * jet[j] * inv_n : 0.0f;
        }
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) sl[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0 && loss) {
        double tot = 0.0;
        for (int w = 0; w < NT_SIMT / 32; ++w) tot += sl[w];
        atomicAdd(loss, tot * inv_n);
    }
}

// Backward deltas of one sample: D3, D2, D1 (n x HID each) from D4.
__global__ void __launch_bounds__(NT_SIMT) k_train_bwd(const float *__restrict__ q, const float *__restrict__ Z,
                                                       const float *__restrict__ D4, int64_t n,
                                                       float *__restrict__ D) {
    extern __shared__ float sq[];
    for (int i = threadIdx.x; i < NPARAM; i += NT_SIMT) sq[i] = q[i];
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * NT_SIMT + threadIdx.x;
    if (s >= n) return;
    const float *z = Z + s * (3 * HID);
    float d4[OUT_USED], d3[HID], d2[HID];
    for (int i = 0; i < OUT_USED; ++i) d4[i] = D4[s * OUT_USED + i];
    for (int k = 0; k < HID; ++k) {
        float g = 0.0f;
        for (int o = 0; o < OUT_USED; ++o) g = fmaf(sq[OFF_W4 + o * HID + k], d4[o], g);
        d3[k] = g * gelu_d(z[2 * HID + k]);
    }
    for (int k = 0; k < HID; ++k) {
        float g = 0.0f;
        for (int o = 0; o < HID; ++o) g = fmaf(sq[OFF_W3 + o * HID + k], d3[o], g);
        d2[k] = g * gelu_d(z[HID + k]);
    }
    float *out = D + s * (3 * HID);
    for (int k = 0; k < HID; ++k) {
        float g = 0.0f;
        for (int o = 0; o < HID; ++o) g = fmaf(sq[OFF_W2 + o * HID + k], d2[o], g);
        out[k] = g * gelu_d(z[k]);  // D1
        out[HID + k] = d2[k];
        out[2 * HID + k] = d3[k];
    }
}

// Gradient of every parameter: one thread per parameter, summing over the batch.
__global__ void k_train_wgrad(const float *__restrict__ A, const float *__restrict__ D, const float *__restrict__ D4,
                              int64_t n, float *__restrict__ G) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    float s = 0.0f;
    if (i < OFF_B1) {  // W1[o][k]: D1[o] * a0[k]
        const int o = i / IN, k = i % IN;
        for (int64_t b = 0; b < n; ++b) s = fmaf(D[b * 3 * HID + o], A[b * ACT + k], s);
    } else if (i < OFF_W2) {
        const int o = i - OFF_B1;
        for (int64_t b = 0; b < n; ++b) s += D[b * 3 * HID + o];
    } else if (i < OFF_B2) {
        const int o = (i - OFF_W2) / HID, k = (i - OFF_W2) % HID;
        for (int64_t b = 0; b < n; ++b) s = fmaf(D[b * 3 * HID + HID + o], A[b * ACT + IN + k], s);
    } else if (i < OFF_W3) {
        const int o = i - OFF_B2;
        for (int64_t b = 0; b < n; ++b) s += D[b * 3 * HID + HID + o];
    } else if (i < OFF_B3) {
        const int o = (i - OFF_W3) / HID, k = (i - OFF_W3) % HID;
        for (int64_t b = 0; b < n; ++b) s = fmaf(D[b * 3 * HID + 2 * HID + o], A[b * ACT + IN + HID + k], s);
    } else if (i < OFF_W4) {
        const int o = i - OFF_B3;
        for (int64_t b = 0; b < n; ++b) s += D[b * 3 * HID + 2 * HID + o];
    } else if (i < OFF_B4) {
        const int o = (i - OFF_W4) / HID, k = (i - OFF_W4) % HID;
        if (o < OUT_USED)
            for (int64_t b = 0; b < n; ++b) s = fmaf(D4[b * OUT_USED + o], A[b * ACT + IN + 2 * HID + k], s);
    } else {
        const int o = i - OFF_B4;
        if (o < OUT_USED)
            for (int64_t b = 0; b < n; ++b) s += D4[b * OUT_USED + o];
    }
    G[i] = s;
}

__global__ void k_adam(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

size_t infer_smem_bytes() { return sizeof(InferSmem) + 1024; }

cudaError_t launch_infer_tc(const float *params, const float *X, int64_t n, float *Y, int nj, int *err, int grid,
                            cudaStream_t st) {
    if (nj != NJ_SL && nj != NJ_DL) return cudaErrorInvalidValue;
    const size_t smem = infer_smem_bytes();
    auto kern = nj == NJ_SL ? k_mlp_infer_tc<NJ_SL> : k_mlp_infer_tc<NJ_DL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, TILE, smem, st>>>(params, X, n, Y, err);
    return cudaGetLastError();
}

namespace {
// The timeout path of the bounded waits: an mbarrier that expects one arrival, which thread 0
// makes only when `arrive` is set; every thread polls at most `limit` times, and a wait that
// runs out sets *flag and returns (no asynchronous operation is tied to this barrier).
__global__ void k_wait_probe(int arrive, uint32_t limit, int *flag) {
    __shared__ uint64_t mbar;
    if (threadIdx.x == 0) {
        mbar_init(&mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (arrive && threadIdx.x == 0)
        asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}\n" ::"r"(smem_u32(&mbar))
                     : "memory");
    const bool ok = mbar_wait_bounded(&mbar, 0u, limit);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicExch(flag, 1);
}
}  // namespace

cudaError_t launch_wait_probe(int arrive, uint32_t limit, int *flag, cudaStream_t st) {
    k_wait_probe<<<1, 128, 0, st>>>(arrive, limit, flag);
    return cudaGetLastError();
}

cudaError_t launch_quantize(const float *p, float *q, cudaStream_t st) {
    k_quantize<<<(NPARAM + 255) / 256, 256, 0, st>>>(p, q);
    return cudaGetLastError();
}

cudaError_t launch_infer_ref(const float *q, const float *X, int64_t n, float *Y, int nj, cudaStream_t st) {
    if (nj != NJ_SL && nj != NJ_DL) return cudaErrorInvalidValue;
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_infer_ref, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SIMT_SMEM);
    if (e != cudaSuccess) return e;
    k_mlp_infer_ref<<<(unsigned)((n + NT_SIMT - 1) / NT_SIMT), NT_SIMT, SIMT_SMEM, st>>>(q, X, n, nj, Y);
    return cudaGetLastError();
}

cudaError_t launch_train_grad(const float *q, const float *X, const float *T, const int *idx, int64_t n, int nj,
                              float *Z, float *A, float *D4, float *D, float *G, double *loss, cudaStream_t st) {
    if (nj != NJ_SL && nj != NJ_DL) return cudaErrorInvalidValue;
    const unsigned nb = (unsigned)((n + NT_SIMT - 1) / NT_SIMT);
    const float inv_n = 1.0f / (float)n;
    cudaError_t e = cudaFuncSetAttribute(k_train_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SIMT_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_train_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SIMT_SMEM);
    if (e != cudaSuccess) return e;
    k_train_fwd<<<nb, NT_SIMT, SIMT_SMEM, st>>>(q, X, T, idx, n, nj, inv_n, Z, A, D4, loss);
    k_train_bwd<<<nb, NT_SIMT, SIMT_SMEM, st>>>(q, Z, D4, n, D);
    k_train_wgrad<<<(NPARAM + 127) / 128, 128, 0, st>>>(A, D, D4, n, G);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *p, float *m, float *v, const float *g, float lr, int step, cudaStream_t st) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    k_adam<<<(NPARAM + 255) / 256, 256, 0, st>>>(p, m, v, g, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError();
}

}  // namespace mlp
}  // namespace ers
