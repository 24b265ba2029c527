// Layout of the closure network's parameters and the launchers of k_mlp.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ers {
namespace mlp {

constexpr int IN = 16;        // 13 features used, padded to one K step of the tensor-core MMA
constexpr int HID = 64;
constexpr int OUT = 16;       // N of the last MMA; 3 outputs used
constexpr int OUT_USED = 3;
constexpr int OUT_STRIDE = 4; // row stride of the output array
constexpr int ACT = IN + 3 * HID;  // stored activations per sample (training)
// FP32 parameters, weights row-major W[out][in]
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + HID * IN;
constexpr int OFF_W2 = OFF_B1 + HID;
constexpr int OFF_B2 = OFF_W2 + HID * HID;
constexpr int OFF_W3 = OFF_B2 + HID;
constexpr int OFF_B3 = OFF_W3 + HID * HID;
constexpr int OFF_W4 = OFF_B3 + HID;
constexpr int OFF_B4 = OFF_W4 + OUT * HID;
constexpr int NPARAM = OFF_B4 + OUT;  // 10448

size_t infer_smem_bytes();
cudaError_t launch_infer_tc(const float *params, const float *X, int64_t n, float *Y, int *err, int grid,
                            cudaStream_t st);
cudaError_t launch_quantize(const float *p, float *q, cudaStream_t st);
cudaError_t launch_infer_ref(const float *q, const float *X, int64_t n, float *Y, cudaStream_t st);
cudaError_t launch_train_grad(const float *q, const float *X, const float *T, const int *idx, int64_t n, float *Z,
                              float *A, float *D4, float *D, float *G, double *loss, cudaStream_t st);
cudaError_t launch_adam(float *p, float *m, float *v, const float *g, float lr, int step, cudaStream_t st);
// One CTA whose bounded mbarrier wait completes (arrive != 0) or runs out after `limit` polls
// (then *flag = 1): the timeout path of the tensor-core and treecode waits, tested on its own.
cudaError_t launch_wait_probe(int arrive, uint32_t limit, int *flag, cudaStream_t st);

}  // namespace mlp
}  // namespace ers
