// Layout of the closure network's parameters and samples, and the launchers of k_mlp.cu.
//
// The network maps the local geometry of a target (lambda_0, the principal curvatures times h,
// rho_0, rho_1) to the coefficients of a linear map from the density jets to the correction:
//   A = MLP(geometry) (OUT_USED = 3 J values used of OUT), c_e = sum_j A[e J + j] jet_j, e = 0..2,
// with J = NJ_SL jets for the single layer and NJ_DL for the double layer.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ers {
namespace mlp {

constexpr int IN = 16;        // network inputs (NGEOM used), one K step of the tensor-core MMA
constexpr int NGEOM = 5;      // lambda_0, kappa_1 h, kappa_2 h, rho_0, rho_1
constexpr int JET_OFF = 16;   // offset of the jets in a sample record
constexpr int NJ_SL = 18;     // single layer: orders 0..2 of 3 components (6 x 3)
constexpr int NJ_DL = 27;     // double layer: orders 1..3 of 3 components (9 x 3)
constexpr int NJ_MAX = 32;    // jet slots of a sample record
constexpr int XSTR = JET_OFF + NJ_MAX;  // floats per sample record: [geometry | pad | jets | pad]
constexpr int HID = 64;
constexpr int OUT = 96;       // N of the last MMA
constexpr int OUT_USED = 3 * NJ_DL;  // 81 coefficients at most (54 for the single layer)
constexpr int OUT_STRIDE = 4; // output rows: c_0, c_1, c_2, unused
constexpr int TSTR = 4;       // training targets: c_0, c_1, c_2, sample weight
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
constexpr int NPARAM = OFF_B4 + OUT;  // 15648

__host__ __device__ constexpr int jets_of_layer(int layer) { return layer == 0 ? NJ_SL : NJ_DL; }

size_t infer_smem_bytes();
// Inference: Y (n, OUT_STRIDE) = the contraction of the network's coefficients with the jets of
// the sample records X (n, XSTR); nj = jets_of_layer(layer).
cudaError_t launch_infer_tc(const float *params, const float *X, int64_t n, float *Y, int nj, int *err, int grid,
                            cudaStream_t st);
cudaError_t launch_quantize(const float *p, float *q, cudaStream_t st);
cudaError_t launch_infer_ref(const float *q, const float *X, int64_t n, float *Y, int nj, cudaStream_t st);
cudaError_t launch_train_grad(const float *q, const float *X, const float *T, const int *idx, int64_t n, int nj,
                              float *Z, float *A, float *D4, float *D, float *G, double *loss, cudaStream_t st);
cudaError_t launch_adam(float *p, float *m, float *v, const float *g, float lr, int step, cudaStream_t st);
// One CTA whose bounded mbarrier wait completes (arrive != 0) or runs out after `limit` polls
// (then *flag = 1): the timeout path of the tensor-core and treecode waits, tested on its own.
cudaError_t launch_wait_probe(int arrive, uint32_t limit, int *flag, cudaStream_t st);

}  // namespace mlp
}  // namespace ers
