// Shared between the surrogate's FP32 SIMT kernels (mlp.cu) and its
// tensor-core kernels (mlp_tc.cu).
#pragma once

#include <cuda_runtime.h>

namespace bsi {

struct MlpDev {
  int d, w;
  float *p;       // master FP32 params, flat: W1 [w][d] | b1 | W2 [w][w] | b2 | w3 | b3
  float *g;       // gradient, same layout
  float *m, *v;   // Adam moments
  float *norm;    // mu_x [d] | sd_x [d] | mu_y | sd_y
};

// Tensor-core (mma.sync BF16, FP32 accumulation) forms of the forward, the
// per-row backward and the weight gradients, with the same inputs, outputs
// and scratch layouts as the SIMT kernels: store rows [xn (d) | h1 (w) |
// h2 (w) | yn], bw rows [dz1 (w) | dz2 (w) | dyn].  Width 128, d <= 64.
bool mlp_tc_supported(int d, int w);
cudaError_t mlp_tc_forward(const MlpDev &M, const float *x, int n, const int *idx, int nrows,
                           float *y, float *store, cudaStream_t s);
cudaError_t mlp_tc_backward_rows(const MlpDev &M, const float *t, const int *idx, int nrows,
                                 const float *store, float *bw, float *loss, cudaStream_t s);
cudaError_t mlp_tc_wgrad(const MlpDev &M, int nrows, const float *store, const float *bw,
                         cudaStream_t s);

}  // namespace bsi
