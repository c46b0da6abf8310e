// Measured arithmetic ceilings for roofline fractions (the paper has no
// counterpart): the FP32 FMA and FP64 FMA rates this GPU sustains on
// register-resident operands.
//
// Kernel: every thread runs kChains independent FMA chains x <- x * a + b for
// `iters` steps (no memory traffic inside the loop; the chains hide the FMA
// latency), and writes one value derived from all chains so that nothing is
// optimised away.  The grid holds kBlocksPerSM blocks of kThreads threads on
// every SM.  The rate is 2 x FMAs / elapsed time between CUDA events on the
// caller's stream.
#include <algorithm>

#include "bs_internal.h"

namespace bsi {

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 4;

template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_peak(int iters, T a, T b, T *out) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = x[c] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)-12345.0) out[blockIdx.x] = s;  // practically never taken; keeps the chains live
}

template <class T>
cudaError_t time_peak(int iters, cudaStream_t s, double *rate) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int grid = nsm * kBlocksPerSM;
  cudaEvent_t e0, e1;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  // a = 1 - 2^-20, b = 2^-20: x stays bounded, no denormals or overflow
  const T a = (T)(1.0 - 1.0 / 1048576.0), b = (T)(1.0 / 1048576.0);
  k_fma_peak<T><<<grid, kThreads, 0, s>>>(std::max(1, iters / 8), a, b, nullptr);  // warm-up
  cudaEventRecord(e0, s);
  k_fma_peak<T><<<grid, kThreads, 0, s>>>(iters, a, b, nullptr);
  cudaEventRecord(e1, s);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  const double fmas = (double)grid * kThreads * kChains * (double)iters;
  *rate = 2.0 * fmas / (ms * 1e-3);
  return cudaSuccess;
}

}  // namespace

}  // namespace bsi

extern "C" bs_status bs_measure_peak(int kind, int iters, double *flops_per_s, void *stream) {
  BS_NVTX("bs_measure_peak");
  using namespace bsi;
  if (!flops_per_s || (kind != 0 && kind != 1) || iters < 1) return BS_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cudaError_t e = kind == 0 ? time_peak<float>(iters, s, flops_per_s)
                                  : time_peak<double>(iters, s, flops_per_s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver ? BS_ERR_NO_DEVICE
                                                                      : BS_ERR_CUDA;
  }
  return BS_OK;
}
