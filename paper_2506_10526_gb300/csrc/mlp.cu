// Error-bar surrogate: a 3-layer MLP that predicts log Var of each 3D
// bispectrum bin from triangle and flag features, trained on the per-bin
// variances the batched Monte Carlo path produces.  Not in the paper (which
// estimates error bars by brute Monte Carlo over 250 realisations); the
// Monte Carlo stays the fallback and the reference the surrogate's error is
// measured against.
//
//   xn = (x - mu_x)/sd_x;  h1 = tanh(W1 xn + b1);  h2 = tanh(W2 h1 + b2)
//   yn = w3 . h2 + b3;     y = mu_y + sd_y yn
// W1, W2, w3 are used as BF16 values (rounded from FP32 master weights when
// they are staged in shared memory); every sum accumulates in FP32.  Loss:
// mean squared error on the normalised target; Adam on the FP32 masters.
//
// Kernels: features per bin, column statistics, forward (one thread per row),
// per-row backward (dz2, dz1), weight gradients (tiled reductions over rows
// with FP32 atomics), Adam.  Width 128 runs the forward, backward and weight
// gradients on the tensor cores instead (mlp_tc.cu); these FP32 SIMT kernels
// remain for other widths and as the checker (bs_mlp_set_kernels).  Minibatch rows come from a counter-based hash of
// (seed, step, slot).
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "mlp_internal.h"
#include "plan_internal.h"

using namespace bsi;

namespace {

constexpr int kMaxD = 64, kMaxW = 128, kRows = 128;

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__host__ __device__ inline long long n_params(int d, int w) {
  return (long long)w * d + w + (long long)w * w + w + w + 1;
}

// SplitMix64-style hash: independent uniform row index per (seed, step, slot).
__device__ __forceinline__ unsigned long long mix(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Stage the BF16-rounded weights and FP32 biases of one network in shared memory.
__device__ void stage_weights(const MlpDev &M, float *W1, float *b1, float *W2, float *b2,
                              float *w3, float *b3) {
  const int d = M.d, w = M.w;
  const float *p = M.p;
  for (int q = threadIdx.x; q < w * d; q += blockDim.x) W1[q] = bf(p[q]);
  p += w * d;
  for (int q = threadIdx.x; q < w; q += blockDim.x) b1[q] = p[q];
  p += w;
  for (int q = threadIdx.x; q < w * w; q += blockDim.x) W2[q] = bf(p[q]);
  p += w * w;
  for (int q = threadIdx.x; q < w; q += blockDim.x) b2[q] = p[q];
  p += w;
  for (int q = threadIdx.x; q < w; q += blockDim.x) w3[q] = bf(p[q]);
  p += w;
  if (threadIdx.x == 0) *b3 = p[0];
}

// Forward for rows[r] = idx ? idx[r] : r0 + r.  Writes y (denormalised) and,
// when store != null, per row [xn (d) | h1 (w) | h2 (w) | yn] for the backward.
__global__ void __launch_bounds__(kRows) k_mlp_forward(MlpDev M, const float *__restrict__ x, int n,
                                                       const int *__restrict__ idx, int nrows,
                                                       float *__restrict__ y,
                                                       float *__restrict__ store) {
  extern __shared__ float sm[];
  const int d = M.d, w = M.w;
  float *W1 = sm, *b1 = W1 + w * d, *W2 = b1 + w, *b2 = W2 + w * w, *w3 = b2 + w, *b3 = w3 + w;
  float *h1 = b3 + 1;  // [kRows][w + 1]
  stage_weights(M, W1, b1, W2, b2, w3, b3);
  __syncthreads();
  const int r = blockIdx.x * kRows + threadIdx.x;
  if (r >= nrows) return;
  const int row = idx ? idx[r] : r;
  if (row < 0 || row >= n) return;
  const float *mu = M.norm, *sd = M.norm + d;
  float xn[kMaxD];
  for (int k = 0; k < d; ++k) xn[k] = (x[(long long)row * d + k] - mu[k]) / sd[k];
  float *hr = h1 + threadIdx.x * (w + 1);
  for (int j = 0; j < w; ++j) {
    float z = b1[j];
    for (int k = 0; k < d; ++k) z = fmaf(W1[j * d + k], xn[k], z);
    hr[j] = tanhf(z);
  }
  float *st = store ? store + (long long)r * (d + 2 * w + 1) : nullptr;
  float yn = *b3;
  for (int j = 0; j < w; ++j) {
    float z = b2[j];
    for (int k = 0; k < w; ++k) z = fmaf(W2[j * w + k], hr[k], z);
    const float h = tanhf(z);
    yn = fmaf(w3[j], h, yn);
    if (st) st[d + w + j] = h;
  }
  if (st) {
    for (int k = 0; k < d; ++k) st[k] = xn[k];
    for (int k = 0; k < w; ++k) st[d + k] = hr[k];
    st[d + 2 * w] = yn;
  }
  if (y) y[r] = M.norm[2 * d] + M.norm[2 * d + 1] * yn;
}

// Per-row backward: dyn, dz2 = dyn w3 (1 - h2^2), dz1 = (W2^T dz2)(1 - h1^2).
// bw row layout: [dz1 (w) | dz2 (w) | dyn].
__global__ void __launch_bounds__(kRows) k_mlp_backward_rows(MlpDev M, const float *__restrict__ t,
                                                             const int *__restrict__ idx, int nrows,
                                                             const float *__restrict__ store,
                                                             float *__restrict__ bw,
                                                             float *__restrict__ loss) {
  extern __shared__ float sm[];
  const int d = M.d, w = M.w;
  float *W2 = sm, *w3 = W2 + w * w, *dz = w3 + w;  // dz: [kRows][w + 1]
  const float *p = M.p + (long long)w * d + w;
  for (int q = threadIdx.x; q < w * w; q += blockDim.x) W2[q] = bf(p[q]);
  for (int q = threadIdx.x; q < w; q += blockDim.x) w3[q] = bf(p[w * w + w + q]);
  __syncthreads();
  const int r = blockIdx.x * kRows + threadIdx.x;
  float l2 = 0.f;
  if (r < nrows) {
    const int row = idx ? idx[r] : r;
    const float *st = store + (long long)r * (d + 2 * w + 1);
    const float tn = (t[row] - M.norm[2 * d]) / M.norm[2 * d + 1];
    const float res = st[d + 2 * w] - tn;
    l2 = res * res;
    const float dyn = 2.f * res / (float)nrows;
    float *dr = dz + threadIdx.x * (w + 1);
    float *o = bw + (long long)r * (2 * w + 1);
    for (int j = 0; j < w; ++j) {
      const float h = st[d + w + j];
      dr[j] = dyn * w3[j] * (1.f - h * h);
      o[w + j] = dr[j];
    }
    o[2 * w] = dyn;
    for (int k = 0; k < w; ++k) {
      float s = 0.f;
      for (int j = 0; j < w; ++j) s = fmaf(W2[j * w + k], dr[j], s);
      const float h = st[d + k];
      o[k] = s * (1.f - h * h);
    }
  }
  // loss = mean of squared residuals
  for (int off = 16; off > 0; off >>= 1) l2 += __shfl_xor_sync(0xffffffffu, l2, off);
  if (loss && (threadIdx.x & 31) == 0) atomicAdd(loss, l2 / (float)nrows);
}

// Weight gradients: for an output block of 32 rows j of W (layer selected by
// blockIdx.z) and a chunk of batch rows, each thread accumulates one (j, k)
// over the chunk and adds it to the global gradient.  Layer 0: dW1 = dz1^T xn
// (+ db1), layer 1: dW2 = dz2^T h1 (+ db2), layer 2: dw3 = dyn h2 (+ db3).
__global__ void k_mlp_wgrad(MlpDev M, int nrows, const float *__restrict__ store,
                            const float *__restrict__ bw, int chunk) {
  const int d = M.d, w = M.w;
  const int layer = blockIdx.z;
  const int r0 = blockIdx.x * chunk, r1 = min(nrows, r0 + chunk);
  const int sw = d + 2 * w + 1, bwid = 2 * w + 1;
  const int K = layer == 0 ? d : w;  // inputs of the layer
  const int J = layer == 2 ? 1 : w;  // outputs of the layer
  const int jb = blockIdx.y * 32;
  float *gW1 = M.g, *gb1 = gW1 + w * d, *gW2 = gb1 + w, *gb2 = gW2 + w * w, *gw3 = gb2 + w,
        *gb3 = gw3 + w;
  for (int e = threadIdx.x; e < 32 * (K + 1); e += blockDim.x) {
    const int jj = e / (K + 1), k = e - jj * (K + 1);  // k == K: bias
    const int j = jb + jj;
    if (j >= J) continue;
    float acc = 0.f;
    for (int r = r0; r < r1; ++r) {
      const float *st = store + (long long)r * sw;
      const float *b = bw + (long long)r * bwid;
      float dz, in;
      if (layer == 0) {
        dz = b[j];
        in = k < K ? st[k] : 1.f;
      } else if (layer == 1) {
        dz = b[w + j];
        in = k < K ? st[d + k] : 1.f;
      } else {
        dz = b[2 * w];
        in = k < K ? st[d + w + k] : 1.f;
      }
      acc = fmaf(dz, in, acc);
    }
    float *dst;
    if (layer == 0)
      dst = k < K ? gW1 + j * d + k : gb1 + j;
    else if (layer == 1)
      dst = k < K ? gW2 + j * w + k : gb2 + j;
    else
      dst = k < K ? gw3 + k : gb3;
    atomicAdd(dst, acc);
  }
}

__global__ void k_mlp_adam(MlpDev M, long long np, float lr, float b1, float b2, float eps, int step) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < np;
       q += (long long)gridDim.x * blockDim.x) {
    const float g = M.g[q];
    const float m = b1 * M.m[q] + (1.f - b1) * g;
    const float v = b2 * M.v[q] + (1.f - b2) * g * g;
    M.m[q] = m;
    M.v[q] = v;
    M.p[q] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    M.g[q] = 0.f;
  }
}

__global__ void k_mlp_sample(int *idx, int nrows, int n, unsigned long long seed, int step) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nrows)
    idx[r] = (int)(mix(seed ^ mix(((unsigned long long)step << 32) | (unsigned)r)) % (unsigned long long)n);
}

// Column mean and standard deviation (FP64 sums) of x [n][d] and t [n].
__global__ void k_mlp_colstats(const float *__restrict__ x, const float *__restrict__ t, int n, int d,
                               float *norm) {
  const int c = blockIdx.x;  // 0..d-1: features, d: target
  double s = 0, s2 = 0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const double v = c < d ? x[(long long)r * d + c] : t[r];
    s += v;
    s2 += v * v;
  }
  __shared__ double a[256], b[256];
  a[threadIdx.x] = s;
  b[threadIdx.x] = s2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      a[threadIdx.x] += a[threadIdx.x + o];
      b[threadIdx.x] += b[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double mean = a[0] / n, var = fmax(b[0] / n - mean * mean, 0.0);
    const float sd = var > 1e-24 ? (float)sqrt(var) : 1.f;
    if (c < d) {
      norm[c] = (float)mean;
      norm[d + c] = sd;
    } else {
      norm[2 * d] = (float)mean;
      norm[2 * d + 1] = sd;
    }
  }
}

// Features of every 3D-bispectrum bin (trip, a, b); NaN rows for ring triples
// without closed triangles.  tab[trip] = (log T, k_perp i, k_perp j, k_perp l).
__global__ void k_mlp_features(int ntrip, int nc, const float4 *__restrict__ tab,
                               const float *__restrict__ flagf, float kpar_unit,
                               float *__restrict__ out) {
  const long long nbin = (long long)ntrip * nc * nc;
  const int h = nc / 2;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nbin;
       q += (long long)gridDim.x * blockDim.x) {
    const int trip = (int)(q / ((long long)nc * nc));
    const int rem = (int)(q - (long long)trip * nc * nc);
    const int ia = rem / nc, ib = rem - ia * nc;
    float *o = out + q * BS_MLP_FEATURES;
    const float4 tb = tab[trip];
    if (!(tb.x == tb.x)) {
      for (int k = 0; k < BS_MLP_FEATURES; ++k) o[k] = __int_as_float(0x7fc00000);
      continue;
    }
    const float ka = kpar_unit * (float)(ia - h), kb = kpar_unit * (float)(ib - h), kc = -(ka + kb);
    float k1 = sqrtf(tb.y * tb.y + ka * ka), k2 = sqrtf(tb.z * tb.z + kb * kb),
          k3 = sqrtf(tb.w * tb.w + kc * kc);
    // sort descending
    if (k1 < k2) { const float s = k1; k1 = k2; k2 = s; }
    if (k2 < k3) { const float s = k2; k2 = k3; k3 = s; }
    if (k1 < k2) { const float s = k1; k1 = k2; k2 = s; }
    o[0] = logf(k1);
    o[1] = k2 / k1;
    o[2] = (k1 * k1 + k2 * k2 - k3 * k3) / (2.f * k1 * k2);
    o[3] = flagf[0];
    o[4] = tb.x;
    o[5] = fabsf(ka);
    o[6] = fabsf(kb);
    o[7] = logf(tb.y);
    o[8] = logf(tb.z);
    o[9] = logf(tb.w);
    for (int k = 0; k < 32; ++k) o[10 + k] = flagf[1 + k];
    for (int k = 0; k < 3; ++k) o[42 + k] = flagf[33 + k];
  }
}

size_t fwd_smem(int d, int w) { return sizeof(float) * ((size_t)w * d + 3 * w + (size_t)w * w + 1 + (size_t)kRows * (w + 1)); }
size_t bwd_smem(int w) { return sizeof(float) * ((size_t)w * w + w + (size_t)kRows * (w + 1)); }

}  // namespace

struct bs_mlp_s {
  MlpDev dev{};
  int *idx = nullptr;
  float *store = nullptr, *bw = nullptr, *loss = nullptr;
  int cap = 0;  // rows of the training scratch
  int step = 0;
  bool tc = false;  // tensor-core kernels (width 128), else FP32 SIMT
  std::string err = "no error";
};

namespace {

bs_status lfail(bs_mlp m, bs_status s, const std::string &msg) {
  if (m) m->err = msg;
  return s;
}

#define ML_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t e__ = (call);                                                                  \
    if (e__ != cudaSuccess) return lfail(m, BS_ERR_CUDA, std::string(#call) + ": " +           \
                                                          cudaGetErrorString(e__));             \
  } while (0)

bs_status ensure_scratch(bs_mlp m, int rows) {
  if (rows <= m->cap) return BS_OK;
  cudaFree(m->idx);
  cudaFree(m->store);
  cudaFree(m->bw);
  const int d = m->dev.d, w = m->dev.w;
  ML_CUDA(cudaMalloc(&m->idx, (size_t)rows * sizeof(int)));
  ML_CUDA(cudaMalloc(&m->store, (size_t)rows * (d + 2 * w + 1) * sizeof(float)));
  ML_CUDA(cudaMalloc(&m->bw, (size_t)rows * (2 * w + 1) * sizeof(float)));
  m->cap = rows;
  return BS_OK;
}

// Loss and gradient of a batch of rows (idx or the first nrows rows) into dev.g.
bs_status grad_batch(bs_mlp m, const float *x, const float *t, int n, const int *idx, int nrows,
                     cudaStream_t s) {
  const int d = m->dev.d, w = m->dev.w;
  if (m->tc) {
    ML_CUDA(mlp_tc_forward(m->dev, x, n, idx, nrows, nullptr, m->store, s));
    ML_CUDA(mlp_tc_backward_rows(m->dev, t, idx, nrows, m->store, m->bw, m->loss, s));
    ML_CUDA(mlp_tc_wgrad(m->dev, nrows, m->store, m->bw, s));
    return BS_OK;
  }
  const int blocks = (nrows + kRows - 1) / kRows;
  k_mlp_forward<<<blocks, kRows, fwd_smem(d, w), s>>>(m->dev, x, n, idx, nrows, nullptr, m->store);
  ML_CUDA(cudaGetLastError());
  k_mlp_backward_rows<<<blocks, kRows, bwd_smem(w), s>>>(m->dev, t, idx, nrows, m->store, m->bw,
                                                         m->loss);
  ML_CUDA(cudaGetLastError());
  const int chunk = 256;
  dim3 g((nrows + chunk - 1) / chunk, (w + 31) / 32, 3);
  k_mlp_wgrad<<<g, 256, 0, s>>>(m->dev, nrows, m->store, m->bw, chunk);
  ML_CUDA(cudaGetLastError());
  return BS_OK;
}

}  // namespace

extern "C" {

const char *bs_mlp_last_error(bs_mlp m) { return m ? m->err.c_str() : "no surrogate"; }

bs_status bs_mlp_create(int d_in, int width, uint64_t seed, bs_mlp *out) {
  BS_NVTX("bs_mlp_create");
  if (!out || d_in < 1 || d_in > kMaxD || width < 1 || width > kMaxW) return BS_ERR_ARG;
  *out = nullptr;
  bs_mlp m = new bs_mlp_s();
  m->dev.d = d_in;
  m->dev.w = width;
  const long long np = n_params(d_in, width);
  std::vector<float> p(np);
  // Glorot-uniform weights from a SplitMix64 stream, zero biases
  unsigned long long z = seed;
  auto uni = [&]() {
    z += 0x9E3779B97F4A7C15ULL;
    unsigned long long q = z;
    q = (q ^ (q >> 30)) * 0xBF58476D1CE4E5B9ULL;
    q = (q ^ (q >> 27)) * 0x94D049BB133111EBULL;
    q ^= q >> 31;
    return (double)(q >> 11) * (1.0 / 9007199254740992.0);
  };
  long long o = 0;
  const double a1 = std::sqrt(6.0 / (d_in + width)), a2 = std::sqrt(6.0 / (2.0 * width)),
               a3 = std::sqrt(6.0 / (width + 1.0));
  for (long long q = 0; q < (long long)width * d_in; ++q) p[o++] = (float)(a1 * (2 * uni() - 1));
  for (int q = 0; q < width; ++q) p[o++] = 0.f;
  for (long long q = 0; q < (long long)width * width; ++q) p[o++] = (float)(a2 * (2 * uni() - 1));
  for (int q = 0; q < width; ++q) p[o++] = 0.f;
  for (int q = 0; q < width; ++q) p[o++] = (float)(a3 * (2 * uni() - 1));
  p[o++] = 0.f;
  std::vector<float> norm(2 * d_in + 2, 0.f);
  for (int k = 0; k < d_in; ++k) norm[d_in + k] = 1.f;
  norm[2 * d_in + 1] = 1.f;
  if (inject_fail("mlp_alloc") || cudaMalloc(&m->dev.p, np * 4) != cudaSuccess ||
      cudaMalloc(&m->dev.g, np * 4) != cudaSuccess ||
      cudaMalloc(&m->dev.m, np * 4) != cudaSuccess || cudaMalloc(&m->dev.v, np * 4) != cudaSuccess ||
      cudaMalloc(&m->dev.norm, norm.size() * 4) != cudaSuccess ||
      cudaMalloc(&m->loss, sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    bs_mlp_destroy(m);
    return BS_ERR_OOM;
  }
  cudaMemcpy(m->dev.p, p.data(), np * 4, cudaMemcpyHostToDevice);
  cudaMemset(m->dev.g, 0, np * 4);
  cudaMemset(m->dev.m, 0, np * 4);
  cudaMemset(m->dev.v, 0, np * 4);
  cudaMemcpy(m->dev.norm, norm.data(), norm.size() * 4, cudaMemcpyHostToDevice);
  m->tc = mlp_tc_supported(d_in, width);
  if (smem_optin_once<k_mlp_forward>() != cudaSuccess ||
      smem_optin_once<k_mlp_backward_rows>() != cudaSuccess) {
    cudaGetLastError();
    bs_mlp_destroy(m);
    return BS_ERR_CUDA;
  }
  *out = m;
  return BS_OK;
}

bs_status bs_mlp_destroy(bs_mlp m) {
  BS_NVTX("bs_mlp_destroy");
  if (!m) return BS_OK;
  cudaFree(m->dev.p);
  cudaFree(m->dev.g);
  cudaFree(m->dev.m);
  cudaFree(m->dev.v);
  cudaFree(m->dev.norm);
  cudaFree(m->idx);
  cudaFree(m->store);
  cudaFree(m->bw);
  cudaFree(m->loss);
  delete m;
  return BS_OK;
}

bs_status bs_mlp_params(bs_mlp m, float *params_host, int64_t n, int set) {
  BS_NVTX("bs_mlp_params");
  if (!m || !params_host) return BS_ERR_ARG;
  const long long np = n_params(m->dev.d, m->dev.w);
  const long long nn = np + 2 * m->dev.d + 2;
  if (n != nn) return lfail(m, BS_ERR_ARG, "expected " + std::to_string(nn) + " values");
  if (set) {
    ML_CUDA(cudaMemcpy(m->dev.p, params_host, np * 4, cudaMemcpyHostToDevice));
    ML_CUDA(cudaMemcpy(m->dev.norm, params_host + np, (nn - np) * 4, cudaMemcpyHostToDevice));
    m->step = 0;
    ML_CUDA(cudaMemset(m->dev.m, 0, np * 4));
    ML_CUDA(cudaMemset(m->dev.v, 0, np * 4));
  } else {
    ML_CUDA(cudaMemcpy(params_host, m->dev.p, np * 4, cudaMemcpyDeviceToHost));
    ML_CUDA(cudaMemcpy(params_host + np, m->dev.norm, (nn - np) * 4, cudaMemcpyDeviceToHost));
  }
  return BS_OK;
}

bs_status bs_mlp_fit_norm(bs_mlp m, const float *x_dev, const float *t_dev, int n, void *stream) {
  BS_NVTX("bs_mlp_fit_norm");
  if (!m || !x_dev || !t_dev || n < 2) return BS_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_mlp_colstats<<<m->dev.d + 1, 256, 0, s>>>(x_dev, t_dev, n, m->dev.d, m->dev.norm);
  ML_CUDA(cudaGetLastError());
  return BS_OK;
}

bs_status bs_mlp_forward(bs_mlp m, const float *x_dev, int n, float *y_dev, void *stream) {
  BS_NVTX("bs_mlp_forward");
  if (!m || !x_dev || !y_dev || n < 0) return BS_ERR_ARG;
  if (n == 0) return BS_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (m->tc) {
    ML_CUDA(mlp_tc_forward(m->dev, x_dev, n, nullptr, n, y_dev, nullptr, s));
    return BS_OK;
  }
  k_mlp_forward<<<(n + kRows - 1) / kRows, kRows, fwd_smem(m->dev.d, m->dev.w), s>>>(
      m->dev, x_dev, n, nullptr, n, y_dev, nullptr);
  ML_CUDA(cudaGetLastError());
  return BS_OK;
}

bs_status bs_mlp_set_kernels(bs_mlp m, int kind) {
  BS_NVTX("bs_mlp_set_kernels");
  if (!m || (kind != 0 && kind != 1)) return BS_ERR_ARG;
  if (kind == 0 && !mlp_tc_supported(m->dev.d, m->dev.w))
    return lfail(m, BS_ERR_UNSUPPORTED, "tensor-core kernels need width 128 and d_in <= 64");
  m->tc = kind == 0;
  return BS_OK;
}

bs_status bs_mlp_grad(bs_mlp m, const float *x_dev, const float *t_dev, int n, float *grad_host,
                      float *loss_host, void *stream) {
  BS_NVTX("bs_mlp_grad");
  if (!m || !x_dev || !t_dev || n < 1) return BS_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bs_status st = ensure_scratch(m, n);
  if (st != BS_OK) return st;
  const long long np = n_params(m->dev.d, m->dev.w);
  ML_CUDA(cudaMemsetAsync(m->dev.g, 0, np * 4, s));
  ML_CUDA(cudaMemsetAsync(m->loss, 0, 4, s));
  st = grad_batch(m, x_dev, t_dev, n, nullptr, n, s);
  if (st != BS_OK) return st;
  if (grad_host) ML_CUDA(cudaMemcpyAsync(grad_host, m->dev.g, np * 4, cudaMemcpyDeviceToHost, s));
  if (loss_host) ML_CUDA(cudaMemcpyAsync(loss_host, m->loss, 4, cudaMemcpyDeviceToHost, s));
  ML_CUDA(cudaStreamSynchronize(s));
  ML_CUDA(cudaMemsetAsync(m->dev.g, 0, np * 4, s));
  return BS_OK;
}

bs_status bs_mlp_train(bs_mlp m, const float *x_dev, const float *t_dev, int n, int steps,
                       int batch, float lr, uint64_t seed, float *loss_host, void *stream) {
  BS_NVTX("bs_mlp_train");
  if (!m || !x_dev || !t_dev || n < 1 || steps < 0 || batch < 1) return BS_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bs_status st = ensure_scratch(m, batch);
  if (st != BS_OK) return st;
  const long long np = n_params(m->dev.d, m->dev.w);
  for (int k = 0; k < steps; ++k) {
    ++m->step;
    k_mlp_sample<<<(batch + 255) / 256, 256, 0, s>>>(m->idx, batch, n, seed, m->step);
    ML_CUDA(cudaGetLastError());
    if (k == steps - 1) ML_CUDA(cudaMemsetAsync(m->loss, 0, 4, s));
    st = grad_batch(m, x_dev, t_dev, n, m->idx, batch, s);
    if (st != BS_OK) return st;
    k_mlp_adam<<<(int)std::min<long long>((np + 255) / 256, 1024), 256, 0, s>>>(
        m->dev, np, lr, 0.9f, 0.999f, 1e-8f, m->step);
    ML_CUDA(cudaGetLastError());
  }
  if (loss_host) {
    ML_CUDA(cudaMemcpyAsync(loss_host, m->loss, 4, cudaMemcpyDeviceToHost, s));
    ML_CUDA(cudaStreamSynchronize(s));
  }
  return BS_OK;
}

#define BS_CUDA(call)                                            \
  do {                                                           \
    cudaError_t e__ = (call);                                    \
    if (e__ != cudaSuccess) return cuda_fail(p, e__, #call);     \
  } while (0)

bs_status bs_mlp_features(bs_plan p, const uint8_t *flags_host, float *feat_dev, void *stream) {
  BS_NVTX("bs_mlp_features");
  if (!p || !feat_dev) return BS_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bs_status st = prepare(p, s);
  if (st != BS_OK) return st;
  if (!p->counts_ready) {
    st = run_counts(p, p->at<int8_t>(p->L.label), s);
    if (st != BS_OK) return st;
    p->counts_default = true;
  }
  const double r = p->d.r > 0 ? p->d.r : 1.0, rp = p->d.rprime > 0 ? p->d.rprime : 1.0,
               dnu = p->d.dnu_c > 0 ? p->d.dnu_c : 1.0;
  std::vector<float> tab((size_t)p->ntrip * 4 + 36);
  for (int t = 0; t < p->ntrip; ++t) {
    const int i = p->trips[3 * t], j = p->trips[3 * t + 1], l = p->trips[3 * t + 2];
    const bool ok = p->T[t] > 0;
    tab[4 * t] = ok ? (float)std::log((double)p->T[t]) : std::nanf("");
    tab[4 * t + 1] = (float)(2 * M_PI * p->umean[i] / r);
    tab[4 * t + 2] = (float)(2 * M_PI * p->umean[j] / r);
    tab[4 * t + 3] = (float)(2 * M_PI * p->umean[l] / r);
  }
  float *ff = tab.data() + (size_t)p->ntrip * 4;
  int nfl = 0;
  std::vector<int> pos_n(32, 0), pos_f(32, 0);
  for (int c = 0; c < p->nc; ++c) {
    const int f = flags_host && flags_host[c] ? 1 : 0;
    nfl += f;
    pos_n[c % 32] += 1;
    pos_f[c % 32] += f;
  }
  ff[0] = (float)nfl / p->nc;
  for (int q = 0; q < 32; ++q) ff[1 + q] = pos_n[q] ? (float)pos_f[q] / pos_n[q] : 0.f;
  // sampling of the Eq. (dft) square under this mask: folded counts N(d) of valid
  // channel triples at the separations -nc/2 <= d1, d2 < nc/2
  {
    const int nc = p->nc, n2 = 2 * nc - 1, h = nc / 2;
    std::vector<uint8_t> valid(nc);
    for (int c = 0; c < nc; ++c) valid[c] = (flags_host && flags_host[c]) ? 0 : 1;
    std::vector<long long> plane((size_t)n2 * n2, 0);
    const int full[6] = {0, nc, 0, nc, 0, nc};
    add_block_sampling(nc, valid, full, plane.data());
    double sinv = 0, ssum = 0;
    long long nsamp = 0;
    for (int d1 = -h; d1 < nc - h; ++d1)
      for (int d2 = -h; d2 < nc - h; ++d2) {
        long long c = plane[(size_t)(d1 + nc - 1) * n2 + d2 + nc - 1];
        if (d1 != 0 || d2 != 0) c += plane[(size_t)((long long)(nc - 1 - d1) * n2 + (nc - 1 - d2))];
        if (c > 0) {
          sinv += 1.0 / (double)c;
          ssum += (double)c;
          ++nsamp;
        }
      }
    ff[33] = nsamp ? (float)std::log(sinv) : 0.f;
    ff[34] = (float)nsamp / ((float)nc * nc);
    ff[35] = nsamp ? (float)std::log(ssum / nsamp) : 0.f;
  }
  float *dtab = p->at<float>(p->L.mlptab);
  BS_CUDA(cudaMemcpyAsync(dtab, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, s));
  const float kpar_unit = (float)(2 * M_PI / (rp * p->nc * dnu));
  const long long nbin = (long long)p->ntrip * p->nc * p->nc;
  k_mlp_features<<<(int)std::min<long long>((nbin + 255) / 256, 4096), 256, 0, s>>>(
      p->ntrip, p->nc, reinterpret_cast<const float4 *>(dtab), dtab + (size_t)p->ntrip * 4,
      kpar_unit, feat_dev);
  BS_CUDA(cudaGetLastError());
  BS_CUDA(cudaStreamSynchronize(s));  // the host table above is a temporary
  return BS_OK;
}

}  // extern "C"
