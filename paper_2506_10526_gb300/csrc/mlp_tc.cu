// Error-bar surrogate on the tensor cores: the forward pass, the per-row
// backward and the weight gradients of the width-128 network as BF16
// mma.sync (m16n8k16, FP32 accumulation).  The FP32 SIMT kernels of mlp.cu
// compute the same quantities and serve as the checker.
//
// Precision.  The network's weights are BF16 values by definition (the FP32
// masters rounded when staged), so a weight operand is exact in BF16.  Every
// other operand x (activations, normalised inputs, back-propagated dz) is
// split x = hi + lo, hi = bf16(x), lo = bf16(x - hi): 16 significant bits.
// Forward and dz1 products take W hi + W lo (two MMAs); the weight gradients
// (both operands split) take hi hi + hi lo + lo hi (three MMAs; lo lo is
// below 2^-16 of the term).  Accumulation is FP32 throughout.
//
// Fragment layouts (PTX ISA, mma.m16n8k16 with .bf16 operands): g = lane / 4,
// t = lane % 4.  A (16 x 16, row major): a0 = (g, 2t..2t+1), a1 = (g + 8,
// 2t..), a2 = (g, 2t + 8..), a3 = (g + 8, 2t + 8..).  B (16 x 8, K x N):
// b0 = (k = 2t..2t+1, n = g), b1 = (k = 2t + 8.., n = g).  C (16 x 8):
// c0, c1 = (g, 2t..2t+1), c2, c3 = (g + 8, 2t..).  The lower half of each
// 32-bit register holds the element with the smaller index.  A C tile pair
// (n-tiles 2kk, 2kk + 1) is exactly the A fragment of k-step kk of the next
// layer, so activations stay in registers between the layers.
//
// Kernels (8 warps, 16 rows per warp, 128 rows per CTA):
//   forward       h1 = tanh(W1 xn + b1), h2 = tanh(W2 h1 + b2), yn = w3.h2 + b3
//   backward rows dz2 = dyn w3 (1 - h2^2), dz1 = (W2^T dz2)(1 - h1^2)
//   wgrad         dW1 = dz1^T xn, dW2 = dz2^T h1 over a 128-row chunk per CTA
//                 (operands staged transposed in shared memory), FP32 atomics
//                 into the gradient; biases and the output layer in FP32.
#include <cuda_bf16.h>

#include "bs_internal.h"
#include "mlp_internal.h"

namespace bsi {

namespace {

constexpr int W = 128;           // hidden width of the tensor-core kernels
constexpr int kWarps = 8, kThreads = 32 * kWarps, kRowsPerCta = 16 * kWarps;
constexpr int LD2 = W + 8;       // bf16 pitch of the staged W2 (conflict-free fragments)
constexpr int LDR = kRowsPerCta + 8;  // bf16 pitch of the transposed wgrad operands

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}
// hi / lo BF16 parts of two consecutive elements, packed
__device__ __forceinline__ void split2(float x0, float x1, uint32_t &hi, uint32_t &lo) {
  const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
  const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
  const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
  hi = pack2(h0, h1);
  lo = pack2(l0, l1);
}

__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// W1 [W][d] as BF16 rows of pitch K1 + 8 (zero beyond d), W2 [W][W] of pitch
// LD2, biases and w3 in FP32 (w3 BF16-rounded, as the network defines it).
template <int K1>
__device__ void stage_net(const MlpDev &M, __nv_bfloat16 *W1s, __nv_bfloat16 *W2s, float *b1,
                          float *b2, float *w3) {
  constexpr int LD1 = K1 + 8;
  const int d = M.d;
  const float *p = M.p;
  for (int q = threadIdx.x; q < W * K1; q += blockDim.x) {
    const int j = q / K1, k = q - j * K1;
    W1s[j * LD1 + k] = __float2bfloat16_rn(k < d ? p[j * d + k] : 0.f);
  }
  p += W * d;
  for (int q = threadIdx.x; q < W; q += blockDim.x) b1[q] = p[q];
  p += W;
  for (int q = threadIdx.x; q < W * W; q += blockDim.x) {
    const int j = q / W, k = q - j * W;
    W2s[j * LD2 + k] = __float2bfloat16_rn(p[q]);
  }
  p += W * W;
  for (int q = threadIdx.x; q < W; q += blockDim.x) b2[q] = p[q];
  p += W;
  for (int q = threadIdx.x; q < W; q += blockDim.x) w3[q] = __bfloat162float(__float2bfloat16_rn(p[q]));
}

// B fragment (k = 2t.., n = g) of a weight matrix stored [n][k] with pitch ld:
// two consecutive k of one row, one 32-bit load
__device__ __forceinline__ uint32_t bfrag_nk(const __nv_bfloat16 *Ws, int ld, int n, int k) {
  return *reinterpret_cast<const uint32_t *>(Ws + n * ld + k);
}

// Forward for rows[r] = idx ? idx[r] : r.  y (denormalised) and, when store
// is set, per row [xn (d) | h1 (W) | h2 (W) | yn].
template <int K1>
__global__ void __launch_bounds__(kThreads) k_mlp_tc_forward(MlpDev M, const float *__restrict__ x,
                                                             int n, const int *__restrict__ idx,
                                                             int nrows, float *__restrict__ y,
                                                             float *__restrict__ store) {
  constexpr int LD1 = K1 + 8, KS1 = K1 / 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __nv_bfloat16 *W1s = reinterpret_cast<__nv_bfloat16 *>(smem_raw);
  __nv_bfloat16 *W2s = W1s + W * LD1;
  float *b1 = reinterpret_cast<float *>(W2s + W * LD2), *b2 = b1 + W, *w3 = b2 + W;
  stage_net<K1>(M, W1s, W2s, b1, b2, w3);
  __syncthreads();
  const int d = M.d, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  // the warp's rows g and g + 8
  const int r0 = blockIdx.x * kRowsPerCta + warp * 16 + g, r1 = r0 + 8;
  int row0 = -1, row1 = -1;
  if (r0 < nrows) row0 = idx ? idx[r0] : r0;
  if (r1 < nrows) row1 = idx ? idx[r1] : r1;
  const bool ok0 = row0 >= 0 && row0 < n, ok1 = row1 >= 0 && row1 < n;
  const float *mu = M.norm, *sd = M.norm + d;
  const int sw = d + 2 * W + 1;
  float *st0 = (store && ok0) ? store + (long long)r0 * sw : nullptr;
  float *st1 = (store && ok1) ? store + (long long)r1 * sw : nullptr;
  // layer 1: A = xn (hi, lo), B = W1^T
  float c[16][4];
#pragma unroll
  for (int j = 0; j < 16; ++j) c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.f;
#pragma unroll
  for (int kk = 0; kk < KS1; ++kk) {
    float v[8];  // (row, col): (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1), then cols + 8
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int col = 16 * kk + 2 * t + (q & 1) + ((q >> 2) << 3);
      const bool hi_row = (q >> 1) & 1;
      const bool okr = hi_row ? ok1 : ok0;
      const int row = hi_row ? row1 : row0;
      float xv = 0.f;
      if (okr && col < d) {
        xv = (x[(long long)row * d + col] - mu[col]) / sd[col];
        float *st = hi_row ? st1 : st0;
        if (st) st[col] = xv;
      }
      v[q] = xv;
    }
    uint32_t ah[4], al[4];
    split2(v[0], v[1], ah[0], al[0]);
    split2(v[2], v[3], ah[1], al[1]);
    split2(v[4], v[5], ah[2], al[2]);
    split2(v[6], v[7], ah[3], al[3]);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint32_t b0 = bfrag_nk(W1s, LD1, 8 * j + g, 16 * kk + 2 * t);
      const uint32_t bb = bfrag_nk(W1s, LD1, 8 * j + g, 16 * kk + 2 * t + 8);
      mma16816(c[j], ah, b0, bb);
      mma16816(c[j], al, b0, bb);
    }
  }
  // h1 = tanh(z1 + b1) -> A fragments of layer 2
  uint32_t a2h[8][4], a2l[8][4];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int col = 8 * j + 2 * t;
    const float h00 = tanhf(c[j][0] + b1[col]), h01 = tanhf(c[j][1] + b1[col + 1]);
    const float h10 = tanhf(c[j][2] + b1[col]), h11 = tanhf(c[j][3] + b1[col + 1]);
    if (st0) {
      st0[d + col] = h00;
      st0[d + col + 1] = h01;
    }
    if (st1) {
      st1[d + col] = h10;
      st1[d + col + 1] = h11;
    }
    const int kk = j >> 1, hs = (j & 1) * 2;  // n-tile 2kk -> a0, a1; 2kk + 1 -> a2, a3
    split2(h00, h01, a2h[kk][hs], a2l[kk][hs]);
    split2(h10, h11, a2h[kk][hs + 1], a2l[kk][hs + 1]);
  }
  // layer 2 in two halves of 8 n-tiles; yn accumulates on the fly
  float y0 = 0.f, y1 = 0.f;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    float c2[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) c2[j][0] = c2[j][1] = c2[j][2] = c2[j][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int nrow = 8 * (8 * half + j) + g;
        const uint32_t b0 = bfrag_nk(W2s, LD2, nrow, 16 * kk + 2 * t);
        const uint32_t bb = bfrag_nk(W2s, LD2, nrow, 16 * kk + 2 * t + 8);
        mma16816(c2[j], a2h[kk], b0, bb);
        mma16816(c2[j], a2l[kk], b0, bb);
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int col = 8 * (8 * half + j) + 2 * t;
      const float h00 = tanhf(c2[j][0] + b2[col]), h01 = tanhf(c2[j][1] + b2[col + 1]);
      const float h10 = tanhf(c2[j][2] + b2[col]), h11 = tanhf(c2[j][3] + b2[col + 1]);
      y0 = fmaf(w3[col], h00, fmaf(w3[col + 1], h01, y0));
      y1 = fmaf(w3[col], h10, fmaf(w3[col + 1], h11, y1));
      if (st0) {
        st0[d + W + col] = h00;
        st0[d + W + col + 1] = h01;
      }
      if (st1) {
        st1[d + W + col] = h10;
        st1[d + W + col + 1] = h11;
      }
    }
  }
  // the four threads of a group hold the row's partial dot products
  y0 += __shfl_xor_sync(0xffffffffu, y0, 1);
  y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
  y1 += __shfl_xor_sync(0xffffffffu, y1, 1);
  y1 += __shfl_xor_sync(0xffffffffu, y1, 2);
  if (t == 0) {
    const float b3 = M.p[(long long)W * d + W + W * W + W + W];
    const float yn0 = y0 + b3, yn1 = y1 + b3;
    const float my = M.norm[2 * d], sy = M.norm[2 * d + 1];
    if (ok0) {
      if (st0) st0[d + 2 * W] = yn0;
      if (y) y[r0] = my + sy * yn0;
    }
    if (ok1) {
      if (st1) st1[d + 2 * W] = yn1;
      if (y) y[r1] = my + sy * yn1;
    }
  }
}

// Per-row backward: dyn = 2 (yn - tn) / nrows, dz2 = dyn w3 (1 - h2^2),
// dz1 = (W2^T dz2)(1 - h1^2).  bw rows [dz1 (W) | dz2 (W) | dyn]; loss += mean
// of squared residuals.
__global__ void __launch_bounds__(kThreads) k_mlp_tc_backward_rows(
    MlpDev M, const float *__restrict__ tgt, const int *__restrict__ idx, int nrows,
    const float *__restrict__ store, float *__restrict__ bw, float *__restrict__ loss) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __nv_bfloat16 *W2s = reinterpret_cast<__nv_bfloat16 *>(smem_raw);  // [j][k], pitch LD2
  float *w3 = reinterpret_cast<float *>(W2s + W * LD2);
  const int d = M.d;
  {
    const float *p = M.p + (long long)W * d + W;
    for (int q = threadIdx.x; q < W * W; q += blockDim.x) {
      const int j = q / W, k = q - j * W;
      W2s[j * LD2 + k] = __float2bfloat16_rn(p[q]);
    }
    for (int q = threadIdx.x; q < W; q += blockDim.x)
      w3[q] = __bfloat162float(__float2bfloat16_rn(p[W * W + W + q]));
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int r0 = blockIdx.x * kRowsPerCta + warp * 16 + g, r1 = r0 + 8;
  const bool ok0 = r0 < nrows, ok1 = r1 < nrows;
  const int sw = d + 2 * W + 1, bwid = 2 * W + 1;
  const float *s0 = store + (long long)(ok0 ? r0 : 0) * sw;
  const float *s1 = store + (long long)(ok1 ? r1 : 0) * sw;
  float *o0 = bw + (long long)(ok0 ? r0 : 0) * bwid;
  float *o1 = bw + (long long)(ok1 ? r1 : 0) * bwid;
  const float my = M.norm[2 * d], sy = M.norm[2 * d + 1];
  float dyn0 = 0.f, dyn1 = 0.f, l2 = 0.f;
  if (ok0) {
    const float res = s0[d + 2 * W] - (tgt[idx ? idx[r0] : r0] - my) / sy;
    dyn0 = 2.f * res / (float)nrows;
    if (t == 0) l2 += res * res;
  }
  if (ok1) {
    const float res = s1[d + 2 * W] - (tgt[idx ? idx[r1] : r1] - my) / sy;
    dyn1 = 2.f * res / (float)nrows;
    if (t == 0) l2 += res * res;
  }
  // dz2 in A-fragment order (k-step kk covers j = 16 kk .. 16 kk + 15)
  uint32_t ah[8][4], al[8][4];
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {  // a0: (g, 2t), a1: (g+8, 2t), a2: (g, 2t+8), a3: (g+8, 2t+8)
      const int j = 16 * kk + 2 * t + ((q >> 1) << 3);
      const bool hi_row = q & 1;
      const float *sr = hi_row ? s1 : s0;
      const float dyn = hi_row ? dyn1 : dyn0;
      const bool okr = hi_row ? ok1 : ok0;
      float z0 = 0.f, z1 = 0.f;
      if (okr) {
        const float h0 = sr[d + W + j], h1 = sr[d + W + j + 1];
        z0 = dyn * w3[j] * (1.f - h0 * h0);
        z1 = dyn * w3[j + 1] * (1.f - h1 * h1);
        float *o = hi_row ? o1 : o0;
        o[W + j] = z0;
        o[W + j + 1] = z1;
      }
      split2(z0, z1, ah[kk][q], al[kk][q]);
    }
  }
  // dz1 pre-activation: sum_j dz2_j W2[j][k]; B = W2 as (K = j) x (N = k), two
  // 16-bit loads per register (consecutive j are a row apart)
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    float c[8][4];
#pragma unroll
    for (int n = 0; n < 8; ++n) c[n][0] = c[n][1] = c[n][2] = c[n][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
#pragma unroll
      for (int n = 0; n < 8; ++n) {
        const int kcol = 8 * (8 * half + n) + g;
        const int j = 16 * kk + 2 * t;
        const uint32_t b0 = pack2(W2s[j * LD2 + kcol], W2s[(j + 1) * LD2 + kcol]);
        const uint32_t bb = pack2(W2s[(j + 8) * LD2 + kcol], W2s[(j + 9) * LD2 + kcol]);
        mma16816(c[n], ah[kk], b0, bb);
        mma16816(c[n], al[kk], b0, bb);
      }
    }
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const int k = 8 * (8 * half + n) + 2 * t;
      if (ok0) {
        const float h0 = s0[d + k], h1 = s0[d + k + 1];
        o0[k] = c[n][0] * (1.f - h0 * h0);
        o0[k + 1] = c[n][1] * (1.f - h1 * h1);
      }
      if (ok1) {
        const float h0 = s1[d + k], h1 = s1[d + k + 1];
        o1[k] = c[n][2] * (1.f - h0 * h0);
        o1[k + 1] = c[n][3] * (1.f - h1 * h1);
      }
    }
  }
  if (t == 0) {
    if (ok0) o0[2 * W] = dyn0;
    if (ok1) o1[2 * W] = dyn1;
  }
  for (int off = 16; off > 0; off >>= 1) l2 += __shfl_xor_sync(0xffffffffu, l2, off);
  if (loss && lane == 0) atomicAdd(loss, l2 / (float)nrows);
}

// Weight gradients over one 128-row chunk: blockIdx.y = 0: dW1 = dz1^T xn and
// db1; 1: dW2 = dz2^T h1, db2, and the output layer dw3 = dyn^T h2, db3 (FP32).
// A = dz^T [W][r] and B = in^T [KN][r] are staged in shared memory, r
// contiguous, as BF16 hi / lo.
template <int K1>
__global__ void __launch_bounds__(kThreads) k_mlp_tc_wgrad(MlpDev M, int nrows,
                                                           const float *__restrict__ store,
                                                           const float *__restrict__ bw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int layer = blockIdx.y;
  const int d = M.d;
  const int KN = layer == 0 ? K1 : W;  // inputs of the layer (padded)
  __nv_bfloat16 *Ah = reinterpret_cast<__nv_bfloat16 *>(smem_raw);
  __nv_bfloat16 *Al = Ah + W * LDR;
  __nv_bfloat16 *Bh = Al + W * LDR;
  __nv_bfloat16 *Bl = Bh + KN * LDR;
  const int r0 = blockIdx.x * kRowsPerCta;
  const int sw = d + 2 * W + 1, bwid = 2 * W + 1;
  float *gW1 = M.g, *gb1 = gW1 + W * d, *gW2 = gb1 + W, *gb2 = gW2 + W * W, *gw3 = gb2 + W,
        *gb3 = gw3 + W;
  const int zoff = layer == 0 ? 0 : W, ioff = layer == 0 ? 0 : d;
  // stage dz^T (and the bias sums: each thread keeps one j)
  float bsum = 0.f;
  for (int e = threadIdx.x; e < kRowsPerCta * W; e += blockDim.x) {
    const int r = e / W, j = e - r * W;
    const float z = (r0 + r < nrows) ? bw[(long long)(r0 + r) * bwid + zoff + j] : 0.f;
    bsum += z;
    const __nv_bfloat16 h = __float2bfloat16_rn(z);
    Ah[j * LDR + r] = h;
    Al[j * LDR + r] = __float2bfloat16_rn(z - __bfloat162float(h));
  }
  atomicAdd((layer == 0 ? gb1 : gb2) + (threadIdx.x % W), bsum);
  for (int e = threadIdx.x; e < kRowsPerCta * KN; e += blockDim.x) {
    const int r = e / KN, k = e - r * KN;
    const bool live = r0 + r < nrows && (layer == 1 || k < d);
    const float v = live ? store[(long long)(r0 + r) * sw + ioff + k] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    Bh[k * LDR + r] = h;
    Bl[k * LDR + r] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
  if (layer == 1 && threadIdx.x < W) {  // output layer, FP32
    const int k = threadIdx.x;
    float acc = 0.f, db = 0.f;
    for (int r = r0; r < min(nrows, r0 + kRowsPerCta); ++r) {
      const float dyn = bw[(long long)r * bwid + 2 * W];
      acc = fmaf(dyn, store[(long long)r * sw + d + W + k], acc);
      db += dyn;
    }
    atomicAdd(gw3 + k, acc);
    if (k == 0) atomicAdd(gb3, db);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int jr = 16 * warp + g;  // output rows jr, jr + 8
  float c[W / 8][4];
#pragma unroll
  for (int n = 0; n < W / 8; ++n) c[n][0] = c[n][1] = c[n][2] = c[n][3] = 0.f;
  const int NT = KN / 8;
#pragma unroll
  for (int kk = 0; kk < kRowsPerCta / 16; ++kk) {
    const int rc = 16 * kk + 2 * t;
    uint32_t ah[4], al[4];
    ah[0] = *reinterpret_cast<const uint32_t *>(Ah + jr * LDR + rc);
    ah[1] = *reinterpret_cast<const uint32_t *>(Ah + (jr + 8) * LDR + rc);
    ah[2] = *reinterpret_cast<const uint32_t *>(Ah + jr * LDR + rc + 8);
    ah[3] = *reinterpret_cast<const uint32_t *>(Ah + (jr + 8) * LDR + rc + 8);
    al[0] = *reinterpret_cast<const uint32_t *>(Al + jr * LDR + rc);
    al[1] = *reinterpret_cast<const uint32_t *>(Al + (jr + 8) * LDR + rc);
    al[2] = *reinterpret_cast<const uint32_t *>(Al + jr * LDR + rc + 8);
    al[3] = *reinterpret_cast<const uint32_t *>(Al + (jr + 8) * LDR + rc + 8);
#pragma unroll
    for (int n = 0; n < W / 8; ++n) {
      if (n < NT) {
        const int kb = (8 * n + g) * LDR + rc;
        const uint32_t bh0 = *reinterpret_cast<const uint32_t *>(Bh + kb);
        const uint32_t bh1 = *reinterpret_cast<const uint32_t *>(Bh + kb + 8);
        const uint32_t bl0 = *reinterpret_cast<const uint32_t *>(Bl + kb);
        const uint32_t bl1 = *reinterpret_cast<const uint32_t *>(Bl + kb + 8);
        mma16816(c[n], ah, bh0, bh1);
        mma16816(c[n], ah, bl0, bl1);
        mma16816(c[n], al, bh0, bh1);
      }
    }
  }
  float *gW = layer == 0 ? gW1 : gW2;
  const int ldw = layer == 0 ? d : W;
#pragma unroll
  for (int n = 0; n < W / 8; ++n) {
    if (n < NT) {
      const int k = 8 * n + 2 * t;
      if (k < ldw) {
        atomicAdd(gW + jr * ldw + k, c[n][0]);
        atomicAdd(gW + (jr + 8) * ldw + k, c[n][2]);
      }
      if (k + 1 < ldw) {
        atomicAdd(gW + jr * ldw + k + 1, c[n][1]);
        atomicAdd(gW + (jr + 8) * ldw + k + 1, c[n][3]);
      }
    }
  }
}

template <int K1>
size_t fwd_smem_tc() {
  return (size_t)W * (K1 + 8) * 2 + (size_t)W * LD2 * 2 + 3 * W * sizeof(float);
}
size_t bwd_smem_tc() { return (size_t)W * LD2 * 2 + W * sizeof(float); }
size_t wgrad_smem_tc() { return (size_t)4 * W * LDR * 2; }

template <int K1>
cudaError_t forward_k(const MlpDev &M, const float *x, int n, const int *idx, int nrows, float *y,
                      float *store, cudaStream_t s) {
  cudaError_t e = smem_optin_once<k_mlp_tc_forward<K1>>();
  if (e != cudaSuccess) return e;
  k_mlp_tc_forward<K1><<<(nrows + kRowsPerCta - 1) / kRowsPerCta, kThreads, fwd_smem_tc<K1>(), s>>>(
      M, x, n, idx, nrows, y, store);
  return cudaGetLastError();
}

template <int K1>
cudaError_t wgrad_k(const MlpDev &M, int nrows, const float *store, const float *bw,
                    cudaStream_t s) {
  cudaError_t e = smem_optin_once<k_mlp_tc_wgrad<K1>>();
  if (e != cudaSuccess) return e;
  dim3 grid((nrows + kRowsPerCta - 1) / kRowsPerCta, 2);
  k_mlp_tc_wgrad<K1><<<grid, kThreads, wgrad_smem_tc(), s>>>(M, nrows, store, bw);
  return cudaGetLastError();
}

}  // namespace

bool mlp_tc_supported(int d, int w) { return w == W && d >= 1 && d <= 64; }

cudaError_t mlp_tc_forward(const MlpDev &M, const float *x, int n, const int *idx, int nrows,
                           float *y, float *store, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  const int k1 = (M.d + 15) / 16 * 16;
  switch (k1) {
    case 16: return forward_k<16>(M, x, n, idx, nrows, y, store, s);
    case 32: return forward_k<32>(M, x, n, idx, nrows, y, store, s);
    case 48: return forward_k<48>(M, x, n, idx, nrows, y, store, s);
    default: return forward_k<64>(M, x, n, idx, nrows, y, store, s);
  }
}

cudaError_t mlp_tc_backward_rows(const MlpDev &M, const float *t, const int *idx, int nrows,
                                 const float *store, float *bw, float *loss, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  cudaError_t e = smem_optin_once<k_mlp_tc_backward_rows>();
  if (e != cudaSuccess) return e;
  k_mlp_tc_backward_rows<<<(nrows + kRowsPerCta - 1) / kRowsPerCta, kThreads, bwd_smem_tc(), s>>>(
      M, t, idx, nrows, store, bw, loss);
  return cudaGetLastError();
}

cudaError_t mlp_tc_wgrad(const MlpDev &M, int nrows, const float *store, const float *bw,
                         cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  const int k1 = (M.d + 15) / 16 * 16;
  switch (k1) {
    case 16: return wgrad_k<16>(M, nrows, store, bw, s);
    case 32: return wgrad_k<32>(M, nrows, store, bw, s);
    case 48: return wgrad_k<48>(M, nrows, store, bw, s);
    default: return wgrad_k<64>(M, nrows, store, bw, s);
  }
}

}  // namespace bsi
