// Shared-memory Stockham autosort FFT (radix 8, 4, 2, 3, 5), FP32, used by the
// image-plane field kernels (Eq. iFT) and by the delay transform (Eq. dft).
//
// Formulation: for a length-N transform with radices R_1 ... R_s and
// p = R_1 ... R_{t-1} before stage t, every butterfly index i in [0, N/R)
// reads x[i + q N/R] (q < R), multiplies input q by w^(q k), k = i mod p,
// w = exp(sign 2 pi i / (p R)), applies the radix-R DFT and writes
// y[(i - k) R + k + q p].  Input and output of a stage ping-pong between two
// shared buffers; the result needs no bit reversal.  Twiddles come from a
// table tw[t] = exp(+2 pi i t / N) (FP64 on the host, rounded to FP32);
// sign = -1 uses the conjugate.
#pragma once

#include <cuda_runtime.h>

#include "bs_internal.h"

namespace bsi {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// multiply by sign * i
__device__ __forceinline__ float2 cmuli(float2 a, float sign) { return make_float2(-sign * a.y, sign * a.x); }

template <int R>
__device__ __forceinline__ void butterfly(float2 *u, float sign);

template <>
__device__ __forceinline__ void butterfly<2>(float2 *u, float) {
  float2 a = u[0], b = u[1];
  u[0] = cadd(a, b);
  u[1] = csub(a, b);
}

template <>
__device__ __forceinline__ void butterfly<4>(float2 *u, float sign) {
  float2 s02 = cadd(u[0], u[2]), d02 = csub(u[0], u[2]);
  float2 s13 = cadd(u[1], u[3]), d13 = cmuli(csub(u[1], u[3]), sign);
  u[0] = cadd(s02, s13);
  u[2] = csub(s02, s13);
  u[1] = cadd(d02, d13);
  u[3] = csub(d02, d13);
}

// Radix 8 as two radix-4 DFTs of the even and odd inputs, combined with
// w^k, w = exp(sign 2 pi i / 8): w = sqrt(1/2) (1 + sign i), w^2 = sign i,
// w^3 = sqrt(1/2) (-1 + sign i).
template <>
__device__ __forceinline__ void butterfly<8>(float2 *u, float sign) {
  float2 e[4] = {u[0], u[2], u[4], u[6]}, o[4] = {u[1], u[3], u[5], u[7]};
  butterfly<4>(e, sign);
  butterfly<4>(o, sign);
  const float h = 0.70710678118654752440f;
  const float2 o1 = make_float2(h * (o[1].x - sign * o[1].y), h * (o[1].y + sign * o[1].x));
  const float2 o2 = cmuli(o[2], sign);
  const float2 o3 = make_float2(h * (-o[3].x - sign * o[3].y), h * (sign * o[3].x - o[3].y));
  u[0] = cadd(e[0], o[0]);
  u[4] = csub(e[0], o[0]);
  u[1] = cadd(e[1], o1);
  u[5] = csub(e[1], o1);
  u[2] = cadd(e[2], o2);
  u[6] = csub(e[2], o2);
  u[3] = cadd(e[3], o3);
  u[7] = csub(e[3], o3);
}

template <>
__device__ __forceinline__ void butterfly<3>(float2 *u, float sign) {
  // w = exp(sign 2 pi i / 3) = -1/2 + sign i sqrt(3)/2
  const float c = -0.5f, s = 0.86602540378443864676f * sign;
  float2 a = u[0], b = u[1], d = u[2];
  float2 t = cadd(b, d);
  float2 m = make_float2(a.x + c * t.x, a.y + c * t.y);
  float2 q = csub(b, d);
  float2 rq = make_float2(-s * q.y, s * q.x);  // i s (b - d)
  u[0] = cadd(a, t);
  u[1] = cadd(m, rq);
  u[2] = csub(m, rq);
}

template <>
__device__ __forceinline__ void butterfly<5>(float2 *u, float sign) {
  // cos(2pi/5) = (sqrt5 - 1)/4, cos(4pi/5) = -(sqrt5 + 1)/4,
  // sin(2pi/5), sin(4pi/5) from sin^2 = 1 - cos^2.
  const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;
  const float s1 = 0.95105651629515357212f * sign, s2 = 0.58778525229247312917f * sign;
  float2 a = u[0];
  float2 t1 = cadd(u[1], u[4]), t2 = cadd(u[2], u[3]);
  float2 d1 = csub(u[1], u[4]), d2 = csub(u[2], u[3]);
  float2 m1 = make_float2(a.x + c1 * t1.x + c2 * t2.x, a.y + c1 * t1.y + c2 * t2.y);
  float2 m2 = make_float2(a.x + c2 * t1.x + c1 * t2.x, a.y + c2 * t1.y + c1 * t2.y);
  // i (s1 d1 + s2 d2) and i (s2 d1 - s1 d2)
  float2 e1 = make_float2(-(s1 * d1.y + s2 * d2.y), s1 * d1.x + s2 * d2.x);
  float2 e2 = make_float2(-(s2 * d1.y - s1 * d2.y), s2 * d1.x - s1 * d2.x);
  u[0] = cadd(a, cadd(t1, t2));
  u[1] = cadd(m1, e1);
  u[4] = csub(m1, e1);
  u[2] = cadd(m2, e2);
  u[3] = csub(m2, e2);
}

// Quotient n / d for 0 <= n < 2^20 from the FP32 reciprocal of d: the product
// is within 1/8 of the true quotient, so one correction step makes it exact
// (checked exhaustively for every stage divisor of the lengths up to 4096).
__device__ __forceinline__ int quot(int n, float inv_d, int d) {
  int q = __float2int_rz(__fmul_rn((float)n, inv_d));
  const int r = n - q * d;
  q += (r >= d) - (r < 0);
  return q;
}

template <int R>
__device__ __forceinline__ void stockham_stage(const float2 *__restrict__ x, float2 *__restrict__ y,
                                               int nrows, int N, int ld, int p, const float2 *tw,
                                               float sign) {
  const int NR = N / R;
  const int tstride = N / (p * R);
  const int total = nrows * NR;
  const float inv_nr = __fdiv_rn(1.0f, (float)NR), inv_p = __fdiv_rn(1.0f, (float)p);
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int row = quot(idx, inv_nr, NR);
    const int i = idx - row * NR;
    const float2 *xr = x + row * ld;
    float2 *yr = y + row * ld;
    const int k = i - quot(i, inv_p, p) * p;
    float2 u[R];
#pragma unroll
    for (int q = 0; q < R; ++q) u[q] = xr[i + q * NR];
    if (k != 0) {
#pragma unroll
      for (int q = 1; q < R; ++q) {
        float2 w = tw[q * k * tstride];
        w.y *= sign;
        u[q] = cmul(u[q], w);
      }
    }
    butterfly<R>(u, sign);
    const int j = (i - k) * R + k;
#pragma unroll
    for (int q = 0; q < R; ++q) yr[j + q * p] = u[q];
  }
}

// Compile-time stage sequence of a length N (the same radices, in the same
// order, as factor_radices: 8s, then 4s, 2s, 3s, 5s).  With N, R and p known at
// compile time the row / butterfly / twiddle index arithmetic of a stage
// reduces to constant multiplies and shifts, and the stages unroll.
__host__ __device__ constexpr int ct_radix(int N, int s) {
  int m = N, k = 0;
  const int rs[5] = {8, 4, 2, 3, 5};
  for (int t = 0; t < 5; ++t)
    while (m % rs[t] == 0) {
      if (k == s) return rs[t];
      m /= rs[t];
      ++k;
    }
  return 0;
}
__host__ __device__ constexpr int ct_nstages(int N) {
  int s = 0;
  while (ct_radix(N, s)) ++s;
  return s;
}

template <int N, int R, int P>
__device__ __forceinline__ void stockham_stage_ct(const float2 *__restrict__ x,
                                                  float2 *__restrict__ y, int nrows, int ld,
                                                  const float2 *tw, float sign) {
  constexpr int NR = N / R;
  constexpr int tstride = N / (P * R);
  const int total = nrows * NR;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int row = idx / NR;
    const int i = idx - row * NR;
    const float2 *xr = x + row * ld;
    float2 *yr = y + row * ld;
    const int k = i % P;
    float2 u[R];
#pragma unroll
    for (int q = 0; q < R; ++q) u[q] = xr[i + q * NR];
    if constexpr (P > 1) {
      if (k != 0) {
        const int kt = k * tstride;
#pragma unroll
        for (int q = 1; q < R; ++q) {
          float2 w = tw[q * kt];
          w.y *= sign;
          u[q] = cmul(u[q], w);
        }
      }
    }
    butterfly<R>(u, sign);
    const int j = (i - k) * R + k;
#pragma unroll
    for (int q = 0; q < R; ++q) yr[j + q * P] = u[q];
  }
}

template <int N, int S, int P>
__device__ __forceinline__ float2 *stockham_ct(float2 *x, float2 *y, int nrows, int ld,
                                               const float2 *tw, float sign) {
  if constexpr (S < ct_nstages(N)) {
    constexpr int R = ct_radix(N, S);
    stockham_stage_ct<N, R, P>(x, y, nrows, ld, tw, sign);
    __syncthreads();
    return stockham_ct<N, S + 1, P * R>(y, x, nrows, ld, tw, sign);
  } else {
    return x;
  }
}

// Runtime stage loop for the lengths without a compiled sequence.
__device__ __forceinline__ float2 *stockham_rt(float2 *x, float2 *y, int nrows, int N, int ld,
                                               const Radices &rad, const float2 *tw, float sign) {
  int p = 1;
  for (int s = 0; s < rad.n; ++s) {
    const int R = rad.r[s];
    switch (R) {
      case 8: stockham_stage<8>(x, y, nrows, N, ld, p, tw, sign); break;
      case 4: stockham_stage<4>(x, y, nrows, N, ld, p, tw, sign); break;
      case 2: stockham_stage<2>(x, y, nrows, N, ld, p, tw, sign); break;
      case 3: stockham_stage<3>(x, y, nrows, N, ld, p, tw, sign); break;
      default: stockham_stage<5>(x, y, nrows, N, ld, p, tw, sign); break;
    }
    __syncthreads();
    float2 *t = x;
    x = y;
    y = t;
    p *= R;
  }
  return x;
}

// In-place (ping-pong) transform of nrows rows of length N, row r at x + r ld
// (ld >= N; ld = N + 1 keeps column-wise accesses of power-of-two rows off a
// single bank); y is scratch of the same size.  All threads of the block must
// call it.  Returns the buffer that holds the result.  The image sides of
// per-triple planes (2^a x {8, 12}) and the usual channel counts take the
// compiled stage sequences.
__device__ __forceinline__ float2 *stockham(float2 *x, float2 *y, int nrows, int N, int ld,
                                            const Radices &rad, const float2 *tw, float sign) {
  switch (N) {
    case 16: return stockham_ct<16, 0, 1>(x, y, nrows, ld, tw, sign);
    case 24: return stockham_ct<24, 0, 1>(x, y, nrows, ld, tw, sign);
    case 32: return stockham_ct<32, 0, 1>(x, y, nrows, ld, tw, sign);
    case 48: return stockham_ct<48, 0, 1>(x, y, nrows, ld, tw, sign);
    case 64: return stockham_ct<64, 0, 1>(x, y, nrows, ld, tw, sign);
    case 96: return stockham_ct<96, 0, 1>(x, y, nrows, ld, tw, sign);
    case 128: return stockham_ct<128, 0, 1>(x, y, nrows, ld, tw, sign);
    case 192: return stockham_ct<192, 0, 1>(x, y, nrows, ld, tw, sign);
    case 256: return stockham_ct<256, 0, 1>(x, y, nrows, ld, tw, sign);
    case 384: return stockham_ct<384, 0, 1>(x, y, nrows, ld, tw, sign);
    case 512: return stockham_ct<512, 0, 1>(x, y, nrows, ld, tw, sign);
    case 768: return stockham_ct<768, 0, 1>(x, y, nrows, ld, tw, sign);
    default: return stockham_rt(x, y, nrows, N, ld, rad, tw, sign);
  }
}
__device__ __forceinline__ float2 *stockham(float2 *x, float2 *y, int nrows, int N,
                                            const Radices &rad, const float2 *tw, float sign) {
  return stockham(x, y, nrows, N, N, rad, tw, sign);
}

}  // namespace bsi
