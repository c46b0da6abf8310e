// Exact FP32 <-> FP64 conversions from the IEEE 754 bit fields, for host and
// device.  GB300 executes FP64 arithmetic and FP32 <-> FP64 conversions on a
// narrow pipe (1.05 TFLOP/s FP64 FMA measured), so the delay-transform passes
// convert with these integer operations instead.
#pragma once

#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

namespace bsi {
namespace fpb {

__host__ __device__ __forceinline__ uint32_t bits_f(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  uint32_t b;
  std::memcpy(&b, &x, 4);
  return b;
#endif
}
__host__ __device__ __forceinline__ float from_f(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float x;
  std::memcpy(&x, &b, 4);
  return x;
#endif
}
__host__ __device__ __forceinline__ uint64_t bits_d(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  std::memcpy(&b, &x, 8);
  return b;
#endif
}
__host__ __device__ __forceinline__ double from_d(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  std::memcpy(&x, &b, 8);
  return x;
#endif
}
__host__ __device__ __forceinline__ int clz32(uint32_t x) {
#ifdef __CUDA_ARCH__
  return __clz((int)x);
#else
  return __builtin_clz(x);
#endif
}

// x * 2^e2 as FP64, exact for finite x (FP32 subnormals normalised by their
// leading bit) as long as the result stays within FP64's normal range;
// zeros keep their sign, infinities and NaNs map to their FP64 kind.
__host__ __device__ __forceinline__ double f32_to_f64_pow2(float x, int e2) {
  const uint32_t b = bits_f(x);
  const uint64_t sign = (uint64_t)(b >> 31) << 63;
  const uint32_t ex = (b >> 23) & 0xffu, m = b & 0x7fffffu;
  uint64_t bits;
  if (ex == 0xffu) {
    bits = sign | (0x7ffull << 52) | ((uint64_t)m << 29);
  } else if (ex == 0u) {
    if (m == 0u) {
      bits = sign;
    } else {  // m 2^-149 with the leading bit of m at position p
      const int p = 31 - clz32(m);
      const uint64_t man = ((uint64_t)m << (52 - p)) & ((1ull << 52) - 1);
      bits = sign | ((uint64_t)(p - 149 + 1023 + e2) << 52) | man;
    }
  } else {
    bits = sign | ((uint64_t)((int)ex - 127 + 1023 + e2) << 52) | ((uint64_t)m << 29);
  }
  return from_d((uint64_t)bits);
}

// x rounded to the nearest FP32 (ties to even), as the IEEE conversion
// defines it, from the FP64 bit fields.
__host__ __device__ __forceinline__ float f64_to_f32_rn(double x) {
  const uint64_t b = bits_d(x);
  const uint32_t sign = (uint32_t)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7ffu);
  const uint64_t m = b & ((1ull << 52) - 1);
  if (e == 0x7ff) return from_f(sign | 0x7f800000u | (m ? 0x400000u : 0u));
  const int E = e - 1023 + 127;  // FP32 biased exponent
  if (E >= 255) return from_f(sign | 0x7f800000u);
  uint64_t M;
  int sh;
  if (E >= 1) {  // normal: drop 29 bits
    M = m;
    sh = 29;
  } else {  // FP32 subnormal or zero: the implicit bit joins, 29 + 1 - E bits go
    if (E < -25 || e == 0) return from_f(sign);
    M = m | (1ull << 52);
    sh = 30 - E;
  }
  const uint64_t keep = M >> sh, rem = M & ((1ull << sh) - 1), half = 1ull << (sh - 1);
  const uint32_t up = (rem > half || (rem == half && (keep & 1ull))) ? 1u : 0u;
  // a carry out of the mantissa raises the exponent field (to infinity at the top)
  const uint32_t body = (E >= 1 ? ((uint32_t)E << 23) | (uint32_t)(keep & 0x7fffffu)
                                : (uint32_t)keep) + up;
  return from_f(sign | body);
}

}  // namespace fpb
}  // namespace bsi
