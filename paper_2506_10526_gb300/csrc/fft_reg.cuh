// Register-resident FFT of lengths N = N1 x N2 (N1, N2 <= 32), FP32, for the
// image-plane field passes (Eq. iFT).
//
// Four-step form: with input index n = n2 + N2 n1 and output index
// k = k1 + N1 k2,
//   X[k1 + N1 k2] = sum_{n2} w_N2^(n2 k2) [ w_N^(n2 k1) sum_{n1} x[n2 + N2 n1] w_N1^(n1 k1) ],
// w_L = exp(S 2 pi i / L).  Pass 1: one thread per (row, n2) takes the N1
// inputs of stride N2 into registers, applies the length-N1 DFT, multiplies by
// w_N^(n2 k1) (a shared table in [k1][n2] order) and writes row k1 of a padded
// shared tile.  Pass 2: one thread per (row, k1) reads the N2 values of tile row
// k1 and applies the length-N2 DFT; its outputs are X[k1 + N1 k2].  One
// shared-memory exchange per transform, instead of one per radix stage.
//
// The inter-pass twiddles w_N^(n2 k1) are entries (n2 k1 mod N) of the level's
// table exp(+2 pi i t / N) (FP64 on the host, rounded to FP32).
//
// The in-register DFTs (lengths 2, 3, 4, 5 and their products up to 32: 6, 8,
// 9, 10, 12, 15, 16, 18, 20, 24, 25, 27, 30, 32) split L = a b
// the same way, with every index and twiddle known at compile time; the
// twiddles are cos / sin of 2 pi j / L evaluated at compile time by a Taylor
// series (reduced to the first quadrant by exact symmetries) and rounded to
// FP32.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

namespace bsi {
namespace freg {

// ---------------------------------------------------------------- compile-time twiddles

__host__ __device__ constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 14; ++k) {
    term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 14; ++k) {
    term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    sum += term;
  }
  return sum;
}
// cos and sin of 2 pi j / L for integers j, L > 0: j reduced modulo L, the
// quadrant split off exactly (4 j' = q L + r), the remainder angle 2 pi r / (4 L)
// in [0, pi / 2) by the series.
__host__ __device__ constexpr double cos2pi(int j, int L) {
  const int jr = ((j % L) + L) % L;
  const int q = (4 * jr) / L, r = 4 * jr - q * L;
  const double x = 3.14159265358979323846 * r / (2.0 * L);
  const double c = taylor_cos(x), s = taylor_sin(x);
  return q == 0 ? c : q == 1 ? -s : q == 2 ? -c : s;
}
__host__ __device__ constexpr double sin2pi(int j, int L) {
  const int jr = ((j % L) + L) % L;
  const int q = (4 * jr) / L, r = 4 * jr - q * L;
  const double x = 3.14159265358979323846 * r / (2.0 * L);
  const double c = taylor_cos(x), s = taylor_sin(x);
  return q == 0 ? s : q == 1 ? c : q == 2 ? -s : -c;
}

template <int I>
using ic = std::integral_constant<int, I>;

template <int I, int N, class F>
__host__ __device__ __forceinline__ void sfor(F &&f) {
  if constexpr (I < N) {
    f(ic<I>{});
    sfor<I + 1, N>(f);
  }
}

__host__ __device__ __forceinline__ float2 add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// x * w_L^J, w_L = exp(S 2 pi i / L), with the exact cases (1, +-i, -1) as
// swaps and negations
template <int L, int J, int S>
__host__ __device__ __forceinline__ float2 twiddle(float2 x) {
  constexpr int j = ((J % L) + L) % L;
  if constexpr (j == 0) {
    return x;
  } else if constexpr (2 * j == L) {
    return make_float2(-x.x, -x.y);
  } else if constexpr (4 * j == L) {  // S i
    return S > 0 ? make_float2(-x.y, x.x) : make_float2(x.y, -x.x);
  } else if constexpr (4 * j == 3 * L) {  // -S i
    return S > 0 ? make_float2(x.y, -x.x) : make_float2(-x.y, x.x);
  } else {
    constexpr float c = (float)cos2pi(j, L);
    constexpr float s = (float)(S * sin2pi(j, L));
    return make_float2(x.x * c - x.y * s, x.x * s + x.y * c);
  }
}

__host__ __device__ constexpr int first_factor(int L) {
  return L % 8 == 0 && L > 8   ? 8
         : L % 4 == 0 && L > 4 ? 4
         : L % 2 == 0 && L > 2 ? 2
         : L % 3 == 0 && L > 3 ? 3
                               : 5;
}

// In-place DFT of length L held in registers, natural order in and out.
template <int L, int S>
__host__ __device__ __forceinline__ void dft(float2 (&v)[L]) {
  if constexpr (L == 1) {
  } else if constexpr (L == 2) {
    const float2 a = v[0], b = v[1];
    v[0] = add(a, b);
    v[1] = sub(a, b);
  } else if constexpr (L == 3) {
    constexpr float c = -0.5f, s = (float)(S * 0.86602540378443864676);
    const float2 a = v[0], t = add(v[1], v[2]), q = sub(v[1], v[2]);
    const float2 m = make_float2(a.x + c * t.x, a.y + c * t.y);
    const float2 rq = make_float2(-s * q.y, s * q.x);
    v[0] = add(a, t);
    v[1] = add(m, rq);
    v[2] = sub(m, rq);
  } else if constexpr (L == 5) {
    // c1 = cos(2 pi / 5), c2 = cos(4 pi / 5), s1, s2 the sines (times S)
    constexpr float c1 = (float)cos2pi(1, 5), c2 = (float)cos2pi(2, 5);
    constexpr float s1 = (float)(S * sin2pi(1, 5)), s2 = (float)(S * sin2pi(2, 5));
    const float2 a = v[0], t1 = add(v[1], v[4]), t2 = add(v[2], v[3]);
    const float2 d1 = sub(v[1], v[4]), d2 = sub(v[2], v[3]);
    const float2 m1 = make_float2(a.x + c1 * t1.x + c2 * t2.x, a.y + c1 * t1.y + c2 * t2.y);
    const float2 m2 = make_float2(a.x + c2 * t1.x + c1 * t2.x, a.y + c2 * t1.y + c1 * t2.y);
    // i (s1 d1 + s2 d2) and i (s2 d1 - s1 d2)
    const float2 e1 = make_float2(-(s1 * d1.y + s2 * d2.y), s1 * d1.x + s2 * d2.x);
    const float2 e2 = make_float2(-(s2 * d1.y - s1 * d2.y), s2 * d1.x - s1 * d2.x);
    v[0] = add(a, add(t1, t2));
    v[1] = add(m1, e1);
    v[4] = sub(m1, e1);
    v[2] = add(m2, e2);
    v[3] = sub(m2, e2);
  } else if constexpr (L == 4) {
    const float2 s02 = add(v[0], v[2]), d02 = sub(v[0], v[2]);
    const float2 s13 = add(v[1], v[3]), d13 = twiddle<4, 1, S>(sub(v[1], v[3]));
    v[0] = add(s02, s13);
    v[2] = sub(s02, s13);
    v[1] = add(d02, d13);
    v[3] = sub(d02, d13);
  } else {
    constexpr int a = first_factor(L), b = L / a;
    static_assert(a * b == L && b > 1, "unsupported register DFT length");
    // length-a DFTs over the stride-b subsequences, twiddled, then length-b
    // DFTs over each output frequency of the first step
    float2 T[b][a];
    sfor<0, b>([&](auto M2) {
      constexpr int m2 = decltype(M2)::value;
      float2 t[a];
      sfor<0, a>([&](auto M1) { t[decltype(M1)::value] = v[m2 + b * decltype(M1)::value]; });
      dft<a, S>(t);
      sfor<0, a>([&](auto K1) {
        constexpr int k1 = decltype(K1)::value;
        T[m2][k1] = twiddle<L, m2 * k1, S>(t[k1]);
      });
    });
    sfor<0, a>([&](auto K1) {
      constexpr int k1 = decltype(K1)::value;
      float2 u[b];
      sfor<0, b>([&](auto M2) { u[decltype(M2)::value] = T[decltype(M2)::value][k1]; });
      dft<b, S>(u);
      sfor<0, b>([&](auto K2) { v[k1 + a * decltype(K2)::value] = u[decltype(K2)::value]; });
    });
  }
}

// ---------------------------------------------------------------- the two-pass split

// N = N1 x N2 for the lengths with a register plan; N1 = 0 for the others.
template <int N>
struct Split {
  static constexpr int N1 = N == 16 ? 4 : N == 24 ? 4 : N == 32 ? 4 : N == 48 ? 6 : N == 64 ? 8
                          : N == 96 ? 8 : N == 128 ? 8 : N == 192 ? 12 : N == 256 ? 16
                          : N == 384 ? 16 : N == 512 ? 16 : N == 768 ? 24
                          // channel counts with factors 3 and 5
                          : N == 540 ? 20 : N == 675 ? 25 : N == 729 ? 27 : N == 750 ? 25 : 0;
  static constexpr int N2 = N1 ? N / N1 : 0;
  static constexpr int LDY = N2 + 1;  // odd row pitch of the exchange tile
};

}  // namespace freg
}  // namespace bsi
