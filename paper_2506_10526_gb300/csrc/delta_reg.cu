// Delay transform of Eq. (dft) on the register FFT (fft_reg.cuh) for the
// channel counts with a register plan: the same periodic placement, fold
// normalisation and centred real-part output as delta.cu, with one
// shared-memory exchange per transform and an intermediate laid out so that
// both passes read and write along rows.
//
// rows pass: CTA = R consecutive rows n of one plane.  Pass 1 threads take
//   m fastest, so the folded-plane reads (two separations per element) are
//   consecutive; pass 2 writes tmp[n][k] (k the frequency along m, k <= N/2:
//   the rows are real) along k.
//   Rows with no sampled separation in any plane (row flags from the fold
//   table) are neither transformed nor written.
// cols pass: CTA = CB consecutive columns k <= N/2.  Threads take columns
//   fastest: pass 1 reads rows of tmp (flagged rows only), pass 2 writes the
//   centred output along its columns and, since the plane is real and the
//   output its transform's real part, out(-a, -b) = out(a, b) for the mirror
//   columns N - k.  The FP64 output is formed from the FP32 result
//   by exact bit arithmetic (x 2^e of the scale's binary exponent), so that
//   the store needs no FP64 multiply or conversion.
#include <cmath>

#include "bs_internal.h"
#include "fft_reg.cuh"
#include "fp_bits.cuh"

namespace bsi {

namespace {

using freg::Split;
using fpb::f32_to_f64_pow2;
using fpb::f64_to_f32_rn;

constexpr int kDelThreads = 128;
constexpr int kColsCB = 8;     // columns per cols-pass CTA
constexpr int kColsPad = 8;    // per-k1 pad of the cols exchange tile (half the banks)

template <int N>
struct DelCfg {
  // rows per rows-pass CTA: few for long rows, so that more CTAs are resident
  // to cover the latency of the dependent sampling / accumulator reads
  static constexpr int R = N <= 64 ? N : N < 256 ? 8 : 4;
};

template <int N>
__global__ void __launch_bounds__(kDelThreads) k_bs3d_rows_reg(
    const double *__restrict__ dsum, const float *__restrict__ rinv,
    const uint8_t *__restrict__ rowflag, const double *__restrict__ tnorm,
    float2 *__restrict__ tmp, int ntrip, const float2 *__restrict__ twN,
    const int *__restrict__ list) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, LDY = Split<N>::LDY;
  constexpr int R = DelCfg<N>::R, n2s = 2 * N - 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *tw2 = reinterpret_cast<float2 *>(smem_raw);  // [N1][N2], conjugated
  float2 *Y = tw2 + N;                                   // [R][N1][LDY]
  const int n0 = blockIdx.x * R, trip = list ? list[blockIdx.y] : blockIdx.y, b = blockIdx.z;
  const double tn = tnorm[trip];
  if (tn == 0.0) return;  // no closed triangle: the cols pass writes zeros
  const float tnf = f64_to_f32_rn(tn);
  int any = 0;
  for (int r = threadIdx.x; r < R; r += blockDim.x) any |= (n0 + r < N) && rowflag[n0 + r];
  if (!__syncthreads_or(any)) return;  // nothing sampled in these rows of any plane
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    const int k1 = t / N2, n2 = t - k1 * N2;
    const float2 w = twN[(n2 * k1) % N];
    tw2[t] = make_float2(w.x, -w.y);
  }
  __syncthreads();
  const double *ds = dsum + ((long long)b * ntrip + trip) * (long long)n2s * n2s;
  // pass 1: (row, n2) items, n2 fastest
  for (int it = threadIdx.x; it < R * N2; it += blockDim.x) {
    const int r = it / N2, n2 = it - r * N2;
    const int nidx = n0 + r;
    float2 v[N1];
    const bool live = nidx < N && rowflag[nidx];
    // one period of the N-periodic kernel: separations -N/2 <= n, m < N/2
    const int np = (2 * nidx < N) ? nidx : nidx - N;
    const int i1 = np + N - 1, j1 = n2s - 1 - i1;
    // in groups of G elements: the reciprocal sampling first, then the two
    // separations of every sampled element (unsampled ones hold no sums and are
    // not read), so that each group's loads are in flight together
    constexpr int G = N1 % 8 == 0 ? 8 : N1 % 6 == 0 ? 6 : N1 % 4 == 0 ? 4 : 1;
    const float *rrow = rinv + (long long)nidx * N;
#pragma unroll
    for (int g0 = 0; g0 < N1; g0 += G) {
      float ri[G];
      double da[G], db[G];
#pragma unroll
      for (int q = 0; q < G; ++q) ri[q] = live ? rrow[n2 + N2 * (g0 + q)] : 0.f;
#pragma unroll
      for (int q = 0; q < G; ++q) {
        const int m = n2 + N2 * (g0 + q);
        const int mp = (2 * m < N) ? m : m - N;
        const int i2 = mp + N - 1, j2 = n2s - 1 - i2;
        da[q] = 0.0;
        db[q] = 0.0;
        if (ri[q] != 0.f && BS_CHK((long long)i1 * n2s + i2, (long long)n2s * n2s, 11) &&
            BS_CHK((long long)j1 * n2s + j2, (long long)n2s * n2s, 11)) {
          da[q] = ds[(long long)i1 * n2s + i2];
          if (j1 != i1 || j2 != i2) db[q] = ds[(long long)j1 * n2s + j2];
        }
      }
#pragma unroll
      for (int q = 0; q < G; ++q) {
        const float sv = f64_to_f32_rn(da[q]) + f64_to_f32_rn(db[q]);
        v[g0 + q] = make_float2(sv * (tnf * ri[q]), 0.f);
      }
    }
    freg::dft<N1, -1>(v);
    float2 *Yr = Y + r * (N1 * LDY);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      const float2 w = tw2[k1 * N2 + n2];
      const float2 a = v[k1];
      Yr[k1 * LDY + n2] = make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
    }
  }
  __syncthreads();
  float2 *tb = tmp + ((long long)b * ntrip + trip) * (long long)N * N;
  // pass 2: (row, k1) items, k1 fastest; tmp[n][k1 + N1 k2]
  for (int it = threadIdx.x; it < R * N1; it += blockDim.x) {
    const int r = it / N1, k1 = it - r * N1;
    const int nidx = n0 + r;
    if (nidx >= N || !rowflag[nidx]) continue;
    float2 v[N2];
    const float2 *Yr = Y + r * (N1 * LDY) + k1 * LDY;
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) v[n2] = Yr[n2];
    freg::dft<N2, -1>(v);
    float2 *row = tb + (long long)nidx * N;
    // the input is real: only k <= N/2 is kept (the cols pass mirrors the rest)
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2)
      if (k1 + N1 * k2 <= N / 2 && BS_CHK((long long)nidx * N + k1 + N1 * k2, (long long)N * N, 12))
        row[k1 + N1 * k2] = v[k2];
  }
}

template <int N>
__global__ void __launch_bounds__(kDelThreads) k_bs3d_cols_reg(
    const float2 *__restrict__ tmp, const uint8_t *__restrict__ rowflag, double *__restrict__ out,
    int ntrip, const float2 *__restrict__ twN, float scale_m, int scale_e,
    const double *__restrict__ tnorm, const int *__restrict__ list) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, CB = kColsCB;
  constexpr int PK = N2 * CB + kColsPad;  // pitch of one k1 slab of the exchange tile
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *tw2 = reinterpret_cast<float2 *>(smem_raw);  // [N1][N2], conjugated
  float2 *Y = tw2 + N;                                   // [N1][PK]
  uint8_t *fl = reinterpret_cast<uint8_t *>(Y + N1 * PK);
  const int k0 = blockIdx.x * CB, trip = list ? list[blockIdx.y] : blockIdx.y, b = blockIdx.z;
  const int nout = list ? gridDim.y : ntrip;
  const int h = N / 2;
  double *ob = out + ((long long)b * nout + blockIdx.y) * (long long)N * N;
  auto centred = [&](int k) { return (k < N - h) ? k + h : k - N + h; };
  // columns b = k0 + c in [0, N/2]; b in (0, N/2) also writes its mirror N - b
  const int ncol = min(CB, N / 2 + 1 - k0);
  auto mirrored = [&](int bcol) { return bcol != 0 && 2 * bcol != N; };
  if (tnorm[trip] == 0.0) {
    for (int e = threadIdx.x; e < N * CB; e += blockDim.x) {
      const int a = e / CB, c = e - a * CB;
      if (c >= ncol) continue;
      const int bcol = k0 + c;
      ob[(long long)centred(a) * N + centred(bcol)] = 0.0;
      if (mirrored(bcol)) ob[(long long)centred(a) * N + centred(N - bcol)] = 0.0;
    }
    return;
  }
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    const int k1 = t / N2, n2 = t - k1 * N2;
    const float2 w = twN[(n2 * k1) % N];
    tw2[t] = make_float2(w.x, -w.y);
    fl[t] = rowflag[t];
  }
  __syncthreads();
  const float2 *tb = tmp + ((long long)b * ntrip + trip) * (long long)N * N + k0;
  // pass 1: (n2, column) items, columns fastest; rows of tmp without a flag are zero
  for (int it = threadIdx.x; it < N2 * CB; it += blockDim.x) {
    const int n2 = it / CB, c = it - n2 * CB;
    float2 v[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
      const int n = n2 + N2 * n1;
      v[n1] = (fl[n] && c < ncol && BS_CHK((long long)n * N + k0 + c, (long long)N * N, 13))
                  ? tb[(long long)n * N + c]
                  : make_float2(0.f, 0.f);
    }
    freg::dft<N1, -1>(v);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      const float2 w = tw2[k1 * N2 + n2];
      const float2 a = v[k1];
      Y[k1 * PK + n2 * CB + c] = make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
    }
  }
  __syncthreads();
  // pass 2: (k1, column) items, columns fastest; out[a + N/2][b + N/2] = scale Re
  for (int it = threadIdx.x; it < N1 * CB; it += blockDim.x) {
    const int k1 = it / CB, c = it - k1 * CB;
    float2 v[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) v[n2] = Y[k1 * PK + n2 * CB + c];
    freg::dft<N2, -1>(v);
    if (c < ncol) {
      // Re of the transform of a real plane: out(-a, -b) = out(a, b)
      const int bcol = k0 + c;
      double *oc = ob + centred(bcol);
      double *om = ob + centred((N - bcol) % N);
      const bool mir = mirrored(bcol);
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        const int a = k1 + N1 * k2;
        const double val = f32_to_f64_pow2(v[k2].x * scale_m, scale_e);
        if (BS_CHK((long long)centred(a) * N + centred(bcol), (long long)N * N, 14))
          oc[(long long)centred(a) * N] = val;
        if (mir && BS_CHK((long long)centred((N - a) % N) * N + centred((N - bcol) % N),
                          (long long)N * N, 14))
          om[(long long)centred((N - a) % N) * N] = val;
      }
    }
  }
}

template <int N>
cudaError_t bs3d_n(const double *dsum, const float *rinv, const uint8_t *rowflag,
                   const double *tnorm, float2 *tmp, double *out, int batch, int ntrip,
                   const float2 *twN, double scale, const int *list, int ny, cudaStream_t s) {
  constexpr int R = DelCfg<N>::R;
  const size_t smem_r = (size_t)(N + R * Split<N>::N1 * Split<N>::LDY) * sizeof(float2);
  const size_t smem_c = (size_t)(N + Split<N>::N1 * (Split<N>::N2 * kColsCB + kColsPad)) *
                            sizeof(float2) + (size_t)N;
  cudaError_t e = smem_optin_once<k_bs3d_rows_reg<N>>();
  if (e != cudaSuccess) return e;
  e = smem_optin_once<k_bs3d_cols_reg<N>>();
  if (e != cudaSuccess) return e;
  // scale = m 2^e with m in [1, 2): the FP32 product v m keeps 24 bits, 2^e is exact
  int se = 0;
  const double sm = std::frexp(scale, &se);  // scale = sm 2^se, sm in [0.5, 1)
  const float scale_m = (float)(2.0 * sm);
  const int scale_e = se - 1;
  dim3 gr((N + R - 1) / R, ny, batch);
  k_bs3d_rows_reg<N><<<gr, kDelThreads, smem_r, s>>>(dsum, rinv, rowflag, tnorm, tmp, ntrip, twN,
                                                     list);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 gc((N / 2 + 1 + kColsCB - 1) / kColsCB, ny, batch);
  k_bs3d_cols_reg<N><<<gc, kDelThreads, smem_c, s>>>(tmp, rowflag, out, ntrip, twN, scale_m,
                                                     scale_e, tnorm, list);
  return cudaGetLastError();
}

}  // namespace

bool has_reg_dft(int nc) {
  switch (nc) {
    case 16: case 24: case 32: case 48: case 64: case 96: case 128: case 192: case 256:
    case 384: case 512: case 768: case 540: case 675: case 729: case 750:
      return true;
    default:
      return false;
  }
}

cudaError_t launch_bs3d_reg(const double *dsum, const float *rinv, const uint8_t *rowflag,
                            const double *tnorm, float2 *tmp, double *out, int batch, int ntrip,
                            int nc, const float2 *twN, double scale, const int *list, int ny,
                            cudaStream_t s) {
  switch (nc) {
#define BS_DEL_CASE(n) \
  case n: return bs3d_n<n>(dsum, rinv, rowflag, tnorm, tmp, out, batch, ntrip, twN, scale, list, ny, s);
    BS_DEL_CASE(16) BS_DEL_CASE(24) BS_DEL_CASE(32) BS_DEL_CASE(48) BS_DEL_CASE(64)
    BS_DEL_CASE(96) BS_DEL_CASE(128) BS_DEL_CASE(192) BS_DEL_CASE(256) BS_DEL_CASE(384)
    BS_DEL_CASE(512) BS_DEL_CASE(768) BS_DEL_CASE(540) BS_DEL_CASE(675) BS_DEL_CASE(729)
    BS_DEL_CASE(750)
#undef BS_DEL_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bsi
