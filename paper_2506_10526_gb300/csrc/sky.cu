// Monte Carlo validation sky of Section 4 on the GPU (bs_sky_*).
//
// One realisation r is the non-Gaussian field of Eq. (mb1) on the periodic
// (nc, nt, nt) box, g = IDFT( sqrt(P) DFT(w) ), delta = g + f (g^2 - sigma^2),
// and its centred per-channel visibilities V = fftshift(DFT2(delta)).  The
// white noise w comes from Philox4x32-10 (Salmon, Moraes, Dror & Shaw 2011)
// with Box-Muller normals: cell c = (z nt + y) nt + x takes normal c mod 4 of
// Philox call q = c / 4 with counter (q lo, q hi, r lo, r hi) and key (seed lo,
// seed hi); outputs (o0, o1) give cells 4q, 4q+1 as sqrt(-2 ln a)(cos, sin)
// (2 pi b), a = (o0 + 1/2) 2^-32, b = (o1 + 1/2) 2^-32, (o2, o3) cells 4q+2, 4q+3.
//
// Two realisations share every transform: both the noise and the filter
// sqrt(P) are real and P(k) = P(-k), so one complex field z = w_a + i w_b
// carries g_a + i g_b through the 3D filter, delta_a + i delta_b through the
// quadratic map, and the 2D transform of it splits into the two (Hermitian)
// visibility sets as V_a(k) = (Z(k) + Z(-k)^*)/2, V_b(k) = (Z(k) - Z(-k)^*)/(2i).
//
// Passes over a pair buffer [pair][z][y][x] (complex64, in place): each CTA
// moves UB whole lines of one axis into shared memory and runs the Stockham
// FFT of fft_smem.cuh there.
//   x  noise -> DFT_x
//   y  DFT_y
//   z  DFT_z, times sqrt(P)/N, IDFT_z
//   y  IDFT_y
//   x  IDFT_x, quadratic map, DFT_x
//   y  DFT_y
//   separate + fftshift into the caller's visibility buffer.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "bs_internal.h"
#include "fft_reg.cuh"
#include "fft_smem.cuh"

namespace bsi {
namespace {

constexpr int kSkyThreads = 256;
constexpr int kSkySmemBudget = 100 * 1024;  // two CTAs per SM

struct LineGeom {
  int n;              // line length
  int ni;             // lines per outer index
  int UB;             // lines per CTA
  long long tstride;  // element stride along a line
  long long istride;  // stride between neighbouring lines
  long long ostride;  // stride of the outer index (blockIdx.y)
  long long pstride;  // stride of a pair (blockIdx.z)
};

enum SkyPre { PRE_LOAD = 0, PRE_NOISE = 1 };
enum SkyMid { MID_NONE = 0, MID_FILTER = 1, MID_QUAD = 2 };

struct SkyParams {
  int nt;
  unsigned long long seed, r0;
  float f_ng, sigma2;
  const float *sqrtp;  // [nc][nt][nt], sqrt(P) / N
};

// One Philox4x32 round count of 10, multipliers and Weyl key increments of
// the published generator.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ float2 box_muller(uint32_t o0, uint32_t o1) {
  const float a = fmaf((float)o0, 2.3283064365386963e-10f, 1.1641532182693481e-10f);
  const float b = fmaf((float)o1, 2.3283064365386963e-10f, 1.1641532182693481e-10f);
  const float rad = sqrtf(fmaxf(-2.0f * logf(a), 0.0f));
  float s, c;
  sincospif(2.0f * b, &s, &c);
  return make_float2(rad * c, rad * s);
}

// Four normals of cells 4q .. 4q+3 of realisation r.
__device__ __forceinline__ float4 normals4(unsigned long long q, unsigned long long r,
                                           unsigned long long seed) {
  const uint4 o = philox4x32_10(make_uint4((uint32_t)q, (uint32_t)(q >> 32), (uint32_t)r,
                                           (uint32_t)(r >> 32)),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const float2 n01 = box_muller(o.x, o.y), n23 = box_muller(o.z, o.w);
  return make_float4(n01.x, n01.y, n23.x, n23.y);
}

// In-place transform of nl lines of length N (line r at buf + r LD) on the
// register FFT (fft_reg.cuh), sign -1 by conjugating input and output:
// pass 1 reads the lines along n2 into registers, the exchange tile Y takes
// [line][k1][n2] (odd pitch), pass 2 writes X[k1 + N1 k2] back along the line.
template <int N>
__device__ __forceinline__ void reg_lines(float2 *buf, float2 *Y, const float2 *tw2, int nl, int LD,
                                          float sign) {
  constexpr int N1 = freg::Split<N>::N1, N2 = freg::Split<N>::N2, LDY = freg::Split<N>::LDY;
  const float cj = sign < 0.f ? -1.f : 1.f;
  for (int it = threadIdx.x; it < nl * N2; it += blockDim.x) {
    const int r = it / N2, n2 = it - r * N2;
    float2 v[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
      const float2 x = buf[r * LD + n2 + N2 * n1];
      v[n1] = make_float2(x.x, cj * x.y);
    }
    freg::dft<N1, 1>(v);
    float2 *Yr = Y + r * (N1 * LDY);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      const float2 w = tw2[k1 * N2 + n2], a = v[k1];
      Yr[k1 * LDY + n2] = make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
    }
  }
  __syncthreads();
  for (int it = threadIdx.x; it < nl * N1; it += blockDim.x) {
    const int r = it / N1, k1 = it - r * N1;
    float2 v[N2];
    const float2 *Yr = Y + r * (N1 * LDY) + k1 * LDY;
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) v[n2] = Yr[n2];
    freg::dft<N2, 1>(v);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) buf[r * LD + k1 + N1 * k2] = make_float2(v[k2].x, cj * v[k2].y);
  }
  __syncthreads();
}

// NR > 0: line length NR on the register FFT; NR = 0: Stockham stages.
template <int PRE, int MID, int NR>
__global__ void __launch_bounds__(kSkyThreads, 2) k_sky_lines(LineGeom g, SkyParams sp, float2 *data,
                                                             const float2 *__restrict__ twg,
                                                             Radices rad, float sign1) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = NR > 0 ? NR : g.n, UB = g.UB;
  const int LD = n + 1;  // padded lines: strided (line-major) accesses spread over the banks
  float2 *tw = reinterpret_cast<float2 *>(smem_raw);
  float2 *bufA = tw + n;
  float2 *bufB = bufA + UB * LD;  // Stockham ping-pong buffer, or the register FFT's Y and tw2
  float2 *tw2 = bufB + (NR > 0 ? UB * (n + freg::Split<(NR > 0 ? NR : 16)>::N1) : 0);
  for (int t = threadIdx.x; t < n; t += blockDim.x) tw[t] = twg[t];
  if constexpr (NR > 0) {
    constexpr int N2 = freg::Split<NR>::N2;
    for (int t = threadIdx.x; t < NR; t += blockDim.x) {
      const int k1 = t / N2, n2 = t - k1 * N2;
      tw2[t] = twg[(n2 * k1) % NR];
    }
  }
  const int i0 = blockIdx.x * UB;
  const int nl = min(UB, g.ni - i0);
  const long long base =
      (long long)blockIdx.z * g.pstride + (long long)blockIdx.y * g.ostride + (long long)i0 * g.istride;
  const bool rowmajor = (g.tstride == 1);  // lines are contiguous rows of length n
  if (PRE == PRE_NOISE) {
    // x lines only (tstride 1, istride n, one outer index): the CTA's cells are
    // the contiguous range [c0, c0 + nl n) of the box.
    const unsigned long long c0 = (unsigned long long)i0 * n;
    const unsigned long long c1 = c0 + (unsigned long long)nl * n;
    const unsigned long long q0 = c0 >> 2, q1 = (c1 + 3) >> 2;
    const unsigned long long ra = sp.r0 + 2ull * blockIdx.z, rb = ra + 1;
    for (unsigned long long q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
      const float4 a = normals4(q, ra, sp.seed), b = normals4(q, rb, sp.seed);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const unsigned long long c = 4 * q + s;
        if (c >= c0 && c < c1) {
          const int l = (int)((c - c0) / n), t = (int)(c - c0) - l * n;
          bufA[l * LD + t] = make_float2(av[s], bv[s]);
        }
      }
    }
  } else {
    const int tot = nl * n;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
      int l, t;
      if (rowmajor) {
        l = e / n;
        t = e - l * n;
      } else {
        t = e / nl;
        l = e - t * nl;
      }
      bufA[l * LD + t] = data[base + (long long)l * g.istride + (long long)t * g.tstride];
    }
  }
  __syncthreads();
  float2 *res;
  if constexpr (NR > 0) {
    reg_lines<NR>(bufA, bufB, tw2, nl, LD, sign1);
    res = bufA;
  } else {
    res = stockham(bufA, bufB, nl, n, LD, rad, tw, sign1);
  }
  if (MID != MID_NONE) {
    float2 *oth = (res == bufA) ? bufB : bufA;
    const int tot = nl * n;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
      const int l = e / n, t = e - l * n;
      float2 v = res[l * LD + t];
      if (MID == MID_FILTER) {
        // offset of the element inside its pair = its box cell (kz, ky, kx)
        const long long cell =
            (long long)blockIdx.y * g.ostride + (long long)(i0 + l) * g.istride + (long long)t * g.tstride;
        const float s = sp.sqrtp[cell];
        v = make_float2(v.x * s, v.y * s);
      } else {
        v = make_float2(v.x + sp.f_ng * (v.x * v.x - sp.sigma2), v.y + sp.f_ng * (v.y * v.y - sp.sigma2));
      }
      res[l * LD + t] = v;
    }
    __syncthreads();
    if constexpr (NR > 0)
      reg_lines<NR>(res, bufB, tw2, nl, LD, -sign1);
    else
      res = stockham(res, oth, nl, n, LD, rad, tw, -sign1);
  }
  const int tot = nl * n;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    int l, t;
    if (rowmajor) {
      l = e / n;
      t = e - l * n;
    } else {
      t = e / nl;
      l = e - t * nl;
    }
    data[base + (long long)l * g.istride + (long long)t * g.tstride] = res[l * LD + t];
  }
}

// Z = DFT2 of (delta_a + i delta_b) per channel -> centred V_a, V_b.
__global__ void k_sky_separate(const float2 *__restrict__ Z, int nt, int nc, long long N, int batch,
                               float2 *__restrict__ vis) {
  const long long plane = (long long)nt * nt;
  const long long total = (long long)((batch + 1) / 2) * N;
  const int h = nt / 2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long p = e / N;
    const long long rem = e - p * N;
    const long long z = rem / plane;
    const int cell = (int)(rem - z * plane);
    const int ky = cell / nt, kx = cell - ky * nt;
    const int my = ky ? nt - ky : 0, mx = kx ? nt - kx : 0;
    const float2 a = Z[p * N + z * plane + cell];
    const float2 b = Z[p * N + z * plane + my * nt + mx];  // Z(-k)
    const int sy = ky + h >= nt ? ky + h - nt : ky + h;
    const int sx = kx + h >= nt ? kx + h - nt : kx + h;
    const long long o = z * plane + (long long)sy * nt + sx;
    // V_a = (a + conj b)/2 ; V_b = (a - conj b)/(2i)
    vis[(2 * p) * N + o] = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
    if (2 * p + 1 < batch) vis[(2 * p + 1) * N + o] = make_float2(0.5f * (a.y + b.y), -0.5f * (a.x - b.x));
  }
}

// first-pass length N1 of the register plan of n (0: none in the sky's set)
int sky_reg_n1(int n) {
  switch (n) {
    case 64: return freg::Split<64>::N1;
    case 128: return freg::Split<128>::N1;
    case 256: return freg::Split<256>::N1;
    case 384: return freg::Split<384>::N1;
    case 512: return freg::Split<512>::N1;
    case 768: return freg::Split<768>::N1;
    case 540: return freg::Split<540>::N1;
    case 675: return freg::Split<675>::N1;
    case 729: return freg::Split<729>::N1;
    case 750: return freg::Split<750>::N1;
    default: return 0;
  }
}

// tables + lines + (Stockham: a second line buffer; register FFT: the
// exchange tile of ub (n + N1) and the split twiddles)
size_t sky_smem(int n, int ub) {
  const int n1 = sky_reg_n1(n);
  if (n1) return (size_t)8 * (2 * (size_t)n + (size_t)ub * (n + 1) + (size_t)ub * (n + n1));
  return (size_t)8 * (n + 2 * (size_t)ub * (n + 1));
}

int pick_ub(int n) {
  for (int ub = 16; ub > 1; ub >>= 1)
    if (sky_smem(n, ub) <= (size_t)kSkySmemBudget) return ub;
  return 1;
}

thread_local std::string g_sky_create_error = "no error";

}  // namespace
}  // namespace bsi

using namespace bsi;

struct bs_sky_s {
  int device = 0, nt = 0, nc = 0, max_batch = 0;
  double sigma = 0, f_ng = 0;
  long long N = 0;
  float *sqrtp = nullptr;
  float2 *work = nullptr, *twT = nullptr, *twC = nullptr;
  Radices radT, radC;
  bool broken = false;
  std::string err = "no error";
};

namespace {

bs_status sky_fail(bs_sky s, bs_status st, const std::string &msg) {
  if (s) {
    s->err = msg;
    if (st == BS_ERR_CUDA) s->broken = true;
  } else {
    bsi::g_sky_create_error = msg;
  }
  return st;
}

template <int PRE, int MID, int NR>
cudaError_t launch_lines_n(const bs_sky_s *s, const LineGeom &g, const SkyParams &sp, int npair,
                           const float2 *tw, const Radices &rad, float sign1, cudaStream_t st) {
  const size_t smem = sky_smem(g.n, g.UB);
  cudaError_t e = cudaFuncSetAttribute(k_sky_lines<PRE, MID, NR>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long outer = g.ostride ? (long long)s->N / g.ostride : 1;
  dim3 grid((g.ni + g.UB - 1) / g.UB, (unsigned)outer, npair);
  k_sky_lines<PRE, MID, NR><<<grid, kSkyThreads, smem, st>>>(g, sp, s->work, tw, rad, sign1);
  return cudaGetLastError();
}

// x and y lines (length nt) of every pass kind, z lines (length nchan) with the
// filter: the register FFT for the lengths of sky_reg_n1, else Stockham
template <int PRE, int MID>
cudaError_t launch_lines(const bs_sky_s *s, const LineGeom &g, const SkyParams &sp, int npair,
                         const float2 *tw, const Radices &rad, float sign1, cudaStream_t st) {
  if constexpr (MID == MID_FILTER) {
    switch (g.n) {
      case 256: return launch_lines_n<PRE, MID, 256>(s, g, sp, npair, tw, rad, sign1, st);
      case 384: return launch_lines_n<PRE, MID, 384>(s, g, sp, npair, tw, rad, sign1, st);
      case 768: return launch_lines_n<PRE, MID, 768>(s, g, sp, npair, tw, rad, sign1, st);
      case 540: return launch_lines_n<PRE, MID, 540>(s, g, sp, npair, tw, rad, sign1, st);
      case 675: return launch_lines_n<PRE, MID, 675>(s, g, sp, npair, tw, rad, sign1, st);
      case 729: return launch_lines_n<PRE, MID, 729>(s, g, sp, npair, tw, rad, sign1, st);
      case 750: return launch_lines_n<PRE, MID, 750>(s, g, sp, npair, tw, rad, sign1, st);
      default: break;
    }
  } else {
    switch (g.n) {
      case 64: return launch_lines_n<PRE, MID, 64>(s, g, sp, npair, tw, rad, sign1, st);
      case 128: return launch_lines_n<PRE, MID, 128>(s, g, sp, npair, tw, rad, sign1, st);
      case 256: return launch_lines_n<PRE, MID, 256>(s, g, sp, npair, tw, rad, sign1, st);
      case 512: return launch_lines_n<PRE, MID, 512>(s, g, sp, npair, tw, rad, sign1, st);
      default: break;
    }
  }
  return launch_lines_n<PRE, MID, 0>(s, g, sp, npair, tw, rad, sign1, st);
}

}  // namespace

extern "C" {

const char *bs_sky_last_error(bs_sky s) { return s ? s->err.c_str() : bsi::g_sky_create_error.c_str(); }

bs_status bs_sky_create(int nt, int nchan, double slope, double sigma, double f_ng, int max_batch,
                        bs_sky *out) {
  BS_NVTX("bs_sky_create");
  if (!out) return sky_fail(nullptr, BS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (nt < 8 || nt > 4096 || nt % 2) return sky_fail(nullptr, BS_ERR_ARG, "nt must be even, 8..4096");
  if (nchan < 1 || nchan > 4096) return sky_fail(nullptr, BS_ERR_ARG, "nchan must be 1..4096");
  if (max_batch < 1 || max_batch > 131070)
    return sky_fail(nullptr, BS_ERR_ARG, "max_batch must be 1..131070");
  if (!std::isfinite(slope) || !(sigma > 0) || !std::isfinite(sigma) || !std::isfinite(f_ng))
    return sky_fail(nullptr, BS_ERR_ARG, "slope, sigma and f_ng must be finite, sigma > 0");
  Radices rt, rc;
  if (!factor_radices(nt, rt) || !factor_radices(nchan, rc))
    return sky_fail(nullptr, BS_ERR_UNSUPPORTED, "nt and nchan must factor into 2, 3 and 5");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return sky_fail(nullptr, BS_ERR_NO_DEVICE, "no CUDA device is available");
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return sky_fail(nullptr, BS_ERR_NO_DEVICE, "cannot query the CUDA device");
  }
  if (!(prop.major == 10 && prop.minor == 3))
    return sky_fail(nullptr, BS_ERR_NO_DEVICE, "libbs is built for sm_103a (GB300)");

  bs_sky s = new bs_sky_s();
  s->device = dev;
  s->nt = nt;
  s->nc = nchan;
  s->max_batch = max_batch;
  s->sigma = sigma;
  s->f_ng = f_ng;
  s->N = (long long)nchan * nt * nt;
  s->radT = rt;
  s->radC = rc;
  // P(k) ~ |k|^slope, P(0) = 0, scaled so that (1/N) sum_k P(k) = sigma^2;
  // stored as sqrt(P) / N (the 1/N of the inverse transform folded in).
  std::vector<double> k2z(nchan), k2t(nt);
  auto freq2 = [](int i, int n) {
    const double f = (double)(i <= (n - 1) / 2 ? i : i - n) / (double)n;
    const double k = 2.0 * M_PI * f;
    return k * k;
  };
  for (int i = 0; i < nchan; ++i) k2z[i] = freq2(i, nchan);
  for (int i = 0; i < nt; ++i) k2t[i] = freq2(i, nt);
  std::vector<double> P(s->N);
  double sum = 0;
  for (int z = 0; z < nchan; ++z)
    for (int y = 0; y < nt; ++y)
      for (int x = 0; x < nt; ++x) {
        const double k2 = k2z[z] + k2t[y] + k2t[x];
        const double p = k2 > 0 ? std::pow(k2, 0.5 * slope) : 0.0;
        P[((long long)z * nt + y) * nt + x] = p;
        sum += p;
      }
  std::vector<float> sp(s->N);
  const double scale = sum > 0 ? sigma * sigma * (double)s->N / sum : 0.0;
  for (long long c = 0; c < s->N; ++c) sp[c] = (float)(std::sqrt(P[c] * scale) / (double)s->N);
  const long long npair = (max_batch + 1) / 2;
  if (inject_fail("sky_alloc") || cudaMalloc(&s->sqrtp, s->N * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&s->work, npair * s->N * sizeof(float2)) != cudaSuccess ||
      cudaMalloc(&s->twT, nt * sizeof(float2)) != cudaSuccess ||
      cudaMalloc(&s->twC, nchan * sizeof(float2)) != cudaSuccess) {
    cudaGetLastError();
    bs_sky_destroy(s);
    return sky_fail(nullptr, BS_ERR_OOM, "cannot allocate the generator's device buffers");
  }
  const std::vector<float2> twt = twiddles(nt), twc = twiddles(nchan);
  if (cudaMemcpy(s->sqrtp, sp.data(), s->N * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->twT, twt.data(), nt * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->twC, twc.data(), nchan * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    bs_sky_destroy(s);
    return sky_fail(nullptr, BS_ERR_CUDA, "cannot upload the generator's tables");
  }
  *out = s;
  return BS_OK;
}

bs_status bs_sky_destroy(bs_sky s) {
  BS_NVTX("bs_sky_destroy");
  if (!s) return BS_OK;
  cudaFree(s->sqrtp);
  cudaFree(s->work);
  cudaFree(s->twT);
  cudaFree(s->twC);
  delete s;
  return BS_OK;
}

bs_status bs_sky_generate(bs_sky s, uint64_t seed, uint64_t realisation0, int batch, void *vis_dev,
                          void *cuda_stream) {
  BS_NVTX("bs_sky_generate");
  if (!s) return BS_ERR_ARG;
  if (s->broken) return sky_fail(s, BS_ERR_STATE, "generator is in an error state: " + s->err);
  if (batch < 1 || batch > s->max_batch) return sky_fail(s, BS_ERR_ARG, "batch must be 1..max_batch");
  if (!vis_dev) return sky_fail(s, BS_ERR_ARG, "vis_dev is NULL");
  if (((uintptr_t)vis_dev) % 8) return sky_fail(s, BS_ERR_ARG, "vis_dev must be 8-byte aligned");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int nt = s->nt, nc = s->nc, npair = (batch + 1) / 2;
  const long long plane = (long long)nt * nt;
  SkyParams sp{nt, seed, realisation0, (float)s->f_ng, (float)(s->sigma * s->sigma), s->sqrtp};
  // x lines: rows (z, y) of length nt, contiguous
  LineGeom gx{nt, nc * nt, pick_ub(nt), 1, nt, 0, s->N};
  // y lines: outer z, inner x, stride nt along the line
  LineGeom gy{nt, nt, pick_ub(nt), nt, 1, plane, s->N};
  // z lines: inner (y, x), stride nt^2 along the line
  LineGeom gz{nc, (int)plane, pick_ub(nc), plane, 1, 0, s->N};
  cudaError_t e;
  if ((e = launch_lines<PRE_NOISE, MID_NONE>(s, gx, sp, npair, s->twT, s->radT, -1.f, st)) ||
      (e = launch_lines<PRE_LOAD, MID_NONE>(s, gy, sp, npair, s->twT, s->radT, -1.f, st)) ||
      (e = launch_lines<PRE_LOAD, MID_FILTER>(s, gz, sp, npair, s->twC, s->radC, -1.f, st)) ||
      (e = launch_lines<PRE_LOAD, MID_NONE>(s, gy, sp, npair, s->twT, s->radT, +1.f, st)) ||
      (e = launch_lines<PRE_LOAD, MID_QUAD>(s, gx, sp, npair, s->twT, s->radT, +1.f, st)) ||
      (e = launch_lines<PRE_LOAD, MID_NONE>(s, gy, sp, npair, s->twT, s->radT, -1.f, st)))
    return sky_fail(s, BS_ERR_CUDA, std::string("sky line pass: ") + cudaGetErrorString(e));
  const long long total = (long long)npair * s->N;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
  k_sky_separate<<<blocks, 256, 0, st>>>(s->work, nt, nc, s->N, batch, (float2 *)vis_dev);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return sky_fail(s, BS_ERR_CUDA, std::string("sky separate: ") + cudaGetErrorString(e));
  return BS_OK;
}

}  // extern "C"
