// Monopole of the 3D bispectrum binned in triangle size and shape
// (Section 2: Eq. shape and Eq. bs_lm at l = m = 0; the (k1, mu, t) binning
// of Section 5; Eq. bsana for the binned analytic prediction).
//
// Samples: every closable ring triple (i, j, l) x every delay pair (a, b) of
// the Eq. (dft) output.  The three sides are k_n = sqrt(kperp_n^2 + kpar_n^2)
// with kpar_1 = kpar(a) (ring i), kpar_2 = kpar(b) (ring j) and
// kpar_3 = -(kpar_1 + kpar_2) (ring l).  With S1 >= S2 >= S3 the squared
// sides, the size is k1 = sqrt(S1) and the shape t = k2 / k1,
// mu = (S1 + S2 - S3) / (2 k1 k2) (the closure k1 + k2 + k3 = 0 turns
// -k1.k2 into squared lengths).  A bin holds the sum of the values and the
// number of samples; the caller divides.
//
// The bin is decided in FP32 on squared quantities, with no square root and
// no division on the exact path:
//   k1 in bin q          <=>  E_q <= S1 < E_{q+1},  E_q = fl32(e_q^2)
//   t >= tau             <=>  S2 >= tau^2 S1
//   mu >= m              <=>  N^2 >= 4 m^2 P,  N = S1 + S2 - S3 >= S1 > 0,
//                                              P = S1 S2
// A fast approximate t and mu (reciprocal square root, fast divide) picks a
// first bin, and the exact comparisons above move it to the right one.  The
// squared sides carry at most 16 units u = 2^-24 of relative error
// (including the rounding of the FP64 inputs and of k_par3 = -(k_par1 +
// k_par2)), so the decisions equal the FP64 ones except for samples whose k1
// lies within about 9u relative of a k1 edge, t within 17u or mu within 68u
// of a shape edge or an acceptance limit.  Values and sums are FP64; the
// model of Eq. (bsana) takes FP64 squared lengths from FP64 tables.
//
// The bin of a sample depends only on the geometry (k tables, edges, bin
// counts, closable ring triples), not on the values, so the plan keeps an
// int16 table of the bins of every sample and rebuilds it only when the
// geometry changes (k_mono_bins: one thread per sample).  The summing kernel
// (k_mono_sum) then streams the table and the values with coalesced loads:
// each warp walks a contiguous range 32 samples at a time; when all 32 share
// the warp's running bin each lane adds its value to its own per-realisation
// running sums, which are reduced across the warp and flushed to the CTA's
// shared-memory histogram only when the bin changes (neighbouring delay modes
// mostly share a bin); mixed groups add per lane.  One FP64 add per sample
// and realisation remains: the GB300 FP64 rate (about 0.5e12 adds/s
// measured), not HBM, is what bounds the kernel.  The CTA adds its non-empty
// bins to the global sums with FP64 atomics.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "plan_internal.h"

namespace bsi {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBatch = 8;  // realisations per launch (the host loops over more)
constexpr int kMonoMaxK1 = 1024;
constexpr int kMonoMaxShape = 1024;
// Sides from ring-mean k_perp close only approximately: mu and t within
// kShapeTol outside [0.5, 1] are clamped into it, samples further out dropped.
constexpr double kShapeTol = 1e-2;

struct MonoArgs {
  const double *b3d;     // [batch_total][n_planes][nc][nc] or null (model)
  long long bstride;     // n_planes * nc * nc
  int b0, nbatch;        // realisations [b0, b0 + nbatch) of this launch
  const int *rings;      // [n_planes][3]
  const float *kperp;    // [nb], rounded to FP32
  const float *kpar;     // [nc], rounded to FP32
  const double *kperp64; // [nb] (model values)
  const double *kpar64;  // [nc]
  const float *thr;      // E [n_k1 + 1] | cmu [n_mu + 1] | ct [n_t + 1]
  int nc, n_k1, n_mu, n_t, nbin;
  int chunk;             // samples per CTA, a multiple of 256 (nc^2 < 2^31)
  int model;
  double f2, p_amp, p_half;  // 2 f_NG, amplitude, p_index / 2
  double *sums;          // [batch_total][nbin]
  unsigned long long *cnt;  // [nbin], or null (counted by an earlier launch)
};

// Bin of one sample, -1 when it is dropped.  E, cmu, ct: squared thresholds
// (cmu[0] and cmu[n_mu], ct[0]: the acceptance limits of mu and t).
__device__ __forceinline__ int bin_of(const MonoArgs &a, const float *E, const float *cmu,
                                      const float *ct, float kpi, float kpj, float kpl, float ka,
                                      float kb) {
  const float kc = -(ka + kb);
  float s1 = kpi * kpi + ka * ka, s2 = kpj * kpj + kb * kb, s3 = kpl * kpl + kc * kc, tmp;
  if (s1 < s2) { tmp = s1; s1 = s2; s2 = tmp; }
  if (s2 < s3) { tmp = s2; s2 = s3; s3 = tmp; }
  if (s1 < s2) { tmp = s1; s1 = s2; s2 = tmp; }
  if (!(s1 >= E[0] && s1 < E[a.n_k1] && s1 > 0.0f)) return -1;
  if (!(s2 >= ct[0] * s1)) return -1;  // t below its acceptance limit
  const float N = (s1 + s2) - s3, P = s1 * s2, N2 = N * N;
  if (!(N2 >= cmu[0] * P && N2 <= cmu[a.n_mu] * P)) return -1;  // mu outside its limits
  int lo = 0, hi = a.n_k1;  // E[lo] <= S1 < E[hi]
  while (hi - lo > 1) {
    const int m = (lo + hi) >> 1;
    if (E[m] <= s1) lo = m; else hi = m;
  }
  const float r = __fdividef(s2, s1);
  const float ta = r * rsqrtf(r);              // ~ t
  const float ma = 0.5f * N * rsqrtf(P);       // ~ mu
  int qt = min(max((int)((ta - 0.5f) * (float)(2 * a.n_t)), 0), a.n_t - 1);
  while (qt > 0 && s2 < ct[qt] * s1) --qt;
  while (qt < a.n_t - 1 && s2 >= ct[qt + 1] * s1) ++qt;
  int qm = min(max((int)((ma - 0.5f) * (float)(2 * a.n_mu)), 0), a.n_mu - 1);
  while (qm > 0 && N2 < cmu[qm] * P) --qm;
  while (qm < a.n_mu - 1 && N2 >= cmu[qm + 1] * P) ++qm;
  return (lo * a.n_mu + qm) * a.n_t + qt;
}

// Eq. (bsana) at one sample from FP64 squared lengths.
__device__ __forceinline__ double model_value(const MonoArgs &a, int i, int j, int l, int ia,
                                              int ib) {
  const double za = a.kpar64[ia], zb = a.kpar64[ib], zc = -(za + zb);
  const double pi_ = a.kperp64[i], pj = a.kperp64[j], pl = a.kperp64[l];
  const double P1 = a.p_amp * pow(pi_ * pi_ + za * za, a.p_half),
               P2 = a.p_amp * pow(pj * pj + zb * zb, a.p_half),
               P3 = a.p_amp * pow(pl * pl + zc * zc, a.p_half);
  return a.f2 * (P1 * P2 + P2 * P3 + P3 * P1);
}

// Bin of every sample of every closable plane: bins[p][e], e = (a + nc/2) nc + b + nc/2.
__global__ void __launch_bounds__(kThreads) k_mono_bins(const MonoArgs a, long long total,
                                                        int16_t *__restrict__ bins) {
  __shared__ float thr_s[3 * (kMonoMaxShape + 1) + kMonoMaxK1 + 1];
  const int nthr = a.n_k1 + a.n_mu + a.n_t + 3;
  for (int q = threadIdx.x; q < nthr; q += blockDim.x) thr_s[q] = a.thr[q];
  __syncthreads();
  const float *E = thr_s, *cmu = thr_s + a.n_k1 + 1, *ct = cmu + a.n_mu + 1;
  const long long n = (long long)a.nc * a.nc;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
       x += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(x / n);
    const int e = (int)(x - (long long)p * n);
    const int ia = e / a.nc, ib = e - ia * a.nc;
    const int i = a.rings[3 * p], j = a.rings[3 * p + 1], l = a.rings[3 * p + 2];
    bins[x] = (int16_t)bin_of(a, E, cmu, ct, a.kperp[i], a.kperp[j], a.kperp[l], a.kpar[ia],
                              a.kpar[ib]);
  }
}

constexpr int kSumUnroll = 8;  // groups of 32 samples loaded ahead per warp

template <int NB>  // realisations per launch held in registers (a.nbatch <= NB)
__global__ void __launch_bounds__(kThreads) k_mono_sum(const MonoArgs a,
                                                       const int16_t *__restrict__ bins) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *hs = reinterpret_cast<double *>(smem_raw);                             // [nbatch][nbin]
  unsigned *hc = reinterpret_cast<unsigned *>(hs + (size_t)a.nbatch * a.nbin);  // [nbin]
  const int p = blockIdx.y;
  for (int q = threadIdx.x; q < a.nbatch * a.nbin; q += blockDim.x) hs[q] = 0.0;
  for (int q = threadIdx.x; q < a.nbin; q += blockDim.x) hc[q] = 0u;
  __syncthreads();
  const int nb = a.model ? 1 : a.nbatch;
  const int i = a.rings[3 * p], j = a.rings[3 * p + 1], l = a.rings[3 * p + 2];
  const int n = a.nc * a.nc;
  const int c0 = blockIdx.x * a.chunk, c1 = min(n, c0 + a.chunk);
  // this warp's contiguous range
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kThreads / 32;
  const int per = ((c1 - c0 + nw - 1) / nw + 31) / 32 * 32;
  const int w0 = min(c1, c0 + warp * per), w1 = min(c1, w0 + per);
  const int16_t *bp = bins + (long long)p * n;
  const double *vb = a.b3d ? a.b3d + (long long)a.b0 * a.bstride + (long long)p * n : nullptr;

  // The warp's running bin (uniform across the warp) and count; each lane keeps
  // its own per-realisation running sums (one FP64 add per sample: the FP64 rate
  // of the part bounds this kernel), reduced across the warp only when flushed.
  int cur = -1;
  unsigned cnt = 0;
  double run[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) run[b] = 0.0;
  auto flush = [&]() {
    if (cur >= 0) {
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        if (b >= nb) break;
        double x = run[b];
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) atomicAdd(hs + (size_t)b * a.nbin + cur, x);
      }
      if (lane == 0) atomicAdd(hc + cur, cnt);
    }
    cnt = 0;
#pragma unroll
    for (int b = 0; b < NB; ++b) run[b] = 0.0;
  };
  for (int g0 = w0; g0 < w1; g0 += 32 * kSumUnroll) {
    int q[kSumUnroll];
    double v[kSumUnroll][NB];
    // bins and values are loaded together (no load waits on another)
#pragma unroll
    for (int u = 0; u < kSumUnroll; ++u) {
      const int e = g0 + 32 * u + lane;
      q[u] = e < w1 ? (int)bp[e] : -1;
      if (q[u] >= 0 && !BS_CHK(q[u], a.nbin, 41)) q[u] = -1;  // a bin outside the histogram
#pragma unroll
      for (int b = 0; b < NB; ++b)
        v[u][b] = (!a.model && b < nb && e < w1) ? __ldg(vb + (long long)b * a.bstride + e) : 0.0;
    }
    if (a.model) {
#pragma unroll
      for (int u = 0; u < kSumUnroll; ++u) {
        const int e = g0 + 32 * u + lane;
        if (q[u] >= 0) {
          const int ia = e / a.nc;
          v[u][0] = model_value(a, i, j, l, ia, e - ia * a.nc);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kSumUnroll; ++u) {
      const int q0 = __shfl_sync(0xffffffffu, q[u], 0);
      if (__all_sync(0xffffffffu, q[u] == q0)) {
        if (q0 != cur) {
          flush();
          cur = q0;
        }
        if (cur >= 0) {
          cnt += 32;
#pragma unroll
          for (int b = 0; b < NB; ++b)
            if (b < nb) run[b] += v[u][b];
        }
      } else {  // mixed bins: close the run, then every lane adds its own sample
        flush();
        cur = -1;
        if (q[u] >= 0) {
          atomicAdd(hc + q[u], 1u);
#pragma unroll
          for (int b = 0; b < NB; ++b)
            if (b < nb) atomicAdd(hs + (size_t)b * a.nbin + q[u], v[u][b]);
        }
      }
    }
  }
  flush();
  __syncthreads();
  for (int q = threadIdx.x; q < a.nbin; q += blockDim.x) {
    const unsigned c = hc[q];
    if (!c) continue;
    if (a.cnt) atomicAdd(a.cnt + q, (unsigned long long)c);
    for (int b = 0; b < a.nbatch; ++b)
      atomicAdd(a.sums + (size_t)(a.b0 + b) * a.nbin + q, hs[(size_t)b * a.nbin + q]);
  }
}

// m = 0 multipoles (Eq. bs_lm): per bin the sums of (2l+1) P_l(mu_1) B over the
// paired samples, l = 0..LMAX, with mu_1 = k_par / k of the largest side (the
// first of sides 1, 2, 3 on ties) and P_l by Bonnet's recursion, in FP64 with
// the same operation order as the oracle.  Bins come from the plan's table.
// Layout as k_mono_sum: warps walk 32 consecutive samples; lane-private
// running sums while the warp's bin is unchanged.
constexpr int kMaxL = 4;

template <int NB, int LMAX>
__global__ void __launch_bounds__(kThreads) k_mono_multipole(const MonoArgs a,
                                                             const int16_t *__restrict__ bins,
                                                             int skip0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *hs = reinterpret_cast<double *>(smem_raw);  // [nbatch][LMAX + 1][nbin]
  unsigned *hc = reinterpret_cast<unsigned *>(hs + (size_t)a.nbatch * (LMAX + 1) * a.nbin);
  const int p = blockIdx.y;
  for (int q = threadIdx.x; q < a.nbatch * (LMAX + 1) * a.nbin; q += blockDim.x) hs[q] = 0.0;
  for (int q = threadIdx.x; q < a.nbin; q += blockDim.x) hc[q] = 0u;
  __syncthreads();
  const int i = a.rings[3 * p], j = a.rings[3 * p + 1], l = a.rings[3 * p + 2];
  const double pi2 = __dmul_rn(a.kperp64[i], a.kperp64[i]),
               pj2 = __dmul_rn(a.kperp64[j], a.kperp64[j]),
               pl2 = __dmul_rn(a.kperp64[l], a.kperp64[l]);
  const int n = a.nc * a.nc;
  const int c0 = blockIdx.x * a.chunk, c1 = min(n, c0 + a.chunk);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kThreads / 32;
  const int per = ((c1 - c0 + nw - 1) / nw + 31) / 32 * 32;
  const int w0 = min(c1, c0 + warp * per), w1 = min(c1, w0 + per);
  const int16_t *bp = bins + (long long)p * n;
  const double *vb = a.b3d + (long long)a.b0 * a.bstride + (long long)p * n;
  int cur = -1;
  unsigned cnt = 0;
  double run[NB][LMAX + 1];
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int q = 0; q <= LMAX; ++q) run[b][q] = 0.0;
  auto flush = [&]() {
    if (cur >= 0) {
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        if (b >= a.nbatch) break;
#pragma unroll
        for (int q = 0; q <= LMAX; ++q) {
          double x = run[b][q];
          for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
          if (lane == 0) atomicAdd(hs + ((size_t)b * (LMAX + 1) + q) * a.nbin + cur, x);
        }
      }
      if (lane == 0) atomicAdd(hc + cur, cnt);
    }
    cnt = 0;
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int q = 0; q <= LMAX; ++q) run[b][q] = 0.0;
  };
  for (int g0 = w0; g0 < w1; g0 += 32) {
    const int e = g0 + lane;
    int q = -1;
    double wl[LMAX + 1];
    if (e < w1) {
      const int ia = e / a.nc, ib = e - ia * a.nc;
      q = (skip0 && (ia == 0 || ib == 0)) ? -1 : (int)bp[e];
      if (q >= 0 && !BS_CHK(q, a.nbin, 42)) q = -1;
      if (q >= 0) {
        const double za = a.kpar64[ia], zb = a.kpar64[ib], zc = -__dadd_rn(za, zb);
        const double s1 = __dadd_rn(pi2, __dmul_rn(za, za)), s2 = __dadd_rn(pj2, __dmul_rn(zb, zb)),
                     s3 = __dadd_rn(pl2, __dmul_rn(zc, zc));
        double sm = s1, zm = za;
        if (s2 > sm) { sm = s2; zm = zb; }
        if (s3 > sm) { sm = s3; zm = zc; }
        const double x = zm / sqrt(sm);
        double pm1 = 1.0, p0 = x;
        wl[0] = 1.0;
        if (LMAX >= 1) wl[1] = 3.0 * x;
#pragma unroll
        for (int ll = 1; ll < LMAX; ++ll) {
          const double pn = ((2 * ll + 1) * x * p0 - ll * pm1) / (ll + 1);
          pm1 = p0;
          p0 = pn;
          wl[ll + 1] = (2 * ll + 3) * pn;
        }
      }
    }
    double v[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b)
      v[b] = (b < a.nbatch && e < w1) ? __ldg(vb + (long long)b * a.bstride + e) : 0.0;
    const int qq = __shfl_sync(0xffffffffu, q, 0);
    if (__all_sync(0xffffffffu, q == qq)) {
      if (qq != cur) {
        flush();
        cur = qq;
      }
      if (cur >= 0) {
        cnt += 32;
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int ll = 0; ll <= LMAX; ++ll)
            if (b < a.nbatch) run[b][ll] += wl[ll] * v[b];
      }
    } else {
      flush();
      cur = -1;
      if (q >= 0) {
        atomicAdd(hc + q, 1u);
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int ll = 0; ll <= LMAX; ++ll)
            if (b < a.nbatch)
              atomicAdd(hs + ((size_t)b * (LMAX + 1) + ll) * a.nbin + q, wl[ll] * v[b]);
      }
    }
  }
  flush();
  __syncthreads();
  for (int q = threadIdx.x; q < a.nbin; q += blockDim.x) {
    const unsigned c = hc[q];
    if (!c) continue;
    if (a.cnt) atomicAdd(a.cnt + q, (unsigned long long)c);
    for (int b = 0; b < a.nbatch; ++b)
      for (int ll = 0; ll <= LMAX; ++ll)
        atomicAdd(a.sums + ((size_t)(a.b0 + b) * (LMAX + 1) + ll) * a.nbin + q,
                  hs[((size_t)b * (LMAX + 1) + ll) * a.nbin + q]);
  }
}

// The 3D bispectrum of each plane binned on an n x n grid in the (k_par1,
// k_par2) plane (Section 5, the binning behind Fig. cylbs).  k_par grows with
// the delay index, so the bins of rows (and of columns) are contiguous index
// ranges; qa[a] is the bin of index a (-1 outside), seg[r] the index range
// of bin r.  One CTA owns one (plane, realisation) and each thread CPT
// columns: walking the rows in order, a thread keeps running column sums in
// registers while the row bin stays the same.  When it changes (the same
// row for the whole CTA), the threads write their column sums to a shared
// row buffer and thread r adds bin r's range of it to acc[q][r]: no atomics.
// Loads are coalesced row segments.  The rows of a plane are split over
// gridDim.z CTAs, which add their n x n partial sums into the (zeroed)
// output.
constexpr int kCylThreads = 256;
template <int CPT>
__global__ void __launch_bounds__(kCylThreads) k_bs_cylindrical(
    const double *__restrict__ b3d, long long bstride, int nc, int n, const int *__restrict__ qa,
    const int2 *__restrict__ seg, double *__restrict__ sums) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *acc = reinterpret_cast<double *>(smem_raw);  // [n][n]
  double *colsum = acc + n * n;                         // [nc]
  const int p = blockIdx.x, b = blockIdx.y, npl = gridDim.x;
  const int rows = (nc + gridDim.z - 1) / gridDim.z;
  const int ra = blockIdx.z * rows, rb = min(nc, ra + rows);
  for (int q = threadIdx.x; q < n * n; q += blockDim.x) acc[q] = 0.0;
  __syncthreads();
  const double *pl = b3d + (long long)b * bstride + (long long)p * nc * nc;
  int qc[CPT];
  double run[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int c = threadIdx.x + k * kCylThreads;
    qc[k] = c < nc ? qa[c] : -1;
    run[k] = 0.0;
  }
  int qcur = -1;
  auto flush = [&]() {  // CTA-uniform: every thread sees the same row bins
    if (qcur >= 0) {
#pragma unroll
      for (int k = 0; k < CPT; ++k)
        if (qc[k] >= 0) colsum[threadIdx.x + k * kCylThreads] = run[k];
      __syncthreads();
      for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const int2 sg = seg[r];
        double v = 0.0;
        for (int c = sg.x; c < sg.y; ++c) v += colsum[c];
        acc[qcur * n + r] += v;
      }
      __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < CPT; ++k) run[k] = 0.0;
  };
  constexpr int U = 8;  // rows loaded ahead
  for (int a0 = ra; a0 < rb; a0 += U) {
    double v[U][CPT];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int a = a0 + u;
      const bool rowok = a < rb && qa[a] >= 0;
#pragma unroll
      for (int k = 0; k < CPT; ++k)
        v[u][k] = (rowok && qc[k] >= 0) ? pl[(long long)a * nc + threadIdx.x + k * kCylThreads] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int a = a0 + u;
      if (a >= rb) break;
      const int q = qa[a];
      if (q != qcur) {
        flush();
        qcur = q;
      }
      if (q < 0) continue;
#pragma unroll
      for (int k = 0; k < CPT; ++k) run[k] += v[u][k];
    }
  }
  flush();
  __syncthreads();
  double *out = sums + ((long long)b * npl + p) * n * n;
  for (int q = threadIdx.x; q < n * n; q += blockDim.x)
    if (acc[q] != 0.0) atomicAdd(out + q, acc[q]);
}

// General plans: the binnings are linear in the 3D bispectrum, so its complex
// values are binned as two real realisations per realisation b: 2b the real
// part and 2b + 1 the imaginary part of in[b] ([ub][per] double2).
__global__ void k_split_complex(const double2 *__restrict__ in, long long per, int ub,
                                double *__restrict__ out) {
  const long long total = (long long)ub * per;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const long long b = q / per, k = q - b * per;
    const double2 v = in[q];
    out[2 * b * per + k] = v.x;
    out[(2 * b + 1) * per + k] = v.y;
  }
}

// ... and the real sums of the two parts, [2 ub][rest], back as complex sums
// [ub][rest].
__global__ void k_join_complex(const double *__restrict__ in, long long rest, int ub,
                               double2 *__restrict__ out) {
  const long long total = (long long)ub * rest;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const long long b = q / rest, k = q - b * rest;
    out[q] = make_double2(in[2 * b * rest + k], in[(2 * b + 1) * rest + k]);
  }
}

int grid_of(long long total) {
  return (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 152LL * 32));
}

}  // namespace

// Bytes of shared memory the summing kernel needs for nbatch realisations.
static size_t mono_smem(int nbin, int nbatch) {
  return (size_t)nbatch * nbin * 8 + (size_t)nbin * 4;
}

}  // namespace bsi

#define MONO_CUDA(call)                                          \
  do {                                                           \
    cudaError_t e__ = (call);                                    \
    if (e__ != cudaSuccess) return cuda_fail(p, e__, #call);     \
  } while (0)

// A general plan's complex closable 3D bispectrum (per = planes x nc^2 values
// per realisation) split into real planes in the plan's scratch, followed by
// zeroed room for the real sums (rest per part); *planes and *sums point there.
static bs_status split_general(bs_plan p, const double *b3d, long long per, long long rest,
                               const double **planes, double **sums, cudaStream_t s) {
  using namespace bsi;
  const long long ub = p->ubatch;
  bs_status st = general_scratch(p, &p->gbin, &p->gbin_cap, (size_t)(2 * ub * (per + rest)));
  if (st != BS_OK) return st;
  double *pl = p->gbin, *sm = p->gbin + 2 * ub * per;
  if (ub * per > 0) {
    k_split_complex<<<grid_of(ub * per), 256, 0, s>>>(reinterpret_cast<const double2 *>(b3d), per,
                                                     (int)ub, pl);
    MONO_CUDA(cudaGetLastError());
  }
  MONO_CUDA(cudaMemsetAsync(sm, 0, (size_t)(2 * ub * rest) * sizeof(double), s));
  *planes = pl;
  *sums = sm;
  return BS_OK;
}

// The real sums of split_general's parts into the caller's complex sums.
static bs_status join_general(bs_plan p, const double *sums, long long rest, double *out,
                              cudaStream_t s) {
  using namespace bsi;
  const long long ub = p->ubatch;
  if (ub * rest == 0) return BS_OK;
  k_join_complex<<<grid_of(ub * rest), 256, 0, s>>>(sums, rest, (int)ub,
                                                   reinterpret_cast<double2 *>(out));
  MONO_CUDA(cudaGetLastError());
  return BS_OK;
}

// Complex values are read and written as double2: 16-byte aligned pointers.
static bool aligned16(const void *ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15) == 0; }

// Geometry of the (k1, mu, t) binning shared by the monopole and the
// multipoles: FP64 and FP32 k tables and the squared thresholds uploaded to
// the plan, the argument fields that describe them, and the plan's cached bin
// table (rebuilt when the geometry changed).
static bs_status mono_geometry(bs_plan p, const double *kperp_host, const double *kpar_host,
                               const double *k1_edges_host, int n_k1, int n_mu, int n_t,
                               cudaStream_t s, MonoArgs &a) {
  const int npl = (int)p->clos.size();
  // constants: FP64 kperp [nb], kpar [nc]; FP32 kperp, kpar (rounded to nearest);
  // squared thresholds E_q = e_q^2 [n_k1 + 1], cmu_q = 4 m_q^2 [n_mu + 1],
  // ct_q = tau_q^2 [n_t + 1], with the acceptance limits at both ends of the
  // shape tables (a pageable source is staged before the copy call returns)
  const int nb = p->nb, nc = p->nc, nthr = n_k1 + n_mu + n_t + 3;
  std::vector<unsigned char> &tab = p->mono_tab;
  const size_t off32 = (size_t)(nb + nc) * 8;
  tab.assign(off32 + (size_t)(nb + nc + nthr) * 4, 0);
  std::vector<float> f32((size_t)nb + nc + nthr);
  for (int m = 0; m < nb; ++m) f32[m] = (float)kperp_host[m];
  for (int c = 0; c < nc; ++c) f32[nb + c] = (float)kpar_host[c];
  float *thr = f32.data() + nb + nc;
  const double lo = 0.5 - kShapeTol, hi = 1.0 + kShapeTol;
  for (int q = 0; q <= n_k1; ++q) thr[q] = (float)(k1_edges_host[q] * k1_edges_host[q]);
  thr[0] = k1_edges_host[0] > 0.0 ? thr[0] : 0.0f;  // k1 >= e_0 for every k1 > 0
  float *cmu = thr + n_k1 + 1, *ct = cmu + n_mu + 1;
  for (int q = 0; q <= n_mu; ++q) {
    const double m = q == 0 ? lo : q == n_mu ? hi : 0.5 + 0.5 * q / n_mu;
    cmu[q] = (float)(4.0 * m * m);
  }
  for (int q = 0; q <= n_t; ++q) {
    const double t = q == 0 ? lo : q == n_t ? hi : 0.5 + 0.5 * q / n_t;
    ct[q] = (float)(t * t);
  }
  std::memcpy(tab.data(), kperp_host, (size_t)nb * 8);
  std::memcpy(tab.data() + (size_t)nb * 8, kpar_host, (size_t)nc * 8);
  std::memcpy(tab.data() + off32, f32.data(), f32.size() * 4);
  unsigned char *dtab = p->at<unsigned char>(p->L.mono);
  MONO_CUDA(cudaMemcpyAsync(dtab, tab.data(), tab.size(), cudaMemcpyHostToDevice, s));
  a.bstride = (long long)npl * nc * nc;
  a.rings = p->at<int>(p->L.closrings);
  a.kperp64 = reinterpret_cast<const double *>(dtab);
  a.kpar64 = a.kperp64 + nb;
  a.kperp = reinterpret_cast<const float *>(dtab + off32);
  a.kpar = a.kperp + nb;
  a.thr = a.kpar + nc;
  a.nc = nc;
  a.n_k1 = n_k1;
  a.n_mu = n_mu;
  a.n_t = n_t;
  a.nbin = n_k1 * n_mu * n_t;
  // the bin table: rebuilt only when the geometry (tables, bin counts, planes) changed
  std::vector<unsigned char> key(tab);
  const int dims[3] = {n_k1, n_mu, n_t};
  key.insert(key.end(), reinterpret_cast<const unsigned char *>(dims),
             reinterpret_cast<const unsigned char *>(dims) + sizeof(dims));
  key.insert(key.end(), reinterpret_cast<const unsigned char *>(p->clos.data()),
             reinterpret_cast<const unsigned char *>(p->clos.data() + p->clos.size()));
  const long long total = (long long)npl * nc * nc;
  if (!p->mono_bins || key != p->mono_key) {
    if ((size_t)total > p->mono_bins_cap) {
      if (p->mono_bins) MONO_CUDA(cudaFree(p->mono_bins));
      p->mono_bins = nullptr;
      p->mono_bins_cap = 0;
      void *m = nullptr;
      const cudaError_t e = cudaMalloc(&m, (size_t)total * sizeof(int16_t));
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(p, BS_ERR_OOM, "bin table allocation failed");
      }
      p->mono_bins = static_cast<int16_t *>(m);
      p->mono_bins_cap = (size_t)total;
    }
    const int grid = (int)std::min<long long>((total + kThreads - 1) / kThreads, 152LL * 64);
    k_mono_bins<<<grid, kThreads, 0, s>>>(a, total, p->mono_bins);
    MONO_CUDA(cudaGetLastError());
    p->mono_key.swap(key);
  }
  // CTAs of 64 Ki samples (8 Ki per warp): few flushes, several CTAs per plane
  const int n = nc * nc;
  const int per_cta = 65536;
  const int nx = std::max(1, (n + per_cta - 1) / per_cta);
  a.chunk = ((n + nx - 1) / nx + 255) / 256 * 256;
  return BS_OK;
}


extern "C" {

bs_status bs_plan_ring_umean(bs_plan p, double *umean_host) {
  BS_NVTX("bs_plan_ring_umean");
  if (!p || !umean_host) return fail(p, BS_ERR_ARG, "umean_host must not be NULL");
  for (int m = 0; m < p->nb; ++m) umean_host[m] = p->umean[m];
  return BS_OK;
}

bs_status bs_bs_monopole(bs_plan p, const double *b3d, const double *kperp_host,
                         const double *kpar_host, const double *k1_edges_host, int n_k1, int n_mu,
                         int n_t, double f_ng, double p_amp, double p_index, double *sum_dev,
                         int64_t *count_dev, void *stream) {
  BS_NVTX("bs_bs_monopole");
  using namespace bsi;
  if (!p || !kperp_host || !kpar_host || !k1_edges_host || !sum_dev || !count_dev)
    return fail(p, BS_ERR_ARG, "bs_bs_monopole: NULL argument");
  if (n_k1 < 1 || n_k1 > kMonoMaxK1 || n_mu < 1 || n_t < 1 || n_mu > kMonoMaxShape ||
      n_t > kMonoMaxShape)
    return fail(p, BS_ERR_ARG, "bs_bs_monopole: bin counts out of range");
  for (int q = 0; q < n_k1; ++q)
    if (!(k1_edges_host[q + 1] > k1_edges_host[q]) || !std::isfinite(k1_edges_host[q + 1]))
      return fail(p, BS_ERR_ARG, "bs_bs_monopole: k1 edges must be finite and ascending");
  // a general plan's complex values: real and imaginary parts binned as two realisations
  const bool cplx = p->general && b3d;
  if (cplx && !(aligned16(b3d) && aligned16(sum_dev)))
    return fail(p, BS_ERR_ARG, "bs_bs_monopole: complex b3d and sums must be 16-byte aligned");
  if (!p->counts_ready) return fail(p, BS_ERR_STATE, "bs_bs_monopole before the ring-triple counts");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bs_status st = prepare(p, s);
  if (st != BS_OK) return st;
  for (int m = 0; m < p->nb; ++m)
    if (!(kperp_host[m] >= 1e-8 && kperp_host[m] <= 1e8))
      return fail(p, BS_ERR_ARG, "bs_bs_monopole: k_perp must lie in [1e-8, 1e8]");
  for (int c = 0; c < p->nc; ++c)
    if (!(std::fabs(kpar_host[c]) <= 1e8))
      return fail(p, BS_ERR_ARG, "bs_bs_monopole: |k_par| must not exceed 1e8");
  const int nbin = n_k1 * n_mu * n_t;
  const int batch = b3d ? (cplx ? 2 * p->ubatch : p->ubatch) : 1;
  const int per = std::min(batch, kMaxBatch);
  if (mono_smem(nbin, per) > (size_t)200 * 1024)
    return fail(p, BS_ERR_UNSUPPORTED, "bs_bs_monopole: too many bins for one CTA's histogram");
  MONO_CUDA(cudaMemsetAsync(sum_dev, 0, (size_t)batch * nbin * sizeof(double), s));
  MONO_CUDA(cudaMemsetAsync(count_dev, 0, (size_t)nbin * sizeof(int64_t), s));
  const int npl = (int)p->clos.size();
  if (npl == 0) return BS_OK;
  MONO_CUDA(smem_optin_once<k_mono_sum<1>>());
  MONO_CUDA(smem_optin_once<k_mono_sum<2>>());
  MONO_CUDA(smem_optin_once<k_mono_sum<4>>());
  MONO_CUDA(smem_optin_once<k_mono_sum<kMaxBatch>>());
  MonoArgs a{};
  a.b3d = b3d;
  st = mono_geometry(p, kperp_host, kpar_host, k1_edges_host, n_k1, n_mu, n_t, s, a);
  if (st != BS_OK) return st;
  a.model = b3d ? 0 : 1;
  a.f2 = 2.0 * f_ng;
  a.p_amp = p_amp;
  a.p_half = 0.5 * p_index;
  a.sums = sum_dev;
  if (cplx) {
    st = split_general(p, b3d, a.bstride, nbin, &a.b3d, &a.sums, s);
    if (st != BS_OK) return st;
  }
  a.cnt = reinterpret_cast<unsigned long long *>(count_dev);
  const int n = p->nc * p->nc;
  const int gx = (n + a.chunk - 1) / a.chunk;
  for (int b0 = 0; b0 < batch; b0 += per) {
    a.b0 = b0;
    a.nbatch = std::min(per, batch - b0);
    if (b0 > 0) a.cnt = nullptr;  // the same samples: counted by the first launch
    const dim3 grid(gx, npl);
    const size_t sm = mono_smem(nbin, a.nbatch);
    if (a.nbatch == 1)
      k_mono_sum<1><<<grid, kThreads, sm, s>>>(a, p->mono_bins);
    else if (a.nbatch == 2)
      k_mono_sum<2><<<grid, kThreads, sm, s>>>(a, p->mono_bins);
    else if (a.nbatch <= 4)
      k_mono_sum<4><<<grid, kThreads, sm, s>>>(a, p->mono_bins);
    else
      k_mono_sum<kMaxBatch><<<grid, kThreads, sm, s>>>(a, p->mono_bins);
    MONO_CUDA(cudaGetLastError());
  }
  if (cplx) return join_general(p, a.sums, nbin, sum_dev, s);
  return BS_OK;
}

bs_status bs_bs_multipoles(bs_plan p, const double *b3d, const double *kperp_host,
                           const double *kpar_host, const double *k1_edges_host, int n_k1,
                           int n_mu, int n_t, int lmax, double *sum_dev, int64_t *count_dev,
                           void *stream) {
  BS_NVTX("bs_bs_multipoles");
  using namespace bsi;
  if (!p || !b3d || !kperp_host || !kpar_host || !k1_edges_host || !sum_dev || !count_dev)
    return fail(p, BS_ERR_ARG, "bs_bs_multipoles: NULL argument");
  if (lmax < 0 || lmax > kMaxL) return fail(p, BS_ERR_ARG, "bs_bs_multipoles: lmax must be in [0, 4]");
  if (n_k1 < 1 || n_k1 > kMonoMaxK1 || n_mu < 1 || n_t < 1 || n_mu > kMonoMaxShape ||
      n_t > kMonoMaxShape)
    return fail(p, BS_ERR_ARG, "bs_bs_multipoles: bin counts out of range");
  for (int q = 0; q < n_k1; ++q)
    if (!(k1_edges_host[q + 1] > k1_edges_host[q]) || !std::isfinite(k1_edges_host[q + 1]))
      return fail(p, BS_ERR_ARG, "bs_bs_multipoles: k1 edges must be finite and ascending");
  const bool cplx = p->general;  // complex values: real and imaginary parts as two realisations
  if (cplx && !(aligned16(b3d) && aligned16(sum_dev)))
    return fail(p, BS_ERR_ARG, "bs_bs_multipoles: complex b3d and sums must be 16-byte aligned");
  if (!p->counts_ready) return fail(p, BS_ERR_STATE, "bs_bs_multipoles before the ring-triple counts");
  for (int m = 0; m < p->nb; ++m)
    if (!(kperp_host[m] >= 1e-8 && kperp_host[m] <= 1e8))
      return fail(p, BS_ERR_ARG, "bs_bs_multipoles: k_perp must lie in [1e-8, 1e8]");
  for (int c = 0; c < p->nc; ++c)
    if (!(std::fabs(kpar_host[c]) <= 1e8))
      return fail(p, BS_ERR_ARG, "bs_bs_multipoles: |k_par| must not exceed 1e8");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bs_status st = prepare(p, s);
  if (st != BS_OK) return st;
  const int nbin = n_k1 * n_mu * n_t;
  const int batch = cplx ? 2 * p->ubatch : p->ubatch;
  const int per = std::min(batch, 4);
  if ((size_t)per * (lmax + 1) * nbin * 8 + (size_t)nbin * 4 > (size_t)200 * 1024)
    return fail(p, BS_ERR_UNSUPPORTED, "bs_bs_multipoles: too many bins for one CTA's histogram");
  MONO_CUDA(cudaMemsetAsync(sum_dev, 0, (size_t)batch * (lmax + 1) * nbin * sizeof(double), s));
  MONO_CUDA(cudaMemsetAsync(count_dev, 0, (size_t)nbin * sizeof(int64_t), s));
  const int npl = (int)p->clos.size();
  if (npl == 0) return BS_OK;
  MonoArgs a{};
  a.b3d = b3d;
  st = mono_geometry(p, kperp_host, kpar_host, k1_edges_host, n_k1, n_mu, n_t, s, a);
  if (st != BS_OK) return st;
  a.sums = sum_dev;
  if (cplx) {
    st = split_general(p, b3d, a.bstride, (long long)(lmax + 1) * nbin, &a.b3d, &a.sums, s);
    if (st != BS_OK) return st;
  }
  a.cnt = reinterpret_cast<unsigned long long *>(count_dev);
  const int n = p->nc * p->nc;
  const int gx = (n + a.chunk - 1) / a.chunk;
  const int skip0 = p->nc % 2 == 0;  // delay index -nc/2 has no reflection on the grid
  for (int b0 = 0; b0 < batch; b0 += per) {
    a.b0 = b0;
    a.nbatch = std::min(per, batch - b0);
    if (b0 > 0) a.cnt = nullptr;
    const dim3 grid(gx, npl);
    const size_t sm = (size_t)a.nbatch * (lmax + 1) * nbin * 8 + (size_t)nbin * 4;
#define MULTIPOLE_LAUNCH(NB, L)                                                        \
  do {                                                                                 \
    const cudaError_t eo__ = smem_optin_once<k_mono_multipole<NB, L>>();              \
    if (eo__ != cudaSuccess) return cuda_fail(p, eo__, "multipole smem opt-in");      \
    k_mono_multipole<NB, L><<<grid, kThreads, sm, s>>>(a, p->mono_bins, skip0);       \
  } while (0)
    const int nbt = a.nbatch == 1 ? 1 : 4;
    switch (lmax * 10 + nbt) {
      case 1: MULTIPOLE_LAUNCH(1, 0); break;
      case 4: MULTIPOLE_LAUNCH(4, 0); break;
      case 11: MULTIPOLE_LAUNCH(1, 1); break;
      case 14: MULTIPOLE_LAUNCH(4, 1); break;
      case 21: MULTIPOLE_LAUNCH(1, 2); break;
      case 24: MULTIPOLE_LAUNCH(4, 2); break;
      case 31: MULTIPOLE_LAUNCH(1, 3); break;
      case 34: MULTIPOLE_LAUNCH(4, 3); break;
      case 41: MULTIPOLE_LAUNCH(1, 4); break;
      default: MULTIPOLE_LAUNCH(4, 4); break;
    }
#undef MULTIPOLE_LAUNCH
    MONO_CUDA(cudaGetLastError());
  }
  if (cplx) return join_general(p, a.sums, (long long)(lmax + 1) * nbin, sum_dev, s);
  return BS_OK;
}

bs_status bs_bs_cylindrical(bs_plan p, const double *b3d, const double *kpar_host,
                            const double *edges_host, int n, double *sum_dev, int64_t *count_dev,
                            void *stream) {
  BS_NVTX("bs_bs_cylindrical");
  using namespace bsi;
  if (!p || !b3d || !kpar_host || !edges_host || !sum_dev || !count_dev)
    return fail(p, BS_ERR_ARG, "bs_bs_cylindrical: NULL argument");
  if (n < 1 || n > 64) return fail(p, BS_ERR_ARG, "bs_bs_cylindrical: n must be in [1, 64]");
  for (int q = 0; q < n; ++q)
    if (!(edges_host[q + 1] > edges_host[q]))
      return fail(p, BS_ERR_ARG, "bs_bs_cylindrical: edges must be ascending");
  for (int c = 1; c < p->nc; ++c)
    if (!(kpar_host[c] > kpar_host[c - 1]))
      return fail(p, BS_ERR_ARG, "bs_bs_cylindrical: k_par must grow with the delay index");
  const bool cplx = p->general;  // complex values: real and imaginary parts as two realisations
  if (cplx && !(aligned16(b3d) && aligned16(sum_dev)))
    return fail(p, BS_ERR_ARG, "bs_bs_cylindrical: complex b3d and sums must be 16-byte aligned");
  if (!p->counts_ready) return fail(p, BS_ERR_STATE, "bs_bs_cylindrical before the ring-triple counts");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bs_status st = prepare(p, s);
  if (st != BS_OK) return st;
  const int nc = p->nc, npl = (int)p->clos.size();
  // bins along one axis: q = (number of edges <= k_par) - 1, decided on the host
  std::vector<int> &tab = p->cyl_tab;  // qa [nc], then seg [n] as (start, end)
  tab.assign((size_t)nc + 2 * n, 0);
  std::vector<long long> na(n, 0);
  for (int c = 0; c < nc; ++c) {
    int q = (int)(std::upper_bound(edges_host, edges_host + n + 1, kpar_host[c]) - edges_host) - 1;
    if (q >= n) q = -1;
    tab[c] = q;
    if (q >= 0) {
      if (na[q]++ == 0) tab[nc + 2 * q] = c;
      tab[nc + 2 * q + 1] = c + 1;
    }
  }
  std::vector<long long> &cnt = p->cyl_cnt;
  cnt.assign((size_t)n * n, 0);
  for (int q = 0; q < n; ++q)
    for (int r = 0; r < n; ++r) cnt[(size_t)q * n + r] = na[q] * na[r];
  MONO_CUDA(cudaMemcpyAsync(count_dev, cnt.data(), cnt.size() * sizeof(long long),
                            cudaMemcpyHostToDevice, s));
  if (npl == 0) return BS_OK;
  int *dtab = p->at<int>(p->L.cyl);
  MONO_CUDA(cudaMemcpyAsync(dtab, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  const size_t sm = ((size_t)n * n + nc) * sizeof(double);
  MONO_CUDA(smem_optin_once<k_bs_cylindrical<16>>());
  const int batch = cplx ? 2 * p->ubatch : p->ubatch;
  const long long bst = (long long)npl * nc * nc, rest = (long long)npl * n * n;
  double *sums = sum_dev;
  if (cplx) {
    st = split_general(p, b3d, bst, rest, &b3d, &sums, s);
    if (st != BS_OK) return st;
  } else {
    MONO_CUDA(cudaMemsetAsync(sum_dev, 0, (size_t)batch * rest * sizeof(double), s));
  }
  const dim3 grid(npl, batch, 2);  // two row ranges per plane
  const int2 *seg = reinterpret_cast<const int2 *>(dtab + nc);
  if (nc <= kCylThreads)
    k_bs_cylindrical<1><<<grid, kCylThreads, sm, s>>>(b3d, bst, nc, n, dtab, seg, sums);
  else if (nc <= 2 * kCylThreads)
    k_bs_cylindrical<2><<<grid, kCylThreads, sm, s>>>(b3d, bst, nc, n, dtab, seg, sums);
  else if (nc <= 3 * kCylThreads)
    k_bs_cylindrical<3><<<grid, kCylThreads, sm, s>>>(b3d, bst, nc, n, dtab, seg, sums);
  else if (nc <= 8 * kCylThreads)
    k_bs_cylindrical<8><<<grid, kCylThreads, sm, s>>>(b3d, bst, nc, n, dtab, seg, sums);
  else
    k_bs_cylindrical<16><<<grid, kCylThreads, sm, s>>>(b3d, bst, nc, n, dtab, seg, sums);
  MONO_CUDA(cudaGetLastError());
  if (cplx) return join_general(p, sums, rest, sum_dev, s);
  return BS_OK;
}

}  // extern "C"
