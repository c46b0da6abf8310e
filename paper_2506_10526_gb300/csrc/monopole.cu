// Monopole of the 3D bispectrum binned in triangle size and shape
// (Section 2: Eq. shape and Eq. bs_lm at l = m = 0; the (k1, mu, t) binning
// of Section 5; Eq. bsana for the binned analytic prediction).
//
// Samples: every closable ring triple (i, j, l) x every delay pair (a, b) of
// the Eq. (dft) output.  The three sides are k_n = sqrt(kperp_n^2 + kpar_n^2)
// with kpar_1 = kpar(a) (ring i), kpar_2 = kpar(b) (ring j) and
// kpar_3 = -(kpar_1 + kpar_2) (ring l).  With S1 >= S2 >= S3 the squared
// sides, the size is K1 = sqrt(S1) and the shape t = K2 / K1,
// mu = ((S1 + S2) - S3) / (2 K1 K2) (the closure k1 + k2 + k3 = 0 turns
// -k1.k2 into squared lengths).  A bin holds the sum of the values and the
// number of samples; the caller divides.
//
// The bin is decided in FP32 with every operation rounded once, in a fixed
// order and without fused multiply-adds, so that bin indices are a
// deterministic function of the inputs; values and sums are FP64.  The k1
// edges are compared in FP32 too: for a float x and a double e, x >= e
// exactly when x >= the smallest float not below e, so the host rounds each
// edge up to FP32 once and the comparisons stay on the FP32 pipe (the GB300
// FP64 rate is a small fraction of its FP32 rate).
//
// Kernel: grid (chunks of one plane, planes).  Each thread walks runs of kRun
// consecutive samples and keeps a running (bin, sums, count) in registers,
// flushing to the CTA's shared-memory histogram only when the bin changes
// (neighbouring delay modes mostly share a bin).  The CTA then adds its
// non-empty bins to the global sums with FP64 atomics.
#include <algorithm>
#include <cmath>
#include <limits>
#include <vector>

#include "plan_internal.h"

namespace bsi {

namespace {

constexpr int kRun = 16;      // consecutive samples per thread and pass
constexpr int kThreads = 256;
constexpr int kMaxBatch = 8;  // realisations per launch (the host loops over more)
constexpr int kMonoMaxK1 = 1024;

struct MonoArgs {
  const double *b3d;     // [batch_total][n_planes][nc][nc] or null (model)
  long long bstride;     // n_planes * nc * nc
  int b0, nbatch;        // realisations [b0, b0 + nbatch) of this launch
  const int *rings;      // [n_planes][3]
  const float *kperp;    // [nb], rounded to FP32
  const float *kpar;     // [nc], rounded to FP32
  const float *edges;    // [n_k1 + 1], each rounded up to FP32
  int nc, n_k1, n_mu, n_t, nbin;
  int chunk;             // samples per CTA (nc^2 < 2^31)
  float lo, hi;          // accepted mu, t range before clamping
  int model;
  double f2, p_amp, p_half;  // 2 f_NG, amplitude, p_index / 2
  double *sums;          // [batch_total][nbin]
  unsigned long long *cnt;  // [nbin], or null (counted by an earlier launch)
};

__device__ __forceinline__ int bin_of(const MonoArgs &a, const float *edges, float kpi, float kpj,
                                      float kpl, float ka, float kb, float (&S)[3]) {
  const float kc = -__fadd_rn(ka, kb);
  S[0] = __fadd_rn(__fmul_rn(kpi, kpi), __fmul_rn(ka, ka));
  S[1] = __fadd_rn(__fmul_rn(kpj, kpj), __fmul_rn(kb, kb));
  S[2] = __fadd_rn(__fmul_rn(kpl, kpl), __fmul_rn(kc, kc));
  float s1 = S[0], s2 = S[1], s3 = S[2], tmp;
  if (s1 < s2) { tmp = s1; s1 = s2; s2 = tmp; }
  if (s2 < s3) { tmp = s2; s2 = s3; s3 = tmp; }
  if (s1 < s2) { tmp = s1; s1 = s2; s2 = tmp; }
  const float K1 = __fsqrt_rn(s1), K2 = __fsqrt_rn(s2);
  const float t = __fdiv_rn(K2, K1);
  const float mu = __fdiv_rn(__fsub_rn(__fadd_rn(s1, s2), s3), __fmul_rn(2.0f, __fmul_rn(K1, K2)));
  if (!(mu >= a.lo && mu <= a.hi && t >= a.lo && t <= a.hi)) return -1;
  if (!(K1 >= edges[0] && K1 < edges[a.n_k1])) return -1;
  int lo = 0, hi = a.n_k1;  // edges[lo] <= K1 < edges[hi]
  while (hi - lo > 1) {
    const int m = (lo + hi) >> 1;
    if (edges[m] <= K1) lo = m; else hi = m;
  }
  const float muc = fminf(fmaxf(mu, 0.5f), 1.0f), tc = fminf(fmaxf(t, 0.5f), 1.0f);
  const int qm = min((int)floorf(__fmul_rn(__fsub_rn(muc, 0.5f), (float)(2 * a.n_mu))), a.n_mu - 1);
  const int qt = min((int)floorf(__fmul_rn(__fsub_rn(tc, 0.5f), (float)(2 * a.n_t))), a.n_t - 1);
  return (lo * a.n_mu + qm) * a.n_t + qt;
}

template <int NB>  // realisations held in registers (a.nbatch <= NB)
__global__ void __launch_bounds__(kThreads) k_bs_monopole(const MonoArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *hs = reinterpret_cast<double *>(smem_raw);                  // [nbatch][nbin]
  unsigned *hc = reinterpret_cast<unsigned *>(hs + (size_t)a.nbatch * a.nbin);  // [nbin]
  float *edges = reinterpret_cast<float *>(hc + a.nbin);                          // [n_k1 + 1]
  const int p = blockIdx.y;
  for (int q = threadIdx.x; q < a.nbatch * a.nbin; q += blockDim.x) hs[q] = 0.0;
  for (int q = threadIdx.x; q < a.nbin; q += blockDim.x) hc[q] = 0u;
  for (int q = threadIdx.x; q <= a.n_k1; q += blockDim.x) edges[q] = a.edges[q];
  __syncthreads();
  const int i = a.rings[3 * p], j = a.rings[3 * p + 1], l = a.rings[3 * p + 2];
  const float kpi = a.kperp[i], kpj = a.kperp[j], kpl = a.kperp[l];
  const int n = a.nc * a.nc;
  const int e0 = blockIdx.x * a.chunk, e1 = min(n, e0 + a.chunk);
  const double *vb = a.b3d ? a.b3d + (long long)a.b0 * a.bstride + (long long)p * n : nullptr;

  int cur = -1;
  unsigned run_n = 0;
  double run_s[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) run_s[b] = 0.0;
  auto flush = [&]() {
    if (cur >= 0 && run_n) {
      atomicAdd(hc + cur, run_n);
#pragma unroll
      for (int b = 0; b < NB; ++b)
        if (b < a.nbatch) atomicAdd(hs + (size_t)b * a.nbin + cur, run_s[b]);
    }
    run_n = 0;
#pragma unroll
    for (int b = 0; b < NB; ++b) run_s[b] = 0.0;
  };
  for (int base = e0 + threadIdx.x * kRun; base < e1; base += blockDim.x * kRun) {
    const int stop = min(e1, base + kRun);
    int ia = base / a.nc, ib = base - ia * a.nc;  // row a + nc/2, column b + nc/2
    float ka = a.kpar[ia];
    for (int e = base; e < stop; ++e, ++ib) {
      if (ib == a.nc) {
        ib = 0;
        ka = a.kpar[++ia];
      }
      float S[3];
      const int q = bin_of(a, edges, kpi, kpj, kpl, ka, a.kpar[ib], S);
      if (q < 0) continue;
      if (q != cur) {
        flush();
        cur = q;
      }
      ++run_n;
      if (a.model) {
        const double P1 = a.p_amp * pow((double)S[0], a.p_half),
                     P2 = a.p_amp * pow((double)S[1], a.p_half),
                     P3 = a.p_amp * pow((double)S[2], a.p_half);
        run_s[0] += a.f2 * (P1 * P2 + P2 * P3 + P3 * P1);
      } else {
#pragma unroll
        for (int b = 0; b < NB; ++b)
          if (b < a.nbatch) run_s[b] += vb[(long long)b * a.bstride + e];
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

}  // namespace

// Bytes of shared memory the kernel needs for nbatch realisations.
static size_t mono_smem(int nbin, int nbatch, int n_k1) {
  return (size_t)nbatch * nbin * 8 + (size_t)nbin * 4 + (size_t)(n_k1 + 1) * 4;
}

// The smallest float not below e (x >= e  <=>  x >= up_f32(e) for floats x).
static float up_f32(double e) {
  float f = (float)e;
  if ((double)f < e) f = std::nextafter(f, std::numeric_limits<float>::infinity());
  return f;
}

}  // namespace bsi

#define MONO_CUDA(call)                                          \
  do {                                                           \
    cudaError_t e__ = (call);                                    \
    if (e__ != cudaSuccess) return cuda_fail(p, e__, #call);     \
  } while (0)

extern "C" {

bs_status bs_plan_ring_umean(bs_plan p, double *umean_host) {
  if (!p || !umean_host) return fail(p, BS_ERR_ARG, "umean_host must not be NULL");
  for (int m = 0; m < p->nb; ++m) umean_host[m] = p->umean[m];
  return BS_OK;
}

bs_status bs_bs_monopole(bs_plan p, const double *b3d, const double *kperp_host,
                         const double *kpar_host, const double *k1_edges_host, int n_k1, int n_mu,
                         int n_t, double f_ng, double p_amp, double p_index, double *sum_dev,
                         int64_t *count_dev, void *stream) {
  using namespace bsi;
  if (!p || !kperp_host || !kpar_host || !k1_edges_host || !sum_dev || !count_dev)
    return fail(p, BS_ERR_ARG, "bs_bs_monopole: NULL argument");
  if (n_k1 < 1 || n_k1 > kMonoMaxK1 || n_mu < 1 || n_t < 1 || n_mu > 1024 || n_t > 1024)
    return fail(p, BS_ERR_ARG, "bs_bs_monopole: bin counts out of range");
  for (int q = 0; q < n_k1; ++q)
    if (!(k1_edges_host[q + 1] > k1_edges_host[q]) || !std::isfinite(k1_edges_host[q + 1]))
      return fail(p, BS_ERR_ARG, "bs_bs_monopole: k1 edges must be finite and ascending");
  if (!p->counts_ready) return fail(p, BS_ERR_STATE, "bs_bs_monopole before the ring-triple counts");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bs_status st = prepare(p, s);
  if (st != BS_OK) return st;
  const int nbin = n_k1 * n_mu * n_t;
  const int batch = b3d ? p->batch : 1;
  const int per = std::min(batch, kMaxBatch);
  if (mono_smem(nbin, per, n_k1) > (size_t)160 * 1024)
    return fail(p, BS_ERR_UNSUPPORTED, "bs_bs_monopole: too many bins for one CTA's histogram");
  MONO_CUDA(cudaMemsetAsync(sum_dev, 0, (size_t)batch * nbin * sizeof(double), s));
  MONO_CUDA(cudaMemsetAsync(count_dev, 0, (size_t)nbin * sizeof(int64_t), s));
  const int npl = (int)p->clos.size();
  if (npl == 0) return BS_OK;
  // FP32 constants: kperp [nb] and kpar [nc] rounded to nearest, the k1 edges
  // [n_k1 + 1] rounded up (a pageable source is staged before the copy call returns)
  std::vector<float> &ftab = p->mono_tab;
  ftab.assign((size_t)p->nb + p->nc + n_k1 + 1, 0.f);
  for (int m = 0; m < p->nb; ++m) ftab[m] = (float)kperp_host[m];
  for (int c = 0; c < p->nc; ++c) ftab[p->nb + c] = (float)kpar_host[c];
  for (int q = 0; q <= n_k1; ++q) ftab[p->nb + p->nc + q] = up_f32(k1_edges_host[q]);
  float *tab = p->at<float>(p->L.mono);
  MONO_CUDA(cudaMemcpyAsync(tab, ftab.data(), ftab.size() * sizeof(float), cudaMemcpyHostToDevice, s));
  MONO_CUDA(smem_optin_once<k_bs_monopole<1>>());
  MONO_CUDA(smem_optin_once<k_bs_monopole<2>>());
  MONO_CUDA(smem_optin_once<k_bs_monopole<4>>());
  MONO_CUDA(smem_optin_once<k_bs_monopole<kMaxBatch>>());
  MonoArgs a{};
  a.b3d = b3d;
  a.bstride = (long long)npl * p->nc * p->nc;
  a.rings = p->at<int>(p->L.closrings);
  a.kperp = tab;
  a.kpar = tab + p->nb;
  a.edges = tab + p->nb + p->nc;
  a.nc = p->nc;
  a.n_k1 = n_k1;
  a.n_mu = n_mu;
  a.n_t = n_t;
  a.nbin = nbin;
  a.lo = (float)(0.5 - 1e-6);
  a.hi = (float)(1.0 + 1e-6);
  a.model = b3d ? 0 : 1;
  a.f2 = 2.0 * f_ng;
  a.p_amp = p_amp;
  a.p_half = 0.5 * p_index;
  a.sums = sum_dev;
  a.cnt = reinterpret_cast<unsigned long long *>(count_dev);
  // about 64 Ki samples per CTA: few global flushes, several CTAs per plane
  const int n = p->nc * p->nc;
  const int per_cta = kThreads * kRun * 16;
  const int nx = std::max(1, (n + per_cta - 1) / per_cta);
  a.chunk = ((n + nx - 1) / nx + kRun - 1) / kRun * kRun;
  for (int b0 = 0; b0 < batch; b0 += per) {
    a.b0 = b0;
    a.nbatch = std::min(per, batch - b0);
    if (b0 > 0) a.cnt = nullptr;  // the same samples: counted by the first launch
    const dim3 grid(nx, npl);
    const size_t sm = mono_smem(nbin, a.nbatch, n_k1);
    if (a.nbatch == 1)
      k_bs_monopole<1><<<grid, kThreads, sm, s>>>(a);
    else if (a.nbatch == 2)
      k_bs_monopole<2><<<grid, kThreads, sm, s>>>(a);
    else if (a.nbatch <= 4)
      k_bs_monopole<4><<<grid, kThreads, sm, s>>>(a);
    else
      k_bs_monopole<kMaxBatch><<<grid, kThreads, sm, s>>>(a);
    MONO_CUDA(cudaGetLastError());
  }
  return BS_OK;
}

bs_status bs_bs_cylindrical(bs_plan p, const double *b3d, const double *kpar_host,
                            const double *edges_host, int n, double *sum_dev, int64_t *count_dev,
                            void *stream) {
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
  MONO_CUDA(cudaMemsetAsync(sum_dev, 0, (size_t)p->batch * npl * n * n * sizeof(double), s));
  const dim3 grid(npl, p->batch, 2);  // two row ranges per plane
  const int2 *seg = reinterpret_cast<const int2 *>(dtab + nc);
  const long long bst = (long long)npl * nc * nc;
  if (nc <= kCylThreads)
    k_bs_cylindrical<1><<<grid, kCylThreads, sm, s>>>(b3d, bst, nc, n, dtab, seg, sum_dev);
  else if (nc <= 2 * kCylThreads)
    k_bs_cylindrical<2><<<grid, kCylThreads, sm, s>>>(b3d, bst, nc, n, dtab, seg, sum_dev);
  else if (nc <= 3 * kCylThreads)
    k_bs_cylindrical<3><<<grid, kCylThreads, sm, s>>>(b3d, bst, nc, n, dtab, seg, sum_dev);
  else if (nc <= 8 * kCylThreads)
    k_bs_cylindrical<8><<<grid, kCylThreads, sm, s>>>(b3d, bst, nc, n, dtab, seg, sum_dev);
  else
    k_bs_cylindrical<16><<<grid, kCylThreads, sm, s>>>(b3d, bst, nc, n, dtab, seg, sum_dev);
  MONO_CUDA(cudaGetLastError());
  return BS_OK;
}

}  // extern "C"
