// Bound on the rounding error of the MABS estimates of Eq. (estimator_t).
//
// The estimate of ring triple (i, j, l) at channels (nu1, nu2, nu3) is
// S / (A M^2 T) with S = sum_x F_i F_j F_l over the M^2 image pixels.  The
// computed S differs from the exact one through (1) the FP32 transforms that
// make the fields, (2) the rounding of each product term (the pair product
// in FP32, and in the split modes the hi + lo operand parts), and (3) the
// FP32 accumulation of the terms before the FP64 sums.  To first order:
//
//   |dS| <= (c_term + c_acc) sum_x |F_i F_j F_l|
//           + sum_x |dF_i F_j F_l| + the two permutations (dF: field error)
//
// and, by Hoelder's and Cauchy-Schwarz's inequalities,
//   sum_x |F_i F_j F_l| <= ||F_i||_3 ||F_j||_3 ||F_l||_3,
//   sum_x |dF_i F_j F_l| <= ||dF_i||_2 min(||F_j||_inf ||F_l||_2, ||F_j||_2 ||F_l||_inf),
//   ||dF||_2 <= eps_fft ||F||_2                 (normwise FFT error).
// Constants, with u = 2^-24:
//   c_term  FP32 u (pair product); split BF16 3 2^-16 + u (each operand
//           split into hi + lo keeps 16 bits, and lo.lo is dropped); split
//           FP16 3 2^-22 + u, plus an absolute term 2^-25 (2^14 + 2^7) M^2
//           2^-(k_i + k_j + k_l) for the FP16 subnormal floor of the scaled
//           operands (|scaled field| < 2^7, |scaled pair| < 2^14)
//   c_acc   FP32 SIMT: (1024 + ceil(M^2 / 1024) + 1) u (runs of 1024 FMAs,
//           folded into a second FP32 register set); tensor cores:
//           2 u (3 ceil(M^2 / 16) + 1) (every K16 MMA adds into the FP32
//           accumulator, three products per K step; 2 u covers truncation)
//   eps_fft (2 (ceil(log2 M) + 2) 8 + 2) u: two 1D passes, each stage adding
//           at most 8 u of normwise relative error (Higham, Accuracy and
//           Stability of Numerical Algorithms, Thm 24.2, with computed
//           twiddles; mixed-radix stages counted generously), plus the
//           weights and the final store
// The norms are the largest over the channels of each ring's fields (at the
// image side of the triple), so one bound covers every estimate of the ring
// triple: every entry of the full cube, and every mean of the collapsed,
// folded plane.  A factor 1.01 covers second-order terms and the FP32
// rounding of the norms themselves.  These are worst-case bounds: the
// measured errors lie well below them.
//
// General (non-Hermitian) plans evaluate the real path four times, on the
// Hermitian inputs X_H + t Y with t = 0, 1, -1, 2, and combine the results as
// Re S = 2 S(0) - (S(1) + S(-1)) / 2 and Im S = (9 S(1) - S(-1) - 2 S(2) -
// 6 S(0)) / 6.  Each S(t) is an ordinary real evaluation with its own
// computed fields, so its error has the bound above (beta_t, from the norms
// of that evaluation's fields); the combination's weights are exact, so
//   |d Re S| <= 2 beta_0 + (beta_1 + beta_-1) / 2,
//   |d Im S| <= (9 beta_1 + beta_-1 + 2 beta_2 + 6 beta_0) / 6,
// and the bound on the complex error |dS| is the hypot of the two.
//
// Per-channel sampling plans estimate R = S_D / (A S_I) per channel triple,
// with S_I the triple sum of the occupancy fields, and collapse as the ratio
// of the summed numerators and denominators over the K channel triples of a
// bin.  With computed sums S^ = S + dS and |dS_D| <= beta_D, |dS_I| <= beta_I
// per channel triple (the bound above on each component's own fields),
//   R^ - R = (dS_D - A R dS_I) / (A S^_I)   (exactly), so
//   |R^ - R| <= (beta_D / A + |R^| beta_I) / (<S^_I> - beta_I)
// for a bin whose mean computed denominator <S^_I> exceeds beta_I (infinite
// otherwise).  The bound is per bin of the folded plane; per ring triple the
// largest over its bins is reported.
#include <cmath>

#include "plan_internal.h"

namespace bsi {

namespace {

constexpr double kU = 1.0 / 16777216.0;  // 2^-24
constexpr int kNormThreads = 512;

// Per-field norms of one level's FP32 fields [nfield][m2]: out[3 f + 0..2] =
// max |F|, ||F||_2, ||F||_3.  One CTA per field: pass 1 finds the maximum,
// pass 2 sums (|F| / 2^e)^2 and (|F| / 2^e)^3 with 2^e > max, so that every
// term is below 1 (no FP32 overflow), per thread in FP32 and across the CTA
// in FP64.
__global__ void __launch_bounds__(kNormThreads) k_field_norms(const float *__restrict__ F,
                                                               long long m2,
                                                               double *__restrict__ out) {
  __shared__ float smax[kNormThreads / 32];
  __shared__ double s2s[kNormThreads / 32], s3s[kNormThreads / 32];
  __shared__ float bmax;
  const float *f = F + (long long)blockIdx.x * m2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float mx = 0.f;
  for (long long x = threadIdx.x; x < m2; x += blockDim.x) mx = fmaxf(mx, fabsf(f[x]));
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) smax[warp] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.f;
    for (int w = 0; w < kNormThreads / 32; ++w) m = fmaxf(m, smax[w]);
    bmax = m;
  }
  __syncthreads();
  const float m = bmax;
  int e = 0;
  frexpf(m, &e);  // m = g 2^e with g in [0.5, 1): 2^e > m
  const float sc = ldexpf(1.f, -e);
  float a2 = 0.f, a3 = 0.f;
  for (long long x = threadIdx.x; x < m2; x += blockDim.x) {
    const float a = fabsf(f[x]) * sc, q = a * a;
    a2 += q;
    a3 += q * a;
  }
  double d2 = a2, d3 = a3;
  for (int o = 16; o; o >>= 1) {
    d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    d3 += __shfl_xor_sync(0xffffffffu, d3, o);
  }
  if (lane == 0) {
    s2s[warp] = d2;
    s3s[warp] = d3;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t2 = 0.0, t3 = 0.0;
    for (int w = 0; w < kNormThreads / 32; ++w) {
      t2 += s2s[w];
      t3 += s3s[w];
    }
    double *o = out + 3ll * blockIdx.x;
    o[0] = m;
    o[1] = m > 0.f ? ldexp(sqrt(t2), e) : 0.0;
    o[2] = m > 0.f ? ldexp(cbrt(t3), e) : 0.0;
  }
}

struct BoundLevel {
  const double *norms;  // [batch][nslot][nc][3] of this level
  const int *slot_of;   // [nb]
  const int *kexp;      // [batch][nslot] scale exponents (split FP16), else null
  int level, nslot, nc, ntrip;
  int batch;            // realisations written (the caller's, or internal for mode 2)
  int mode;             // 0 bound of S / (A M^2 T); 1 general plan: four evaluations per
                        // realisation (t = 0, 1, -1, 2); 2 bound of each internal
                        // evaluation's S, not normalised
  double c1;            // c_term + c_acc
  double cf;            // eps_fft
  double floor16;       // 2^-25 (2^14 + 2^7) M^2 (split FP16), else 0
};

// Largest norm k (0 max, 1 2-norm, 2 3-norm) over the channels of ring r's fields.
__device__ double ring_max(const BoundLevel &L, int b, int r, int k) {
  const int slot = L.slot_of[r];
  const double *n = L.norms + ((long long)b * L.nslot + slot) * L.nc * 3;
  double m = 0.0;
  for (int c = 0; c < L.nc; ++c) m = fmax(m, n[3 * c + k]);
  return m;
}

// First-order bound on |dS| of one real evaluation (internal realisation b) of
// the ring triple with rings r.
__device__ double trip_beta(const BoundLevel &L, int b, const int r[3]) {
  double ninf[3], n2[3], n3[3];
  for (int q = 0; q < 3; ++q) {
    ninf[q] = ring_max(L, b, r[q], 0);
    n2[q] = ring_max(L, b, r[q], 1);
    n3[q] = ring_max(L, b, r[q], 2);
  }
  double fft = 0.0;
  for (int q = 0; q < 3; ++q) {
    const int a = (q + 1) % 3, c = (q + 2) % 3;
    fft += n2[q] * fmin(ninf[a] * n2[c], n2[a] * ninf[c]);
  }
  double beta = L.c1 * n3[0] * n3[1] * n3[2] + L.cf * fft;
  if (L.kexp) {
    const int *k = L.kexp + (long long)b * L.nslot;
    const int ks = k[L.slot_of[r[0]]] + k[L.slot_of[r[1]]] + k[L.slot_of[r[2]]];
    beta += ldexp(L.floor16, -ks);
  }
  return beta;
}

// bound[b][trip] for the ring triples of one level (table: i, j, l, level).
__global__ void k_trip_bound(BoundLevel L, const int *__restrict__ tab,
                             const double *__restrict__ tnorm, double *__restrict__ bound) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= L.batch * L.ntrip) return;
  const int b = t / L.ntrip, trip = t - b * L.ntrip;
  if (tab[4 * trip + 3] != L.level || !(tnorm[trip] > 0.0)) return;
  const int r[3] = {tab[4 * trip], tab[4 * trip + 1], tab[4 * trip + 2]};
  if (L.mode == 2) {
    bound[(long long)b * L.ntrip + trip] = 1.01 * trip_beta(L, b, r);
    return;
  }
  double beta;
  if (L.mode == 0) {
    beta = trip_beta(L, b, r);
  } else {  // evaluations t = 0, 1, -1, 2 of realisation b are internal 4b .. 4b + 3
    const double b0 = trip_beta(L, 4 * b, r), b1 = trip_beta(L, 4 * b + 1, r),
                 bm = trip_beta(L, 4 * b + 2, r), b2 = trip_beta(L, 4 * b + 3, r);
    const double re = 2.0 * b0 + 0.5 * (b1 + bm);
    const double im = (9.0 * b1 + bm + 2.0 * b2 + 6.0 * b0) / 6.0;
    beta = sqrt(re * re + im * im);
  }
  bound[(long long)b * L.ntrip + trip] = 1.01 * beta * tnorm[trip];
}

// relerr[b][pl][d] = bound[b][trip(pl)] / |delta[b][pl][d]|; trip(pl) = pl, or
// clos[pl] for the closable layout; delta complex (modulus) for general plans.
// NaN where the estimate is undefined.
template <bool CPLX>
__global__ void k_delta_relerr(const double *__restrict__ delta, const double *__restrict__ bound,
                               const int *__restrict__ clos, int nplanes, int ntrip, long long n2,
                               long long total, double *__restrict__ relerr) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const long long bp = q / n2;
    const int b = (int)(bp / nplanes), pl = (int)(bp - (long long)b * nplanes);
    const int trip = clos ? clos[pl] : pl;
    const double mag = CPLX ? hypot(delta[2 * q], delta[2 * q + 1]) : fabs(delta[q]);
    relerr[q] = bound[(long long)b * ntrip + trip] / mag;
  }
}

// bound[b][trip] = 0 for ring triples with a closed triangle (the largest bin
// bound is taken into it), NaN for the others.
__global__ void k_bound_init(const double *__restrict__ tnorm, int ub, int ntrip,
                             double *__restrict__ bound) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ub * ntrip) return;
  bound[q] = tnorm[q % ntrip] > 0.0 ? 0.0 : __longlong_as_double(0x7ff8000000000000LL);
}

// Per-channel sampling plans: relerr[b][pl][d] of the ratio R = delta[b][pl][d]
// from the mean denominator comp[2b + 1][pl][d] (normalised by tnorm) and the
// per-evaluation bounds beta[2b][trip] (numerator), beta[2b + 1][trip]
// (denominator); the largest absolute bound of each ring triple into bound.
__global__ void k_ratio_relerr(const double *__restrict__ delta, const double *__restrict__ comp,
                               const double *__restrict__ beta, const double *__restrict__ tnorm,
                               const int *__restrict__ clos, int nplanes, int ntrip,
                               long long n2, long long total, double inv_a,
                               double *__restrict__ relerr, double *__restrict__ bound) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const long long bp = q / n2, d = q - bp * n2;
    const int b = (int)(bp / nplanes), pl = (int)(bp - (long long)b * nplanes);
    const int trip = clos ? clos[pl] : pl;
    const double R = delta[q];
    if (!(R == R)) {  // undefined estimate
      relerr[q] = R;
      continue;
    }
    const double tn = tnorm[trip];
    const double bd = beta[(2ll * b) * ntrip + trip] * tn,
                 bi = beta[(2ll * b + 1) * ntrip + trip] * tn;
    const double den = comp[((2ll * b + 1) * nplanes + pl) * n2 + d] - bi;
    const double e = den > 0.0 ? (bd * inv_a + fabs(R) * bi) / den : INFINITY;
    relerr[q] = e / fabs(R);
    atomicMax(reinterpret_cast<unsigned long long *>(bound + (long long)b * ntrip + trip),
              (unsigned long long)__double_as_longlong(e));  // e >= 0: bit order = value order
  }
}

int ceil_log2(int m) {
  int k = 0;
  while ((1 << k) < m) ++k;
  return k;
}

}  // namespace

}  // namespace bsi

#define EB_CUDA(call)                                        \
  do {                                                       \
    cudaError_t e__ = (call);                                \
    if (e__ != cudaSuccess) return cuda_fail(p, e__, #call); \
  } while (0)

extern "C" bs_status bs_mabs_error_bound(bs_plan p, double *bound_dev, const double *delta_dev,
                                         int closable, double *relerr_dev, void *stream) {
  BS_NVTX("bs_mabs_error_bound");
  using namespace bsi;
  if (!p || !bound_dev) return fail(p, BS_ERR_ARG, "bs_mabs_error_bound: bound_dev must not be NULL");
  if ((delta_dev == nullptr) != (relerr_dev == nullptr))
    return fail(p, BS_ERR_ARG, "bs_mabs_error_bound: give both delta_dev and relerr_dev, or neither");
  if (closable != 0 && closable != 1)
    return fail(p, BS_ERR_ARG, "bs_mabs_error_bound: closable must be 0 or 1");
  if (p->chans && !delta_dev)
    return fail(p, BS_ERR_ARG,
                "bs_mabs_error_bound: a per-channel sampling plan bounds a folded plane "
                "(give delta_dev and relerr_dev)");
  if (!p->loaded || !p->counts_ready)
    return fail(p, BS_ERR_STATE, "bs_mabs_error_bound before bs_grid_load");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bs_status st = prepare(p, s);
  if (st != BS_OK) return st;
  const int prec = p->d.precision;
  const double c_term = prec == BS_PREC_FP32         ? kU
                        : prec == BS_PREC_SPLIT_BF16 ? 3.0 * std::ldexp(1.0, -16) + kU
                                                     : 3.0 * std::ldexp(1.0, -22) + kU;
  // ring triples: rings and level
  std::vector<int> &tab = p->err_tab;
  tab.assign((size_t)p->ntrip * 4, -1);
  for (int t = 0; t < p->ntrip; ++t) {
    for (int k = 0; k < 3; ++k) tab[4 * t + k] = p->trips[3 * t + k];
    tab[4 * t + 3] = p->T[t] > 0 ? p->lev_of_trip[t] : -1;
  }
  int *dtab = p->at<int>(p->L.errtab);
  EB_CUDA(cudaMemcpyAsync(dtab, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  // the caller's realisations (a general plan holds four internal ones per
  // realisation, a per-channel sampling plan two)
  const int out_batch = p->general || p->chans ? p->ubatch : p->batch;
  double *beta_int = nullptr;  // per-channel sampling: per-evaluation bounds [batch][ntrip]
  if (p->chans) {
    st = general_scratch(p, &p->gerr, &p->gerr_cap, (size_t)p->batch * p->ntrip);
    if (st != BS_OK) return st;
    beta_int = p->gerr;
  }
  // NaN (all bits set) for every ring triple without a closed triangle
  EB_CUDA(cudaMemsetAsync(bound_dev, 0xFF, (size_t)out_batch * p->ntrip * sizeof(double), s));
  double *norms = p->at<double>(p->L.errn);
  for (int li = 0; li < (int)p->levels.size(); ++li) {
    const Level &lv = p->levels[li];
    if (lv.nslot == 0) continue;
    const long long m2 = (long long)lv.M * lv.M;
    const int nfield = p->batch * lv.nslot * p->nc;
    k_field_norms<<<nfield, kNormThreads, 0, s>>>(p->at<float>(lv.offF), m2, norms);
    EB_CUDA(cudaGetLastError());
    BoundLevel B{};
    B.norms = norms;
    B.slot_of = p->at<int>(lv.offSlot);
    B.kexp = prec == BS_PREC_SPLIT_FP16 ? p->at<int>(lv.offKexp) : nullptr;
    B.level = li;
    B.nslot = lv.nslot;
    B.nc = p->nc;
    B.batch = p->chans ? p->batch : out_batch;
    B.mode = p->chans ? 2 : p->general ? 1 : 0;
    B.ntrip = p->ntrip;
    const double c_acc = prec == BS_PREC_FP32
                             ? (1024.0 + std::ceil((double)m2 / 1024.0) + 1.0) * kU
                             : 2.0 * kU * (3.0 * std::ceil((double)m2 / 16.0) + 1.0);
    B.c1 = c_term + c_acc;
    B.cf = (2.0 * (ceil_log2(lv.M) + 2) * 8.0 + 2.0) * kU;
    B.floor16 = prec == BS_PREC_SPLIT_FP16 ? std::ldexp(1.0, -25) * (16384.0 + 128.0) * (double)m2
                                           : 0.0;
    const int nt = B.batch * p->ntrip;
    k_trip_bound<<<(nt + 255) / 256, 256, 0, s>>>(B, dtab, p->at<double>(p->L.tnorm),
                                                  p->chans ? beta_int : bound_dev);
    EB_CUDA(cudaGetLastError());
    norms += (size_t)nfield * 3;
  }
  if (p->chans) {
    const int npl = closable ? (int)p->clos.size() : p->ntrip;
    const long long n2 = (long long)(2 * p->nc - 1) * (2 * p->nc - 1);
    const long long total = (long long)out_batch * npl * n2;
    const int nb = out_batch * p->ntrip;
    k_bound_init<<<(nb + 255) / 256, 256, 0, s>>>(p->at<double>(p->L.tnorm), out_batch, p->ntrip,
                                                 bound_dev);
    EB_CUDA(cudaGetLastError());
    const double *comp = nullptr;
    st = chans_components(p, closable != 0, s, &comp);
    if (st != BS_OK) return st;
    if (total > 0) {
      const int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 32);
      k_ratio_relerr<<<grid, 256, 0, s>>>(delta_dev, comp, beta_int, p->at<double>(p->L.tnorm),
                                          closable ? p->at<int>(p->L.clos) : nullptr, npl,
                                          p->ntrip, n2, total, 1.0 / p->normA, relerr_dev,
                                          bound_dev);
      EB_CUDA(cudaGetLastError());
    }
    return BS_OK;
  }
  if (delta_dev) {
    const int npl = closable ? (int)p->clos.size() : p->ntrip;
    const long long n2 = (long long)(2 * p->nc - 1) * (2 * p->nc - 1);
    const long long total = (long long)out_batch * npl * n2;
    if (total > 0) {
      const int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 32);
      const int *clos = closable ? p->at<int>(p->L.clos) : nullptr;
      if (p->general)
        k_delta_relerr<true><<<grid, 256, 0, s>>>(delta_dev, bound_dev, clos, npl, p->ntrip, n2,
                                                  total, relerr_dev);
      else
        k_delta_relerr<false><<<grid, 256, 0, s>>>(delta_dev, bound_dev, clos, npl, p->ntrip, n2,
                                                   total, relerr_dev);
      EB_CUDA(cudaGetLastError());
    }
  }
  return BS_OK;
}
