// Image-plane fields of Eq. (iFT): for ring m and channel nu,
//   F_{m,nu}(x, y) = sum_{g in ring m} W_g V_g(nu) exp(+2 pi i (u x + v y) / M),
// an unnormalised inverse 2D DFT of side M, real because the ring and the
// visibilities are Hermitian.  Two passes through the plan workspace:
//
//  colpass  (shell mask + weights + FFT along v)
//           G_{m,nu}(u, y) = sum_v X(u, v) exp(+2 pi i v y / M),  u >= 0,
//           X = W V restricted to ring m (W = 1/N_g, 0 for an empty cell or a
//           flagged channel).  One CTA: one channel, UB consecutive u columns,
//           all rings; the visibility tile is read once and masked per ring.
//           Output G[b][m][nu][y][u] (u fastest, UC columns).
//  rowpass  (Hermitian C2R along u)
//           F(x, y) = sum_{|u| < uext(m)} G(u, y) exp(+2 pi i u x / M) with
//           G(-u, y) = conj G(u, y); two rows y, y+1 share one complex FFT
//           (z = A + i B, F(., y) = Re z, F(., y+1) = Im z).  Output
//           F[b][m*nc+nu][y*M + x]; in split-BF16 plans also the BF16
//           hi / lo parts (hi = round(F), lo = round(F - hi)); in split-FP16
//           plans the largest |F| of each (realisation, slot) instead.
//  split16  (split-FP16 plans) F * 2^k in FP16 hi / lo, with k per
//           (realisation, slot) chosen from that largest |F| so that the
//           scaled field stays below 2^7 in magnitude.
//
// Also: exact closed-triangle counts and the Hermitian check.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "bs_internal.h"
#include "fft_smem.cuh"

namespace bsi {

namespace {

__global__ void __launch_bounds__(256) k_colpass(GridGeom g, int UB, const float2 *__restrict__ vis,
                                                 const float *__restrict__ ngrid,
                                                 const uint8_t *__restrict__ valid,
                                                 const int8_t *__restrict__ label,
                                                 const int *__restrict__ uext,
                                                 const float2 *__restrict__ twM, Radices radM,
                                                 float2 *__restrict__ G) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M = g.M, nt = g.nt, h = nt / 2;
  const int u0 = blockIdx.x * UB;
  const int nu = blockIdx.y;
  const int b = blockIdx.z;
  if (!valid[nu]) return;  // fields of a flagged channel are written as zeros by rowpass
  const int LD = M + 1;  // padded column rows: column-wise accesses spread over the banks
  float2 *tw = reinterpret_cast<float2 *>(smem_raw);
  float2 *bufA = tw + M;
  float2 *bufB = bufA + UB * LD;
  float2 *xt = bufB + UB * LD;                                  // [nt][UB] weighted visibilities
  int8_t *lt = reinterpret_cast<int8_t *>(xt + nt * UB);        // [nt][UB] ring labels
  for (int t = threadIdx.x; t < M; t += blockDim.x) tw[t] = twM[t];
  const float2 *vb = vis + ((long long)b * g.nc + nu) * (long long)nt * nt;
  for (int t = threadIdx.x; t < nt * UB; t += blockDim.x) {
    const int iv = t / UB, c = t - iv * UB;
    const int u = u0 + c;
    float2 x = make_float2(0.f, 0.f);
    int8_t lab = -1;
    if (u < h) {
      const int cell = iv * nt + (u + h);
      lab = label[cell];
      if (lab >= 0) {
        const float n = ngrid ? ngrid[cell] : 1.0f;
        if (n > 0.f) {
          const float w = 1.0f / n;
          const float2 v = vb[cell];
          x = make_float2(w * v.x, w * v.y);
        } else {
          lab = -1;
        }
      }
    }
    xt[t] = x;
    lt[t] = lab;
  }
  __syncthreads();
  for (int m = 0; m < g.nb; ++m) {
    const int ue = uext[m];
    const int slot = g.slot_of[m];
    if (slot < 0 || u0 >= ue) continue;  // block-uniform
    for (int t = threadIdx.x; t < UB * LD; t += blockDim.x) bufA[t] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int t = threadIdx.x; t < nt * UB; t += blockDim.x) {
      if (lt[t] == m) {
        const int iv = t / UB, c = t - iv * UB;
        int y = iv - h;
        if (y < 0) y += M;
        bufA[c * LD + y] = xt[t];
      }
    }
    __syncthreads();
    float2 *res = stockham(bufA, bufB, UB, M, LD, radM, tw, +1.0f);
    float2 *Gm = G + (((long long)b * g.nslot + slot) * g.nc + nu) * (long long)M * g.UC;
    const int ncols = min(UB, g.UC - u0);
    for (int t = threadIdx.x; t < M * UB; t += blockDim.x) {
      const int y = t / UB, c = t - y * UB;
      if (c < ncols) Gm[(long long)y * g.UC + u0 + c] = res[c * LD + y];
    }
    __syncthreads();
  }
}

__device__ __forceinline__ uint16_t bf16_bits(float x) {
  __nv_bfloat16 h = __float2bfloat16_rn(x);
  return *reinterpret_cast<uint16_t *>(&h);
}
__device__ __forceinline__ float bf16_val(uint16_t b) {
  return __uint_as_float(((uint32_t)b) << 16);
}

__global__ void __launch_bounds__(256) k_rowpass(GridGeom g, int RPB, const float2 *__restrict__ G,
                                                 const uint8_t *__restrict__ valid,
                                                 const int *__restrict__ uext,
                                                 const float2 *__restrict__ twM, Radices radM,
                                                 float *__restrict__ F, uint16_t *__restrict__ Fhi,
                                                 uint16_t *__restrict__ Flo,
                                                 unsigned *__restrict__ fmax) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M = g.M;
  const int f = blockIdx.y;  // slot * nc + nu
  const int slot = f / g.nc, nu = f - slot * g.nc;
  const int m = g.ring_of[slot];
  const int b = blockIdx.z;
  const int y0 = blockIdx.x * 2 * RPB;
  const int npair = min(RPB, (M - y0) / 2);
  const long long fbase = ((long long)b * g.nslot * g.nc + f) * (long long)M * M;
  const int ue = min(uext[m], g.UC);
  if (!valid[nu] || ue == 0) {
    for (int t = threadIdx.x; t < 2 * npair * M; t += blockDim.x) {
      const long long o = fbase + (long long)y0 * M + t;
      F[o] = 0.f;
      if (Fhi) {
        Fhi[o] = 0;
        Flo[o] = 0;
      }
    }
    return;
  }
  float2 *tw = reinterpret_cast<float2 *>(smem_raw);
  float2 *bufA = tw + M;
  float2 *bufB = bufA + RPB * M;
  for (int t = threadIdx.x; t < M; t += blockDim.x) tw[t] = twM[t];
  for (int t = threadIdx.x; t < RPB * M; t += blockDim.x) bufA[t] = make_float2(0.f, 0.f);
  __syncthreads();
  const float2 *Gm = G + (((long long)b * g.nslot + slot) * g.nc + nu) * (long long)M * g.UC;
  for (int t = threadIdx.x; t < npair * ue; t += blockDim.x) {
    const int p = t / ue, u = t - p * ue;
    const int y = y0 + 2 * p;
    const float2 a = Gm[(long long)y * g.UC + u];
    const float2 c = Gm[(long long)(y + 1) * g.UC + u];
    float2 *z = bufA + p * M;
    if (u == 0) {
      z[0] = make_float2(a.x, c.x);
    } else {
      z[u] = make_float2(a.x - c.y, a.y + c.x);      // A(u) + i B(u)
      z[M - u] = make_float2(a.x + c.y, c.x - a.y);  // conj A(u) + i conj B(u)
    }
  }
  __syncthreads();
  float2 *res = stockham(bufA, bufB, RPB, M, radM, tw, +1.0f);
  // four pixels per thread: 16-byte FP32 stores, 8-byte BF16 hi / lo stores (M % 4 == 0)
  const int M4 = M / 4;
  unsigned amax = 0;  // largest |F| written by this thread, as float bits (order-preserving)
  for (int t = threadIdx.x; t < npair * 2 * M4; t += blockDim.x) {
    const int p = t / (2 * M4), r = t - p * 2 * M4;
    const int which = r / M4, x = 4 * (r - which * M4);
    const float4 z01 = *reinterpret_cast<const float4 *>(res + p * M + x);
    const float4 z23 = *reinterpret_cast<const float4 *>(res + p * M + x + 2);
    const float4 v = which ? make_float4(z01.y, z01.w, z23.y, z23.w)
                           : make_float4(z01.x, z01.z, z23.x, z23.z);
    const long long o = fbase + (long long)(y0 + 2 * p + which) * M + x;
    *reinterpret_cast<float4 *>(F + o) = v;
    amax = max(amax, __float_as_uint(fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w)))));
    if (Fhi) {
      const uint16_t h0 = bf16_bits(v.x), h1 = bf16_bits(v.y), h2 = bf16_bits(v.z),
                     h3 = bf16_bits(v.w);
      const uint16_t l0 = bf16_bits(v.x - bf16_val(h0)), l1 = bf16_bits(v.y - bf16_val(h1)),
                     l2 = bf16_bits(v.z - bf16_val(h2)), l3 = bf16_bits(v.w - bf16_val(h3));
      *reinterpret_cast<uint2 *>(Fhi + o) =
          make_uint2((uint32_t)h0 | ((uint32_t)h1 << 16), (uint32_t)h2 | ((uint32_t)h3 << 16));
      *reinterpret_cast<uint2 *>(Flo + o) =
          make_uint2((uint32_t)l0 | ((uint32_t)l1 << 16), (uint32_t)l2 | ((uint32_t)l3 << 16));
    }
  }
  if (fmax) {  // one atomic per CTA: warp maxima, then the block's
    __shared__ unsigned wmax[8];
    amax = __reduce_max_sync(0xffffffffu, amax);
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = amax;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned m = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, wmax[w]);
      if (m) atomicMax(fmax + (size_t)b * g.nslot + slot, m);
    }
  }
}

// Exponent k of the power-of-two scale of a field whose largest |value| has
// float bits mb: with 2^(E-1) <= max < 2^E, k = 7 - E, so |F| 2^k < 2^7 and a
// pair product of two scaled fields stays below 2^14 (FP16 holds 65504).  An
// all-zero field takes k = 0; k is clamped to [-100, 100] so that 2^k and the
// pair scale 2^(k_i + k_j) of the contraction stay finite FP32 factors.
__device__ __forceinline__ int f16_scale_exp(unsigned mb) {
  if (mb == 0) return 0;
  const int be = (int)((mb >> 23) & 0xffu);
  const int E = be == 0 ? -126 : be - 126;
  return min(100, max(-100, 7 - E));
}
// 2^k as FP32, |k| <= 126
__device__ __forceinline__ float exp2i_f32(int k) { return __uint_as_float((uint32_t)(k + 127) << 23); }

__device__ __forceinline__ uint32_t f16x2_bits(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t *>(&h);
}

// One CTA: 1024 float4 of one field row (F[b][slot*nc + nu][0, M^2)).
__global__ void __launch_bounds__(256) k_split16(int nslot, int nc, int M2, int nrows,
                                                 const float *__restrict__ F,
                                                 const unsigned *__restrict__ fmax,
                                                 int *__restrict__ kexp,
                                                 uint16_t *__restrict__ Fhi,
                                                 uint16_t *__restrict__ Flo) {
  const int nf = nslot * nc;
  for (int row = blockIdx.y; row < nrows; row += gridDim.y) {
    const int b = row / nf, f = row - b * nf;
    const int slot = f / nc;
    const int k = f16_scale_exp(fmax[b * nslot + slot]);
    if (blockIdx.x == 0 && f == slot * nc && threadIdx.x == 0) kexp[b * nslot + slot] = k;
    const float sc = exp2i_f32(k);
    const long long base = (long long)row * M2;
    const int n4 = M2 / 4;
    for (int q = blockIdx.x * 1024 + threadIdx.x; q < min(n4, (int)(blockIdx.x + 1) * 1024); q += 256) {
      const float4 v = *reinterpret_cast<const float4 *>(F + base + 4 * (long long)q);
      const float x0 = v.x * sc, x1 = v.y * sc, x2 = v.z * sc, x3 = v.w * sc;
      const uint32_t h01 = f16x2_bits(x0, x1), h23 = f16x2_bits(x2, x3);
      const __half2 a01 = *reinterpret_cast<const __half2 *>(&h01);
      const __half2 a23 = *reinterpret_cast<const __half2 *>(&h23);
      const float2 r01 = __half22float2(a01), r23 = __half22float2(a23);
      const uint32_t l01 = f16x2_bits(x0 - r01.x, x1 - r01.y), l23 = f16x2_bits(x2 - r23.x, x3 - r23.y);
      *reinterpret_cast<uint2 *>(Fhi + base + 4 * (long long)q) = make_uint2(h01, h23);
      *reinterpret_cast<uint2 *>(Flo + base + 4 * (long long)q) = make_uint2(l01, l23);
    }
  }
}

// Effective ring labels: the plan's labels with empty cells (N_g <= 0) removed.
__global__ void k_effective_label(int ncell, const int8_t *__restrict__ label,
                                  const float *__restrict__ ngrid, int8_t *__restrict__ out) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ncell; t += gridDim.x * blockDim.x)
    out[t] = (ngrid && !(ngrid[t] > 0.f)) ? (int8_t)-1 : label[t];
}

// Closed-triangle counts: every ordered pair (g1, g2) of binned, filled cells
// is tested once; the closing point g3 = -g1 - g2 is looked up in the label
// table; when (ring(g1), ring(g2), ring(g3)) is a listed triple i <= j <= l its
// counter is incremented.  A CTA takes P1 first corners and sweeps all second
// corners; 32-bit shared counters, 64-bit global sums.
constexpr int kCountP1 = 32;

__global__ void __launch_bounds__(256) k_counts(int nt, int nb, const int8_t *__restrict__ label,
                                                const int *__restrict__ cells, int ncells,
                                                const int *__restrict__ trip_of,
                                                unsigned long long *__restrict__ T, int ntrip,
                                                int label_in_smem) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned int *cnt = reinterpret_cast<unsigned int *>(smem_raw);
  int *tof = reinterpret_cast<int *>(cnt + ntrip);
  int8_t *lab_s = reinterpret_cast<int8_t *>(tof + nb * nb * nb);
  __shared__ int su1[kCountP1], sv1[kCountP1], sr1[kCountP1];
  const int h = nt / 2;
  const int nb3 = nb * nb * nb;
  for (int t = threadIdx.x; t < ntrip; t += blockDim.x) cnt[t] = 0;
  for (int t = threadIdx.x; t < nb3; t += blockDim.x) tof[t] = trip_of[t];
  if (label_in_smem)
    for (int t = threadIdx.x; t < nt * nt; t += blockDim.x) lab_s[t] = label[t];
  const int8_t *lab = label_in_smem ? lab_s : label;
  if (threadIdx.x < kCountP1) {
    const int p = blockIdx.x * kCountP1 + threadIdx.x;
    int r = -1, u = 0, v = 0;
    if (p < ncells) {
      const int c = cells[p];
      u = (c & 0xffff) - 32768;
      v = ((c >> 16) & 0xffff) - 32768;
      r = label[(v + h) * nt + (u + h)];
    }
    su1[threadIdx.x] = u;
    sv1[threadIdx.x] = v;
    sr1[threadIdx.x] = r;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < ncells; q += blockDim.x) {
    const int c2 = cells[q];
    const int u2 = (c2 & 0xffff) - 32768, v2 = ((c2 >> 16) & 0xffff) - 32768;
    const int r2 = lab[(v2 + h) * nt + (u2 + h)];
    if (r2 < 0) continue;
#pragma unroll 4
    for (int p = 0; p < kCountP1; ++p) {
      const int r1 = sr1[p];
      if (r1 < 0) continue;
      const int u3 = -su1[p] - u2, v3 = -sv1[p] - v2;
      if (u3 <= -h || u3 >= h || v3 <= -h || v3 >= h) continue;
      const int r3 = lab[(v3 + h) * nt + (u3 + h)];
      if (r3 < 0) continue;
      const int t = tof[(r1 * nb + r2) * nb + r3];
      if (t >= 0 && BS_CHK(t, ntrip, 51)) atomicAdd(&cnt[t], 1u);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < ntrip; t += blockDim.x)
    if (cnt[t]) atomicAdd(&T[t], (unsigned long long)cnt[t]);
}

__device__ __forceinline__ void atomic_max_float(float *addr, float v) {
  // v >= 0: the IEEE bit pattern orders like an unsigned integer
  atomicMax(reinterpret_cast<unsigned int *>(addr), __float_as_uint(v));
}

__global__ void k_hermitian(const float2 *__restrict__ vis, int nc, int nt,
                            const int8_t *__restrict__ label, float *maxdiff, float *maxabs) {
  const int h = nt / 2;
  float md = 0.f, ma = 0.f;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)nc * nt * nt;
       t += (long long)gridDim.x * blockDim.x) {
    const int cell = (int)(t % ((long long)nt * nt));
    const long long base = (long long)blockIdx.y * nc * nt * nt + (t - cell);
    const float2 a = vis[base + cell];
    ma = fmaxf(ma, fabsf(a.x) + fabsf(a.y));
    if (label[cell] < 0) continue;
    const int iu = cell % nt, iv = cell / nt;
    const int mirror = (2 * h - iv) * nt + (2 * h - iu);
    const float2 c = vis[base + mirror];
    md = fmaxf(md, fabsf(a.x - c.x) + fabsf(a.y + c.y));
  }
  for (int o = 16; o > 0; o >>= 1) {
    md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
    ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_float(maxdiff, md);
    atomic_max_float(maxabs, ma);
  }
}

}  // namespace

cudaError_t launch_colpass(const GridGeom &g, const float2 *vis, const float *ngrid,
                           const uint8_t *valid, const int8_t *label, const int *uext,
                           const float2 *twM, const Radices &radM, float2 *G, cudaStream_t s) {
  if (has_reg_fft(g.M, g.nt)) return launch_colpass_reg(g, vis, ngrid, valid, label, uext, twM, G, s);
  // at least two CTAs per SM (shared memory below ~110 KB)
  int UB = 16;
  auto bytes = [&](int ub) {
    return (size_t)(g.M + 2 * ub * (g.M + 1) + g.nt * ub) * sizeof(float2) + (size_t)g.nt * ub;
  };
  while (UB > 1 && bytes(UB) > (size_t)110 * 1024) UB /= 2;
  const size_t smem = bytes(UB);
  cudaError_t e = smem_optin_once<k_colpass>();
  if (e != cudaSuccess) return e;
  dim3 grid((g.UC + UB - 1) / UB, g.nc, g.batch);
  k_colpass<<<grid, 256, smem, s>>>(g, UB, vis, ngrid, valid, label, uext, twM, radM, G);
  return cudaGetLastError();
}

cudaError_t launch_rowpass(const GridGeom &g, const float2 *G, const uint8_t *valid,
                           const int *uext, const float2 *twM, const Radices &radM, float *F,
                           uint16_t *Fhi, uint16_t *Flo, unsigned *fmax, cudaStream_t s) {
  if (has_reg_fft(g.M, g.nt)) return launch_rowpass_reg(g, G, valid, uext, twM, F, Fhi, Flo, fmax, s);
  int RPB = 8;
  while (RPB > 1 && (size_t)(2 * RPB * g.M + g.M) * sizeof(float2) > (size_t)96 * 1024) RPB /= 2;
  const size_t smem = (size_t)(2 * RPB * g.M + g.M) * sizeof(float2);
  cudaError_t e = smem_optin_once<k_rowpass>();
  if (e != cudaSuccess) return e;
  dim3 grid((g.M / 2 + RPB - 1) / RPB, g.nslot * g.nc, g.batch);
  k_rowpass<<<grid, 256, smem, s>>>(g, RPB, G, valid, uext, twM, radM, F, Fhi, Flo, fmax);
  return cudaGetLastError();
}

cudaError_t launch_split_f16(const GridGeom &g, const float *F, const unsigned *fmax, int *kexp,
                             uint16_t *Fhi, uint16_t *Flo, cudaStream_t s) {
  const int M2 = g.M * g.M;  // a multiple of 4: M % 4 == 0
  const int nrows = g.batch * g.nslot * g.nc;
  if (nrows == 0) return cudaSuccess;
  dim3 grid((M2 / 4 + 1023) / 1024, std::min(nrows, 65535));
  k_split16<<<grid, 256, 0, s>>>(g.nslot, g.nc, M2, nrows, F, fmax, kexp, Fhi, Flo);
  return cudaGetLastError();
}

cudaError_t launch_effective_label(int ncell, const int8_t *label, const float *ngrid,
                                  int8_t *out, cudaStream_t s) {
  k_effective_label<<<(ncell + 255) / 256, 256, 0, s>>>(ncell, label, ngrid, out);
  return cudaGetLastError();
}

cudaError_t launch_counts(int nt, int nb, const int8_t *label, const int *cells, int ncells,
                          const int *trip_of, unsigned long long *T, cudaStream_t s) {
  const int ntrip = nb * (nb + 1) * (nb + 2) / 6;
  if (ncells == 0) return cudaSuccess;
  const size_t base = (size_t)ntrip * sizeof(unsigned int) + (size_t)nb * nb * nb * sizeof(int);
  const int in_smem = base + (size_t)nt * nt <= (size_t)160 * 1024;
  const size_t smem = base + (in_smem ? (size_t)nt * nt : 0);
  cudaError_t e = smem_optin_once<k_counts>();
  if (e != cudaSuccess) return e;
  dim3 grid((ncells + kCountP1 - 1) / kCountP1);
  k_counts<<<grid, 256, smem, s>>>(nt, nb, label, cells, ncells, trip_of, T, ntrip, in_smem);
  return cudaGetLastError();
}

cudaError_t launch_hermitian_check(const float2 *vis, int batch, int nc, int nt,
                                   const int8_t *label, float *maxdiff, float *maxabs,
                                   cudaStream_t s) {
  const long long n = (long long)nc * nt * nt;
  int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
  dim3 grid(blocks, batch);
  k_hermitian<<<grid, 256, 0, s>>>(vis, nc, nt, label, maxdiff, maxabs);
  return cudaGetLastError();
}

}  // namespace bsi
