// Triple contraction of Eq. (estimator_t), plain FP32 path (SIMT FMA):
//
//   S(i nu1, j nu2, l nu3) = sum_x F_{i,nu1}(x) F_{j,nu2}(x) F_{l,nu3}(x)
//
// cast as a GEMM: rows are channel pairs (nu1, nu2) of a ring pair (i, j)
// whose pair operand P(x) = F_{i,nu1}(x) F_{j,nu2}(x) is formed on the fly in
// shared memory; columns are fields (l, nu3) with l >= j and T(i, j, l) > 0;
// K runs over the M^2 image pixels.
//
// CTA tile: 128 rows = a 16 (nu1) x 8 (nu2) rectangle, 128 columns, K chunk
// 16; 256 threads, 8 x 8 accumulators each (rows {4ty..4ty+3, 64+4ty..},
// columns {4tx.., 64+4tx..}).  Partial sums are FP32, folded into a second
// FP32 register set every 64 chunks (two-level summation bounds the rounding
// growth over long K).  The K range can be split across CTAs; tile results
// meet in FP64 global atomics:
//   FULL  out[b][trip][nu1][nu2][nu3] += S / (A M^2 T(trip))
//   DELTA dsum[b][trip][nu1-nu3][nu2-nu3] += S, after a shared-memory
//         pre-reduction keyed by (segment of equal trip, nu1-nu2, nu2-nu3).
#include "bs_internal.h"

namespace bsi {

namespace {

constexpr int TR1 = 16, TR2 = 8, TROWS = TR1 * TR2, TCOLS = 128, KC = 16;
constexpr int KOUTER = 64;       // chunks between folds into the outer accumulators
constexpr int RED_CAP = 6144;    // floats of the DELTA pre-reduction buffer
constexpr int MAX_SEG = 64;

template <bool FULL, bool DELTA>
__global__ void __launch_bounds__(256, 1) k_contract_simt(ContractArgs a) {
  __shared__ __align__(16) float As[KC][TROWS];
  __shared__ __align__(16) float Bs[KC][TCOLS];
  __shared__ float rawI[TR1][KC + 1];
  __shared__ float rawJ[TR2][KC + 1];
  __shared__ int colField[TCOLS], colTrip[TCOLS], colNu3[TCOLS], colSeg[TCOLS];
  __shared__ int segTrip[MAX_SEG], segBase[MAX_SEG], segE[MAX_SEG], segD2min[MAX_SEG];
  __shared__ int nsegS, redTotal;
  __shared__ float red[DELTA ? RED_CAP : 1];

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int rt = blockIdx.x;
  const int r1b = rt / a.n_r2, r2b = rt - r1b * a.n_r2;
  const int nu1_0 = a.nu1_lo + r1b * TR1, nu2_0 = a.nu2_lo + r2b * TR2;
  const PairTile pt = a.ptiles[blockIdx.y];
  const int kseg = blockIdx.z % a.nkseg, b = blockIdx.z / a.nkseg;
  const int k0 = kseg * a.kseg_len;
  const int k1 = min(a.M2, k0 + a.kseg_len);
  const float *Fb = a.F + (long long)b * a.bstride;

  for (int c = tid; c < TCOLS; c += blockDim.x) {
    const int cc = pt.col0 + c;
    if (cc < pt.ncol) {
      const ColEntry e = a.cols[pt.col_off + cc];
      colField[c] = e.field;
      colTrip[c] = e.trip;
      colNu3[c] = e.nu3;
    } else {
      colField[c] = -1;
      colTrip[c] = -1;
      colNu3[c] = 0;
    }
  }
  __syncthreads();
  if (DELTA && tid == 0) {
    // segments of consecutive columns with the same ring triple
    int ns = 0, base = 0, c = 0;
    while (c < TCOLS && colField[c] >= 0) {
      int e = c, lo = colNu3[c], hi = colNu3[c];
      while (e + 1 < TCOLS && colField[e + 1] >= 0 && colTrip[e + 1] == colTrip[c]) {
        ++e;
        lo = min(lo, colNu3[e]);
        hi = max(hi, colNu3[e]);
      }
      if (ns < MAX_SEG) {
        segTrip[ns] = colTrip[c];
        segBase[ns] = base;
        segE[ns] = (TR2 - 1) + (hi - lo) + 1;
        segD2min[ns] = nu2_0 - hi;
        for (int q = c; q <= e; ++q) colSeg[q] = ns;
        base += (TR1 + TR2 - 1) * segE[ns];
      } else {
        base = RED_CAP + 1;  // too many segments: direct atomics
      }
      ++ns;
      c = e + 1;
    }
    nsegS = min(ns, MAX_SEG);
    redTotal = base;
  }
  __syncthreads();

  float acc[8][8], accO[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      acc[i][j] = 0.f;
      accO[i][j] = 0.f;
    }

  const long long fI = (long long)pt.ri * a.nc, fJ = (long long)pt.rj * a.nc;
  int nchunk = 0;
  for (int kc = k0; kc < k1; kc += KC) {
    {  // raw rows of the pair operand: 16 nu1 rows and 8 nu2 rows x 16 pixels
      const int r = tid >> 4, k = tid & 15;
      const int nu1 = nu1_0 + r;
      rawI[r][k] = (nu1 < a.nu1_hi) ? Fb[(fI + nu1) * a.fstride + kc + k] : 0.f;
      if (tid < TR2 * KC) {
        const int nu2 = nu2_0 + r;
        rawJ[r][k] = (nu2 < a.nu2_hi) ? Fb[(fJ + nu2) * a.fstride + kc + k] : 0.f;
      }
    }
    for (int q = tid; q < TCOLS * (KC / 4); q += blockDim.x) {
      const int c = q >> 2, kk = (q & 3) * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (colField[c] >= 0)
        v = *reinterpret_cast<const float4 *>(Fb + (long long)colField[c] * a.fstride + kc + kk);
      Bs[kk][c] = v.x;
      Bs[kk + 1][c] = v.y;
      Bs[kk + 2][c] = v.z;
      Bs[kk + 3][c] = v.w;
    }
    __syncthreads();
    for (int q = tid; q < KC * TROWS; q += blockDim.x) {
      const int k = q >> 7, r = q & 127;
      As[k][r] = rawI[r >> 3][k] * rawJ[r & 7][k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      const float4 a0 = *reinterpret_cast<const float4 *>(&As[k][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4 *>(&As[k][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[k][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[k][64 + tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
    if (++nchunk == KOUTER) {
      nchunk = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          accO[i][j] += acc[i][j];
          acc[i][j] = 0.f;
        }
    }
  }

  if (DELTA) {
    for (int q = tid; q < min(redTotal, RED_CAP); q += blockDim.x) red[q] = 0.f;
    __syncthreads();
  }
  const bool use_red = DELTA && redTotal <= RED_CAP;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
    const int nu1 = nu1_0 + (r >> 3), nu2 = nu2_0 + (r & 7);
    if (nu1 >= a.nu1_hi || nu2 >= a.nu2_hi) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = (j < 4) ? tx * 4 + j : 64 + tx * 4 + (j - 4);
      if (colField[c] < 0) continue;
      const float s = accO[i][j] + acc[i][j];
      const int trip = colTrip[c], nu3 = colNu3[c];
      if (FULL) {
        const long long o = (long long)b * a.full_bstride +
                            (((long long)trip * a.nc + nu1) * a.nc + nu2) * a.nc + nu3;
        atomicAdd(a.out_full + o, (double)s * a.tnorm[trip]);
      }
      if (DELTA) {
        if (use_red) {
          const int sg = colSeg[c];
          const int d = nu1 - nu2 - (nu1_0 - nu2_0 - (TR2 - 1));
          const int e = nu2 - nu3 - segD2min[sg];
          atomicAdd(&red[segBase[sg] + d * segE[sg] + e], s);
        } else {
          const int n2 = 2 * a.nc - 1;
          const long long o = (long long)b * a.dsum_bstride +
                              ((long long)trip * n2 + (nu1 - nu3 + a.nc - 1)) * n2 +
                              (nu2 - nu3 + a.nc - 1);
          atomicAdd(a.dsum + o, (double)s);
        }
      }
    }
  }
  if (use_red) {
    __syncthreads();
    const int n2 = 2 * a.nc - 1;
    const int dmin = nu1_0 - nu2_0 - (TR2 - 1);
    for (int q = tid; q < redTotal; q += blockDim.x) {
      const float v = red[q];
      if (v == 0.f) continue;
      int sg = 0;
      while (sg + 1 < nsegS && segBase[sg + 1] <= q) ++sg;
      const int off = q - segBase[sg];
      const int d = off / segE[sg] + dmin;
      const int d2 = off % segE[sg] + segD2min[sg];
      const int d1 = d + d2;
      const long long o = (long long)b * a.dsum_bstride +
                          ((long long)segTrip[sg] * n2 + (d1 + a.nc - 1)) * n2 + (d2 + a.nc - 1);
      atomicAdd(a.dsum + o, (double)v);
    }
  }
}

}  // namespace

cudaError_t launch_contract_simt(const ContractArgs &a, int ntiles_row, int npt, int batch,
                                 cudaStream_t s) {
  if (ntiles_row == 0 || npt == 0) return cudaSuccess;
  dim3 grid(ntiles_row, npt, a.nkseg * batch);
  const bool full = a.out_full != nullptr, delta = a.dsum != nullptr;
  if (full && delta)
    k_contract_simt<true, true><<<grid, 256, 0, s>>>(a);
  else if (full)
    k_contract_simt<true, false><<<grid, 256, 0, s>>>(a);
  else if (delta)
    k_contract_simt<false, true><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace bsi
