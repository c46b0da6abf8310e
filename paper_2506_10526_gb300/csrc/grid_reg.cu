// Image-plane field passes of Eq. (iFT) on the register FFT (fft_reg.cuh) for
// the image sides with a register plan (2^a x {8, 12} from 16 to 768): the
// same column pass (shell mask, weights, transform along v) and row pass
// (Hermitian C2R along u, two rows per complex transform, FP32 and split
// outputs) as grid.cu, with one shared-memory exchange per transform.
//
// colpass: CTA = (UB = 8 or 16 consecutive u columns, channel, realisation x
//   ring slot).  Threads take columns fastest, so the visibility, label and weight
//   reads (through L1 / L2: the rings of a channel re-read its 16-column
//   tile), the exchange tile and the G stores (u fastest) are all consecutive
//   across a warp.  Only the exchange tile is in shared memory.
// rowpass: CTA = RPB consecutive row pairs of the flattened
//   [realisation][field][pair] order (pairs of several fields for small
//   sides).  Pass 1 reads G straight from global memory (the Hermitian mirror
//   z(M - u) = conj A(u) + i conj B(u) built on the fly); pass 2 threads take
//   output columns fastest, so the F and hi / lo stores are consecutive.
#include <cuda_bf16.h>

#include "bs_internal.h"
#include "fft_reg.cuh"

namespace bsi {

namespace {

using freg::Split;

constexpr int kRegThreads = 128;
// u columns per column-pass CTA: 8 for the long transforms, so that the
// exchange tile (UB x N) leaves room for more resident CTAs
template <int N>
struct ColCfg {
  static constexpr int UB = N >= 256 ? 8 : 16;
};

// row pairs per row-pass CTA for each side (about one pass-2 transform per thread)
template <int N>
struct RowCfg {
  static constexpr int RPB = N <= 32 ? 64 : N == 48 ? 48 : N <= 128 ? 32 : N == 192 ? 16
                           : N == 768 ? 8 : 8;
};

__device__ __forceinline__ uint16_t bf16_bits_r(float x) {
  __nv_bfloat16 h = __float2bfloat16_rn(x);
  return *reinterpret_cast<uint16_t *>(&h);
}
__device__ __forceinline__ float bf16_val_r(uint16_t b) { return __uint_as_float(((uint32_t)b) << 16); }

template <int N>
__global__ void __launch_bounds__(kRegThreads) k_colpass_reg(
    GridGeom g, const float2 *__restrict__ vis, const float *__restrict__ ngrid,
    const uint8_t *__restrict__ valid, const int8_t *__restrict__ label,
    const int *__restrict__ uext, const float2 *__restrict__ twM, float2 *__restrict__ G) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, UB = ColCfg<N>::UB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nt = g.nt, h = nt / 2;
  const int u0 = blockIdx.x * UB;
  const int nu = blockIdx.y;
  const int b = blockIdx.z / g.nslot, slot = blockIdx.z - b * g.nslot;  // one ring per CTA
  const int m = g.ring_of[slot];
  const int ue = uext[m];
  if (!valid[nu] || u0 >= ue) return;  // flagged channels: rowpass writes zeros
  float2 *tw2 = reinterpret_cast<float2 *>(smem_raw);  // [N1][N2]
  float2 *Y = tw2 + N;                                   // [N1][N2][UB]
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    const int k1 = t / N2, n2 = t - k1 * N2;
    tw2[t] = twM[(n2 * k1) % N];
  }
  __syncthreads();
  const float2 *vb = vis + ((long long)b * g.nc + nu) * (long long)nt * nt;
  const int ncols = min(UB, g.UC - u0);
  const long long gtot = (long long)g.batch * g.nslot * g.nc * N * g.UC;  // G extent
  (void)gtot;  // used by the checked build's bounds checks
  // the weighted visibility of cell (v, u) if it belongs to ring m, else 0
  // (read through L1: the 16-column tile of a channel is re-read per ring)
  auto cell_of = [&](int v, int u, int m) {
    float2 x = make_float2(0.f, 0.f);
    const int cell = (v + h) * nt + (u + h);
    if (!BS_CHK(cell, (long long)nt * nt, 1)) return x;
    if (__ldg(label + cell) != m) return x;
    const float n = ngrid ? __ldg(ngrid + cell) : 1.0f;
    if (n > 0.f) {
      const float w = 1.0f / n;
      const float2 vv = __ldg(vb + cell);
      x = make_float2(w * vv.x, w * vv.y);
    }
    return x;
  };
  {
    // pass 1: (n2, column) items, columns fastest
    for (int it = threadIdx.x; it < N2 * UB; it += blockDim.x) {
      const int n2 = it / UB, c = it - n2 * UB;
      const int u = u0 + c;
      float2 v[N1];
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) {
        const int y = n2 + N2 * n1;
        // the rows v = y and v = y - N that reach index y (only one holds
        // cells of ring m when N exceeds the ring's diameter)
        float2 acc = make_float2(0.f, 0.f);
        if (u < h) {
          if (y < h) acc = cell_of(y, u, m);
          if (y - N >= -h) acc = freg::add(acc, cell_of(y - N, u, m));
        }
        v[n1] = acc;
      }
      freg::dft<N1, 1>(v);
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) {
        const float2 w = tw2[k1 * N2 + n2];
        const float2 a = v[k1];
        Y[(k1 * N2 + n2) * UB + c] = make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
      }
    }
    __syncthreads();
    // pass 2: (k1, column) items, columns fastest; G[y][u] stores along u
    float2 *Gm = G + (((long long)b * g.nslot + slot) * g.nc + nu) * (long long)N * g.UC;
    for (int it = threadIdx.x; it < N1 * UB; it += blockDim.x) {
      const int k1 = it / UB, c = it - k1 * UB;
      float2 v[N2];
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) v[n2] = Y[(k1 * N2 + n2) * UB + c];
      freg::dft<N2, 1>(v);
      if (c < ncols) {
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
          const long long o = (long long)(k1 + N1 * k2) * g.UC + u0 + c;
          if (BS_CHK(o + (Gm - G), gtot, 2)) Gm[o] = v[k2];
        }
      }
    }
    __syncthreads();
  }
}

template <int N>
__global__ void __launch_bounds__(kRegThreads) k_rowpass_reg(
    GridGeom g, long long npairs, const float2 *__restrict__ G, const uint8_t *__restrict__ valid,
    const int *__restrict__ uext, const float2 *__restrict__ twM, float *__restrict__ F,
    uint16_t *__restrict__ Fhi, uint16_t *__restrict__ Flo, unsigned *__restrict__ fmax) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, LDY = Split<N>::LDY;
  constexpr int RPB = RowCfg<N>::RPB, HALF = N / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *tw2 = reinterpret_cast<float2 *>(smem_raw);  // [N1][N2]
  float2 *Y = tw2 + N;                                   // [RPB][N1][LDY]
  __shared__ long long gofs[RPB];                        // G row y of the pair
  __shared__ int ue_s[RPB], key_s[RPB];
  const long long q0 = (long long)blockIdx.x * RPB;
  const int nf = g.nslot * g.nc;
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    const int k1 = t / N2, n2 = t - k1 * N2;
    tw2[t] = twM[(n2 * k1) % N];
  }
  for (int r = threadIdx.x; r < RPB; r += blockDim.x) {
    const long long q = q0 + r;
    int ue = 0, key = -1;
    long long go = 0;
    if (q < npairs) {
      const long long fq = q / HALF;  // b * nf + f
      const int p = (int)(q - fq * HALF);
      const int b = (int)(fq / nf), f = (int)(fq - (long long)b * nf);
      const int slot = f / g.nc, nu = f - slot * g.nc;
      ue = valid[nu] ? min(uext[g.ring_of[slot]], g.UC) : 0;
      go = (((long long)b * g.nslot + slot) * g.nc + nu) * (long long)N * g.UC +
           (long long)(2 * p) * g.UC;
      key = b * g.nslot + slot;
    }
    gofs[r] = go;
    ue_s[r] = ue;
    key_s[r] = key;
  }
  __syncthreads();
  const long long gtot = (long long)g.batch * g.nslot * g.nc * N * g.UC;  // G extent
  (void)gtot;  // used by the checked build's bounds checks
  // pass 1: (pair, n2) items, n2 fastest
  for (int it = threadIdx.x; it < RPB * N2; it += blockDim.x) {
    const int r = it / N2, n2 = it - r * N2;
    const int ue0 = ue_s[r];  // reads G rows 2p, 2p + 1 at columns below ue0
    const int ue = (ue0 == 0 || BS_CHK(gofs[r] + g.UC + ue0 - 1, gtot, 3)) ? ue0 : 0;
    const float2 *ga = G + gofs[r];
    const float2 *gc = ga + g.UC;
    float2 v[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
      const int mi = n2 + N2 * n1;
      float2 z = make_float2(0.f, 0.f);
      if (mi == 0) {
        if (ue > 0) {
          const float2 a = __ldg(ga), c = __ldg(gc);
          z = make_float2(a.x, c.x);
        }
      } else if (mi < ue) {  // A(u) + i B(u)
        const float2 a = __ldg(ga + mi), c = __ldg(gc + mi);
        z = make_float2(a.x - c.y, a.y + c.x);
      } else if (N - mi < ue) {  // conj A(u) + i conj B(u), u = N - mi
        const float2 a = __ldg(ga + (N - mi)), c = __ldg(gc + (N - mi));
        z = make_float2(a.x + c.y, c.x - a.y);
      }
      v[n1] = z;
    }
    freg::dft<N1, 1>(v);
    float2 *Yr = Y + r * (N1 * LDY);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      const float2 w = tw2[k1 * N2 + n2];
      const float2 a = v[k1];
      Yr[k1 * LDY + n2] = make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
    }
  }
  __syncthreads();
  // pass 2: (pair, k1) items, k1 fastest; outputs X[k1 + N1 k2] -> columns
  for (int it = threadIdx.x; it < RPB * N1; it += blockDim.x) {
    const int r = it / N1, k1 = it - r * N1;
    const long long q = q0 + r;
    const bool live = q < npairs;
    float2 v[N2];
    const float2 *Yr = Y + r * (N1 * LDY) + k1 * LDY;
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) v[n2] = Yr[n2];
    freg::dft<N2, 1>(v);
    unsigned amax = 0;
    if (live) {
      // F rows 2p, 2p + 1 of field fq = q / HALF: offset (2 q) N
      const long long o0 = 2 * q * N, o1 = o0 + N;
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        const int x = k1 + N1 * k2;
        const float a = v[k2].x, c = v[k2].y;
        if (!BS_CHK(o1 + x, 2 * npairs * N, 4)) continue;
        F[o0 + x] = a;
        F[o1 + x] = c;
        amax = max(amax, __float_as_uint(fmaxf(fabsf(a), fabsf(c))));
        if (Fhi) {
          const uint16_t ha = bf16_bits_r(a), hc = bf16_bits_r(c);
          Fhi[o0 + x] = ha;
          Fhi[o1 + x] = hc;
          Flo[o0 + x] = bf16_bits_r(a - bf16_val_r(ha));
          Flo[o1 + x] = bf16_bits_r(c - bf16_val_r(hc));
        }
      }
    }
    if (fmax) {
      const int key = live ? key_s[r] : -1;
      const int k0 = __shfl_sync(0xffffffffu, key, 0);
      if (__all_sync(0xffffffffu, key == k0)) {  // one (realisation, slot) in the warp
        amax = __reduce_max_sync(0xffffffffu, amax);
        if ((threadIdx.x & 31) == 0 && k0 >= 0 && amax) atomicMax(fmax + k0, amax);
      } else if (key >= 0 && amax) {
        atomicMax(fmax + key, amax);
      }
    }
  }
}

size_t colpass_reg_smem(int M, int nt) {
  (void)nt;
  return (size_t)(M + M * (M >= 256 ? 8 : 16)) * sizeof(float2);  // ColCfg<M>::UB
}

template <int N>
cudaError_t colpass_n(const GridGeom &g, const float2 *vis, const float *ngrid,
                      const uint8_t *valid, const int8_t *label, const int *uext,
                      const float2 *twM, float2 *G, cudaStream_t s) {
  const size_t smem = colpass_reg_smem(N, g.nt);
  cudaError_t e = smem_optin_once<k_colpass_reg<N>>();
  if (e != cudaSuccess) return e;
  if (g.nslot == 0) return cudaSuccess;
  if ((long long)g.batch * g.nslot > 65535) return cudaErrorInvalidValue;
  constexpr int UB = ColCfg<N>::UB;
  dim3 grid((g.UC + UB - 1) / UB, g.nc, g.batch * g.nslot);
  k_colpass_reg<N><<<grid, kRegThreads, smem, s>>>(g, vis, ngrid, valid, label, uext, twM, G);
  return cudaGetLastError();
}

template <int N>
cudaError_t rowpass_n(const GridGeom &g, const float2 *G, const uint8_t *valid, const int *uext,
                      const float2 *twM, float *F, uint16_t *Fhi, uint16_t *Flo, unsigned *fmax,
                      cudaStream_t s) {
  constexpr int RPB = RowCfg<N>::RPB;
  const size_t smem = (size_t)(N + RPB * Split<N>::N1 * Split<N>::LDY) * sizeof(float2);
  cudaError_t e = smem_optin_once<k_rowpass_reg<N>>();
  if (e != cudaSuccess) return e;
  const long long npairs = (long long)g.batch * g.nslot * g.nc * (N / 2);
  if (npairs == 0) return cudaSuccess;
  const long long nblk = (npairs + RPB - 1) / RPB;
  if (nblk > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_rowpass_reg<N><<<(unsigned)nblk, kRegThreads, smem, s>>>(g, npairs, G, valid, uext, twM, F,
                                                             Fhi, Flo, fmax);
  return cudaGetLastError();
}

}  // namespace

bool has_reg_fft(int M, int nt) {
  // the column pass keeps its exchange tile (16 columns of M) in shared memory
  if (colpass_reg_smem(M, nt) > (size_t)200 * 1024) return false;
  switch (M) {
    case 16: case 24: case 32: case 48: case 64: case 96: case 128: case 192: case 256:
    case 384: case 512: case 768:
      return true;
    default:
      return false;
  }
}

#define BS_REG_SIDES(X) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768)

cudaError_t launch_colpass_reg(const GridGeom &g, const float2 *vis, const float *ngrid,
                               const uint8_t *valid, const int8_t *label, const int *uext,
                               const float2 *twM, float2 *G, cudaStream_t s) {
  switch (g.M) {
#define BS_COL_CASE(n) \
  case n: return colpass_n<n>(g, vis, ngrid, valid, label, uext, twM, G, s);
    BS_REG_SIDES(BS_COL_CASE)
#undef BS_COL_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_rowpass_reg(const GridGeom &g, const float2 *G, const uint8_t *valid,
                               const int *uext, const float2 *twM, float *F, uint16_t *Fhi,
                               uint16_t *Flo, unsigned *fmax, cudaStream_t s) {
  switch (g.M) {
#define BS_ROW_CASE(n) \
  case n: return rowpass_n<n>(g, G, valid, uext, twM, F, Fhi, Flo, fmax, s);
    BS_REG_SIDES(BS_ROW_CASE)
#undef BS_ROW_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bsi
