// Collapse, fold and delay transform (Section 3.2, Eq. dft), plus the FULL
// layout fill / finalise of Eq. (estimator_t).
//
// Accumulators: dsum[b][trip][d1+nc-1][d2+nc-1] holds the pixel sums S of all
// accumulated channel triples with (nu1-nu3, nu2-nu3) = (d1, d2); nnu[] the
// number of valid such triples (unfolded).  Every valid triple of a ring
// triple has the same denominator A M^2 T (channel-independent occupancy), so
//   Bbar(d) = (S(d) + S(-d)) / (A M^2 T (N(d) + N(-d)))       (d != 0)
//   Bbar(0) = S(0) / (A M^2 T N(0))
// is the mean of B_A over the valid triples at +-d: the fold of Fig. Nv.
//
// With a ring-triple list (the closable triples), grid row y handles ring
// triple list[y] and writes output plane y: the compact layouts.
//
// Delay transform: the separations -nc/2 <= n, m < nc/2 (one period of the
// nc-periodic kernel) are placed at n mod nc, then a forward 2D DFT of length
// nc (Stockham, FP32) gives
//   B(a, b) = (r^2 r' dnu_c)^2 sum_{n,m} exp(-2 pi i (n a + m b)/nc) Bbar(n, m),
// whose real part is stored (Bbar is point symmetric: the imaginary part is
// the unpaired edge n, m = -nc/2 alone).  Unsampled separations contribute
// zero.  Non-smooth nc use a direct DFT.
#include "bs_internal.h"
#include "fft_smem.cuh"

namespace bsi {

namespace {

// rc[t] = 1 / (N(t) + N(plane - 1 - t)) (N(t) once at the centre), 0 where
// nothing was sampled: the folded sampling of element t of the first half of
// the (2 nc - 1)^2 plane, the same for every ring triple.
__global__ void k_fold_recip(const long long *__restrict__ nnu, long long plane,
                             double *__restrict__ rc) {
  const long long half = (plane + 1) / 2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < half;
       t += (long long)gridDim.x * blockDim.x) {
    const long long j = plane - 1 - t;
    long long c = nnu[t];
    if (j != t) c += nnu[j];
    rc[t] = c > 0 ? 1.0 / (double)c : 0.0;
  }
}

__global__ void k_delta_norm(const double *__restrict__ dsum, const double *__restrict__ rc,
                             const double *__restrict__ tnorm, double *__restrict__ out, int ntrip,
                             int nc, const int *__restrict__ list) {
  const int n2 = 2 * nc - 1;
  const long long plane = (long long)n2 * n2;
  const int trip = list ? list[blockIdx.y] : blockIdx.y, b = blockIdx.z;
  const int nout = list ? gridDim.y : ntrip;
  const double *ds = dsum + ((long long)b * ntrip + trip) * plane;
  double *o = out + ((long long)b * nout + blockIdx.y) * plane;
  const double tn = tnorm[trip];
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  if (tn == 0.0) {  // no closed triangle: undefined everywhere, nothing to read
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < plane;
         t += (long long)gridDim.x * blockDim.x)
      o[t] = nan;
    return;
  }
  // element t pairs with its point reflection plane-1-t; each pair is read once
  const long long half = (plane + 1) / 2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < half;
       t += (long long)gridDim.x * blockDim.x) {
    const long long j = plane - 1 - t;
    if (!BS_CHK(j, plane, 21)) continue;
    const double r = rc[t];
    double v = nan;
    if (r != 0.0) {  // unsampled separations hold no sums: their reads are skipped
      double s = ds[t];
      if (j != t) s += ds[j];
      v = s * (tn * r);
    }
    o[t] = v;
    o[j] = v;
  }
}

// Zero rows [r0, r0 + nr) x columns [c0, c0 + ncol) of the (2nc-1)^2 plane of each
// listed ring triple: the separations accumulated since the last reset.
__global__ void k_zero_planes(double *__restrict__ dsum, const int *__restrict__ trips, int ntr,
                              int ntrip, int n2, int r0, int nr, int c0, int ncol) {
  const int k = blockIdx.y, b = blockIdx.z;
  double *o = dsum + ((long long)b * ntrip + trips[k]) * (long long)n2 * n2;
  const long long n = (long long)nr * ncol;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t / ncol), c = (int)(t - (long long)r * ncol);
    o[(long long)(r0 + r) * n2 + c0 + c] = 0.0;
  }
}

// Channel-symmetric accumulation: the orderings of a repeated ring's channels
// that were not contracted, copied from the ones that were.  list[k] = 2 t + kind:
//   kind 0, ring triple (i, i, l):       S(d1, d2) = S(d2, d1)       where d1 > d2
//   kind 1, ring triple (i, j, j), i < j: S(d1, d2) = S(d1 - d2, -d2) where d2 > 0
// (d1 = nu1 - nu3, d2 = nu2 - nu3; exchanging nu1, nu2 or nu2, nu3).  Sources are
// never targets, so the copy is race-free; a source off the plane is 0.
__global__ void k_symmetrize(double *__restrict__ dsum, const int *__restrict__ list, int ntrip,
                             int nc, int r0, int nr, int c0, int ncol) {
  const int code = list[blockIdx.y], b = blockIdx.z;
  const int n2 = 2 * nc - 1;
  double *o = dsum + ((long long)b * ntrip + (code >> 1)) * (long long)n2 * n2;
  const long long n = (long long)nr * ncol;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int r = r0 + (int)(t / ncol), c = c0 + (int)(t % ncol);
    const int d1 = r - (nc - 1), d2 = c - (nc - 1);
    if ((code & 1) == 0) {
      if (d1 > d2) o[(long long)r * n2 + c] = o[(long long)c * n2 + r];
    } else if (d2 > 0) {
      const int s1 = d1 - d2 + nc - 1;
      o[(long long)r * n2 + c] = s1 >= 0 ? o[(long long)s1 * n2 + (nc - 1 - d2)] : 0.0;
    }
  }
}

__device__ void dft_direct(const float2 *x, float2 *y, int N, const float2 *tw, float sign) {
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    float2 acc = make_float2(0.f, 0.f);
    int idx = 0;
    for (int j = 0; j < N; ++j) {
      float2 w = tw[idx];
      w.y *= sign;
      acc = cadd(acc, cmul(x[j], w));
      idx += k;
      if (idx >= N) idx -= N;
    }
    y[k] = acc;
  }
  __syncthreads();
}

// Reciprocal folded sampling over one period of the Eq. (dft) square, in the
// periodic placement of the row pass: rinv[n][m] = 1 / (N(d) + N(-d)) (N(0)
// once) for the separation d = (n, m) taken in [-nc/2, nc/2), 0 where nothing
// was sampled.  The same for every ring triple, so the row pass multiplies.
// rinvf (optional): the same table in FP32, written instead of rinv; rowflag
// (optional, zeroed by the caller): rows n with a sampled separation.
__global__ void k_fold_rinv(const long long *__restrict__ nnu, int nc, double *__restrict__ rinv,
                            float *__restrict__ rinvf, uint8_t *__restrict__ rowflag) {
  const int n2 = 2 * nc - 1;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nc * nc; e += gridDim.x * blockDim.x) {
    const int nidx = e / nc, m = e - nidx * nc;
    const int np = (2 * nidx < nc) ? nidx : nidx - nc, mp = (2 * m < nc) ? m : m - nc;
    const int i1 = np + nc - 1, i2 = mp + nc - 1, j1 = n2 - 1 - i1, j2 = n2 - 1 - i2;
    long long cnt = nnu[i1 * n2 + i2];
    if (j1 != i1 || j2 != i2) cnt += nnu[j1 * n2 + j2];
    if (rinvf) {
      rinvf[e] = cnt > 0 ? 1.0f / (float)cnt : 0.0f;
    } else {
      rinv[e] = cnt > 0 ? 1.0 / (double)cnt : 0.0;
    }
    if (rowflag && cnt > 0) rowflag[nidx] = 1;  // every writer stores the same value
  }
}

// Rows (columns) of the 2D delay transform per CTA, `rows`: the transposed
// stores of the row pass and the scattered stores of the column pass go out as
// runs of that many consecutive elements.  8, or fewer where 8 padded rows
// (and their ping-pong copies) would not fit one CTA's shared memory.
constexpr int kBsRows = 8;

// First pass: for `rows` consecutive n, the folded plane Bbar(n, m) over one
// period of m, transformed along m; written transposed, tmp[k][n].
__global__ void k_bs3d_rows(const double *__restrict__ dsum, const double *__restrict__ rinv,
                            const double *__restrict__ tnorm, float2 *__restrict__ tmp, int ntrip,
                            int nc, const float2 *__restrict__ twN, Radices radN,
                            const int *__restrict__ list, int rows) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int LD = nc + 1;  // padded rows: the transposed reads spread over the banks
  float2 *tw = reinterpret_cast<float2 *>(smem_raw);
  float2 *bufA = tw + nc;
  float2 *bufB = bufA + rows * LD;
  const int n0 = blockIdx.x * rows, trip = list ? list[blockIdx.y] : blockIdx.y, b = blockIdx.z;
  const int nr = min(rows, nc - n0);
  const int n2 = 2 * nc - 1;
  const double *ds = dsum + ((long long)b * ntrip + trip) * (long long)n2 * n2;
  const double tn = tnorm[trip];
  if (tn == 0.0) return;  // no closed triangle: the column pass writes zeros
  for (int t = threadIdx.x; t < nc; t += blockDim.x) tw[t] = twN[t];
  int nonzero = 0;
  for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
    const int r = e / nc, m = e - r * nc;
    const int nidx = n0 + r;
    // one period of the nc-periodic kernel: separations -nc/2 <= n, m < nc/2,
    // each (nidx, m) of the periodic placement being exactly one of them
    const int np = (2 * nidx < nc) ? nidx : nidx - nc, mp = (2 * m < nc) ? m : m - nc;
    const int i1 = np + nc - 1, i2 = mp + nc - 1, j1 = n2 - 1 - i1, j2 = n2 - 1 - i2;
    const double ri = rinv[(long long)nidx * nc + m];
    double acc = 0.0;  // unsampled separations contribute nothing and are not read
    if (ri != 0.0) {
      double sv = ds[(long long)i1 * n2 + i2];
      if (j1 != i1 || j2 != i2) sv += ds[(long long)j1 * n2 + j2];
      acc = sv * (tn * ri);
    }
    bufA[r * LD + m] = make_float2((float)acc, 0.f);
    nonzero |= acc != 0.0;
  }
  float2 *tb = tmp + ((long long)b * ntrip + trip) * (long long)nc * nc;
  if (!__syncthreads_or(nonzero)) {  // rows with nothing sampled: their transform is zero
    for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
      const int k = e / nr, r = e - k * nr;
      tb[(long long)k * nc + n0 + r] = make_float2(0.f, 0.f);
    }
    return;
  }
  float2 *res;
  if (radN.n > 0) {
    res = stockham(bufA, bufB, nr, nc, LD, radN, tw, -1.0f);
  } else {
    for (int r = 0; r < nr; ++r) dft_direct(bufA + r * LD, bufB + r * LD, nc, tw, -1.0f);
    res = bufB;
  }
  for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
    const int k = e / nr, r = e - k * nr;
    tb[(long long)k * nc + n0 + r] = res[r * LD + k];
  }
}

// Second pass: for `rows` consecutive first-pass frequencies, transform along
// n; out[a + nc/2][b + nc/2] = scale * Re.
__global__ void k_bs3d_cols(const float2 *__restrict__ tmp, double *__restrict__ out, int ntrip,
                            int nc, const float2 *__restrict__ twN, Radices radN, double scale,
                            const double *__restrict__ tnorm, const int *__restrict__ list,
                            int rows) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int LD = nc + 1;
  float2 *tw = reinterpret_cast<float2 *>(smem_raw);
  float2 *bufA = tw + nc;
  float2 *bufB = bufA + rows * LD;
  const int bb0 = blockIdx.x * rows, trip = list ? list[blockIdx.y] : blockIdx.y, b = blockIdx.z;
  const int nr = min(rows, nc - bb0);
  const int h = nc / 2;
  const int nout = list ? gridDim.y : ntrip;
  double *ob = out + ((long long)b * nout + blockIdx.y) * (long long)nc * nc;
  auto centred = [&](int k) { return (k < nc - h) ? k + h : k - nc + h; };
  if (tnorm[trip] == 0.0) {
    for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
      const int k = e / nr, r = e - k * nr;
      ob[(long long)k * nc + centred(bb0 + r)] = 0.0;
    }
    return;
  }
  const float2 *tb = tmp + ((long long)b * ntrip + trip) * (long long)nc * nc + (long long)bb0 * nc;
  for (int t = threadIdx.x; t < nc; t += blockDim.x) tw[t] = twN[t];
  for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
    const int r = e / nc, t = e - r * nc;
    bufA[r * LD + t] = tb[(long long)r * nc + t];
  }
  __syncthreads();
  float2 *res;
  if (radN.n > 0) {
    res = stockham(bufA, bufB, nr, nc, LD, radN, tw, -1.0f);
  } else {
    for (int r = 0; r < nr; ++r) dft_direct(bufA + r * LD, bufB + r * LD, nc, tw, -1.0f);
    res = bufB;
  }
  for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
    const int k = e / nr, r = e - k * nr;
    ob[(long long)centred(k) * nc + centred(bb0 + r)] = scale * (double)res[r * LD + k].x;
  }
}

__global__ void k_full_fill(double *__restrict__ out, long long bstride, int ntrip, int nc, int b0,
                            int b1, int b2, int b3, int b4, int b5, double value) {
  const int trip = blockIdx.y, b = blockIdx.z;
  const int w1 = b1 - b0, w2 = b3 - b2, w3 = b5 - b4;
  const long long n = (long long)w1 * w2 * w3;
  double *o = out + (long long)b * bstride + (long long)trip * nc * nc * nc;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int i3 = (int)(t % w3);
    const long long r = t / w3;
    const int i2 = (int)(r % w2), i1 = (int)(r / w2);
    o[((long long)(b0 + i1) * nc + (b2 + i2)) * nc + (b4 + i3)] = value;
  }
}

__global__ void k_full_finalize(double *__restrict__ out, long long bstride, int ntrip, int nc,
                                int b0, int b1, int b2, int b3, int b4, int b5,
                                const uint8_t *__restrict__ valid,
                                const double *__restrict__ tnorm) {
  const int trip = blockIdx.y, b = blockIdx.z;
  const int w1 = b1 - b0, w2 = b3 - b2, w3 = b5 - b4;
  const long long n = (long long)w1 * w2 * w3;
  double *o = out + (long long)b * bstride + (long long)trip * nc * nc * nc;
  const bool tok = tnorm[trip] != 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int i3 = (int)(t % w3);
    const long long r = t / w3;
    const int i2 = (int)(r % w2), i1 = (int)(r / w2);
    const int n1 = b0 + i1, nn2 = b2 + i2, n3 = b4 + i3;
    if (!tok || !valid[n1] || !valid[nn2] || !valid[n3])
      o[((long long)n1 * nc + nn2) * nc + n3] = __longlong_as_double(0x7ff8000000000000LL);
  }
}

}  // namespace

cudaError_t launch_delta_norm(const double *dsum, const long long *nnu, const double *tnorm,
                              double *out, int batch, int ntrip, int nc, const int *list,
                              int nlist, double *scratch, cudaStream_t s) {
  const long long plane = (long long)(2 * nc - 1) * (2 * nc - 1);
  const int ny = list ? nlist : ntrip;
  if (ny == 0) return cudaSuccess;
  k_fold_recip<<<(unsigned)std::min<long long>((plane / 2 + 256) / 256, 1024), 256, 0, s>>>(
      nnu, plane, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)std::min<long long>((plane + 255) / 256, 1024), ny, batch);
  k_delta_norm<<<grid, 256, 0, s>>>(dsum, scratch, tnorm, out, ntrip, nc, list);
  return cudaGetLastError();
}

cudaError_t launch_zero_planes(double *dsum, const int *trips, int ntr, int batch, int ntrip,
                               int n2, const int *box, cudaStream_t s) {
  const int nr = box[1] - box[0] + 1, ncol = box[3] - box[2] + 1;
  if (ntr == 0 || nr <= 0 || ncol <= 0) return cudaSuccess;
  const long long n = (long long)nr * ncol;
  dim3 grid((unsigned)std::min<long long>((n + 255) / 256, 256), ntr, batch);
  k_zero_planes<<<grid, 256, 0, s>>>(dsum, trips, ntr, ntrip, n2, box[0], nr, box[2], ncol);
  return cudaGetLastError();
}

cudaError_t launch_symmetrize(double *dsum, const int *list, int nlist, int batch, int ntrip,
                              int nc, const int *box, cudaStream_t s) {
  const int nr = box[1] - box[0] + 1, ncol = box[3] - box[2] + 1;
  if (nlist == 0 || nr <= 0 || ncol <= 0) return cudaSuccess;
  const long long n = (long long)nr * ncol;
  dim3 grid((unsigned)std::min<long long>((n + 255) / 256, 256), nlist, batch);
  k_symmetrize<<<grid, 256, 0, s>>>(dsum, list, ntrip, nc, box[0], nr, box[2], ncol);
  return cudaGetLastError();
}

namespace {
// y[k] += x[k] (merging collapse sums of disjoint channel blocks)
__global__ void k_add_f64(double *__restrict__ y, const double *__restrict__ x, long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    y[k] += x[k];
}
}  // namespace

cudaError_t launch_add_f64(double *y, const double *x, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int grid = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
  k_add_f64<<<grid, 256, 0, s>>>(y, x, n);
  return cudaGetLastError();
}

cudaError_t launch_bs3d(const double *dsum, const long long *nnu, const double *tnorm, float2 *tmp,
                        double *out, int batch, int ntrip, int nc, const float2 *twN,
                        const Radices &radN, double scale, const int *list, int nlist,
                        cudaStream_t s) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  int rows = kBsRows;
  auto smem_of = [&](int r) { return (size_t)(nc + 2 * r * (nc + 1)) * sizeof(float2); };
  while (rows > 1 && smem_of(rows) > (size_t)optin) rows /= 2;
  const size_t smem = smem_of(rows);
  if (smem > (size_t)optin) return cudaErrorInvalidValue;  // nc beyond one row per CTA
  cudaError_t e = smem_optin_once<k_bs3d_rows>();
  if (e != cudaSuccess) return e;
  e = smem_optin_once<k_bs3d_cols>();
  if (e != cudaSuccess) return e;
  const int threads = nc >= 64 ? 256 : 64;
  // the reciprocal sampling table and the row flags sit after the batch's
  // complex scratch
  double *rinv = reinterpret_cast<double *>(tmp + (size_t)batch * ntrip * nc * nc);
  float *rinvf = reinterpret_cast<float *>(rinv);  // the register path's FP32 table
  uint8_t *rowflag = reinterpret_cast<uint8_t *>(rinv + (size_t)nc * nc);
  const bool reg = has_reg_dft(nc);
  if (reg) {
    e = cudaMemsetAsync(rowflag, 0, (size_t)nc, s);
    if (e != cudaSuccess) return e;
  }
  k_fold_rinv<<<(nc * nc + 255) / 256, 256, 0, s>>>(nnu, nc, rinv, reg ? rinvf : nullptr,
                                                    reg ? rowflag : nullptr);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int ny = list ? nlist : ntrip;
  if (ny == 0) return cudaSuccess;
  if (reg)
    return launch_bs3d_reg(dsum, rinvf, rowflag, tnorm, tmp, out, batch, ntrip, nc, twN, scale,
                           list, ny, s);
  dim3 grid((nc + rows - 1) / rows, ny, batch);
  k_bs3d_rows<<<grid, threads, smem, s>>>(dsum, rinv, tnorm, tmp, ntrip, nc, twN, radN, list, rows);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_bs3d_cols<<<grid, threads, smem, s>>>(tmp, out, ntrip, nc, twN, radN, scale, tnorm, list, rows);
  return cudaGetLastError();
}

cudaError_t launch_full_fill(double *out, long long bstride, int batch, int ntrip, int nc,
                             const int *blk, double value, cudaStream_t s) {
  const long long n = (long long)(blk[1] - blk[0]) * (blk[3] - blk[2]) * (blk[5] - blk[4]);
  if (n == 0) return cudaSuccess;
  dim3 grid((unsigned)std::min<long long>((n + 255) / 256, 1024), ntrip, batch);
  k_full_fill<<<grid, 256, 0, s>>>(out, bstride, ntrip, nc, blk[0], blk[1], blk[2], blk[3], blk[4],
                                   blk[5], value);
  return cudaGetLastError();
}

cudaError_t launch_full_finalize(double *out, long long bstride, int batch, int ntrip, int nc,
                                 const int *blk, const uint8_t *valid, const double *tnorm,
                                 cudaStream_t s) {
  const long long n = (long long)(blk[1] - blk[0]) * (blk[3] - blk[2]) * (blk[5] - blk[4]);
  if (n == 0) return cudaSuccess;
  dim3 grid((unsigned)std::min<long long>((n + 255) / 256, 1024), ntrip, batch);
  k_full_finalize<<<grid, 256, 0, s>>>(out, bstride, ntrip, nc, blk[0], blk[1], blk[2], blk[3],
                                       blk[4], blk[5], valid, tnorm);
  return cudaGetLastError();
}

}  // namespace bsi
