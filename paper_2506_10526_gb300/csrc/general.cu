// General (non-Hermitian) visibilities and sampling (Section 3.2, Eqs. iFT and
// iFT_I with weights and visibilities that need not satisfy V(-U) = V(U)*).
//
// The image-plane fields are then complex.  The weighted grid X = W V splits
// exactly into two Hermitian parts,
//   X = X_H + i Y,  X_H(g) = (X(g) + X(-g)*) / 2,  Y(g) = -i (X(g) - X(-g)*) / 2,
// so every field is F = F_H + i F_Y with F_H, F_Y the real fields of X_H and Y,
// and the triple pixel sum S = sum_x F_i F_j F_l is the value at t = i of the
// cubic S(t) = sum_x (F_H + t F_Y)_i (F_H + t F_Y)_j (F_H + t F_Y)_l =
// P0 + P1 t + P2 t^2 + P3 t^3.  The real path evaluates S(t) at t = 0, 1, -1, 2
// (four Hermitian inputs X_H + t Y, exact in FP32 since t is a small power of
// two), and
//   Re S = P0 - P2 = 2 S(0) - (S(1) + S(-1)) / 2
//   Im S = P1 - P3 = (9 S(1) - S(-1) - 2 S(2) - 6 S(0)) / 6.
// Every later step (normalisation, collapse, fold, Eq. dft) is linear in S,
// so the same combination applies to their outputs.  The work is that of a
// complex contraction (four real products per term); the denominator is the
// exact count of closed triangles of occupied cells, with no symmetry needed.
//
// Per-channel sampling N_g(nu) (Eq. vg with flags per baseline): the
// denominator of Eq. (estimator_t), sum_theta I1 I2 I3 with I the transform of
// W N = [N_g(nu) > 0] (Eq. iFT_I), then depends on the channel triple.  Each
// realisation becomes two: component 0 the weighted visibilities W V, with
// W = 1/N_g(nu), component 1 the occupancy masks.  The same pipeline gives the
// pixel sums of both, S_D and S_I = M^2 x (closed triangles of cells occupied
// at their channels), and the estimate is S_D / (A S_I) per channel triple.
// The collapse to (dnu1, dnu2) takes the ratio of the summed numerators and
// summed denominators over the channel triples at +-d (with one sampling grid
// this is the mean of the estimates).
#include "bs_internal.h"

namespace bsi {

namespace {

__global__ void k_general_prep(int nt, int nc, int ub, const float2 *__restrict__ vis,
                               const float *__restrict__ ngrid, const int8_t *__restrict__ label,
                               float2 *__restrict__ out) {
  const long long cells = (long long)nt * nt;
  const long long plane = (long long)nc * cells;
  const long long total = (long long)ub * plane;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(q / plane);
    const long long r = q - (long long)b * plane;
    const int cell = (int)(r % cells);
    const int iv = cell / nt, iu = cell - iv * nt;
    float2 xh = make_float2(0.f, 0.f), y = make_float2(0.f, 0.f);
    if (label[cell] >= 0) {  // binned cells have a mirror on the grid
      const int mirror = (nt - iv) * nt + (nt - iu);
      const float n0 = ngrid ? ngrid[cell] : 1.f, n1 = ngrid ? ngrid[mirror] : 1.f;
      const float w0 = n0 > 0.f ? 1.f / n0 : 0.f, w1 = n1 > 0.f ? 1.f / n1 : 0.f;
      const float2 v0 = vis[q], v1 = vis[q - cell + mirror];
      const float2 x = make_float2(w0 * v0.x, w0 * v0.y), xm = make_float2(w1 * v1.x, w1 * v1.y);
      xh = make_float2(0.5f * (x.x + xm.x), 0.5f * (x.y - xm.y));
      // d = X(g) - X(-g)*, Y = -i d / 2
      const float2 d = make_float2(x.x - xm.x, x.y + xm.y);
      y = make_float2(0.5f * d.y, -0.5f * d.x);
    }
    float2 *o = out + 4ll * b * plane + r;
    o[0] = xh;
    o[plane] = make_float2(xh.x + y.x, xh.y + y.y);
    o[2 * plane] = make_float2(xh.x - y.x, xh.y - y.y);
    o[3 * plane] = make_float2(xh.x + 2.f * y.x, xh.y + 2.f * y.y);
  }
}

__device__ __forceinline__ double2 combine(double s0, double s1, double sm, double s2) {
  return make_double2(2.0 * s0 - 0.5 * (s1 + sm), (9.0 * s1 - sm - 2.0 * s2 - 6.0 * s0) / 6.0);
}

__global__ void k_combine4(const double *__restrict__ in, long long n, int ub,
                           double2 *__restrict__ out) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < (long long)ub * n;
       q += (long long)gridDim.x * blockDim.x) {
    const long long b = q / n, k = q - b * n;
    const double *x = in + 4 * b * n + k;
    out[q] = combine(x[0], x[n], x[2 * n], x[3 * n]);
  }
}

__global__ void k_combine4_full(const double *__restrict__ in, int ub, int ntrip, int nc, int b0,
                                int n1b, int b2, int n2b, int b4, int n3b,
                                double2 *__restrict__ out) {
  const long long cube = (long long)nc * nc * nc, per = (long long)ntrip * cube;
  const long long blk = (long long)n1b * n2b * n3b;
  const long long total = (long long)ub * ntrip * blk;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    long long r = q;
    const int k3 = (int)(r % n3b); r /= n3b;
    const int k2 = (int)(r % n2b); r /= n2b;
    const int k1 = (int)(r % n1b); r /= n1b;
    const int t = (int)(r % ntrip);
    const int b = (int)(r / ntrip);
    const long long e = (long long)t * cube + ((long long)(b0 + k1) * nc + (b2 + k2)) * nc + (b4 + k3);
    const double *x = in + 4ll * b * per + e;
    out[(long long)b * per + e] = combine(x[0], x[per], x[2 * per], x[3 * per]);
  }
}

__global__ void k_chans_prep(int nt, int nc, int ub, const float2 *__restrict__ vis,
                             const float *__restrict__ ngrid, const int8_t *__restrict__ label,
                             float2 *__restrict__ out) {
  const long long cells = (long long)nt * nt;
  const long long plane = (long long)nc * cells;
  const long long total = (long long)ub * plane;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(q / plane);
    const long long r = q - (long long)b * plane;  // nu * cells + cell
    const int cell = (int)(r % cells);
    float2 x = make_float2(0.f, 0.f), o = make_float2(0.f, 0.f);
    const float n = ngrid[r];
    if (label[cell] >= 0 && n > 0.f) {
      const float w = 1.f / n;
      const float2 v = vis[q];
      x = make_float2(w * v.x, w * v.y);
      o = make_float2(1.f, 0.f);
    }
    float2 *d = out + 2ll * b * plane + r;
    d[0] = x;
    d[plane] = o;
  }
}

__global__ void k_ratio2(const double *__restrict__ in, long long n, int ub, double inv_a,
                         double *__restrict__ out) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < (long long)ub * n;
       q += (long long)gridDim.x * blockDim.x) {
    const long long b = q / n, k = q - b * n;
    const double *x = in + 2 * b * n + k;
    out[q] = x[0] / x[n] * inv_a;
  }
}

__global__ void k_ratio2_full(const double *__restrict__ in, int ub, int ntrip, int nc, int b0,
                              int n1b, int b2, int n2b, int b4, int n3b, double inv_a,
                              double *__restrict__ out) {
  const long long cube = (long long)nc * nc * nc, per = (long long)ntrip * cube;
  const long long total = (long long)ub * ntrip * n1b * n2b * n3b;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    long long r = q;
    const int k3 = (int)(r % n3b); r /= n3b;
    const int k2 = (int)(r % n2b); r /= n2b;
    const int k1 = (int)(r % n1b); r /= n1b;
    const int t = (int)(r % ntrip);
    const int b = (int)(r / ntrip);
    const long long e = (long long)t * cube + ((long long)(b0 + k1) * nc + (b2 + k2)) * nc + (b4 + k3);
    const double *x = in + 2ll * b * per + e;
    out[(long long)b * per + e] = x[0] / x[per] * inv_a;
  }
}

// The ratio planes R [ub][ntrip][n2][n2] written as collapse sums that the
// delay transform's own normalisation, fold(sums) tnorm / fold(N), turns back
// into R: sums(d) = R(d) fold(N)(d) / (2 tnorm) off the origin (both d and -d
// hold it), R(0) N(0) / tnorm at the origin; 0 where R is undefined.
__global__ void k_ratio_to_sums(const double *__restrict__ R, const long long *__restrict__ nnu,
                                const double *__restrict__ tnorm, int ub, int ntrip, int nc,
                                double *__restrict__ sums) {
  const long long n2 = 2LL * nc - 1, plane = n2 * n2;
  const long long total = (long long)ub * ntrip * plane;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const long long d = q % plane;
    const int t = (int)((q / plane) % ntrip);
    const long long j = plane - 1 - d;
    const long long cnt = nnu[d] + (j != d ? nnu[j] : 0);
    const double r = R[q], tn = tnorm[t];
    double v = 0.0;
    if (cnt > 0 && tn > 0.0 && r == r) v = r * (double)cnt / (tn * (j != d ? 2.0 : 1.0));
    sums[q] = v;
  }
}

int grid_of(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 32); }

}  // namespace

cudaError_t launch_general_prep(int nt, int nc, int ub, const float2 *vis, const float *ngrid,
                                const int8_t *label, float2 *out, cudaStream_t s) {
  const long long n = (long long)ub * nc * nt * nt;
  if (n == 0) return cudaSuccess;
  k_general_prep<<<grid_of(n), 256, 0, s>>>(nt, nc, ub, vis, ngrid, label, out);
  return cudaGetLastError();
}

cudaError_t launch_combine4(const double *in, long long n, int ub, double *out, cudaStream_t s) {
  if (n * ub == 0) return cudaSuccess;
  k_combine4<<<grid_of(n * ub), 256, 0, s>>>(in, n, ub, reinterpret_cast<double2 *>(out));
  return cudaGetLastError();
}

cudaError_t launch_combine4_full(const double *in, int ub, int ntrip, int nc, const int *blk,
                                 double *out, cudaStream_t s) {
  const int n1 = blk[1] - blk[0], n2 = blk[3] - blk[2], n3 = blk[5] - blk[4];
  const long long n = (long long)ub * ntrip * n1 * n2 * n3;
  if (n == 0) return cudaSuccess;
  k_combine4_full<<<grid_of(n), 256, 0, s>>>(in, ub, ntrip, nc, blk[0], n1, blk[2], n2, blk[4], n3,
                                             reinterpret_cast<double2 *>(out));
  return cudaGetLastError();
}

cudaError_t launch_chans_prep(int nt, int nc, int ub, const float2 *vis, const float *ngrid,
                              const int8_t *label, float2 *out, cudaStream_t s) {
  const long long n = (long long)ub * nc * nt * nt;
  if (n == 0) return cudaSuccess;
  k_chans_prep<<<grid_of(n), 256, 0, s>>>(nt, nc, ub, vis, ngrid, label, out);
  return cudaGetLastError();
}

cudaError_t launch_ratio2(const double *in, long long n, int ub, double inv_a, double *out,
                          cudaStream_t s) {
  if (n * ub == 0) return cudaSuccess;
  k_ratio2<<<grid_of(n * ub), 256, 0, s>>>(in, n, ub, inv_a, out);
  return cudaGetLastError();
}

cudaError_t launch_ratio2_full(const double *in, int ub, int ntrip, int nc, const int *blk,
                               double inv_a, double *out, cudaStream_t s) {
  const int n1 = blk[1] - blk[0], n2 = blk[3] - blk[2], n3 = blk[5] - blk[4];
  const long long n = (long long)ub * ntrip * n1 * n2 * n3;
  if (n == 0) return cudaSuccess;
  k_ratio2_full<<<grid_of(n), 256, 0, s>>>(in, ub, ntrip, nc, blk[0], n1, blk[2], n2, blk[4], n3,
                                           inv_a, out);
  return cudaGetLastError();
}

cudaError_t launch_ratio_to_sums(const double *R, const long long *nnu, const double *tnorm,
                                 int ub, int ntrip, int nc, double *sums, cudaStream_t s) {
  const long long n = (long long)ub * ntrip * (2LL * nc - 1) * (2LL * nc - 1);
  if (n == 0) return cudaSuccess;
  k_ratio_to_sums<<<grid_of(n), 256, 0, s>>>(R, nnu, tnorm, ub, ntrip, nc, sums);
  return cudaGetLastError();
}

}  // namespace bsi
