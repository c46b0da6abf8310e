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

}  // namespace bsi
