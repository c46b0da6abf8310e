// Gridding of raw visibilities onto the plan's uv grid (Section 3.2,
// Eq. vg) with channel pre-averaging (Section 4):
//
//   V_g(nu) = sum_i w(U_g - U_i) V(U_i, nu) F(U_i, nu),
//   N_g(nu) = sum_i w(U_g - U_i) F(U_i, nu),
//
// w = 1 at the grid point nearest to U_i (floor(u + 1/2), floor(v + 1/2) in
// FP64, coordinates in grid units), F = 0 for flagged data.  The sky is real,
// so each visibility also adds V* at the mirrored cell -g, which keeps the
// grid Hermitian.  Cells with |u| or |v| >= N_t/2 are dropped.  Input channel
// c feeds output channel c / avg.
//
// One thread per (input channel, baseline), baselines fastest: the threads
// in flight share one or two output channel planes (N_t^2 x 12 bytes), which
// stay in L2 while their atomics land (six FP32 atomics per visibility).
// With channels fastest, the atomics spread over every plane of a grid far
// larger than L2 and nearly all of them missed it (the launch read 1.45 GB
// of DRAM for 50 MB of visibilities).  Mode 1 then turns the sums into
// the estimator's input: the per-channel mean V_g / N_g and an occupancy of
// 1 (0 where N_g = 0), so that bs_grid_load's W = 1 / N_g weighting becomes
// the per-channel 1 / N_g(nu) of Eq. (vg).
#include <algorithm>

#include "plan_internal.h"

namespace bsi {

namespace {

__global__ void k_grid_vis(const double *__restrict__ uv, const float2 *__restrict__ vis,
                           const uint8_t *__restrict__ flag, long long nvis, long long nbl,
                           int nin, int avg, int nt, float2 *__restrict__ vg,
                           float *__restrict__ ng) {
  const int h = nt / 2;
  const long long plane = (long long)nt * nt;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nvis;
       t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t / nbl);
    const long long bl = t - (long long)c * nbl;
    const long long iv_in = bl * nin + c;  // element of vis / flag
    if (flag && flag[iv_in]) continue;
    const long long iu = (long long)floor(uv[2 * bl] + 0.5), iv = (long long)floor(uv[2 * bl + 1] + 0.5);
    if (iu <= -h || iu >= h || iv <= -h || iv >= h) continue;
    const float2 v = vis[iv_in];
    const long long o = (long long)(c / avg) * plane;
    const long long g = o + (iv + h) * nt + (iu + h), gm = o + (h - iv) * nt + (h - iu);
    const long long ntot = (long long)(nin / avg) * plane;  // nin = avg * output channels
    if (!BS_CHK(g, ntot, 61) || !BS_CHK(gm, ntot, 61)) continue;
    atomicAdd(&vg[g].x, v.x);
    atomicAdd(&vg[g].y, v.y);
    atomicAdd(ng + g, 1.0f);
    atomicAdd(&vg[gm].x, v.x);
    atomicAdd(&vg[gm].y, -v.y);
    atomicAdd(ng + gm, 1.0f);
  }
}

__global__ void k_grid_mean(long long n, float2 *__restrict__ vg, float *__restrict__ ng) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const float c = ng[t];
    if (c > 0.f) {
      const float2 v = vg[t];
      vg[t] = make_float2(v.x / c, v.y / c);
      ng[t] = 1.f;
    }
  }
}

}  // namespace

}  // namespace bsi

#define GRID_CUDA(call)                                          \
  do {                                                           \
    cudaError_t e__ = (call);                                    \
    if (e__ != cudaSuccess) return cuda_fail(p, e__, #call);     \
  } while (0)

extern "C" {

bs_status bs_grid_visibilities(bs_plan p, const double *uv_dev, const void *vis_dev,
                               const uint8_t *flag_dev, int64_t nbl, int nchan_in, int avg,
                               int mode, void *out_vis_dev, float *out_ng_dev, void *stream) {
  BS_NVTX("bs_grid_visibilities");
  using namespace bsi;
  if (!p || !uv_dev || !vis_dev || !out_vis_dev || !out_ng_dev)
    return fail(p, BS_ERR_ARG, "bs_grid_visibilities: NULL argument");
  if (nbl < 0 || avg < 1 || nchan_in != avg * p->nc || (mode != 0 && mode != 1))
    return fail(p, BS_ERR_ARG, "bs_grid_visibilities: nchan_in must be avg * nchan, mode 0 or 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bs_status st = prepare(p, s);  // device, sticky-error state (the workspace is not used)
  if (st != BS_OK) return st;
  const long long cells = (long long)p->nc * p->nt * p->nt;
  GRID_CUDA(cudaMemsetAsync(out_vis_dev, 0, (size_t)cells * sizeof(float2), s));
  GRID_CUDA(cudaMemsetAsync(out_ng_dev, 0, (size_t)cells * sizeof(float), s));
  const long long nvis = nbl * nchan_in;
  if (nvis > 0) {
    const int blocks = (int)std::min<long long>((nvis + 255) / 256, (long long)p->nsm * 16);
    k_grid_vis<<<blocks, 256, 0, s>>>(uv_dev, static_cast<const float2 *>(vis_dev), flag_dev, nvis,
                                      nbl, nchan_in, avg, p->nt,
                                      static_cast<float2 *>(out_vis_dev), out_ng_dev);
    GRID_CUDA(cudaGetLastError());
  }
  if (mode == 1) {
    const int blocks = (int)std::min<long long>((cells + 255) / 256, (long long)p->nsm * 16);
    k_grid_mean<<<blocks, 256, 0, s>>>(cells, static_cast<float2 *>(out_vis_dev), out_ng_dev);
    GRID_CUDA(cudaGetLastError());
  }
  return BS_OK;
}

}  // extern "C"
