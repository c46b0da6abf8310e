// C ABI of libbs (include/bs.h): plan construction (host), workspace
// layout, and the orchestration of the device stages of Section 3.2.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "plan_internal.h"

using namespace bsi;

namespace {

thread_local std::string g_create_error = "no error";

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool is_smooth(int n) {
  Radices r;
  return n == 1 || factor_radices(n, r);
}

}  // namespace

namespace bsi {

bool factor_radices(int n, Radices &r) {
  r.n = 0;
  if (n <= 0) return false;
  int m = n;
  while (m % 8 == 0 && r.n < 24) {
    r.r[r.n++] = 8;
    m /= 8;
  }
  while (m % 4 == 0 && r.n < 24) {
    r.r[r.n++] = 4;
    m /= 4;
  }
  while (m % 2 == 0 && r.n < 24) {
    r.r[r.n++] = 2;
    m /= 2;
  }
  while (m % 3 == 0 && r.n < 24) {
    r.r[r.n++] = 3;
    m /= 3;
  }
  while (m % 5 == 0 && r.n < 24) {
    r.r[r.n++] = 5;
    m /= 5;
  }
  if (m != 1) {
    r.n = 0;
    return false;
  }
  return true;
}

// exp(+2 pi i t / n), t in [0, n), FP64 then rounded to FP32
std::vector<float2> twiddles(int n) {
  std::vector<float2> tw(n);
  for (int t = 0; t < n; ++t) {
    const double x = 2.0 * (double)t / (double)n;  // angle / pi
    tw[t] = make_float2((float)std::cos(M_PI * x), (float)std::sin(M_PI * x));
  }
  return tw;
}

bs_status fail(bs_plan p, bs_status s, const std::string &msg) {
  if (p)
    p->err = msg;
  else
    g_create_error = msg;
  return s;
}

bs_status cuda_fail(bs_plan p, cudaError_t e, const char *where) {
  p->sticky = true;
  return fail(p, BS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define BS_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e__ = (call);                           \
    if (e__ != cudaSuccess) return cuda_fail(p, e__, #call); \
  } while (0)

void compute_layout(bs_plan p) {
  WsLayout &L = p->L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o += align256(bytes);
    return r;
  };
  const size_t n2 = (size_t)(2 * p->nc - 1);
  L.label = take((size_t)p->nt * p->nt);
  L.efflabel = take((size_t)p->nt * p->nt);
  L.cells = take(p->cells.size() * sizeof(int) + 4);
  L.uext = take((size_t)p->nb * sizeof(int));
  L.tripof = take((size_t)p->nb * p->nb * p->nb * sizeof(int));
  L.valid = take((size_t)p->nc);
  L.twN = take((size_t)p->nc * sizeof(float2));
  L.tnorm = take((size_t)p->ntrip * sizeof(double));
  L.T = take((size_t)p->ntrip * sizeof(unsigned long long));
  L.nnu = take(n2 * n2 * sizeof(long long));
  L.cols = take(p->max_cols * sizeof(ColEntry));
  L.ptiles = take(p->max_ptiles * sizeof(PairTile));
  L.tctiles = take(p->max_tctiles * sizeof(TcTile));
  size_t gmax = 0;
  const bool split = p->d.precision != BS_PREC_FP32;
  const bool f16 = p->d.precision == BS_PREC_SPLIT_FP16;
  for (Level &lv : p->levels) {
    const size_t nfl = (size_t)lv.nslot * p->nc, m2 = (size_t)lv.M * lv.M;
    gmax = std::max(gmax, (size_t)p->batch * nfl * lv.M * lv.UC * sizeof(float2));
    lv.offF = take((size_t)p->batch * nfl * m2 * sizeof(float));
    lv.offFhi = take(split ? (size_t)p->batch * nfl * m2 * 2 : 0);
    lv.offFlo = take(split ? (size_t)p->batch * nfl * m2 * 2 : 0);
    lv.offTw = take((size_t)lv.M * sizeof(float2));
    lv.offSlot = take((size_t)p->nb * sizeof(int));
    lv.offRing = take((size_t)std::max(1, lv.nslot) * sizeof(int));
    lv.offFmax = take(f16 ? (size_t)p->batch * std::max(1, lv.nslot) * sizeof(unsigned) : 0);
    lv.offKexp = take(f16 ? (size_t)p->batch * std::max(1, lv.nslot) * sizeof(int) : 0);
  }
  L.G = take(gmax);
  // level 0 doubles as the single-level layout of the FP32 path
  L.F = p->levels[0].offF;
  L.Fhi = p->levels[0].offFhi;
  L.Flo = p->levels[0].offFlo;
  L.twM = p->levels[0].offTw;
  L.dsum = take((size_t)p->batch * p->ntrip * n2 * n2 * sizeof(double));
  // delay-transform scratch: complex [batch][T_r][nc][nc], then a double [nc][nc]
  // table and nc row flags
  L.tmp3d = take((size_t)p->batch * p->ntrip * (size_t)p->nc * p->nc * sizeof(float2) +
                 (size_t)p->nc * p->nc * sizeof(double) + (size_t)p->nc);
  L.herm = take(2 * sizeof(float));
  L.err = take(sizeof(int));
  L.maps = take(7 * p->levels.size() * sizeof(CUtensorMap));
  L.tcgroup = take(p->levels.size() * sizeof(TcGroup));
  L.mlptab = take(((size_t)p->ntrip * 4 + 36) * sizeof(float));
  L.ztrips = take((size_t)p->ntrip * sizeof(int));
  L.clos = take((size_t)p->ntrip * sizeof(int));
  L.symtrips = take((size_t)p->ntrip * sizeof(int));
  L.closrings = take((size_t)p->ntrip * 3 * sizeof(int));
  // monopole binning constants: FP64 kperp [nb], kpar [nc]; FP32 kperp, kpar,
  // squared k1 edges [<= 1025], mu and t thresholds [<= 1025 each]
  L.mono = take(((size_t)p->nb + p->nc) * 12 + (size_t)3 * 1025 * 4 + 64);
  L.cyl = take(((size_t)p->nc + 2 * 64) * sizeof(int));  // cylindrical bins (n <= 64)
  // error bound: per-field norms (max |F|, ||F||_2, ||F||_3) of every level, and
  // the ring-triple table (i, j, l, level)
  size_t nfield_all = 0;
  for (const Level &lv : p->levels) nfield_all += (size_t)p->batch * lv.nslot * p->nc;
  L.errn = take(std::max<size_t>(1, nfield_all) * 3 * sizeof(double));
  L.errtab = take((size_t)p->ntrip * 4 * sizeof(int));
  // general plans: the four Hermitian components of the weighted input
  L.gvis = take(p->general || p->chans ? (size_t)p->batch * p->nc * p->nt * p->nt * sizeof(float2)
                                        : 0);
  L.total = o;
}

bool inject_fail(const char *point) {
  const char *env = std::getenv("BS_INJECT_FAIL");
  if (!env || !*env) return false;
  const std::string list = std::string(",") + env + ",";
  return list.find(std::string(",") + point + ",") != std::string::npos;
}

bs_status ensure_workspace(bs_plan p) {
  if (p->ws) return BS_OK;
  if (inject_fail("workspace_alloc"))
    return fail(p, BS_ERR_OOM, "injected failure: workspace allocation (BS_INJECT_FAIL)");
  void *w = nullptr;
  cudaError_t e = cudaMalloc(&w, p->L.total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(p, BS_ERR_OOM, "workspace allocation of " + std::to_string(p->L.total) +
                                   " bytes failed: " + cudaGetErrorString(e));
  }
  p->ws = static_cast<unsigned char *>(w);
  p->ws_owned = true;
  return BS_OK;
}

// Upload the constant tables into a fresh workspace.
bs_status init_tables(bs_plan p, cudaStream_t s) {
  const WsLayout &L = p->L;
  BS_CUDA(cudaMemcpyAsync(p->at<int8_t>(L.label), p->label.data(), p->label.size(),
                          cudaMemcpyHostToDevice, s));
  if (!p->cells.empty())
    BS_CUDA(cudaMemcpyAsync(p->at<int>(L.cells), p->cells.data(), p->cells.size() * sizeof(int),
                            cudaMemcpyHostToDevice, s));
  BS_CUDA(cudaMemcpyAsync(p->at<int>(L.uext), p->uext.data(), p->uext.size() * sizeof(int),
                          cudaMemcpyHostToDevice, s));
  BS_CUDA(cudaMemcpyAsync(p->at<int>(L.tripof), p->trip_of.data(),
                          p->trip_of.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  std::vector<std::vector<float2>> twl;
  for (const Level &lv : p->levels) {
    twl.push_back(twiddles(lv.M));
    BS_CUDA(cudaMemcpyAsync(p->at<float2>(lv.offTw), twl.back().data(),
                            twl.back().size() * sizeof(float2), cudaMemcpyHostToDevice, s));
    BS_CUDA(cudaMemcpyAsync(p->at<int>(lv.offSlot), lv.slot_of.data(), lv.slot_of.size() * sizeof(int),
                            cudaMemcpyHostToDevice, s));
    if (lv.nslot > 0)
      BS_CUDA(cudaMemcpyAsync(p->at<int>(lv.offRing), lv.ring_of.data(),
                              lv.ring_of.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  }
  std::vector<float2> twn = twiddles(p->nc);
  BS_CUDA(cudaMemcpyAsync(p->at<float2>(L.twN), twn.data(), twn.size() * sizeof(float2),
                          cudaMemcpyHostToDevice, s));
  BS_CUDA(cudaMemsetAsync(p->at<int>(L.err), 0, sizeof(int), s));
  BS_CUDA(cudaStreamSynchronize(s));  // host vectors above are temporaries
  return BS_OK;
}

// Read and clear the device error word (synchronises): a bounded wait in a
// kernel gave up since the last check.
bs_status check_device_error(bs_plan p, cudaStream_t s) {
  if (!p->err_pending) return BS_OK;
  BS_CUDA(cudaStreamSynchronize(s));
  p->err_pending = false;
  volatile int *e = p->err_host;
  if (*e != 0) {
    *e = 0;
    return fail(p, BS_ERR_TIMEOUT,
                "a bounded wait in the tensor-core contraction gave up; its results are invalid");
  }
  return BS_OK;
}

// Tensor maps over the field arrays of each level: rows = batch * nf fields,
// inner dimension = M^2 pixels.  hi / lo (BF16, or FP16 in split-FP16
// plans): boxes of 32 pixels x 8, 32 or 128 fields, 64-byte swizzle (the MMA operand layout; the contraction loads
// runs of consecutive fields with the larger boxes).  FP32 F: boxes of 32
// pixels x 8 fields, 128-byte swizzle (the pair producers' input rows).
bs_status ensure_tensor_maps(bs_plan p, cudaStream_t s) {
  if (p->maps_ready) return BS_OK;
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                   cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return fail(p, BS_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the CUDA driver");
  }
  EncodeTiledFn enc = reinterpret_cast<EncodeTiledFn>(fn);
  std::vector<CUtensorMap> all;
  for (Level &lv : p->levels) {
    const cuuint64_t M2 = (cuuint64_t)lv.M * lv.M;
    cuuint64_t dims[2] = {M2, (cuuint64_t)p->batch * std::max(1, lv.nslot) * p->nc};
    cuuint32_t estr[2] = {1, 1};
    for (int w = 0; w < 7; ++w) {
      const bool f32 = (w == 6);
      static const cuuint32_t rows[7] = {8, 8, 32, 32, 128, 128, 8};
      cuuint64_t strides[1] = {M2 * (f32 ? 4 : 2)};
      cuuint32_t box[2] = {32, rows[w]};
      void *base = f32 ? (void *)p->at<float>(lv.offF)
                       : (void *)p->at<uint16_t>(w % 2 == 0 ? lv.offFhi : lv.offFlo);
      const CUtensorMapDataType half_t = p->d.precision == BS_PREC_SPLIT_FP16
                                             ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                             : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
      CUresult r = enc(&lv.maps[w], f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : half_t, 2,
                       base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       f32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS)
        return fail(p, BS_ERR_CUDA,
                    "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
      all.push_back(lv.maps[w]);
    }
  }
  BS_CUDA(cudaMemcpyAsync(p->at<unsigned char>(p->L.maps), all.data(), all.size() * sizeof(CUtensorMap),
                          cudaMemcpyHostToDevice, s));
  BS_CUDA(cudaStreamSynchronize(s));
  p->maps_ready = true;
  return BS_OK;
}

bs_status enqueue_fields(bs_plan p, const void *vis, const float *ngrid, cudaStream_t s) {
  const WsLayout &L = p->L;
  const bool bf16 = p->d.precision == BS_PREC_SPLIT_BF16;
  const bool f16 = p->d.precision == BS_PREC_SPLIT_FP16;
  for (const Level &lv : p->levels) {
    if (lv.nslot == 0) continue;
    GridGeom g{p->nt, p->nc, p->nb, lv.M, lv.UC, p->batch, lv.nslot, p->at<int>(lv.offSlot),
               p->at<int>(lv.offRing)};
    BS_CUDA(launch_colpass(g, static_cast<const float2 *>(vis), ngrid, p->at<uint8_t>(L.valid),
                           p->at<int8_t>(L.label), p->at<int>(L.uext), p->at<float2>(lv.offTw),
                           lv.rad, p->at<float2>(L.G), s));
    if (f16)
      BS_CUDA(cudaMemsetAsync(p->at<unsigned>(lv.offFmax), 0,
                              (size_t)p->batch * lv.nslot * sizeof(unsigned), s));
    BS_CUDA(launch_rowpass(g, p->at<float2>(L.G), p->at<uint8_t>(L.valid), p->at<int>(L.uext),
                           p->at<float2>(lv.offTw), lv.rad, p->at<float>(lv.offF),
                           bf16 ? p->at<uint16_t>(lv.offFhi) : nullptr,
                           bf16 ? p->at<uint16_t>(lv.offFlo) : nullptr,
                           f16 ? p->at<unsigned>(lv.offFmax) : nullptr, s));
    if (f16)
      BS_CUDA(launch_split_f16(g, p->at<float>(lv.offF), p->at<unsigned>(lv.offFmax),
                               p->at<int>(lv.offKexp), p->at<uint16_t>(lv.offFhi),
                               p->at<uint16_t>(lv.offFlo), s));
  }
  return BS_OK;
}

bs_status prepare(bs_plan p, cudaStream_t s) {
  if (p->sticky) return fail(p, BS_ERR_STATE, "plan has a sticky CUDA error: " + p->err);
  BS_CUDA(cudaSetDevice(p->device));
  if (!p->ws) {
    bs_status st = ensure_workspace(p);
    if (st != BS_OK) return st;
    st = init_tables(p, s);
    if (st != BS_OK) return st;
  }
  return BS_OK;
}

// Triangle counts on the device with the given label table; T and tnorm on host.
bs_status run_counts(bs_plan p, const int8_t *lab_dev, cudaStream_t s) {
  unsigned long long *Td = p->at<unsigned long long>(p->L.T);
  BS_CUDA(cudaMemsetAsync(Td, 0, (size_t)p->ntrip * sizeof(unsigned long long), s));
  BS_CUDA(launch_counts(p->nt, p->nb, lab_dev, p->at<int>(p->L.cells), (int)p->cells.size(),
                        p->at<int>(p->L.tripof), Td, s));
  std::vector<unsigned long long> th(p->ntrip);
  BS_CUDA(cudaMemcpyAsync(th.data(), Td, th.size() * sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, s));
  BS_CUDA(cudaStreamSynchronize(s));
  p->T.assign(th.begin(), th.end());
  p->tnorm.resize(p->ntrip);
  for (int t = 0; t < p->ntrip; ++t) {
    const int lv = p->lev_of_trip[t];
    if (p->T[t] > 0 && lv < 0) return fail(p, BS_ERR_STATE, "closable ring triple without a level");
    const double m = lv >= 0 ? (double)p->levels[lv].M : 1.0;
    p->tnorm[t] = p->T[t] > 0 ? 1.0 / (p->normA * m * m * (double)p->T[t]) : 0.0;
  }
  BS_CUDA(cudaMemcpyAsync(p->at<double>(p->L.tnorm), p->tnorm.data(), p->ntrip * sizeof(double),
                          cudaMemcpyHostToDevice, s));
  p->clos.clear();
  p->closrings.clear();
  p->sym_trips.clear();
  for (int t = 0; t < p->ntrip; ++t)
    if (p->T[t] > 0) {
      p->clos.push_back(t);
      for (int k = 0; k < 3; ++k) p->closrings.push_back(p->trips[3 * t + k]);
      const int i = p->trips[3 * t], j = p->trips[3 * t + 1], l = p->trips[3 * t + 2];
      if (i == j)
        p->sym_trips.push_back(2 * t);
      else if (j == l)
        p->sym_trips.push_back(2 * t + 1);
    }
  if (!p->sym_trips.empty())
    BS_CUDA(cudaMemcpyAsync(p->at<int>(p->L.symtrips), p->sym_trips.data(),
                            p->sym_trips.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  if (!p->clos.empty()) {
    BS_CUDA(cudaMemcpyAsync(p->at<int>(p->L.clos), p->clos.data(), p->clos.size() * sizeof(int),
                            cudaMemcpyHostToDevice, s));
    BS_CUDA(cudaMemcpyAsync(p->at<int>(p->L.closrings), p->closrings.data(),
                            p->closrings.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  }
  BS_CUDA(cudaStreamSynchronize(s));
  p->counts_ready = true;
  p->dsum_clean = false;
  return BS_OK;
}

// Unfolded sampling of a channel block: cnt[d1][d2] += #{nu3 in B3 : nu3+d1 in
// B1, nu3+d2 in B2, all three valid}, with 64-bit words of channel bits.
// plane: [2nc-1][2nc-1], index (d1 + nc - 1, d2 + nc - 1).
void add_block_sampling(int nc, const std::vector<uint8_t> &valid, const int *blk,
                        long long *plane) {
  const int n2 = 2 * nc - 1;
  const int W = (nc + 63) / 64;
  auto bits = [&](int lo, int hi) {
    std::vector<uint64_t> b(W, 0);
    for (int c = lo; c < hi; ++c)
      if (valid[c]) b[c >> 6] |= uint64_t(1) << (c & 63);
    return b;
  };
  const std::vector<uint64_t> b1 = bits(blk[0], blk[1]), b2 = bits(blk[2], blk[3]),
                              b3 = bits(blk[4], blk[5]);
  // shifted(src, d)[nu3] = src[nu3 + d]
  auto shifted = [&](const std::vector<uint64_t> &src, int d, uint64_t *out) {
    for (int w = 0; w < W; ++w) {
      const long long s0 = (long long)w * 64 + d;  // source bit of out bit 0 of word w
      uint64_t v = 0;
      const long long q = s0 >= 0 ? s0 / 64 : -((-s0 + 63) / 64);
      const int r = (int)(s0 - q * 64);
      auto word = [&](long long k) -> uint64_t { return (k >= 0 && k < W) ? src[k] : 0; };
      if (r == 0)
        v = word(q);
      else
        v = (word(q) >> r) | (word(q + 1) << (64 - r));
      out[w] = v;
    }
  };
  // reachable separations: d = nu - nu3 with nu in [lo, hi), nu3 in [blk[4], blk[5])
  const int d1lo = std::max(-(nc - 1), blk[0] - blk[5] + 1), d1hi = std::min(nc - 1, blk[1] - 1 - blk[4]);
  const int d2lo = std::max(-(nc - 1), blk[2] - blk[5] + 1), d2hi = std::min(nc - 1, blk[3] - 1 - blk[4]);
  if (d1lo > d1hi || d2lo > d2hi) return;
  std::vector<uint64_t> s2((size_t)n2 * W), p1(W);
  for (int d2 = d2lo; d2 <= d2hi; ++d2) shifted(b2, d2, &s2[(size_t)(d2 + nc - 1) * W]);
  for (int d1 = d1lo; d1 <= d1hi; ++d1) {
    shifted(b1, d1, p1.data());
    bool any = false;
    for (int w = 0; w < W; ++w) {
      p1[w] &= b3[w];
      any |= p1[w] != 0;
    }
    if (!any) continue;
    long long *row = plane + (size_t)(d1 + nc - 1) * n2;
    for (int d2i = d2lo + nc - 1; d2i <= d2hi + nc - 1; ++d2i) {
      const uint64_t *q = &s2[(size_t)d2i * W];
      long long c = 0;
      for (int w = 0; w < W; ++w) c += __builtin_popcountll(p1[w] & q[w]);
      row[d2i] += c;
    }
  }
}

void accumulate_block_nnu(bs_plan p, const int *blk) {
  add_block_sampling(p->nc, p->valid, blk, p->nnu.data());
  p->nnu_dirty = true;
  // the separations this block can write: d = nu - nu3, nu in the block's
  // nu1 (nu2) range, nu3 in its nu3 range
  const int nc = p->nc;
  const int r0 = std::max(0, blk[0] - blk[5] + 1 + nc - 1), r1 = std::min(2 * nc - 2, blk[1] - 1 - blk[4] + nc - 1);
  const int c0 = std::max(0, blk[2] - blk[5] + 1 + nc - 1), c1 = std::min(2 * nc - 2, blk[3] - 1 - blk[4] + nc - 1);
  if (r0 > r1 || c0 > c1) return;
  int *b = p->dbox;
  if (b[1] < b[0] || b[3] < b[2]) {
    b[0] = r0; b[1] = r1; b[2] = c0; b[3] = c1;
  } else {
    b[0] = std::min(b[0], r0); b[1] = std::max(b[1], r1);
    b[2] = std::min(b[2], c0); b[3] = std::max(b[3], c1);
  }
}

bs_status upload_staged(bs_plan p, cudaStream_t s, const StagedUpload *u, int n) {
  size_t total = 0;
  for (int k = 0; k < n; ++k) total += (u[k].bytes + 255) / 256 * 256;
  if (p->stage_pending) {  // the previous uploads from the buffer are done
    BS_CUDA(cudaEventSynchronize(p->stage_ev));
    p->stage_pending = false;
  }
  if (!p->stage_ev) BS_CUDA(cudaEventCreateWithFlags(&p->stage_ev, cudaEventDisableTiming));
  if (total > p->h_stage_cap) {
    if (p->h_stage) cudaFreeHost(p->h_stage);
    p->h_stage = nullptr;
    p->h_stage_cap = 0;
    void *h = nullptr;
    if (cudaHostAlloc(&h, total + total / 4, cudaHostAllocDefault) == cudaSuccess) {
      p->h_stage = static_cast<unsigned char *>(h);
      p->h_stage_cap = total + total / 4;
    } else {
      cudaGetLastError();
    }
  }
  if (!p->h_stage) {  // no pinned memory: ordinary (host-synchronous) copies
    for (int k = 0; k < n; ++k)
      if (u[k].bytes)
        BS_CUDA(cudaMemcpyAsync(u[k].dst, u[k].src, u[k].bytes, cudaMemcpyHostToDevice, s));
    return BS_OK;
  }
  size_t off = 0;
  for (int k = 0; k < n; ++k) {
    if (!u[k].bytes) continue;
    std::memcpy(p->h_stage + off, u[k].src, u[k].bytes);
    BS_CUDA(cudaMemcpyAsync(u[k].dst, p->h_stage + off, u[k].bytes, cudaMemcpyHostToDevice, s));
    off += (u[k].bytes + 255) / 256 * 256;
  }
  BS_CUDA(cudaEventRecord(p->stage_ev, s));
  p->stage_pending = true;
  return BS_OK;
}

bs_status upload_nnu(bs_plan p, cudaStream_t s) {
  if (!p->nnu_dirty) return BS_OK;
  BS_CUDA(cudaMemcpyAsync(p->at<long long>(p->L.nnu), p->nnu.data(),
                          p->nnu.size() * sizeof(long long), cudaMemcpyHostToDevice, s));
  BS_CUDA(cudaStreamSynchronize(s));
  p->nnu_dirty = false;
  return BS_OK;
}

bs_status sym_fill(bs_plan p, cudaStream_t s) {
  if (p->sym_state != 2) return BS_OK;
  BS_CUDA(launch_symmetrize(p->at<double>(p->L.dsum), p->at<int>(p->L.symtrips),
                            (int)p->sym_trips.size(), p->batch, p->ntrip, p->nc, p->dbox, s));
  p->sym_state = 3;
  return BS_OK;
}

bs_status delta_reset(bs_plan p, cudaStream_t s) {
  std::fill(p->nnu.begin(), p->nnu.end(), 0LL);
  p->nnu_dirty = true;
  p->sym_state = 0;
  const size_t n2 = (size_t)(2 * p->nc - 1);
  if (!p->dsum_clean || !p->counts_ready) {
    BS_CUDA(cudaMemsetAsync(p->at<double>(p->L.dsum), 0,
                            (size_t)p->batch * p->ntrip * n2 * n2 * sizeof(double), s));
    p->dsum_clean = p->counts_ready;
    p->dbox[0] = 0; p->dbox[1] = -1; p->dbox[2] = 0; p->dbox[3] = -1;
    p->zero_trips.clear();
    for (int t = 0; t < p->ntrip; ++t)
      if (p->counts_ready && p->T[t] > 0) p->zero_trips.push_back(t);
    if (!p->zero_trips.empty())
      BS_CUDA(cudaMemcpyAsync(p->at<int>(p->L.ztrips), p->zero_trips.data(),
                              p->zero_trips.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    return BS_OK;
  }
  // only ring triples with closed triangles are ever accumulated into, and only
  // at the separations of the blocks accumulated since the last reset
  BS_CUDA(launch_zero_planes(p->at<double>(p->L.dsum), p->at<int>(p->L.ztrips),
                             (int)p->zero_trips.size(), p->batch, p->ntrip, (int)n2, p->dbox, s));
  p->dbox[0] = 0; p->dbox[1] = -1; p->dbox[2] = 0; p->dbox[3] = -1;
  return BS_OK;
}

std::vector<TcGroup> build_tc_work(bs_plan p, const int *blk, int group_base,
                                   std::vector<ColEntry> &cols, const ColEntry *cols_dev,
                                   std::vector<TcTile> &tiles, double *out_full, int accumulate,
                                   int min_tiles) {
  const int nc = p->nc, nb = p->nb;
  const int w3 = blk[5] - blk[4];
  const int run = ((w3 + 7) / 8) * 8;
  const int nlev = (int)p->levels.size();
  std::vector<TcGroup> groups(nlev);
  for (int lv = 0; lv < nlev; ++lv) {
    const Level &L = p->levels[lv];
    const int M2 = L.M * L.M;
    TcGroup &G = groups[lv];
    G.F = p->at<float>(L.offF);
    G.fstride = M2;
    G.bstride = (long long)std::max(1, L.nslot) * nc * M2;
    G.nf = std::max(1, L.nslot) * nc;
    G.batch = p->batch;
    G.M2 = M2;
    G.Kpad = ((M2 + 31) / 32) * 32;
    G.nc = nc;
    G.nu1_hi = blk[1];
    G.nu2_hi = blk[3];
    G.cols = cols_dev;
    G.tnorm = p->at<double>(p->L.tnorm);
    G.out_full = out_full;
    G.full_bstride = (long long)p->ntrip * nc * nc * nc;
    G.dsum = accumulate ? p->at<double>(p->L.dsum) : nullptr;
    G.dsum_bstride = (long long)p->ntrip * (2 * nc - 1) * (2 * nc - 1);
    G.kseg_len = G.Kpad;
    G.kexp = p->d.precision == BS_PREC_SPLIT_FP16 ? p->at<int>(L.offKexp) : nullptr;
    G.nslot = std::max(1, L.nslot);
  }
  if (w3 == 0 || blk[1] <= blk[0] || blk[3] <= blk[2]) return groups;
  // channel-symmetric accumulation of a cube block S x S x S: ring triples with a
  // repeated ring are contracted for one ordering of its channels only (the
  // ring pair (i, i) keeps nu1 <= nu2; the triple (i, j, j), i < j, moves to the
  // ring pair (j, j) as swapped rows (i, nu1) with nu2 <= nu3)
  const bool sym = accumulate == 2;
  // column lists per (level, ring pair): fields (l, nu3) of the level's slots,
  // runs padded to multiples of 8 so TMA boxes of 8 fields never straddle rings
  struct PairList {
    int lv, si, sj, off, n;
  };
  std::vector<PairList> pl;
  for (int lv = 0; lv < nlev; ++lv) {
    const Level &L = p->levels[lv];
    auto add_run = [&](int ring, int t, int swapped) {
      for (int q = 0; q < run; ++q) {
        const int n3 = blk[4] + q;
        cols.push_back(ColEntry{q < w3 ? L.slot_of[ring] * nc + n3 : -1, t, n3, swapped});
      }
    };
    for (int i = 0; i < nb; ++i)
      for (int j = i; j < nb; ++j) {
        if (L.slot_of[i] < 0 || L.slot_of[j] < 0) continue;
        const int off = (int)cols.size();
        if (sym && i == j)
          for (int k = 0; k < i; ++k) {  // ring triples (k, i, i): rows (k, nu1)
            const int t = p->trip_of[((size_t)k * nb + i) * nb + i];
            if (p->T[t] > 0 && p->lev_of_trip[t] == lv) add_run(k, t, 1);
          }
        for (int l = (sym && i < j) ? j + 1 : j; l < nb; ++l) {
          const int t = p->trip_of[((size_t)i * nb + j) * nb + l];
          if (p->T[t] <= 0 || p->lev_of_trip[t] != lv) continue;
          add_run(l, t, 0);
        }
        const int n = (int)cols.size() - off;
        if (n > 0) pl.push_back(PairList{lv, L.slot_of[i], L.slot_of[j], off, n});
      }
  }
  const int n1b = (blk[1] - blk[0] + 31) / 32, n2b = (blk[3] - blk[2] + 15) / 16;
  long long base_tiles = 0;
  // a tile is one CTA pair's work: 256 column entries (128 per CTA) x 32 x 16 pairs
  for (const PairList &q : pl) base_tiles += (long long)n1b * n2b * ((q.n + 255) / 256);
  base_tiles *= p->batch;
  // split K (the same factor on every level) until the launch has min_tiles tiles
  int nk = 1;
  int kmin = 1 << 30;
  for (const TcGroup &G : groups) kmin = std::min(kmin, G.Kpad);
  while (base_tiles * nk < min_tiles && nk < 64 && kmin / (32 * nk * 2) >= 8) nk *= 2;
  std::vector<int> nks(nlev);
  for (int lv = 0; lv < nlev; ++lv) {
    TcGroup &G = groups[lv];
    G.kseg_len = ((G.Kpad / 32 + nk - 1) / nk) * 32;
    nks[lv] = (G.Kpad + G.kseg_len - 1) / G.kseg_len;
  }
  const size_t t0 = tiles.size();
  auto add_tiles = [&](int b, const PairList &q, int c0, int a1, int a2) {
    const int x0 = blk[0] + 32 * a1, y0 = blk[2] + 16 * a2;
    int diag = 0;
    if (sym && q.si == q.sj) {  // one-ring pair operand: keep nu1 <= nu2
      const int x1 = std::min(x0 + 31, blk[1] - 1), y1 = std::min(y0 + 15, blk[3] - 1);
      if (x0 > y1) return;  // every pair has nu1 > nu2
      diag = x1 > y0 ? 1 : 0;
    }
    for (int k = 0; k < nks[q.lv]; ++k)
      tiles.push_back(TcTile{group_base + q.lv, b, q.si, q.sj, x0, y0, q.off, q.n, c0, k, diag, 0});
  };
  for (int b = 0; b < p->batch; ++b)
    for (const PairList &q : pl)
      for (int c0 = 0; c0 < q.n; c0 += 256)
        for (int a1 = 0; a1 < n1b; ++a1)
          for (int a2 = 0; a2 < n2b; ++a2) add_tiles(b, q, c0, a1, a2);
  // heaviest tiles first: static round-robin over persistent CTAs then balances
  std::stable_sort(tiles.begin() + t0, tiles.end(), [&](const TcTile &x, const TcTile &y) {
    return groups[x.group - group_base].kseg_len > groups[y.group - group_base].kseg_len;
  });
  return groups;
}

// Tensor-core contraction of one channel block of one plan (split BF16): one launch.
static bs_status mabs_tc_launch(bs_plan p, const int *blk, double *out_full, int accumulate,
                                cudaStream_t s) {
  bs_status st = BS_OK;
  const WsLayout &L = p->L;
  p->h_cols.clear();
  p->h_tctiles.clear();
  p->h_groups = build_tc_work(p, blk, 0, p->h_cols, p->at<ColEntry>(L.cols), p->h_tctiles,
                              out_full, accumulate, p->nsm);
  if (p->h_tctiles.empty()) return BS_OK;
  if (p->h_tctiles.size() > p->max_tctiles || p->h_cols.size() > p->max_cols)
    return fail(p, BS_ERR_UNSUPPORTED, "tensor-core tile list exceeds the plan's capacity");
  const StagedUpload up[3] = {
      {p->at<ColEntry>(L.cols), p->h_cols.data(), p->h_cols.size() * sizeof(ColEntry)},
      {p->at<TcTile>(L.tctiles), p->h_tctiles.data(), p->h_tctiles.size() * sizeof(TcTile)},
      {p->at<TcGroup>(L.tcgroup), p->h_groups.data(), p->h_groups.size() * sizeof(TcGroup)}};
  st = upload_staged(p, s, up, 3);
  if (st != BS_OK) return st;
  TcArgs a{};
  a.groups = p->at<TcGroup>(L.tcgroup);
  a.maps = p->at<unsigned char>(L.maps);
  a.tiles = p->at<TcTile>(L.tctiles);
  a.ntiles = (int)p->h_tctiles.size();
  a.err = p->err_dev;
  p->err_pending = true;
  a.wait_limit_ns = 2000000000LL;
  const char *inj = std::getenv("BS_INJECT_MMA_STALL");
  a.stall_test = (inj && inj[0] == '1') ? 1 : 0;
  a.f16 = p->d.precision == BS_PREC_SPLIT_FP16 ? 1 : 0;
  if (a.stall_test) a.wait_limit_ns = 50000000LL;
  BS_CUDA(launch_contract_tc(a, p->nsm, s));
  return BS_OK;
}

// A channel-symmetric cube wider than 128 channels runs as one launch per
// 128 x 128 sub-block of its (nu1, nu2) pair plane, rows over the whole cube:
// each launch has the tile structure of an ordinary 128 x 128 x 256 block,
// whose concurrently running CTA pairs share field and FP32 rows in L2
// (measured on the 256-channel MWA-like cube: 25-74 GB of DRAM reads per
// launch, 153-205 GB per cube).
bs_status mabs_tc(bs_plan p, const int *blk, double *out_full, int accumulate, cudaStream_t s) {
  bs_status st = ensure_tensor_maps(p, s);
  if (st != BS_OK) return st;
  constexpr int SUB = 128;
  if (accumulate != 2 || blk[1] - blk[0] <= SUB)
    return mabs_tc_launch(p, blk, out_full, accumulate, s);
  for (int s1 = blk[0]; s1 < blk[1]; s1 += SUB)
    for (int s2 = blk[2]; s2 < blk[3]; s2 += SUB) {
      const int sub[6] = {s1, std::min(blk[1], s1 + SUB), s2, std::min(blk[3], s2 + SUB),
                          blk[4], blk[5]};
      st = mabs_tc_launch(p, sub, out_full, accumulate, s);
      if (st != BS_OK) return st;
    }
  return BS_OK;
}

// Scratch of a general plan for the four real components of an output (grown on
// demand with cudaMalloc, freed with the plan).
bs_status general_scratch(bs_plan p, double **buf, size_t *cap, size_t n) {
  if (*buf && *cap >= n) return BS_OK;
  if (inject_fail("scratch_alloc"))
    return fail(p, BS_ERR_OOM, "injected failure: scratch allocation (BS_INJECT_FAIL)");
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  void *m = nullptr;
  const cudaError_t e = cudaMalloc(&m, std::max<size_t>(1, n) * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(p, BS_ERR_OOM, "scratch of " + std::to_string(n * sizeof(double)) +
                                   " bytes for the general-input components failed");
  }
  *buf = static_cast<double *>(m);
  *cap = n;
  return BS_OK;
}

}  // namespace bsi

extern "C" {

int bs_abi_version(void) { return BS_ABI_VERSION; }

const char *bs_last_error(bs_plan plan) {
  return plan ? plan->err.c_str() : g_create_error.c_str();
}

bs_status bs_plan_create(const bs_plan_desc *desc, bs_plan *out) {
  BS_NVTX("bs_plan_create");
  if (!desc || !out) return fail(nullptr, BS_ERR_ARG, "desc and out must not be NULL");
  *out = nullptr;
  if (inject_fail("plan_create"))
    return fail(nullptr, BS_ERR_OOM, "injected failure: plan creation (BS_INJECT_FAIL)");
  const bs_plan_desc &d = *desc;
  if (d.nt < 8 || d.nt > 1024 || (d.nt & 1))
    return fail(nullptr, BS_ERR_ARG, "nt must be even and in [8, 1024]");
  if (d.nchan < 1 || d.nchan > 4096) return fail(nullptr, BS_ERR_ARG, "nchan must be in [1, 4096]");
  if (d.nbins < 1 || d.nbins > 32) return fail(nullptr, BS_ERR_ARG, "nbins must be in [1, 32]");
  if (!d.bin_edges) return fail(nullptr, BS_ERR_ARG, "bin_edges must not be NULL");
  if (d.batch < 1) return fail(nullptr, BS_ERR_ARG, "batch must be >= 1");
  if (d.general != 0 && d.general != 1) return fail(nullptr, BS_ERR_ARG, "general must be 0 or 1");
  if (d.general && (long long)d.batch * 4 > 65535)
    return fail(nullptr, BS_ERR_ARG, "batch too large for a general plan");
  if (d.chan_sampling != 0 && d.chan_sampling != 1)
    return fail(nullptr, BS_ERR_ARG, "chan_sampling must be 0 or 1");
  if (d.chan_sampling && d.general)
    return fail(nullptr, BS_ERR_UNSUPPORTED, "chan_sampling with general input");
  if (d.chan_sampling && (long long)d.batch * 2 > 65535)
    return fail(nullptr, BS_ERR_ARG, "batch too large for a per-channel sampling plan");
  if (d.precision != BS_PREC_FP32 && d.precision != BS_PREC_SPLIT_BF16 &&
      d.precision != BS_PREC_SPLIT_FP16)
    return fail(nullptr, BS_ERR_ARG, "unknown precision");
  for (int m = 0; m <= d.nbins; ++m)
    if (!std::isfinite(d.bin_edges[m]) || d.bin_edges[m] < 0 ||
        (m > 0 && !(d.bin_edges[m] > d.bin_edges[m - 1])))
      return fail(nullptr, BS_ERR_ARG, "bin_edges must be finite, >= 0 and strictly ascending");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(nullptr, BS_ERR_NO_DEVICE, "no CUDA device is available");
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, BS_ERR_NO_DEVICE, "cannot query the CUDA device");
  }
  if (!(prop.major == 10 && prop.minor == 3))
    return fail(nullptr, BS_ERR_NO_DEVICE,
                "libbs is built for sm_103a (GB300); device is sm_" + std::to_string(prop.major) +
                    std::to_string(prop.minor));

  bs_plan p = new bs_plan_s();
  p->d = d;
  p->device = dev;
  p->nt = d.nt;
  p->nc = d.nchan;
  p->nb = d.nbins;
  // general input: four Hermitian components per realisation, processed as
  // realisations of their own and combined into complex results
  p->general = d.general != 0;
  p->chans = d.chan_sampling != 0;
  p->ubatch = d.batch;
  p->batch = p->general ? 4 * d.batch : p->chans ? 2 * d.batch : d.batch;
  if (cudaHostAlloc(&p->err_host, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer(&p->err_dev, p->err_host, 0) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return fail(nullptr, BS_ERR_OOM, "cannot allocate the mapped error word");
  }
  *p->err_host = 0;
  p->edges.assign(d.bin_edges, d.bin_edges + d.nbins + 1);
  p->d.bin_edges = nullptr;
  p->normA = d.norm_A > 0 ? d.norm_A : 1.0;
  const double r = d.r > 0 ? d.r : 1.0, rp = d.rprime > 0 ? d.rprime : 1.0,
               dnu = d.dnu_c > 0 ? d.dnu_c : 1.0;
  p->scale3d = (r * r * rp * dnu) * (r * r * rp * dnu);

  // ring labels: e_m <= |U| < e_{m+1}, |U|^2 (exact integer) against e^2 (FP64)
  const int nt = p->nt, h = nt / 2;
  p->label.assign((size_t)nt * nt, -1);
  p->uext.assign(p->nb, 0);
  int cmax = 0;
  std::vector<double> e2(p->nb + 1);
  for (int m = 0; m <= p->nb; ++m) e2[m] = p->edges[m] * p->edges[m];
  for (int iv = 1; iv < nt; ++iv)
    for (int iu = 1; iu < nt; ++iu) {
      const int u = iu - h, v = iv - h;
      if (u == 0 && v == 0) continue;
      const double q = (double)((long long)u * u + (long long)v * v);
      int ring = -1;
      for (int m = 0; m < p->nb; ++m)
        if (q >= e2[m] && q < e2[m + 1]) {
          ring = m;
          break;
        }
      if (ring < 0) continue;
      p->label[(size_t)iv * nt + iu] = (int8_t)ring;
      p->cells.push_back(pack_cell(u, v));
      p->uext[ring] = std::max(p->uext[ring], std::abs(u) + 1);
      cmax = std::max(cmax, std::max(std::abs(u), std::abs(v)));
    }
  p->umean.assign(p->nb, 0.0);
  {
    std::vector<long long> nin(p->nb, 0);
    for (int c : p->cells) {
      const int u = (c & 0xffff) - 32768, v = ((c >> 16) & 0xffff) - 32768;
      const int m = p->label[(size_t)(v + h) * nt + (u + h)];
      p->umean[m] += std::sqrt((double)u * u + (double)v * v);
      ++nin[m];
    }
    for (int m = 0; m < p->nb; ++m)
      p->umean[m] = nin[m] ? p->umean[m] / nin[m] : 0.5 * (p->edges[m] + p->edges[m + 1]);
  }
  p->UC = 0;
  for (int m = 0; m < p->nb; ++m) p->UC = std::max(p->UC, p->uext[m]);
  p->UC = std::max(p->UC, 1);
  // alias-free image side: M > 3 cmax, M % 4 == 0, smooth
  if (d.fft_m > 0) {
    if (d.fft_m % 4 || !factor_radices(d.fft_m, p->radM) || d.fft_m <= 3 * cmax || d.fft_m > 4096) {
      delete p;
      return fail(nullptr, BS_ERR_ARG,
                  "fft_m must be a multiple of 4, a product of 2, 3, 5, at most 4096 and > 3 * " +
                      std::to_string(cmax));
    }
    p->M = d.fft_m;
  } else {
    int m = std::max(8, 3 * cmax + 1);
    m = (m + 3) & ~3;
    while (!is_smooth(m)) m += 4;
    p->M = m;
    factor_radices(p->M, p->radM);
  }
  if (p->M > 4096) {
    delete p;
    return fail(nullptr, BS_ERR_UNSUPPORTED, "image side M above 4096");
  }
  if (!factor_radices(p->nc, p->radN)) p->radN.n = 0;  // direct DFT for non-smooth nchan
  // ring triples i <= j <= l, lexicographic
  p->trip_of.assign((size_t)p->nb * p->nb * p->nb, -1);
  for (int i = 0; i < p->nb; ++i)
    for (int j = i; j < p->nb; ++j)
      for (int l = j; l < p->nb; ++l) {
        p->trip_of[((size_t)i * p->nb + j) * p->nb + l] = (int)(p->trips.size() / 3);
        p->trips.push_back(i);
        p->trips.push_back(j);
        p->trips.push_back(l);
      }
  p->ntrip = (int)(p->trips.size() / 3);
  p->nf = p->nb * p->nc;
  // image levels
  p->cring.assign(p->nb, -1);
  std::vector<double> rmin(p->nb, 1e300), rmax(p->nb, -1.0);
  for (int c : p->cells) {
    const int u = (c & 0xffff) - 32768, v = ((c >> 16) & 0xffff) - 32768;
    const int m = p->label[(size_t)(v + h) * nt + (u + h)];
    p->cring[m] = std::max(p->cring[m], std::max(std::abs(u), std::abs(v)));
    const double r = std::sqrt((double)u * u + (double)v * v);
    rmin[m] = std::min(rmin[m], r);
    rmax[m] = std::max(rmax[m], r);
  }
  p->multires = d.multires != 0;
  p->lev_of_trip.assign(p->ntrip, -1);
  if (!p->multires) {
    Level lv;
    lv.M = p->M;
    lv.rad = p->radM;
    lv.UC = p->UC;
    lv.nslot = p->nb;
    for (int m = 0; m < p->nb; ++m) {
      lv.slot_of.push_back(m);
      lv.ring_of.push_back(m);
    }
    p->levels.push_back(lv);
    std::fill(p->lev_of_trip.begin(), p->lev_of_trip.end(), 0);
  } else {
    // per ring triple the smallest M = 2^a x {8, 12} with M > c_i + c_j + c_l (exact
    // closure) and M > 2 max(c) (Hermitian halves of a ring never overlap); triples
    // whose annuli cannot form a triangle (|g3| <= |g1| + |g2| and permutations)
    // have no closed triangle and get no level
    std::vector<int> cand;
    for (int b = 8; b <= 4096; b *= 2) {
      cand.push_back(b);
      if (b * 3 / 2 <= 4096) cand.push_back(b * 3 / 2);
    }
    std::sort(cand.begin(), cand.end());
    std::vector<int> tripM(p->ntrip, 0);
    for (int t = 0; t < p->ntrip; ++t) {
      const int i = p->trips[3 * t], j = p->trips[3 * t + 1], l = p->trips[3 * t + 2];
      if (p->cring[i] < 0 || p->cring[j] < 0 || p->cring[l] < 0) continue;
      if (rmin[l] > rmax[i] + rmax[j] + 1e-9 || rmin[i] > rmax[j] + rmax[l] + 1e-9 ||
          rmin[j] > rmax[i] + rmax[l] + 1e-9)
        continue;
      const int need = std::max(p->cring[i] + p->cring[j] + p->cring[l],
                                2 * std::max(p->cring[i], std::max(p->cring[j], p->cring[l])));
      int M = 0;
      for (int c : cand)
        if (c > need) {
          M = c;
          break;
        }
      if (M == 0) {
        delete p;
        return fail(nullptr, BS_ERR_UNSUPPORTED, "a ring triple needs an image side above 4096");
      }
      tripM[t] = M;
    }
    std::vector<int> used;
    for (int M : tripM)
      if (M && std::find(used.begin(), used.end(), M) == used.end()) used.push_back(M);
    std::sort(used.begin(), used.end());
    for (int M : used) {
      Level lv;
      lv.M = M;
      factor_radices(M, lv.rad);
      lv.slot_of.assign(p->nb, -1);
      p->levels.push_back(lv);
    }
    for (int t = 0; t < p->ntrip; ++t) {
      if (!tripM[t]) continue;
      const int lvi = (int)(std::find(used.begin(), used.end(), tripM[t]) - used.begin());
      p->lev_of_trip[t] = lvi;
      Level &lv = p->levels[lvi];
      for (int q = 0; q < 3; ++q) {
        const int m = p->trips[3 * t + q];
        if (lv.slot_of[m] < 0) {
          lv.slot_of[m] = lv.nslot++;
          lv.ring_of.push_back(m);
          lv.UC = std::max(lv.UC, p->uext[m]);
        }
      }
    }
    if (p->levels.empty()) {  // nothing can close: one empty level keeps the layout valid
      Level lv;
      lv.M = 8;
      factor_radices(8, lv.rad);
      lv.slot_of.assign(p->nb, -1);
      p->levels.push_back(lv);
    }
  }
  p->valid.assign(p->nc, 1);
  p->nnu.assign((size_t)(2 * p->nc - 1) * (2 * p->nc - 1), 0);
  const int npairs = p->nb * (p->nb + 1) / 2;
  p->max_cols = (size_t)npairs * p->nb * p->nc;
  p->max_ptiles = (size_t)npairs * ((size_t)p->nb * p->nc / 128 + 1);
  // tensor-core tiles: pair rectangles (32 x 16) x 256-entry column windows (runs padded to 8)
  cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (p->d.precision != BS_PREC_FP32) {
    // largest block: the full cube; K splitting only happens while tiles < 2 per SM
    const size_t runs = (size_t)p->nb * (((p->nc + 7) / 8) * 8);
    const size_t full = (size_t)npairs * ((p->nc + 31) / 32) * ((p->nc + 15) / 16) * ((runs + 127) / 128);
    p->max_tctiles = std::min<size_t>(full + 4 * (size_t)p->nsm, (size_t)1 << 22);
    p->max_cols = (size_t)npairs * runs;
  }
  compute_layout(p);
  *out = p;
  return BS_OK;
}

bs_status bs_plan_destroy(bs_plan p) {
  BS_NVTX("bs_plan_destroy");
  if (!p) return BS_OK;
  if (p->ws && p->ws_owned) {
    cudaSetDevice(p->device);
    cudaFree(p->ws);
  }
  if (p->mono_bins) {
    cudaSetDevice(p->device);
    cudaFree(p->mono_bins);
  }
  for (double *g : {p->gfull, p->gdelta, p->g3d, p->gbin, p->gerr})
    if (g) {
      cudaSetDevice(p->device);
      cudaFree(g);
    }
  delete p;
  return BS_OK;
}

bs_status bs_plan_info(bs_plan p, int64_t *info, int n) {
  BS_NVTX("bs_plan_info");
  if (!p || !info || n < 0) return fail(p, BS_ERR_ARG, "bad arguments");
  int64_t v[7] = {p->M, p->ntrip, p->nf, (int64_t)p->L.total, p->UC, -1,
                  (int64_t)p->levels.size()};
  if (p->counts_ready) {
    int64_t c = 0;
    for (long long t : p->T) c += t > 0;
    v[5] = c;
  }
  for (int k = 0; k < n && k < 7; ++k) info[k] = v[k];
  return BS_OK;
}

bs_status bs_plan_trip_sides(bs_plan p, int64_t *side_host) {
  BS_NVTX("bs_plan_trip_sides");
  if (!p || !side_host) return fail(p, BS_ERR_ARG, "side_host must not be NULL");
  for (int t = 0; t < p->ntrip; ++t) {
    const int lv = p->lev_of_trip[t];
    side_host[t] = lv >= 0 ? p->levels[lv].M : 0;
  }
  return BS_OK;
}

bs_status bs_plan_set_workspace(bs_plan p, void *ws, size_t bytes) {
  BS_NVTX("bs_plan_set_workspace");
  if (!p) return BS_ERR_ARG;
  if (p->ws) return fail(p, BS_ERR_STATE, "workspace already in place");
  if (!ws || bytes < p->L.total || (reinterpret_cast<uintptr_t>(ws) & 255))
    return fail(p, BS_ERR_ARG, "workspace must be 256-byte aligned and at least " +
                                   std::to_string(p->L.total) + " bytes");
  p->ws = static_cast<unsigned char *>(ws);
  p->ws_owned = false;
  cudaStream_t s = nullptr;
  cudaSetDevice(p->device);
  return init_tables(p, s);
}

bs_status bs_grid_load(bs_plan p, const void *vis, const float *ngrid, const uint8_t *flags,
                       void *stream) {
  BS_NVTX("bs_grid_load");
  if (!p) return BS_ERR_ARG;
  if (!vis || (reinterpret_cast<uintptr_t>(vis) & 7))
    return fail(p, BS_ERR_ARG, "vis_dev must be a non-NULL 8-byte aligned device pointer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bs_status st = prepare(p, s);
  if (st != BS_OK) return st;
  const WsLayout &L = p->L;
  for (int c = 0; c < p->nc; ++c) p->valid[c] = flags ? (flags[c] ? 0 : 1) : 1;
  BS_CUDA(cudaMemcpyAsync(p->at<uint8_t>(L.valid), p->valid.data(), p->nc,
                          cudaMemcpyHostToDevice, s));
  const int8_t *lab = p->at<int8_t>(L.label);
  if (p->chans && !ngrid)
    return fail(p, BS_ERR_ARG, "a per-channel sampling plan needs ngrid_dev [nchan][nt][nt]");
  if (ngrid && !p->chans) {
    BS_CUDA(launch_effective_label(p->nt * p->nt, lab, ngrid, p->at<int8_t>(L.efflabel), s));
    st = run_counts(p, p->at<int8_t>(L.efflabel), s);
    if (st != BS_OK) return st;
    p->counts_default = false;
  } else if (!p->counts_ready || !p->counts_default) {
    // geometric counts: with per-channel sampling they decide only which ring
    // triples can close; the denominators come from the occupancy component
    st = run_counts(p, lab, s);
    if (st != BS_OK) return st;
    p->counts_default = true;
  }
  if (p->general) {
    // weights and the Hermitian split applied here; the fields see unit weights
    float2 *gv = p->at<float2>(L.gvis);
    BS_CUDA(launch_general_prep(p->nt, p->nc, p->ubatch, static_cast<const float2 *>(vis), ngrid,
                                lab, gv, s));
    st = enqueue_fields(p, gv, nullptr, s);
  } else if (p->chans) {
    // per-channel weights W V and occupancy masks, as two realisations each
    float2 *gv = p->at<float2>(L.gvis);
    BS_CUDA(launch_chans_prep(p->nt, p->nc, p->ubatch, static_cast<const float2 *>(vis), ngrid,
                              lab, gv, s));
    st = enqueue_fields(p, gv, nullptr, s);
  } else {
    st = enqueue_fields(p, vis, ngrid, s);
  }
  if (st != BS_OK) return st;
  st = delta_reset(p, s);
  if (st != BS_OK) return st;
  p->loaded = true;
  return BS_OK;
}

bs_status bs_counts(bs_plan p, int64_t *tri, int64_t *nnu_host) {
  BS_NVTX("bs_counts");
  if (!p) return BS_ERR_ARG;
  if (p->sticky) return fail(p, BS_ERR_STATE, "plan has a sticky CUDA error: " + p->err);
  if (!p->counts_ready) {
    cudaStream_t s = nullptr;
    bs_status st = prepare(p, s);
    if (st != BS_OK) return st;
    st = run_counts(p, p->at<int8_t>(p->L.label), s);
    if (st != BS_OK) return st;
    p->counts_default = true;
  }
  if (tri)
    for (int t = 0; t < p->ntrip; ++t) tri[t] = p->T[t];
  if (nnu_host) {
    const int nc = p->nc, n2 = 2 * nc - 1;
    for (int i1 = 0; i1 < n2; ++i1)
      for (int i2 = 0; i2 < n2; ++i2) {
        const int j1 = n2 - 1 - i1, j2 = n2 - 1 - i2;
        long long c = p->nnu[(size_t)i1 * n2 + i2];
        if (j1 != i1 || j2 != i2) c += p->nnu[(size_t)j1 * n2 + j2];
        nnu_host[(size_t)i1 * n2 + i2] = c;
      }
  }
  return BS_OK;
}

bs_status bs_mabs(bs_plan p, const int32_t *block, double *out_full, int accumulate, void *stream) {
  BS_NVTX("bs_mabs");
  if (!p) return BS_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!p->loaded) return fail(p, BS_ERR_STATE, "bs_mabs before bs_grid_load");
  bs_status st = prepare(p, s);
  if (st != BS_OK) return st;
  const int nc = p->nc;
  int blk[6] = {0, nc, 0, nc, 0, nc};
  if (block)
    for (int k = 0; k < 6; ++k) blk[k] = block[k];
  for (int k = 0; k < 6; k += 2)
    if (blk[k] < 0 || blk[k + 1] > nc || blk[k] > blk[k + 1])
      return fail(p, BS_ERR_ARG, "channel block out of range");
  if (p->d.precision != BS_PREC_FP32 && p->d.precision != BS_PREC_SPLIT_BF16 &&
      p->d.precision != BS_PREC_SPLIT_FP16)
    return fail(p, BS_ERR_UNSUPPORTED, "precision");
  if (accumulate < 0 || accumulate > 2) return fail(p, BS_ERR_ARG, "accumulate must be 0, 1 or 2");
  if (accumulate == 2) {
    // channel-symmetric accumulation of a cube block S x S x S
    if (out_full) return fail(p, BS_ERR_ARG, "accumulate = 2 writes the collapse sums only (out_full_dev must be NULL)");
    if (blk[0] != blk[2] || blk[0] != blk[4] || blk[1] != blk[3] || blk[1] != blk[5])
      return fail(p, BS_ERR_ARG, "accumulate = 2 needs a cube block (the same range on nu1, nu2, nu3)");
    if (p->d.precision == BS_PREC_FP32 || p->general || p->chans)
      return fail(p, BS_ERR_UNSUPPORTED,
                  "accumulate = 2 needs a split-precision plan without general input or per-channel sampling");
    if (p->sym_state == 1)
      return fail(p, BS_ERR_STATE,
                  "accumulate = 2 after ordinary blocks: reset the collapse sums first");
  } else if (accumulate == 1) {
    bs_status sf = sym_fill(p, s);  // ordinary blocks add to complete sums
    if (sf != BS_OK) return sf;
  }
  if (!out_full && !accumulate) return BS_OK;
  const WsLayout &L = p->L;
  const long long full_bstride = (long long)p->ntrip * nc * nc * nc;
  double *const user_full = out_full;
  if (out_full && (p->general || p->chans)) {  // the real components go to the plan's scratch
    st = general_scratch(p, &p->gfull, &p->gfull_cap, (size_t)p->batch * full_bstride);
    if (st != BS_OK) return st;
    out_full = p->gfull;
  }
  if (out_full) BS_CUDA(launch_full_fill(out_full, full_bstride, p->batch, p->ntrip, nc, blk, 0.0, s));
  if (p->d.precision != BS_PREC_FP32) {
    st = mabs_tc(p, blk, out_full, accumulate, s);
    if (st != BS_OK) return st;
  } else {
    // one launch per image side: work list of ring pairs (i <= j) x column tiles over
    // (l, nu3) with T(i,j,l) > 0 at this side and nu3 valid; rings are this level's slots
    const int nb = p->nb;
    for (int li = 0; li < (int)p->levels.size(); ++li) {
      const Level &lv = p->levels[li];
      if (lv.nslot == 0) continue;
      p->h_cols.clear();
      p->h_ptiles.clear();
      for (int i = 0; i < nb; ++i)
        for (int j = i; j < nb; ++j) {
          const int off = (int)p->h_cols.size();
          for (int l = j; l < nb; ++l) {
            const int t = p->trip_of[((size_t)i * nb + j) * nb + l];
            if (p->T[t] <= 0 || p->lev_of_trip[t] != li) continue;
            for (int n3 = blk[4]; n3 < blk[5]; ++n3)
              if (p->valid[n3]) p->h_cols.push_back(ColEntry{lv.slot_of[l] * nc + n3, t, n3, 0});
          }
          const int ncol = (int)p->h_cols.size() - off;
          for (int c0 = 0; c0 < ncol; c0 += 128)
            p->h_ptiles.push_back(PairTile{lv.slot_of[i], lv.slot_of[j], off, ncol, c0, {0, 0, 0}});
        }
      const int n_r1 = (blk[1] - blk[0] + 15) / 16, n_r2 = (blk[3] - blk[2] + 7) / 8;
      const int npt = (int)p->h_ptiles.size();
      if (npt == 0 || n_r1 == 0 || n_r2 == 0) continue;
      if (npt > 65535) return fail(p, BS_ERR_UNSUPPORTED, "too many column tiles in one block");
      BS_CUDA(cudaMemcpyAsync(p->at<ColEntry>(L.cols), p->h_cols.data(),
                              p->h_cols.size() * sizeof(ColEntry), cudaMemcpyHostToDevice, s));
      BS_CUDA(cudaMemcpyAsync(p->at<PairTile>(L.ptiles), p->h_ptiles.data(),
                              p->h_ptiles.size() * sizeof(PairTile), cudaMemcpyHostToDevice, s));
      ContractArgs a{};
      a.F = p->at<float>(lv.offF);
      a.fstride = (long long)lv.M * lv.M;
      a.bstride = (long long)lv.nslot * nc * lv.M * lv.M;
      a.M2 = lv.M * lv.M;
      a.nc = nc;
      a.cols = p->at<ColEntry>(L.cols);
      a.ptiles = p->at<PairTile>(L.ptiles);
      a.nu1_lo = blk[0];
      a.nu1_hi = blk[1];
      a.nu2_lo = blk[2];
      a.nu2_hi = blk[3];
      a.n_r2 = n_r2;
      // split K until the launch covers several waves of 152 SMs
      const long long ctas = (long long)n_r1 * n_r2 * npt * p->batch;
      int nk = 1;
      const int nchunks = a.M2 / 16;
      while (ctas * nk < 4 * 152 && nk * 2 <= nchunks / 16 && nk < 64) nk *= 2;
      while ((long long)nk * p->batch > 65535) nk /= 2;
      a.nkseg = nk;
      a.kseg_len = ((nchunks + nk - 1) / nk) * 16;
      a.tnorm = p->at<double>(L.tnorm);
      a.out_full = out_full;
      a.full_bstride = full_bstride;
      a.dsum = accumulate ? p->at<double>(L.dsum) : nullptr;
      a.dsum_bstride = (long long)p->ntrip * (2 * nc - 1) * (2 * nc - 1);
      BS_CUDA(launch_contract_simt(a, n_r1 * n_r2, npt, p->batch, s));
    }
  }
  if (out_full)
    BS_CUDA(launch_full_finalize(out_full, full_bstride, p->batch, p->ntrip, nc, blk,
                                 p->at<uint8_t>(L.valid), p->at<double>(L.tnorm), s));
  if (user_full && p->general)
    BS_CUDA(launch_combine4_full(out_full, p->ubatch, p->ntrip, nc, blk, user_full, s));
  if (user_full && p->chans)  // tnorm cancels in the ratio; 1/A stays
    BS_CUDA(launch_ratio2_full(out_full, p->ubatch, p->ntrip, nc, blk, 1.0 / p->normA, user_full, s));
  if (accumulate) {
    accumulate_block_nnu(p, blk);
    p->sym_state = accumulate == 2 ? 2 : 1;
  }
  return BS_OK;
}

bs_status bs_delta_reset(bs_plan p, void *stream) {
  BS_NVTX("bs_delta_reset");
  if (!p) return BS_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bs_status st = prepare(p, s);
  if (st != BS_OK) return st;
  return delta_reset(p, s);
}

bs_status bs_delta_export(bs_plan p, double *sums_dev, int64_t *nnu_host, void *stream) {
  BS_NVTX("bs_delta_export");
  if (!p || (!sums_dev && !nnu_host)) return fail(p, BS_ERR_ARG, "bs_delta_export: nothing to export");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!p->loaded) return fail(p, BS_ERR_STATE, "bs_delta_export before bs_grid_load");
  bs_status st = prepare(p, s);
  if (st != BS_OK) return st;
  st = check_device_error(p, s);
  if (st != BS_OK) return st;
  st = sym_fill(p, s);
  if (st != BS_OK) return st;
  const size_t n2 = (size_t)(2 * p->nc - 1);
  if (sums_dev)
    BS_CUDA(cudaMemcpyAsync(sums_dev, p->at<double>(p->L.dsum),
                            (size_t)p->batch * p->ntrip * n2 * n2 * sizeof(double),
                            cudaMemcpyDeviceToDevice, s));
  if (nnu_host)
    for (size_t k = 0; k < p->nnu.size(); ++k) nnu_host[k] = p->nnu[k];
  return BS_OK;
}

bs_status bs_delta_import(bs_plan p, const double *sums_dev, const int64_t *nnu_host, int add,
                          void *stream) {
  BS_NVTX("bs_delta_import");
  if (!p || !sums_dev || !nnu_host || (add != 0 && add != 1))
    return fail(p, BS_ERR_ARG, "bs_delta_import: sums_dev and nnu_host are required, add is 0 or 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!p->loaded) return fail(p, BS_ERR_STATE, "bs_delta_import before bs_grid_load");
  bs_status st = prepare(p, s);
  if (st != BS_OK) return st;
  st = sym_fill(p, s);  // the imported sums add to complete ones
  if (st != BS_OK) return st;
  p->sym_state = 1;
  const size_t n2 = (size_t)(2 * p->nc - 1);
  const long long n = (long long)p->batch * p->ntrip * n2 * n2;
  double *d = p->at<double>(p->L.dsum);
  if (add)
    BS_CUDA(launch_add_f64(d, sums_dev, n, s));
  else
    BS_CUDA(cudaMemcpyAsync(d, sums_dev, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  for (size_t k = 0; k < p->nnu.size(); ++k) p->nnu[k] = (add ? p->nnu[k] : 0) + nnu_host[k];
  p->nnu_dirty = true;
  // the imported sums may touch any separation and any plane: the next reset zeroes all
  p->dsum_clean = false;
  return BS_OK;
}

// Folded collapsed plane of every (or every closable) ring triple into out; a
// general plan normalises its four real components into scratch and combines
// them into complex planes.
static bs_status delta_out(bs_plan p, double *out, bool closable, cudaStream_t s) {
  const int npl = closable ? (int)p->clos.size() : p->ntrip;
  const long long n2 = 2LL * p->nc - 1, per = (long long)npl * n2 * n2;
  double *dst = out;
  if (p->general || p->chans) {
    bs_status st = general_scratch(p, &p->gdelta, &p->gdelta_cap, (size_t)p->batch * per);
    if (st != BS_OK) return st;
    dst = p->gdelta;
  }
  BS_CUDA(launch_delta_norm(p->at<double>(p->L.dsum), p->at<long long>(p->L.nnu),
                            p->at<double>(p->L.tnorm), dst, p->batch, p->ntrip, p->nc,
                            closable ? p->at<int>(p->L.clos) : nullptr,
                            closable ? npl : 0, p->at<double>(p->L.tmp3d), s));
  if (p->general) BS_CUDA(launch_combine4(dst, per, p->ubatch, out, s));
  // per-channel sampling: (summed numerators) / (A x summed denominators)
  if (p->chans && out) BS_CUDA(launch_ratio2(dst, per, p->ubatch, 1.0 / p->normA, out, s));
  return BS_OK;
}

// Eq. (dft) of every (or every closable) ring triple into out; general plans as above.
static bs_status bs3d_out(bs_plan p, double *out, bool closable, cudaStream_t s) {
  const int npl = closable ? (int)p->clos.size() : p->ntrip;
  if (p->chans) {
    // the ratio planes of every ring triple, rewritten as collapse sums that the
    // delay transform normalises back, then transformed like ordinary planes
    bs_status st = delta_out(p, nullptr, false, s);  // components into gdelta only
    if (st != BS_OK) return st;
    const long long n2 = 2LL * p->nc - 1, per = (long long)p->ntrip * n2 * n2;
    st = general_scratch(p, &p->g3d, &p->g3d_cap, (size_t)2 * p->ubatch * per);
    if (st != BS_OK) return st;
    double *ratio = p->g3d, *sums = p->g3d + (size_t)p->ubatch * per;
    BS_CUDA(launch_ratio2(p->gdelta, per, p->ubatch, 1.0 / p->normA, ratio, s));
    BS_CUDA(launch_ratio_to_sums(ratio, p->at<long long>(p->L.nnu), p->at<double>(p->L.tnorm),
                                 p->ubatch, p->ntrip, p->nc, sums, s));
    BS_CUDA(launch_bs3d(sums, p->at<long long>(p->L.nnu), p->at<double>(p->L.tnorm),
                        p->at<float2>(p->L.tmp3d), out, p->ubatch, p->ntrip, p->nc,
                        p->at<float2>(p->L.twN), p->radN, p->scale3d,
                        closable ? p->at<int>(p->L.clos) : nullptr, closable ? npl : 0, s));
    return BS_OK;
  }
  const long long per = (long long)npl * p->nc * p->nc;
  double *dst = out;
  if (p->general) {
    bs_status st = general_scratch(p, &p->g3d, &p->g3d_cap, (size_t)p->batch * per);
    if (st != BS_OK) return st;
    dst = p->g3d;
  }
  BS_CUDA(launch_bs3d(p->at<double>(p->L.dsum), p->at<long long>(p->L.nnu),
                      p->at<double>(p->L.tnorm), p->at<float2>(p->L.tmp3d), dst, p->batch,
                      p->ntrip, p->nc, p->at<float2>(p->L.twN), p->radN, p->scale3d,
                      closable ? p->at<int>(p->L.clos) : nullptr, closable ? npl : 0, s));
  if (p->general) BS_CUDA(launch_combine4(dst, per, p->ubatch, out, s));
  return BS_OK;
}

bs_status bs_mabs_delta(bs_plan p, double *out, void *stream) {
  BS_NVTX("bs_mabs_delta");
  if (!p || !out) return fail(p, BS_ERR_ARG, "out_dev must not be NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!p->loaded) return fail(p, BS_ERR_STATE, "bs_mabs_delta before bs_grid_load");
  bs_status st = prepare(p, s);
  if (st != BS_OK) return st;
  st = check_device_error(p, s);
  if (st != BS_OK) return st;
  st = upload_nnu(p, s);
  if (st != BS_OK) return st;
  st = sym_fill(p, s);
  if (st != BS_OK) return st;
  return delta_out(p, out, false, s);
}

bs_status bs_mabs_delta_closable(bs_plan p, double *out, void *stream) {
  BS_NVTX("bs_mabs_delta_closable");
  if (!p || !out) return fail(p, BS_ERR_ARG, "out_dev must not be NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!p->loaded) return fail(p, BS_ERR_STATE, "bs_mabs_delta_closable before bs_grid_load");
  bs_status st = prepare(p, s);
  if (st != BS_OK) return st;
  st = check_device_error(p, s);
  if (st != BS_OK) return st;
  st = upload_nnu(p, s);
  if (st != BS_OK) return st;
  st = sym_fill(p, s);
  if (st != BS_OK) return st;
  return delta_out(p, out, true, s);
}

bs_status bs_bs3d(bs_plan p, double *out, void *stream) {
  BS_NVTX("bs_bs3d");
  if (!p || !out) return fail(p, BS_ERR_ARG, "out_dev must not be NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!p->loaded) return fail(p, BS_ERR_STATE, "bs_bs3d before bs_grid_load");
  bs_status st = prepare(p, s);
  if (st != BS_OK) return st;
  st = check_device_error(p, s);
  if (st != BS_OK) return st;
  st = upload_nnu(p, s);
  if (st != BS_OK) return st;
  st = sym_fill(p, s);
  if (st != BS_OK) return st;
  return bs3d_out(p, out, false, s);
}

bs_status bs_bs3d_closable(bs_plan p, double *out, void *stream) {
  BS_NVTX("bs_bs3d_closable");
  if (!p || !out) return fail(p, BS_ERR_ARG, "out_dev must not be NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!p->loaded) return fail(p, BS_ERR_STATE, "bs_bs3d_closable before bs_grid_load");
  bs_status st = prepare(p, s);
  if (st != BS_OK) return st;
  st = check_device_error(p, s);
  if (st != BS_OK) return st;
  st = upload_nnu(p, s);
  if (st != BS_OK) return st;
  st = sym_fill(p, s);
  if (st != BS_OK) return st;
  return bs3d_out(p, out, true, s);
}

bs_status bs_check_hermitian(bs_plan p, const void *vis, double tol, void *stream) {
  BS_NVTX("bs_check_hermitian");
  if (!p || !vis) return fail(p, BS_ERR_ARG, "vis_dev must not be NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bs_status st = prepare(p, s);
  if (st != BS_OK) return st;
  float *hm = p->at<float>(p->L.herm);
  BS_CUDA(cudaMemsetAsync(hm, 0, 2 * sizeof(float), s));
  BS_CUDA(launch_hermitian_check(static_cast<const float2 *>(vis), p->ubatch, p->nc, p->nt,
                                 p->at<int8_t>(p->L.label), hm, hm + 1, s));
  float h[2];
  BS_CUDA(cudaMemcpyAsync(h, hm, sizeof(h), cudaMemcpyDeviceToHost, s));
  BS_CUDA(cudaStreamSynchronize(s));
  if (h[0] > tol * h[1])
    return fail(p, BS_ERR_NOT_HERMITIAN,
                "max |V(-U) - conj V(U)| = " + std::to_string(h[0]) + " exceeds tol * max|V| = " +
                    std::to_string(tol * h[1]));
  return BS_OK;
}

}  // extern "C"

// The normalised collapse components of a per-channel sampling plan (summed
// numerators and denominators, internal realisations 2b and 2b + 1) in the
// full or the closable layout, for the error bound of the ratio.
bs_status bsi::chans_components(bs_plan p, bool closable, cudaStream_t s, const double **comp) {
  bs_status st = delta_out(p, nullptr, closable, s);
  if (st != BS_OK) return st;
  *comp = p->gdelta;
  return BS_OK;
}
