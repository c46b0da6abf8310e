// Batched Monte Carlo over realisations of uneven shapes (Section 4 uses 250
// realisations to estimate the ensemble mean and 1-sigma of the MABS and the
// 3D bispectrum).
//
// An ensemble holds shape groups; each group is a plan (its own grid side,
// channels, rings) processing `batch` realisations per run.  One run enqueues
// only kernel launches and memsets, so it can be captured in a CUDA graph:
//   per group  : shell masks + field FFTs (colpass, rowpass), zero the sums
//   all groups : ONE persistent tensor-core contraction over the tiles of every
//                group and realisation (full channel cube of each group; on a
//                cube of 64 channels or more, one ordering of a repeated
//                ring's channels, the other filled in per group afterwards)
//   per group  : fold/normalise (collapsed plane) and Eq. (dft), then a
//                per-bin Welford update of mean and M2 over the realisations.
// Tile lists, counts and the sampling N_nu depend only on the shapes and are
// built once.  The first run executes eagerly; later runs with use_graph
// replay the captured graph.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <vector>

#include "plan_internal.h"

using namespace bsi;

namespace {

// Welford update over the batch dimension: x[b][n] -> (count, mean, M2)[n].
__global__ void k_welford(const double *__restrict__ x, int batch, long long n, double *cnt,
                          double *mean, double *m2) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    double c = cnt[j], mu = mean[j], s = m2[j];
    for (int b = 0; b < batch; ++b) {
      const double v = x[(long long)b * n + j];
      if (v != v) continue;
      c += 1.0;
      const double d = v - mu;
      mu += d / c;
      s += d * (v - mu);
    }
    cnt[j] = c;
    mean[j] = mu;
    m2[j] = s;
  }
}

__global__ void k_welford_final(long long n, const double *cnt, const double *mean,
                                const double *m2, double *mean_out, double *var_out) {
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    const double c = cnt[j];
    if (mean_out) mean_out[j] = c > 0 ? mean[j] : nan;
    if (var_out) var_out[j] = c > 1 ? m2[j] / (c - 1.0) : nan;
  }
}

struct Group {
  bs_plan plan = nullptr;
  std::vector<uint8_t> flags;   // [nc], 1 = flagged (empty = none)
  const void *vis = nullptr;    // [batch][nc][nt][nt] c64, caller-owned
  double *dout = nullptr;       // [batch][ntrip][n2][n2]
  double *bout = nullptr;       // [batch][ntrip][nc][nc]
  double *stats = nullptr;      // 3 x (delta bins) then 3 x (bs3d bins): cnt, mean, m2
  long long nd = 0, nb3 = 0;    // bins per realisation
  int blk[6] = {0, 0, 0, 0, 0, 0};  // channel block each run contracts (set at create: full cube)
  // channel symmetry of repeated rings (a cube block of 64 channels or more):
  // the contraction covers one ordering, k_symmetrize the other, inside box
  bool sym = false;
  int box[4] = {0, -1, 0, -1};
};

}  // namespace

struct bs_mc_s {
  std::vector<Group> groups;
  std::string err = "no error";
  bool prepared = false, ran_once = false;
  long long runs = 0;
  // concatenated tensor-core work
  ColEntry *cols = nullptr;
  TcTile *tiles = nullptr;
  TcGroup *tcgroups = nullptr;
  unsigned char *maps = nullptr;
  int *errw = nullptr;
  int ntiles = 0, nsm = 152;
  int f16 = 0;                  // 1: split-FP16 groups (two-product contraction)
  int min_tiles_factor = 2;     // autotuner knob: K splitting target (tiles per SM)
  int tile_order = 0;           // autotuner knob: 0 longest K first, 1 ring-pair order
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // graphs are captured and replayed on a private stream (the legacy default
  // stream cannot be captured), ordered with the caller's stream by events
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

namespace {

bs_status mfail(bs_mc m, bs_status s, const std::string &msg) {
  if (m) m->err = msg;  // a NULL handle has nowhere to keep the message
  return s;
}

#define MC_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e__ = (call);                                                              \
    if (e__ != cudaSuccess) return mfail(m, BS_ERR_CUDA, std::string(#call) + ": " +       \
                                                      cudaGetErrorString(e__));             \
  } while (0)

bs_status plan_status(bs_mc m, bs_plan p, bs_status st) {
  if (st != BS_OK) m->err = std::string("group plan: ") + bs_last_error(p);
  return st;
}

// Counts, tensor maps, full-cube sampling and the concatenated tile list.
bs_status mc_prepare(bs_mc m, cudaStream_t s) {
  if (m->prepared) return BS_OK;
  std::vector<ColEntry> cols;
  std::vector<TcTile> tiles;
  std::vector<TcGroup> tgs;
  std::vector<unsigned char> maps;
  // pass 1: per-group setup and column offsets
  std::vector<size_t> col_base;
  for (size_t g = 0; g < m->groups.size(); ++g) {
    bs_plan p = m->groups[g].plan;
    bs_status st = prepare(p, s);
    if (st != BS_OK) return plan_status(m, p, st);
    if (!p->counts_ready || !p->counts_default) {
      st = run_counts(p, p->at<int8_t>(p->L.label), s);
      if (st != BS_OK) return plan_status(m, p, st);
      p->counts_default = true;
    }
    st = ensure_tensor_maps(p, s);
    if (st != BS_OK) return plan_status(m, p, st);
    // channel validity from the group's flags; the full cube is contracted
    const std::vector<uint8_t> &fl = m->groups[g].flags;
    for (int c = 0; c < p->nc; ++c) p->valid[c] = (fl.empty() || !fl[c]) ? 1 : 0;
    MC_CUDA(cudaMemcpyAsync(p->at<uint8_t>(p->L.valid), p->valid.data(), p->nc,
                            cudaMemcpyHostToDevice, s));
    std::fill(p->nnu.begin(), p->nnu.end(), 0LL);
    accumulate_block_nnu(p, m->groups[g].blk);
    st = upload_nnu(p, s);
    if (st != BS_OK) return plan_status(m, p, st);
  }
  // pass 2: tiles of every (group, level); column pointers fixed up after the
  // device buffer exists
  for (size_t g = 0; g < m->groups.size(); ++g) {
    bs_plan p = m->groups[g].plan;
    const size_t c0 = cols.size();
    const int *blk = m->groups[g].blk;
    // a cube block S x S x S is closed under exchanging the channels of a repeated
    // ring: one ordering is contracted.  Below 64 channels every pair rectangle of a
    // one-ring pair operand straddles the diagonal and nothing would be saved.
    Group &gr = m->groups[g];
    const int w = blk[1] - blk[0];
    gr.sym = blk[0] == blk[2] && blk[0] == blk[4] && blk[1] == blk[3] && blk[1] == blk[5] &&
             w >= 64 && !p->sym_trips.empty();
    if (gr.sym) {
      const int nc = p->nc;
      gr.box[0] = gr.box[2] = std::max(0, nc - w);
      gr.box[1] = gr.box[3] = std::min(2 * nc - 2, nc + w - 2);
    }
    std::vector<ColEntry> gc;
    std::vector<TcTile> gt;
    std::vector<TcGroup> G = build_tc_work(p, blk, (int)tgs.size(), gc, nullptr, gt, nullptr,
                                           gr.sym ? 2 : 1, m->min_tiles_factor * m->nsm);
    for (TcTile &t : gt) t.col_off += (int)c0;  // offsets into the concatenated list
    cols.insert(cols.end(), gc.begin(), gc.end());
    tiles.insert(tiles.end(), gt.begin(), gt.end());
    tgs.insert(tgs.end(), G.begin(), G.end());
    for (const Level &lv : p->levels) {
      const unsigned char *mp = reinterpret_cast<const unsigned char *>(lv.maps);
      maps.insert(maps.end(), mp, mp + sizeof(lv.maps));
    }
  }
  // order 0: the longest K ranges first across all groups (balance of the
  // persistent launch); order 1: group, level and ring pair order as built
  // (neighbouring CTA pairs share field rows in L2)
  if (m->tile_order == 0)
    std::stable_sort(tiles.begin(), tiles.end(), [&](const TcTile &x, const TcTile &y) {
      return tgs[x.group].kseg_len > tgs[y.group].kseg_len;
    });
  else
    std::stable_sort(tiles.begin(), tiles.end(), [&](const TcTile &x, const TcTile &y) {
      return x.group < y.group;
    });
  MC_CUDA(cudaMalloc(&m->cols, std::max<size_t>(1, cols.size()) * sizeof(ColEntry)));
  MC_CUDA(cudaMalloc(&m->tiles, std::max<size_t>(1, tiles.size()) * sizeof(TcTile)));
  MC_CUDA(cudaMalloc(&m->tcgroups, tgs.size() * sizeof(TcGroup)));
  MC_CUDA(cudaMalloc(&m->maps, maps.size()));
  MC_CUDA(cudaMalloc(&m->errw, sizeof(int)));
  for (TcGroup &G : tgs) G.cols = m->cols;  // tile col_off are global offsets
  if (!cols.empty())
    MC_CUDA(cudaMemcpy(m->cols, cols.data(), cols.size() * sizeof(ColEntry), cudaMemcpyHostToDevice));
  if (!tiles.empty())
    MC_CUDA(cudaMemcpy(m->tiles, tiles.data(), tiles.size() * sizeof(TcTile), cudaMemcpyHostToDevice));
  MC_CUDA(cudaMemcpy(m->tcgroups, tgs.data(), tgs.size() * sizeof(TcGroup), cudaMemcpyHostToDevice));
  MC_CUDA(cudaMemcpy(m->maps, maps.data(), maps.size(), cudaMemcpyHostToDevice));
  MC_CUDA(cudaMemset(m->errw, 0, sizeof(int)));
  m->ntiles = (int)tiles.size();
  m->prepared = true;
  return BS_OK;
}

// One run: kernel launches and memsets only (capturable).
bs_status mc_enqueue(bs_mc m, cudaStream_t s) {
  for (Group &gr : m->groups) {
    bs_plan p = gr.plan;
    bs_status st = enqueue_fields(p, gr.vis, nullptr, s);
    if (st != BS_OK) return plan_status(m, p, st);
    const size_t n2 = (size_t)(2 * p->nc - 1);
    MC_CUDA(cudaMemsetAsync(p->at<double>(p->L.dsum), 0,
                            (size_t)p->batch * p->ntrip * n2 * n2 * sizeof(double), s));
  }
  TcArgs a{};
  a.groups = m->tcgroups;
  a.maps = m->maps;
  a.tiles = m->tiles;
  a.ntiles = m->ntiles;
  a.err = m->errw;
  a.wait_limit_ns = 2000000000LL;
  a.stall_test = 0;
  a.f16 = m->f16;
  MC_CUDA(launch_contract_tc(a, m->nsm, s));
  for (Group &gr : m->groups) {
    bs_plan p = gr.plan;
    const WsLayout &L = p->L;
    if (gr.sym)
      MC_CUDA(launch_symmetrize(p->at<double>(L.dsum), p->at<int>(L.symtrips),
                                (int)p->sym_trips.size(), p->batch, p->ntrip, p->nc, gr.box, s));
    MC_CUDA(launch_delta_norm(p->at<double>(L.dsum), p->at<long long>(L.nnu),
                              p->at<double>(L.tnorm), gr.dout, p->batch, p->ntrip, p->nc,
                              nullptr, 0, p->at<double>(L.tmp3d), s));
    MC_CUDA(launch_bs3d(p->at<double>(L.dsum), p->at<long long>(L.nnu), p->at<double>(L.tnorm),
                        p->at<float2>(L.tmp3d), gr.bout, p->batch, p->ntrip, p->nc,
                        p->at<float2>(L.twN), p->radN, p->scale3d, nullptr, 0, s));
    const int blocks = (int)std::min<long long>((gr.nd + 255) / 256, 4096);
    k_welford<<<blocks, 256, 0, s>>>(gr.dout, p->batch, gr.nd, gr.stats, gr.stats + gr.nd,
                                     gr.stats + 2 * gr.nd);
    MC_CUDA(cudaGetLastError());
    double *s3 = gr.stats + 3 * gr.nd;
    const int blocks3 = (int)std::min<long long>((gr.nb3 + 255) / 256, 4096);
    k_welford<<<blocks3, 256, 0, s>>>(gr.bout, p->batch, gr.nb3, s3, s3 + gr.nb3, s3 + 2 * gr.nb3);
    MC_CUDA(cudaGetLastError());
  }
  return BS_OK;
}

// Drop the tile lists and the captured graph (tuning changed).
void mc_unprepare(bs_mc m) {
  if (m->exec) cudaGraphExecDestroy(m->exec);
  if (m->graph) cudaGraphDestroy(m->graph);
  m->exec = nullptr;
  m->graph = nullptr;
  cudaFree(m->cols);
  cudaFree(m->tiles);
  cudaFree(m->tcgroups);
  cudaFree(m->maps);
  cudaFree(m->errw);
  m->cols = nullptr;
  m->tiles = nullptr;
  m->tcgroups = nullptr;
  m->maps = nullptr;
  m->errw = nullptr;
  m->prepared = false;
  m->ran_once = false;
}

// Shape signature of the ensemble (cache key of the autotuner).
std::string mc_signature(bs_mc m) {
  std::ostringstream o;
  o << "sm" << m->nsm;
  for (const Group &gr : m->groups) {
    const bs_plan p = gr.plan;
    o << "|nt" << p->nt << "nc" << p->nc << "M" << p->M << "b" << p->batch << "e";
    for (double e : p->edges) o << ":" << e;
    o << "blk";
    for (int k = 0; k < 6; ++k) o << ":" << gr.blk[k];
  }
  return o.str();
}

struct Tuned {
  int tiles_per_sm = 2, order = 0;
  double ms = 0.0;
};

std::map<std::string, Tuned> read_cache(const char *path) {
  std::map<std::string, Tuned> out;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    const size_t q0 = line.find('"');
    const size_t q1 = q0 == std::string::npos ? q0 : line.find('"', q0 + 1);
    const size_t t = line.find("\"tiles_per_sm\":");
    const size_t o = line.find("\"order\":");
    const size_t ms = line.find("\"ms\":");
    if (q1 == std::string::npos || t == std::string::npos || ms == std::string::npos) continue;
    Tuned v;
    v.tiles_per_sm = std::atoi(line.c_str() + t + 15);
    v.order = o == std::string::npos ? 0 : std::atoi(line.c_str() + o + 8);
    v.ms = std::atof(line.c_str() + ms + 5);
    out[line.substr(q0 + 1, q1 - q0 - 1)] = v;
  }
  return out;
}

void write_cache(const char *path, const std::map<std::string, Tuned> &c) {
  const std::string tmp = std::string(path) + ".tmp";
  {
    std::ofstream f(tmp);
    f << "{\n";
    size_t k = 0;
    for (const auto &kv : c)
      f << "\"" << kv.first << "\": {\"tiles_per_sm\": " << kv.second.tiles_per_sm
        << ", \"order\": " << kv.second.order << ", \"ms\": " << kv.second.ms << "}"
        << (++k < c.size() ? "," : "") << "\n";
    f << "}\n";
  }
  std::rename(tmp.c_str(), path);
}

}  // namespace

extern "C" {

bs_status bs_mc_autotune(bs_mc m, const char *cache_path, int *chosen, void *stream) {
  BS_NVTX("bs_mc_autotune");
  if (!m) return BS_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (size_t g = 0; g < m->groups.size(); ++g)
    if (!m->groups[g].vis) return mfail(m, BS_ERR_STATE, "autotune needs every group's input");
  const std::string key = mc_signature(m);
  std::map<std::string, Tuned> cache;
  if (cache_path) cache = read_cache(cache_path);
  auto hit = cache.find(key);
  Tuned best;
  best.ms = -1.0;
  // one candidate: prepare its tiles, one warm-up run, two timed runs
  auto trial = [&](int tps, int order, double *ms_out) -> bs_status {
    mc_unprepare(m);
    m->min_tiles_factor = tps;
    m->tile_order = order;
    bs_status st = mc_prepare(m, s);
    if (st != BS_OK) return st;
    st = mc_enqueue(m, s);
    if (st != BS_OK) return st;
    cudaEvent_t e0, e1;
    MC_CUDA(cudaEventCreate(&e0));
    MC_CUDA(cudaEventCreate(&e1));
    MC_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < 2 && st == BS_OK; ++r) st = mc_enqueue(m, s);
    MC_CUDA(cudaEventRecord(e1, s));
    MC_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    MC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_out = ms / 2;
    return st;
  };
  if (hit != cache.end()) {
    best = hit->second;
  } else {
    // coordinate search: the K extent of the tiles (split target, tiles per SM),
    // then the tile order at the best K extent
    for (int c : {1, 2, 4, 8, 16}) {
      double ms = 0;
      bs_status st = trial(c, 0, &ms);
      if (st != BS_OK) return st;
      if (best.ms < 0 || ms < best.ms) {
        best.tiles_per_sm = c;
        best.order = 0;
        best.ms = ms;
      }
    }
    double ms = 0;
    bs_status st = trial(best.tiles_per_sm, 1, &ms);
    if (st != BS_OK) return st;
    if (ms < best.ms) {
      best.order = 1;
      best.ms = ms;
    }
    if (cache_path) {
      cache[key] = best;
      write_cache(cache_path, cache);
    }
  }
  mc_unprepare(m);
  m->min_tiles_factor = best.tiles_per_sm;
  m->tile_order = best.order;
  bs_status st = mc_prepare(m, s);
  if (st != BS_OK) return st;
  for (Group &gr : m->groups)  // tuning runs do not count as realisations
    MC_CUDA(cudaMemsetAsync(gr.stats, 0, (size_t)3 * (gr.nd + gr.nb3) * 8, s));
  m->runs = 0;
  if (chosen) *chosen = best.tiles_per_sm;
  return BS_OK;
}

bs_status bs_mc_tuning(bs_mc m, int *tiles_per_sm, int *tile_order) {
  BS_NVTX("bs_mc_tuning");
  if (!m) return BS_ERR_ARG;
  if (tiles_per_sm) *tiles_per_sm = m->min_tiles_factor;
  if (tile_order) *tile_order = m->tile_order;
  return BS_OK;
}

bs_status bs_mc_set_block(bs_mc m, int group, const int32_t *block_host) {
  BS_NVTX("bs_mc_set_block");
  if (!m || group < 0 || group >= (int)m->groups.size() || !block_host)
    return mfail(m, BS_ERR_ARG, "bs_mc_set_block: bad arguments");
  Group &gr = m->groups[group];
  const int nc = gr.plan->nc;
  for (int k = 0; k < 6; k += 2)
    if (block_host[k] < 0 || block_host[k + 1] > nc || block_host[k] >= block_host[k + 1])
      return mfail(m, BS_ERR_ARG, "bs_mc_set_block: block out of range");
  for (int k = 0; k < 6; ++k) gr.blk[k] = block_host[k];
  mc_unprepare(m);  // tiles and sampling change: rebuilt (and recaptured) on the next run
  return BS_OK;
}

const char *bs_mc_last_error(bs_mc m) { return m ? m->err.c_str() : bs_last_error(nullptr); }

bs_status bs_mc_create(const bs_plan_desc *descs, int ngroups, bs_mc *out) {
  BS_NVTX("bs_mc_create");
  if (!descs || !out || ngroups < 1 || ngroups > 64) return fail(nullptr, BS_ERR_ARG, "bad arguments");
  *out = nullptr;
  bs_mc m = new bs_mc_s();
  for (int g = 0; g < ngroups; ++g) {
    if ((descs[g].precision != BS_PREC_SPLIT_BF16 && descs[g].precision != BS_PREC_SPLIT_FP16) ||
        descs[g].precision != descs[0].precision) {
      delete m;
      return fail(nullptr, BS_ERR_ARG,
                  "Monte Carlo groups share one tensor-core precision (split BF16 or split FP16)");
    }
    if (descs[g].general || descs[g].chan_sampling) {
      delete m;
      return fail(nullptr, BS_ERR_UNSUPPORTED, "Monte Carlo groups take Hermitian input with one sampling grid");
    }
    m->f16 = descs[0].precision == BS_PREC_SPLIT_FP16 ? 1 : 0;
    Group gr;
    bs_status st = bs_plan_create(&descs[g], &gr.plan);
    if (st != BS_OK) {
      bs_mc_destroy(m);
      return st;
    }
    bs_plan p = gr.plan;
    m->nsm = p->nsm;
    const int full[6] = {0, p->nc, 0, p->nc, 0, p->nc};
    for (int k = 0; k < 6; ++k) gr.blk[k] = full[k];
    const size_t n2 = (size_t)(2 * p->nc - 1);
    gr.nd = (long long)p->ntrip * n2 * n2;
    gr.nb3 = (long long)p->ntrip * p->nc * p->nc;
    if (inject_fail("mc_alloc") ||
        cudaMalloc(&gr.dout, (size_t)p->batch * gr.nd * 8) != cudaSuccess ||
        cudaMalloc(&gr.bout, (size_t)p->batch * gr.nb3 * 8) != cudaSuccess ||
        cudaMalloc(&gr.stats, (size_t)3 * (gr.nd + gr.nb3) * 8) != cudaSuccess) {
      cudaGetLastError();
      m->groups.push_back(gr);
      bs_mc_destroy(m);
      return fail(nullptr, BS_ERR_OOM, "Monte Carlo buffers do not fit on the device");
    }
    cudaMemset(gr.stats, 0, (size_t)3 * (gr.nd + gr.nb3) * 8);
    m->groups.push_back(gr);
  }
  *out = m;
  return BS_OK;
}

bs_status bs_mc_destroy(bs_mc m) {
  BS_NVTX("bs_mc_destroy");
  if (!m) return BS_OK;
  mc_unprepare(m);
  if (m->gstream) {
    cudaStreamSynchronize(m->gstream);
    cudaStreamDestroy(m->gstream);
    cudaEventDestroy(m->ev_in);
    cudaEventDestroy(m->ev_out);
  }
  for (Group &gr : m->groups) {
    cudaFree(gr.dout);
    cudaFree(gr.bout);
    cudaFree(gr.stats);
    bs_plan_destroy(gr.plan);
  }
  delete m;
  return BS_OK;
}

bs_status bs_mc_info(bs_mc m, int group, int64_t *info_host, int n) {
  BS_NVTX("bs_mc_info");
  if (!m || group < 0 || group >= (int)m->groups.size()) return BS_ERR_ARG;
  return bs_plan_info(m->groups[group].plan, info_host, n);
}

bs_status bs_mc_set_input(bs_mc m, int group, const void *vis_dev) {
  BS_NVTX("bs_mc_set_input");
  if (!m || group < 0 || group >= (int)m->groups.size())
    return m ? mfail(m, BS_ERR_ARG, "bad group") : BS_ERR_ARG;
  if (!vis_dev || (reinterpret_cast<uintptr_t>(vis_dev) & 7))
    return mfail(m, BS_ERR_ARG, "vis_dev must be a non-NULL 8-byte aligned device pointer");
  if (m->groups[group].vis != vis_dev && m->exec) {  // the captured graph reads the old buffer
    cudaGraphExecDestroy(m->exec);
    cudaGraphDestroy(m->graph);
    m->exec = nullptr;
    m->graph = nullptr;
  }
  m->groups[group].vis = vis_dev;
  return BS_OK;
}

bs_status bs_mc_set_flags(bs_mc m, int group, const uint8_t *flags_host) {
  BS_NVTX("bs_mc_set_flags");
  if (!m || group < 0 || group >= (int)m->groups.size())
    return m ? mfail(m, BS_ERR_ARG, "bad group") : BS_ERR_ARG;
  Group &gr = m->groups[group];
  if (flags_host)
    gr.flags.assign(flags_host, flags_host + gr.plan->nc);
  else
    gr.flags.clear();
  mc_unprepare(m);  // validity, sampling and the graph depend on the flags
  return BS_OK;
}

bs_status bs_mc_set_tuning(bs_mc m, int tiles_per_sm) {
  BS_NVTX("bs_mc_set_tuning");
  if (!m || tiles_per_sm < 1 || tiles_per_sm > 64) return BS_ERR_ARG;
  if (m->prepared) return mfail(m, BS_ERR_STATE, "tuning must be set before the first run");
  m->min_tiles_factor = tiles_per_sm;
  return BS_OK;
}

bs_status bs_mc_run(bs_mc m, int use_graph, void *stream) {
  BS_NVTX("bs_mc_run");
  if (!m) return BS_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (size_t g = 0; g < m->groups.size(); ++g)
    if (!m->groups[g].vis)
      return mfail(m, BS_ERR_STATE, "group " + std::to_string(g) + " has no input (bs_mc_set_input)");
  bs_status st = mc_prepare(m, s);
  if (st != BS_OK) return st;
  if (!use_graph || !m->ran_once) {
    st = mc_enqueue(m, s);
    if (st != BS_OK) return st;
    m->ran_once = true;
  } else {
    if (!m->gstream) {
      MC_CUDA(cudaStreamCreateWithFlags(&m->gstream, cudaStreamNonBlocking));
      MC_CUDA(cudaEventCreateWithFlags(&m->ev_in, cudaEventDisableTiming));
      MC_CUDA(cudaEventCreateWithFlags(&m->ev_out, cudaEventDisableTiming));
    }
    cudaStream_t gs = m->gstream;
    MC_CUDA(cudaEventRecord(m->ev_in, s));
    MC_CUDA(cudaStreamWaitEvent(gs, m->ev_in, 0));
    if (!m->exec) {
      MC_CUDA(cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal));
      bs_status st2 = mc_enqueue(m, gs);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(gs, &g);
      if (st2 != BS_OK) {
        if (g) cudaGraphDestroy(g);
        return st2;
      }
      MC_CUDA(e);
      m->graph = g;
      MC_CUDA(cudaGraphInstantiate(&m->exec, g, 0));
    }
    MC_CUDA(cudaGraphLaunch(m->exec, gs));
    MC_CUDA(cudaEventRecord(m->ev_out, gs));
    MC_CUDA(cudaStreamWaitEvent(s, m->ev_out, 0));
  }
  ++m->runs;
  return BS_OK;
}

bs_status bs_mc_reset(bs_mc m, void *stream) {
  BS_NVTX("bs_mc_reset");
  if (!m) return BS_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (Group &gr : m->groups)
    MC_CUDA(cudaMemsetAsync(gr.stats, 0, (size_t)3 * (gr.nd + gr.nb3) * 8, s));
  m->runs = 0;
  return BS_OK;
}

// Checkpoint file: "BSMCCKP1", then (little-endian host integers) the signature
// length and the ensemble's shape signature, the caller's counter, the runs,
// the tuning (tiles per SM, order), the number of groups, and per group its bin
// counts nd, nb3 followed by the 3 (nd + nb3) FP64 Welford values (count,
// mean, M2 of the collapsed plane, then of the 3D bispectrum).
static const char kCkptMagic[8] = {'B', 'S', 'M', 'C', 'C', 'K', 'P', '1'};

bs_status bs_mc_checkpoint(bs_mc m, const char *path, uint64_t counter, void *stream) {
  BS_NVTX("bs_mc_checkpoint");
  if (!m || !path) return m ? mfail(m, BS_ERR_ARG, "bs_mc_checkpoint: NULL path") : BS_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MC_CUDA(cudaStreamSynchronize(s));
  const std::string sig = mc_signature(m);
  const std::string tmp = std::string(path) + ".tmp";
  std::ofstream f(tmp, std::ios::binary);
  if (!f) return mfail(m, BS_ERR_ARG, std::string("bs_mc_checkpoint: cannot write ") + tmp);
  const uint64_t siglen = sig.size();
  const int64_t runs = m->runs;
  const int32_t tune[2] = {m->min_tiles_factor, m->tile_order};
  const int32_t ng = (int32_t)m->groups.size();
  f.write(kCkptMagic, 8);
  f.write(reinterpret_cast<const char *>(&siglen), 8);
  f.write(sig.data(), (std::streamsize)siglen);
  f.write(reinterpret_cast<const char *>(&counter), 8);
  f.write(reinterpret_cast<const char *>(&runs), 8);
  f.write(reinterpret_cast<const char *>(tune), 8);
  f.write(reinterpret_cast<const char *>(&ng), 4);
  std::vector<double> h;
  for (const Group &gr : m->groups) {
    const int64_t nd = gr.nd, nb3 = gr.nb3;
    h.resize((size_t)3 * (nd + nb3));
    MC_CUDA(cudaMemcpy(h.data(), gr.stats, h.size() * 8, cudaMemcpyDeviceToHost));
    f.write(reinterpret_cast<const char *>(&nd), 8);
    f.write(reinterpret_cast<const char *>(&nb3), 8);
    f.write(reinterpret_cast<const char *>(h.data()), (std::streamsize)(h.size() * 8));
  }
  f.close();
  if (!f) return mfail(m, BS_ERR_ARG, std::string("bs_mc_checkpoint: write failed: ") + tmp);
  if (std::rename(tmp.c_str(), path) != 0)
    return mfail(m, BS_ERR_ARG, std::string("bs_mc_checkpoint: cannot rename to ") + path);
  return BS_OK;
}

bs_status bs_mc_restore(bs_mc m, const char *path, uint64_t *counter, void *stream) {
  BS_NVTX("bs_mc_restore");
  if (!m || !path) return m ? mfail(m, BS_ERR_ARG, "bs_mc_restore: NULL path") : BS_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::ifstream f(path, std::ios::binary);
  if (!f) return mfail(m, BS_ERR_ARG, std::string("bs_mc_restore: cannot read ") + path);
  char magic[8];
  uint64_t siglen = 0, ctr = 0;
  int64_t runs = 0;
  int32_t tune[2] = {0, 0}, ng = 0;
  f.read(magic, 8);
  f.read(reinterpret_cast<char *>(&siglen), 8);
  if (!f || std::memcmp(magic, kCkptMagic, 8) != 0 || siglen > (1u << 20))
    return mfail(m, BS_ERR_ARG, "bs_mc_restore: not a Monte Carlo checkpoint");
  std::string sig(siglen, '\0');
  f.read(&sig[0], (std::streamsize)siglen);
  f.read(reinterpret_cast<char *>(&ctr), 8);
  f.read(reinterpret_cast<char *>(&runs), 8);
  f.read(reinterpret_cast<char *>(tune), 8);
  f.read(reinterpret_cast<char *>(&ng), 4);
  if (!f || sig != mc_signature(m) || ng != (int32_t)m->groups.size())
    return mfail(m, BS_ERR_ARG, "bs_mc_restore: the checkpoint belongs to other shapes");
  std::vector<std::vector<double>> h(m->groups.size());
  for (size_t g = 0; g < m->groups.size(); ++g) {
    int64_t nd = 0, nb3 = 0;
    f.read(reinterpret_cast<char *>(&nd), 8);
    f.read(reinterpret_cast<char *>(&nb3), 8);
    if (!f || nd != m->groups[g].nd || nb3 != m->groups[g].nb3)
      return mfail(m, BS_ERR_ARG, "bs_mc_restore: bin counts differ");
    h[g].resize((size_t)3 * (nd + nb3));
    f.read(reinterpret_cast<char *>(h[g].data()), (std::streamsize)(h[g].size() * 8));
    if (!f) return mfail(m, BS_ERR_ARG, "bs_mc_restore: truncated checkpoint");
  }
  if (tune[0] != m->min_tiles_factor || tune[1] != m->tile_order) {
    mc_unprepare(m);
    m->min_tiles_factor = tune[0];
    m->tile_order = tune[1];
  }
  MC_CUDA(cudaStreamSynchronize(s));
  for (size_t g = 0; g < m->groups.size(); ++g)
    MC_CUDA(cudaMemcpy(m->groups[g].stats, h[g].data(), h[g].size() * 8, cudaMemcpyHostToDevice));
  m->runs = runs;
  if (counter) *counter = ctr;
  return BS_OK;
}

bs_status bs_mc_stats(bs_mc m, int group, int which, double *mean_dev, double *var_dev,
                      int64_t *runs_host, void *stream) {
  BS_NVTX("bs_mc_stats");
  if (!m || group < 0 || group >= (int)m->groups.size() || (which != 0 && which != 1))
    return m ? mfail(m, BS_ERR_ARG, "bad group or statistic") : BS_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int h = 0;
  if (m->errw) {
    MC_CUDA(cudaMemcpyAsync(&h, m->errw, sizeof(int), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    if (h) return mfail(m, BS_ERR_TIMEOUT, "a bounded wait in the contraction gave up");
  }
  Group &gr = m->groups[group];
  const long long n = which == 0 ? gr.nd : gr.nb3;
  const double *base = gr.stats + (which == 0 ? 0 : 3 * gr.nd);
  const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
  k_welford_final<<<blocks, 256, 0, s>>>(n, base, base + n, base + 2 * n, mean_dev, var_dev);
  MC_CUDA(cudaGetLastError());
  if (runs_host) *runs_host = m->runs * gr.plan->batch;
  return BS_OK;
}

}  // extern "C"
