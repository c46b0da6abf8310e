// Internal plan state shared by the libbs translation units.
#pragma once

#include <cuda.h>

#include <string>
#include <vector>

#include "bs_internal.h"

namespace bsi {

struct WsLayout {
  size_t label, efflabel, cells, uext, tripof, valid, twM, twN, tnorm, T, nnu, cols, ptiles, tctiles,
      G, F, Fhi, Flo, dsum, tmp3d, herm, err, maps, tcgroup, mlptab, ztrips, clos, closrings, mono, cyl,
      errn, errtab, gvis, symtrips, total;
};

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);


// Fields at one image side M: the rings that need it (slots), where they live
// in the workspace, and their tensor maps.
struct Level {
  int M = 0, UC = 1, nslot = 0;
  Radices rad;
  std::vector<int> slot_of;  // [nb], -1: no field at this level
  std::vector<int> ring_of;  // [nslot]
  size_t offF = 0, offFhi = 0, offFlo = 0, offTw = 0, offSlot = 0, offRing = 0;
  // split FP16: per (realisation, slot) largest |F| (float bits) and scale exponent
  size_t offFmax = 0, offKexp = 0;
  // hi, lo (BF16 or FP16) with boxes of 8, 32, 128 rows, then FP32 F (host copies; device at L.maps)
  CUtensorMap maps[7]{};
};

}  // namespace bsi

using namespace bsi;  // internal header: plan state uses the library types unqualified

struct bs_plan_s {
  bs_plan_desc d{};
  std::vector<double> edges;
  int nt = 0, nc = 0, nb = 0, M = 0, UC = 0, batch = 1, ntrip = 0, nf = 0;
  int device = 0;
  double normA = 1, scale3d = 1;
  Radices radM, radN;
  std::vector<int8_t> label;     // [nt*nt]
  std::vector<int> cells;        // packed (u + 32768) | (v + 32768) << 16 of binned cells
  std::vector<int> uext;         // [nb]
  std::vector<double> umean;     // [nb] mean |U| of each ring's cells
  std::vector<int> cring;        // [nb] largest |u| or |v| of a ring's cells
  std::vector<Level> levels;     // image sides; one level holding every ring unless multires
  std::vector<int> lev_of_trip;  // [ntrip] level of each ring triple (-1: cannot close)
  bool multires = false;
  bool dsum_clean = false;        // every plane of a non-closable triple is zero
  // plane indices (d + nc - 1) of the separations accumulated since the last
  // reset: rows [0] .. [1], columns [2] .. [3] (empty when [1] < [0])
  int dbox[4] = {0, -1, 0, -1};
  std::vector<int> zero_trips;    // closable ring triples (the only planes ever accumulated)
  // closable ring triples with a repeated ring, 2 t + kind (0: (i, i, l), 1: (i, j, j),
  // i < j; device copy at L.symtrips), and the state of the collapse sums since the
  // last reset: 0 nothing accumulated, 1 ordinary blocks (or imported sums), 2
  // channel-symmetric cubes with the left-out orderings not yet filled in, 3 the
  // same, filled in
  std::vector<int> sym_trips;
  int sym_state = 0;
  std::vector<int> clos;          // ring triples with T > 0, ascending (device copy at L.clos)
  std::vector<int> closrings;     // [clos.size()][3] rings (i, j, l) of those triples
  std::vector<unsigned char> mono_tab;  // k tables and thresholds of the last monopole call
  // bin of every monopole sample [n_c][nchan][nchan] (int16, -1 dropped) for the
  // geometry in mono_key (k tables, edges, bin counts, closable triples); device,
  // allocated at the first monopole call, freed with the plan
  int16_t *mono_bins = nullptr;
  size_t mono_bins_cap = 0;
  std::vector<unsigned char> mono_key;
  // general (non-Hermitian) input: batch = 4 x ubatch internal realisations (the
  // Hermitian components X_H + t Y, t = 0, 1, -1, 2, of each user realisation) and
  // scratch for their real outputs before they are combined (device, on demand)
  bool general = false;
  // per-channel sampling: batch = 2 x ubatch (weighted visibilities, occupancy)
  bool chans = false;
  int ubatch = 1;
  double *gfull = nullptr, *gdelta = nullptr, *g3d = nullptr;
  size_t gfull_cap = 0, gdelta_cap = 0, g3d_cap = 0;
  // binnings of a general plan's complex 3D bispectrum: its real and imaginary
  // planes, then their real sums (device, on demand)
  double *gbin = nullptr;
  size_t gbin_cap = 0;
  // error bound of a per-channel sampling plan: per-evaluation bounds [batch][ntrip]
  double *gerr = nullptr;
  size_t gerr_cap = 0;
  std::vector<int> cyl_tab;       // row bins and column ranges of the last cylindrical call
  std::vector<long long> cyl_cnt; // its per-bin counts
  std::vector<int> err_tab;       // [ntrip][4] rings (i, j, l) and level, for the error bound
  std::vector<int> trips;        // [ntrip][3]
  std::vector<int> trip_of;      // [nb^3] -> trip index of sorted (i<=j<=l), else -1
  std::vector<long long> T;      // [ntrip] closed-triangle counts
  std::vector<double> tnorm;     // [ntrip]
  std::vector<uint8_t> valid;    // [nc]
  std::vector<long long> nnu;    // [(2nc-1)^2] accumulated unfolded sampling
  bool counts_ready = false, counts_default = false, nnu_dirty = true, loaded = false;
  bool sticky = false;
  // error word of the tensor-core contraction in mapped pinned host memory
  // (read after a stream sync, with no copy engine involved)
  int *err_host = nullptr, *err_dev = nullptr;
  bool err_pending = false;  // a contraction ran since the last check
  // pinned staging of the per-call work lists (tile and column lists), so that
  // their uploads are asynchronous; stage_ev marks the last upload from it
  unsigned char *h_stage = nullptr;
  size_t h_stage_cap = 0;
  cudaEvent_t stage_ev = nullptr;
  bool stage_pending = false;
  ~bs_plan_s() {
    if (err_host) cudaFreeHost(err_host);
    if (stage_pending && stage_ev) cudaEventSynchronize(stage_ev);
    if (h_stage) cudaFreeHost(h_stage);
    if (stage_ev) cudaEventDestroy(stage_ev);
  }
  std::string err = "no error";
  // workspace
  WsLayout L{};
  unsigned char *ws = nullptr;
  bool ws_owned = false;
  size_t max_cols = 0, max_ptiles = 0, max_tctiles = 0;
  std::vector<ColEntry> h_cols;
  std::vector<PairTile> h_ptiles;
  std::vector<TcTile> h_tctiles;

  bool maps_ready = false;
  std::vector<TcGroup> h_groups;
  int nsm = 152;

  template <class T_>
  T_ *at(size_t off) const {
    return reinterpret_cast<T_ *>(ws + off);
  }
};


namespace bsi {
// helpers implemented in plan.cu
bs_status fail(bs_plan p, bs_status s, const std::string &msg);
bs_status cuda_fail(bs_plan p, cudaError_t e, const char *where);
bs_status prepare(bs_plan p, cudaStream_t s);
bs_status run_counts(bs_plan p, const int8_t *lab_dev, cudaStream_t s);
bs_status ensure_tensor_maps(bs_plan p, cudaStream_t s);
bs_status check_device_error(bs_plan p, cudaStream_t s);
void accumulate_block_nnu(bs_plan p, const int *blk);
// Fills in the channel orderings a symmetric accumulation left out (state 2 -> 3).
bs_status sym_fill(bs_plan p, cudaStream_t s);
// Adds the unfolded sampling of channel block blk under the channel validity
// `valid` to plane[(d1 + nc - 1) * (2nc - 1) + d2 + nc - 1].
void add_block_sampling(int nc, const std::vector<uint8_t> &valid, const int *blk,
                        long long *plane);
bs_status upload_nnu(bs_plan p, cudaStream_t s);
// Device scratch of n doubles in *buf (grown with cudaMalloc when *cap < n,
// freed with the plan); BS_ERR_OOM when it cannot be had.
bs_status general_scratch(bs_plan p, double **buf, size_t *cap, size_t n);
// Per-channel sampling plans: the normalised collapse components [2 ubatch]
// [planes][2nc-1][2nc-1] (numerator sums, then denominator sums, of each
// realisation) of the full (closable = false) or closable layout, in plan scratch.
bs_status chans_components(bs_plan p, bool closable, cudaStream_t s, const double **comp);
// Host-to-device uploads of per-call work lists through the plan's pinned
// staging buffer (asynchronous; the buffer is reused once the previous
// uploads from it have completed).  Falls back to ordinary copies when
// pinned memory cannot be had.
struct StagedUpload {
  void *dst;
  const void *src;
  size_t bytes;
};
bs_status upload_staged(bs_plan p, cudaStream_t s, const StagedUpload *u, int n);
// Append the tensor-core work of one channel block of plan p (all
// realisations): one shape group per image level, numbered from group_base.
// Column entries are appended to cols, tiles to tiles (col_off relative to
// the concatenated list at cols_dev).  Returns the group descriptors.
std::vector<TcGroup> build_tc_work(bs_plan p, const int *blk, int group_base,
                                   std::vector<ColEntry> &cols, const ColEntry *cols_dev,
                                   std::vector<TcTile> &tiles, double *out_full, int accumulate,
                                   int min_tiles);
// Enqueue shell masks + field FFTs of every level (kernel launches only).
bs_status enqueue_fields(bs_plan p, const void *vis, const float *ngrid, cudaStream_t s);
}  // namespace bsi
