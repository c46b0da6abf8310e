// Internal declarations shared by the libbs translation units.
#pragma once

#include <cstring>

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "bs.h"

#include <nvtx3/nvToolsExt.h>

namespace bsi {

// ---- checked build (-DBS_CHECKED) -------------------------------------------
// BS_CHK(i, n, site) is true when 0 <= i < n.  In a checked build a false
// check also records the violation in the translation unit's device error
// word (count, first site and index, its bound) and the caller skips the
// access, so an index error is reported instead of faulting; bs_checked_status
// reads and clears the words of every translation unit.  In an ordinary build
// the check is the constant true and compiles away.
#ifdef BS_CHECKED
static __device__ unsigned long long g_chk_word[3];
__device__ __forceinline__ bool chk_index(long long i, long long n, int site) {
  if (i >= 0 && i < n) return true;
  if (atomicAdd(&g_chk_word[0], 1ull) == 0ull) {
    g_chk_word[1] = ((unsigned long long)(unsigned)site << 48) |
                    ((unsigned long long)i & 0xffffffffffffull);
    g_chk_word[2] = (unsigned long long)n;
  }
  return false;
}
#define BS_CHK(i, n, site) ::bsi::chk_index((long long)(i), (long long)(n), (site))
// reads (and with reset, clears) one translation unit's word
using ChkReader = cudaError_t (*)(unsigned long long *w, bool reset);
void register_chk_reader(ChkReader r);
static cudaError_t chk_read_tu(unsigned long long *w, bool reset) {
  cudaError_t e = cudaMemcpyFromSymbol(w, g_chk_word, sizeof(g_chk_word));
  if (e == cudaSuccess && reset) {
    const unsigned long long z[3] = {0, 0, 0};
    e = cudaMemcpyToSymbol(g_chk_word, z, sizeof(z));
  }
  return e;
}
static const bool g_chk_registered = (register_chk_reader(&chk_read_tu), true);
#else
#define BS_CHK(i, n, site) true
#endif

// Mixed-radix factorisation of a transform length (radices 4, 2, 3, 5).
struct Radices {
  int n = 0;
  int r[24] = {0};
};

// n = 8^a 4^b 2^c 3^d 5^e: the Stockham stage radices (8s first, then 4, 2, 3, 5);
// false when n has another prime factor.
bool factor_radices(int n, Radices &r);
// exp(+2 pi i t / n), t in [0, n), computed in FP64 and rounded to FP32.
std::vector<float2> twiddles(int n);

// One column of the triple contraction: field (l, nu3) and its ring triple.
struct ColEntry {
  int field;  // l * nchan + nu3
  int trip;   // ring-triple index of (i, j, l)
  int nu3;
  // 0: the row is (l, nu3) against pairs (nu1, nu2).  1 (channel-symmetric
  // accumulation only): the row is (i, nu1) of ring triple (i, j, j), i < j,
  // against pairs (nu2, nu3) of ring j; `nu3` then holds nu1
  int swapped;
};

// A (ring pair, column tile) work item of the contraction.
struct PairTile {
  int ri, rj;    // rings of the pair operand
  int col_off;   // offset of this pair's column list in the column array
  int ncol;      // columns in the pair's list
  int col0;      // first column of this tile
  int pad[3];
};

// Geometry shared by the field kernels.  A plan may hold fields at several
// image sizes (levels); at each level only some rings have fields, stored in
// slots: slot_of[ring] (-1: no field at this level), ring_of[slot].
struct GridGeom {
  int nt, nc, nb, M, UC;  // UC: u >= 0 columns stored per field
  int batch;
  int nslot;              // rings with fields at this level
  const int *slot_of;     // device [nb]
  const int *ring_of;     // device [nslot]
};

// Contraction launch arguments.
struct ContractArgs {
  const float *F;          // fields [batch][nb*nc][M*M]
  long long fstride;       // M*M
  long long bstride;       // nb*nc*M*M
  int M2, nc;
  const ColEntry *cols;
  const PairTile *ptiles;
  int nu1_lo, nu1_hi, nu2_lo, nu2_hi;
  int n_r2;                // number of nu2 row blocks
  int kseg_len, nkseg;
  const double *tnorm;     // per ring triple: 1/(A M^2 T), 0 when T == 0
  double *out_full;        // [batch][ntrip][nc][nc][nc] or null
  long long full_bstride;  // ntrip*nc^3
  double *dsum;            // [batch][ntrip][2nc-1][2nc-1] or null
  long long dsum_bstride;  // ntrip*(2nc-1)^2
};

// A tensor-core contraction tile: shape group, realisation, ring pair, pair
// rectangle origin, a 128-entry window of the pair's column list, K segment.
struct TcTile {
  int group, b;
  int ri, rj;
  int nu1_0, nu2_0;
  int col_off, ncol, col0;
  int kseg;
  // 1: the pair operand is F_i F_i of one ring and only pairs nu1 <= nu2 are kept
  // (the rectangle straddles the diagonal nu1 = nu2); 0: every pair is kept
  int diag;
  int pad;
};

// Per shape group (one plan): where its fields, lists and outputs live.
struct TcGroup {
  const float *F;          // FP32 fields (pair operand source)
  long long fstride;       // M*M
  long long bstride;       // nf*M*M
  int nf, batch, M2, Kpad, nc;
  int nu1_hi, nu2_hi;      // block upper bounds (pairs beyond are skipped)
  int kseg_len;
  const ColEntry *cols;    // per ring pair: runs of fields (l, nu3), padded to multiples of 8
  const double *tnorm;
  double *out_full;
  long long full_bstride;
  double *dsum;
  long long dsum_bstride;
  // split-FP16 only (null otherwise): per (realisation, slot) exponent k of the
  // power-of-two field scale 2^k, index b * nslot + slot
  const int *kexp;
  int nslot;
};

struct TcArgs {
  const TcGroup *groups;   // device
  const void *maps;        // device: 2 CUtensorMap (hi, lo) per group, 64-byte aligned
  const TcTile *tiles;     // device
  int ntiles;
  int *err;                // device error word: 1 = a bounded wait gave up
  long long wait_limit_ns;
  int stall_test;          // failure injection: the MMA thread waits on a barrier nobody arrives at
  int f16;                 // 1: split-FP16 operands (two products), 0: split BF16 (three)
};

// NVTX range over an entry point, named after it (no cost unless a profiler
// that records NVTX is attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
#define BS_NVTX(name) ::bsi::NvtxRange bs_nvtx_range_(name)

// Host-side failure injection for tests: true when the environment variable
// BS_INJECT_FAIL lists `point` (comma-separated: plan_create, workspace_alloc,
// mc_alloc, sky_alloc, mlp_alloc, scratch_alloc).  The caller then fails as
// the real failure would (BS_ERR_OOM), without touching the device.
bool inject_fail(const char *point);

// Grid cell (u, v) with |u|, |v| < 32768 packed as (u + 32768) | (v + 32768) << 16,
// computed in unsigned arithmetic and stored bit for bit in an int; the
// counting kernel decodes it with c & 0xffff and (c >> 16) & 0xffff.
__host__ __device__ inline int pack_cell(int u, int v) {
  const unsigned w = (unsigned)(u + 32768) | ((unsigned)(v + 32768) << 16);
  int c;
  memcpy(&c, &w, sizeof c);
  return c;
}

// Set a kernel's dynamic shared-memory limit to the device's opt-in maximum,
// once per process (so that launches can be captured in CUDA graphs).  The
// kernel is a template argument: one flag per kernel, not per signature.
template <auto kernel>
inline cudaError_t smem_optin_once() {
  static cudaError_t done = cudaErrorNotReady;
  if (done == cudaErrorNotReady) {
    int dev = 0, mx = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    done = cudaFuncGetAttributes(&fa, kernel);
    if (done == cudaSuccess)  // dynamic + static shared memory must fit the opt-in limit
      done = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  mx - (int)fa.sharedSizeBytes);
  }
  return done;
}

// ---- kernels / launchers (each returns cudaGetLastError after launch) ----
// Register-FFT variants of the two field passes (grid_reg.cu) for the image
// sides with a register plan (has_reg_fft); the launchers below dispatch to them.
bool has_reg_fft(int M, int nt);
cudaError_t launch_colpass_reg(const GridGeom &g, const float2 *vis, const float *ngrid,
                               const uint8_t *valid, const int8_t *label, const int *uext,
                               const float2 *twM, float2 *G, cudaStream_t s);
cudaError_t launch_rowpass_reg(const GridGeom &g, const float2 *G, const uint8_t *valid,
                               const int *uext, const float2 *twM, float *F, uint16_t *Fhi,
                               uint16_t *Flo, unsigned *fmax, cudaStream_t s);
cudaError_t launch_colpass(const GridGeom &g, const float2 *vis, const float *ngrid,
                           const uint8_t *valid, const int8_t *label, const int *uext,
                           const float2 *twM, const Radices &radM, float2 *G,
                           cudaStream_t s);
// fmax (split FP16, else null): per (realisation, slot) largest |F| as float
// bits, combined with atomicMax (zeroed by the caller)
cudaError_t launch_rowpass(const GridGeom &g, const float2 *G, const uint8_t *valid,
                           const int *uext, const float2 *twM, const Radices &radM,
                           float *F, uint16_t *Fhi, uint16_t *Flo, unsigned *fmax,
                           cudaStream_t s);
// Split FP16: kexp[b][slot] = power-of-two scale exponent from fmax, and the
// FP16 hi / lo parts of every scaled field of one level.
cudaError_t launch_split_f16(const GridGeom &g, const float *F, const unsigned *fmax, int *kexp,
                             uint16_t *Fhi, uint16_t *Flo, cudaStream_t s);
cudaError_t launch_effective_label(int ncell, const int8_t *label, const float *ngrid,
                                  int8_t *out, cudaStream_t s);
cudaError_t launch_counts(int nt, int nb, const int8_t *label, const int *cells, int ncells,
                          const int *trip_of, unsigned long long *T, cudaStream_t s);
cudaError_t launch_contract_simt(const ContractArgs &a, int ntiles_row, int npt,
                                 int batch, cudaStream_t s);
cudaError_t launch_full_fill(double *out, long long bstride, int batch, int ntrip, int nc,
                             const int *blk, double value, cudaStream_t s);
cudaError_t launch_full_finalize(double *out, long long bstride, int batch, int ntrip,
                                 int nc, const int *blk, const uint8_t *valid,
                                 const double *tnorm, cudaStream_t s);
// list (nlist entries, or null for every ring triple): ring triples to process;
// output plane y holds list[y] (compact layout), else plane t holds triple t.
// scratch: ((2nc-1)^2 + 1) / 2 doubles for the reciprocal folded sampling.
cudaError_t launch_delta_norm(const double *dsum, const long long *nnu, const double *tnorm,
                              double *out, int batch, int ntrip, int nc, const int *list,
                              int nlist, double *scratch, cudaStream_t s);
// y[k] += x[k], k < n
cudaError_t launch_add_f64(double *y, const double *x, long long n, cudaStream_t s);
// box = {row_lo, row_hi, col_lo, col_hi} (inclusive plane indices) to zero
cudaError_t launch_zero_planes(double *dsum, const int *trips, int ntr, int batch, int ntrip,
                               int n2, const int *box, cudaStream_t s);
// Channel-symmetric accumulation: fills, inside box, the channel orderings of
// the listed ring triples (2 t + kind; kind 0: (i, i, l), kind 1: (i, j, j))
// that the contraction left out, from the ones it computed.
cudaError_t launch_symmetrize(double *dsum, const int *list, int nlist, int batch, int ntrip,
                              int nc, const int *box, cudaStream_t s);
// tmp: batch * ntrip * nc^2 float2 followed by nc^2 doubles of scratch
// Register-FFT delay transform (delta_reg.cu) for the channel counts with a
// register plan (has_reg_dft); launch_bs3d dispatches to it.  rinv [nc][nc]:
// FP32 reciprocal folded sampling; rowflag [nc]: rows of the periodic
// placement with a sampled separation.
bool has_reg_dft(int nc);
cudaError_t launch_bs3d_reg(const double *dsum, const float *rinv, const uint8_t *rowflag,
                            const double *tnorm, float2 *tmp, double *out, int batch, int ntrip,
                            int nc, const float2 *twN, double scale, const int *list, int ny,
                            cudaStream_t s);
cudaError_t launch_bs3d(const double *dsum, const long long *nnu, const double *tnorm,
                        float2 *tmp, double *out, int batch, int ntrip, int nc,
                        const float2 *twN, const Radices &radN, double scale, const int *list,
                        int nlist, cudaStream_t s);
// General (non-Hermitian) input: the four Hermitian components X_H + t Y,
// t = 0, 1, -1, 2, of X = W V (out [4 ub][nc][nt][nt]), and the combination of
// four real results into complex ones (in [4 ub][n] -> out [ub][n][2]; the
// _full form only touches the channel block blk of [.][ntrip][nc^3]).
cudaError_t launch_general_prep(int nt, int nc, int ub, const float2 *vis, const float *ngrid,
                                const int8_t *label, float2 *out, cudaStream_t s);
cudaError_t launch_combine4(const double *in, long long n, int ub, double *out, cudaStream_t s);
cudaError_t launch_combine4_full(const double *in, int ub, int ntrip, int nc, const int *blk,
                                 double *out, cudaStream_t s);
// Per-channel sampling: components W V and [N_g(nu) > 0] (out [2 ub][nc][nt][nt]),
// ratios of the two components (x [2b] / x [2b+1] / A; the _full form only in the
// channel block), and ratio planes rewritten as collapse sums for the delay
// transform (see general.cu).
cudaError_t launch_chans_prep(int nt, int nc, int ub, const float2 *vis, const float *ngrid,
                              const int8_t *label, float2 *out, cudaStream_t s);
cudaError_t launch_ratio2(const double *in, long long n, int ub, double inv_a, double *out,
                          cudaStream_t s);
cudaError_t launch_ratio2_full(const double *in, int ub, int ntrip, int nc, const int *blk,
                               double inv_a, double *out, cudaStream_t s);
cudaError_t launch_ratio_to_sums(const double *R, const long long *nnu, const double *tnorm,
                                 int ub, int ntrip, int nc, double *sums, cudaStream_t s);
int tc_smem_bytes(int f16);
cudaError_t launch_contract_tc(const TcArgs &a, int nsm, cudaStream_t s);
cudaError_t launch_hermitian_check(const float2 *vis, int batch, int nc, int nt,
                                   const int8_t *label, float *maxdiff, float *maxabs,
                                   cudaStream_t s);

}  // namespace bsi
