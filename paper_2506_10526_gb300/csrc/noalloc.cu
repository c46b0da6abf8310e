// bs_counts_noalloc: closed-triangle counts without any device allocation.
//
// Some callers cannot call cudaMalloc: a pipeline that runs under a fixed
// device-memory budget handed out by its own pool, a host that must not
// touch the CUDA allocator while other work owns the device, or code that
// only ever receives pre-allocated buffers.  For them this entry point runs
// the same triangle-count kernel as bs_counts, but its scratch (the ring
// label table, the list of binned cells and the ring-triple index table)
// lives in one file-scope __device__ array of fixed size instead of a plan
// workspace.  Under CUDA's lazy module loading the array is reserved on a
// device by the first call there (which loads this file's module); it then
// stays for the life of the process, or until the device's context is reset.
#include <cuda.h>

#include <mutex>

#include "bs_internal.h"

namespace bsi {

namespace {

constexpr int kNoallocMaxNt = 1024;
constexpr int kNoallocMaxBins = 32;
constexpr size_t kLabelBytes = (size_t)kNoallocMaxNt * kNoallocMaxNt;           // int8 labels
constexpr size_t kCellBytes = (size_t)kNoallocMaxNt * kNoallocMaxNt * 4;        // int32 cells
constexpr size_t kTripBytes = (size_t)kNoallocMaxBins * kNoallocMaxBins * kNoallocMaxBins * 4;
constexpr size_t kCounterBytes = 256;
constexpr size_t kScratchBytes = kLabelBytes + kCellBytes + kTripBytes + kCounterBytes;

// The scratch.  Host code must not take this name as an address: it is a
// host-side stand-in; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_counts_scratch[kScratchBytes];

struct Edges {
  double e2[kNoallocMaxBins + 1];  // squared ring edges
  int nb;
};

// Ring label of every cell (same rule as the plan: e_m^2 <= |U|^2 < e_{m+1}^2,
// U = 0 and cells with a component equal to -nt/2 excluded; empty cells of
// ngrid excluded) and the list of binned cells (occupied or not).
__global__ void k_noalloc_labels(int nt, Edges E, const float *__restrict__ ngrid,
                                 int8_t *__restrict__ label, int *__restrict__ cells,
                                 int *__restrict__ ncells) {
  const int h = nt / 2;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt * nt; t += gridDim.x * blockDim.x) {
    const int iu = t % nt, iv = t / nt;
    const int u = iu - h, v = iv - h;
    int ring = -1;
    if (iu > 0 && iv > 0 && (u != 0 || v != 0)) {
      const double q = (double)((long long)u * u + (long long)v * v);
      for (int m = 0; m < E.nb; ++m)
        if (q >= E.e2[m] && q < E.e2[m + 1]) {
          ring = m;
          break;
        }
    }
    if (ring >= 0) cells[atomicAdd(ncells, 1)] = pack_cell(u, v);
    if (ring >= 0 && ngrid && !(ngrid[t] > 0.f)) ring = -1;
    label[t] = (int8_t)ring;
  }
}

// Index of sorted ring triples i <= j <= l in lexicographic order, -1 otherwise.
__global__ void k_noalloc_tripof(int nb, int *__restrict__ trip_of) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nb * nb * nb; t += gridDim.x * blockDim.x) {
    const int i = t / (nb * nb), j = (t / nb) % nb, l = t % nb;
    int idx = -1;
    if (i <= j && j <= l) {
      int k = 0;
      for (int a = 0; a < nb; ++a)
        for (int b = a; b < nb; ++b)
          for (int c = b; c < nb; ++c) {
            if (a == i && b == j && c == l) idx = k;
            ++k;
          }
    }
    trip_of[t] = idx;
  }
}

// Device address of the array per device, with the id of the context it was
// looked up in: a context reset (cudaDeviceReset) unloads the module and frees
// the array, so an address is reused only while the context id is the same.
struct SymbolCache {
  void *ptr = nullptr;
  unsigned long long ctx = 0;
};
std::mutex g_symbol_mutex;
SymbolCache g_symbol[64];

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current context (0 if none or unknown).
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    looked_up = true;
    void *f1 = nullptr, *f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) ==
            cudaSuccess && q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) ==
            cudaSuccess && q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
      get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    cudaGetLastError();
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx ||
      get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

}  // namespace

}  // namespace bsi

using namespace bsi;

extern "C" bs_status bs_counts_noalloc(int nt, int nbins, const double *bin_edges,
                                       const float *ngrid_dev, int64_t *tri_dev,
                                       void *cuda_stream) {
  BS_NVTX("bs_counts_noalloc");
  if (nt < 8 || nt > kNoallocMaxNt || (nt & 1) || nbins < 1 || nbins > kNoallocMaxBins ||
      !bin_edges || !tri_dev)
    return BS_ERR_ARG;  // sizes beyond the static scratch (nt <= 1024, nbins <= 32)
  for (int m = 0; m <= nbins; ++m)
    if (!(bin_edges[m] >= 0) || (m > 0 && !(bin_edges[m] > bin_edges[m - 1]))) return BS_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return BS_ERR_NO_DEVICE;
  }
  unsigned char *scratch = nullptr;
  {
    // once per device (and again after a reset of its context), with that
    // device current: the device address of the array
    std::lock_guard<std::mutex> lock(g_symbol_mutex);
    SymbolCache &c = g_symbol[dev];
    const unsigned long long ctx = c.ptr ? current_context_id() : 0;
    if (!c.ptr || ctx == 0 || ctx != c.ctx) {
      void *ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_counts_scratch) != cudaSuccess || !ptr) {
        cudaGetLastError();
        c.ptr = nullptr;
        return BS_ERR_CUDA;
      }
      c.ptr = ptr;
      c.ctx = current_context_id();
    }
    scratch = static_cast<unsigned char *>(c.ptr);
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int8_t *label = reinterpret_cast<int8_t *>(scratch);
  int *cells = reinterpret_cast<int *>(scratch + kLabelBytes);
  int *trip_of = reinterpret_cast<int *>(scratch + kLabelBytes + kCellBytes);
  int *ncells_dev = reinterpret_cast<int *>(scratch + kLabelBytes + kCellBytes + kTripBytes);
  // number of binned cells, by the same FP64 rule on the host
  Edges E{};
  E.nb = nbins;
  for (int m = 0; m <= nbins; ++m) E.e2[m] = bin_edges[m] * bin_edges[m];
  int ncells = 0;
  const int h = nt / 2;
  for (int iv = 1; iv < nt; ++iv)
    for (int iu = 1; iu < nt; ++iu) {
      const int u = iu - h, v = iv - h;
      if (u == 0 && v == 0) continue;
      const double q = (double)((long long)u * u + (long long)v * v);
      for (int m = 0; m < nbins; ++m)
        if (q >= E.e2[m] && q < E.e2[m + 1]) {
          ++ncells;
          break;
        }
    }
  const int ntrip = nbins * (nbins + 1) * (nbins + 2) / 6;
  // the array keeps the previous call's contents: clear the counter and the output
  if (cudaMemsetAsync(ncells_dev, 0, sizeof(int), s) != cudaSuccess ||
      cudaMemsetAsync(tri_dev, 0, (size_t)ntrip * sizeof(int64_t), s) != cudaSuccess) {
    cudaGetLastError();
    return BS_ERR_CUDA;
  }
  k_noalloc_labels<<<(nt * nt + 255) / 256, 256, 0, s>>>(nt, E, ngrid_dev, label, cells, ncells_dev);
  k_noalloc_tripof<<<(nbins * nbins * nbins + 255) / 256, 256, 0, s>>>(nbins, trip_of);
  if (cudaGetLastError() != cudaSuccess) return BS_ERR_CUDA;
  cudaError_t e = launch_counts(nt, nbins, label, cells, ncells, trip_of,
                                reinterpret_cast<unsigned long long *>(tri_dev), s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return BS_ERR_CUDA;
  }
  return BS_OK;
}
