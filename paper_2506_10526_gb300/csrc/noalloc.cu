// bs_counts_noalloc: closed-triangle counts without any device allocation.
//
// Some callers cannot call cudaMalloc: a pipeline that runs under a fixed
// device-memory budget handed out by its own pool, a host that must not
// touch the CUDA allocator while other work owns the device, or code that
// only ever receives pre-allocated buffers.  For them this entry point runs
// the same triangle-count kernel as bs_counts, but its scratch (the ring
// label table, the list of binned cells and the ring-triple index table)
// lives in one file-scope __device__ array of fixed size instead of a plan
// workspace.  The array exists on every device that loads the library, for
// the life of the process.
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
    if (ring >= 0) cells[atomicAdd(ncells, 1)] = (u + 32768) | ((v + 32768) << 16);
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

std::mutex g_symbol_mutex;
void *g_symbol_addr[64] = {nullptr};

}  // namespace

}  // namespace bsi

using namespace bsi;

extern "C" bs_status bs_counts_noalloc(int nt, int nbins, const double *bin_edges,
                                       const float *ngrid_dev, int64_t *tri_dev,
                                       void *cuda_stream) {
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
    // once per device, with that device current: the device address of the array
    std::lock_guard<std::mutex> lock(g_symbol_mutex);
    if (!g_symbol_addr[dev]) {
      void *ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_counts_scratch) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return BS_ERR_CUDA;
      }
      g_symbol_addr[dev] = ptr;
    }
    scratch = static_cast<unsigned char *>(g_symbol_addr[dev]);
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
