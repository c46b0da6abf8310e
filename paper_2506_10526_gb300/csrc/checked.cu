// Checked build support: the registry of the translation units' device error
// words, the status call, and a self-test kernel whose one access is guarded
// by the same check as the library's kernels.  In an ordinary build both
// calls return BS_ERR_UNSUPPORTED and launch nothing.
#include <mutex>
#include <vector>

#include "bs_internal.h"

namespace bsi {

#ifdef BS_CHECKED
namespace {
std::vector<ChkReader> &readers() {
  static std::vector<ChkReader> r;
  return r;
}
std::mutex &readers_mu() {
  static std::mutex m;
  return m;
}

constexpr int kSelftestSite = 0x7fff;

__global__ void k_checked_selftest(int *buf, long long n, long long idx) {
  if (BS_CHK(idx, n, kSelftestSite)) buf[idx] += 1;
}
}  // namespace

void register_chk_reader(ChkReader r) {
  std::lock_guard<std::mutex> g(readers_mu());
  readers().push_back(r);
}
#endif

}  // namespace bsi

extern "C" {

int bs_checked_build(void) {
#ifdef BS_CHECKED
  return 1;
#else
  return 0;
#endif
}

bs_status bs_checked_status(int reset, uint64_t *out_host) {
  BS_NVTX("bs_checked_status");
  if (!out_host) return BS_ERR_ARG;
#ifdef BS_CHECKED
  using namespace bsi;
  out_host[0] = out_host[1] = out_host[2] = out_host[3] = 0;
  std::lock_guard<std::mutex> g(readers_mu());
  for (ChkReader r : readers()) {
    unsigned long long w[3] = {0, 0, 0};
    if (r(w, reset != 0) != cudaSuccess) {
      cudaGetLastError();
      return BS_ERR_CUDA;
    }
    if (w[0] && !out_host[0]) {  // the first translation unit that saw a violation
      out_host[1] = w[1] >> 48;
      const unsigned long long low = w[1] & 0xffffffffffffull;  // sign-extend 48 bits
      out_host[2] = (uint64_t)((long long)(low << 16) >> 16);
      out_host[3] = w[2];
    }
    out_host[0] += w[0];
  }
  return BS_OK;
#else
  (void)reset;
  return BS_ERR_UNSUPPORTED;
#endif
}

bs_status bs_checked_selftest(int64_t n, int64_t idx, void *stream) {
  BS_NVTX("bs_checked_selftest");
#ifdef BS_CHECKED
  using namespace bsi;
  if (n < 1 || n > 4096) return BS_ERR_ARG;
  int *buf = nullptr;
  if (cudaMalloc(&buf, (size_t)n * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return BS_ERR_OOM;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(buf, 0, (size_t)n * sizeof(int), s);
  if (e == cudaSuccess) {
    k_checked_selftest<<<1, 1, 0, s>>>(buf, (long long)n, (long long)idx);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(buf);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return BS_ERR_CUDA;
  }
  return BS_OK;
#else
  (void)n;
  (void)idx;
  (void)stream;
  return BS_ERR_UNSUPPORTED;
#endif
}

}  // extern "C"
