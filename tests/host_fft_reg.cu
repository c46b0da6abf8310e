// Host driver for the CPU tests of csrc/fft_reg.cuh and csrc/fp_bits.cuh
// (compiled by tests/test_fft_reg_host.py with nvcc as host code):
//   dft  L S  in out : the in-register DFT of length L, sign S, on L complex
//   fft2 N S  in out : the kernels' four-step N1 x N2 split of length N
//   d2f       in out : doubles -> floats, round to nearest even
//   f2d  E    in out : floats -> doubles times 2^E
// Inputs and outputs are raw little-endian arrays.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "fft_reg.cuh"
#include "fp_bits.cuh"

using namespace bsi;

template <class T>
static std::vector<T> read_all(const char *path) {
  std::vector<T> v;
  FILE *f = std::fopen(path, "rb");
  if (!f) std::exit(2);
  T x;
  while (std::fread(&x, sizeof(T), 1, f) == 1) v.push_back(x);
  std::fclose(f);
  return v;
}
template <class T>
static void write_all(const char *path, const std::vector<T> &v) {
  FILE *f = std::fopen(path, "wb");
  if (!f) std::exit(2);
  std::fwrite(v.data(), sizeof(T), v.size(), f);
  std::fclose(f);
}

template <int L, int S>
static void run_dft(std::vector<float2> &x) {
  for (size_t r = 0; r + L <= x.size(); r += L) {
    float2 v[L];
    for (int j = 0; j < L; ++j) v[j] = x[r + j];
    freg::dft<L, S>(v);
    for (int j = 0; j < L; ++j) x[r + j] = v[j];
  }
}

// the kernels' arithmetic: pass-1 DFTs of length N1 over stride-N2 inputs,
// the table twiddle exp(S 2 pi i (n2 k1 mod N) / N) (FP64 rounded to FP32),
// pass-2 DFTs of length N2, output index k1 + N1 k2
template <int N, int S>
static void run_fft2(std::vector<float2> &x) {
  constexpr int N1 = freg::Split<N>::N1, N2 = freg::Split<N>::N2;
  std::vector<float2> tw(N), Y(N);
  for (int t = 0; t < N; ++t) {
    const double a = 2.0 * 3.14159265358979323846 * t / N;
    tw[t] = make_float2((float)std::cos(a), (float)(S * std::sin(a)));
  }
  for (size_t r = 0; r + N <= x.size(); r += N) {
    for (int n2 = 0; n2 < N2; ++n2) {
      float2 v[N1];
      for (int n1 = 0; n1 < N1; ++n1) v[n1] = x[r + n2 + N2 * n1];
      freg::dft<N1, S>(v);
      for (int k1 = 0; k1 < N1; ++k1) {
        const float2 w = tw[(n2 * k1) % N], a = v[k1];
        Y[k1 * N2 + n2] = make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
      }
    }
    for (int k1 = 0; k1 < N1; ++k1) {
      float2 v[N2];
      for (int n2 = 0; n2 < N2; ++n2) v[n2] = Y[k1 * N2 + n2];
      freg::dft<N2, S>(v);
      for (int k2 = 0; k2 < N2; ++k2) x[r + k1 + N1 * k2] = v[k2];
    }
  }
}

template <int S>
static bool dft_any(int L, std::vector<float2> &x) {
  switch (L) {
    case 2: run_dft<2, S>(x); return true;
    case 3: run_dft<3, S>(x); return true;
    case 4: run_dft<4, S>(x); return true;
    case 5: run_dft<5, S>(x); return true;
    case 6: run_dft<6, S>(x); return true;
    case 9: run_dft<9, S>(x); return true;
    case 10: run_dft<10, S>(x); return true;
    case 15: run_dft<15, S>(x); return true;
    case 18: run_dft<18, S>(x); return true;
    case 20: run_dft<20, S>(x); return true;
    case 25: run_dft<25, S>(x); return true;
    case 27: run_dft<27, S>(x); return true;
    case 30: run_dft<30, S>(x); return true;
    case 8: run_dft<8, S>(x); return true;
    case 12: run_dft<12, S>(x); return true;
    case 16: run_dft<16, S>(x); return true;
    case 24: run_dft<24, S>(x); return true;
    case 32: run_dft<32, S>(x); return true;
    default: return false;
  }
}
template <int S>
static bool fft2_any(int N, std::vector<float2> &x) {
  switch (N) {
    case 16: run_fft2<16, S>(x); return true;
    case 24: run_fft2<24, S>(x); return true;
    case 32: run_fft2<32, S>(x); return true;
    case 48: run_fft2<48, S>(x); return true;
    case 64: run_fft2<64, S>(x); return true;
    case 96: run_fft2<96, S>(x); return true;
    case 128: run_fft2<128, S>(x); return true;
    case 192: run_fft2<192, S>(x); return true;
    case 256: run_fft2<256, S>(x); return true;
    case 384: run_fft2<384, S>(x); return true;
    case 512: run_fft2<512, S>(x); return true;
    case 768: run_fft2<768, S>(x); return true;
    case 540: run_fft2<540, S>(x); return true;
    case 675: run_fft2<675, S>(x); return true;
    case 729: run_fft2<729, S>(x); return true;
    case 750: run_fft2<750, S>(x); return true;
    default: return false;
  }
}

int main(int argc, char **argv) {
  if (argc < 4) return 2;
  const char *mode = argv[1];
  if (!std::strcmp(mode, "dft") || !std::strcmp(mode, "fft2")) {
    if (argc != 6) return 2;
    const int L = std::atoi(argv[2]), S = std::atoi(argv[3]);
    std::vector<float2> x = read_all<float2>(argv[4]);
    const bool two = !std::strcmp(mode, "fft2");
    const bool ok = S > 0 ? (two ? fft2_any<1>(L, x) : dft_any<1>(L, x))
                          : (two ? fft2_any<-1>(L, x) : dft_any<-1>(L, x));
    if (!ok) return 3;
    write_all(argv[5], x);
    return 0;
  }
  if (!std::strcmp(mode, "d2f")) {
    std::vector<double> x = read_all<double>(argv[2]);
    std::vector<float> y(x.size());
    for (size_t i = 0; i < x.size(); ++i) y[i] = fpb::f64_to_f32_rn(x[i]);
    write_all(argv[3], y);
    return 0;
  }
  if (!std::strcmp(mode, "f2d")) {
    if (argc != 5) return 2;
    const int e2 = std::atoi(argv[2]);
    std::vector<float> x = read_all<float>(argv[3]);
    std::vector<double> y(x.size());
    for (size_t i = 0; i < x.size(); ++i) y[i] = fpb::f32_to_f64_pow2(x[i], e2);
    write_all(argv[4], y);
    return 0;
  }
  return 2;
}
