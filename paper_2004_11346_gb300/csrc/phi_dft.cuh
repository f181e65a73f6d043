// phi-direction DFT tables and launcher (internal; see phi_dft.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace sht {

template <class T>
struct C2;

constexpr int kMaxPasses = 16;

template <class T>
struct PhiPlanDev {
  int N, M, npass;
  int radix[kMaxPasses], ns[kMaxPasses], tw_off[kMaxPasses];
  const C2<T>* tw;     // per pass: e^{+2 pi i t / (Ns R)}, t < Ns R
  const C2<T>* shift;  // e^{i pi m / M}, m = -(2N-1) .. 2N-1
  const int* perm;     // digit-reversed position of each input index
};

template <class T>
struct PhiTables {
  int N = 0, M = 0, npass = 0, n_tw = 0;
  int nt = 1;            // rows (adjacent nodes) per CTA
  bool two_buf = false;  // a radix without an in-place butterfly needs a second buffer
  int radix[kMaxPasses] = {0}, ns[kMaxPasses] = {0}, tw_off[kMaxPasses] = {0};
  void* d_tw = nullptr;
  void* d_shift = nullptr;
  void* d_perm = nullptr;
  bool build(int N);  // host tables + device upload
  void release();
  size_t smem_bytes() const;
  // synthesis (analysis = false): g (F x (4N-1) x 2N) -> f (F x 2N x (4N-1));
  // analysis: f -> g.  Complex FP64 interleaved.
  cudaError_t launch(const double* in, double* out, int F, bool analysis, int grid, cudaStream_t st) const;
};

}  // namespace sht
