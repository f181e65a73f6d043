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
  unsigned ns_mul[kMaxPasses];  // floor(n / Ns) = umulhi(n, ns_mul) >> ns_shr (ns_mul 0: Ns = 1)
  int ns_shr[kMaxPasses];
  int chunk;           // split mode: positions per CTA of the cluster
  const C2<T>* tw;     // per pass: e^{+2 pi i t / (Ns R)}, t < Ns R
  const C2<T>* shift;  // e^{i pi m / M}, m = -(2N-1) .. 2N-1
  const int* perm;     // digit-reversed position of each input index
};

template <class T>
struct PhiTables {
  int N = 0, M = 0, npass = 0, n_tw = 0;
  // Whole-row mode: each CTA holds `nt` whole rows (adjacent nodes), cl = 1.
  // Split mode: one row spread over a cluster of `cl` CTAs, `chunk` positions
  // each (rows longer than one CTA's shared memory).
  bool split = false;
  int nt = 1, cl = 1, chunk = 0;
  bool two_buf = false;  // a radix without an in-place butterfly needs a second buffer
  int max_clusters = 0;  // co-resident CTAs (clusters in split mode); 0: no shape fits
  int radix[kMaxPasses] = {0}, ns[kMaxPasses] = {0}, tw_off[kMaxPasses] = {0};
  unsigned ns_mul[kMaxPasses] = {0};
  int ns_shr[kMaxPasses] = {0};
  void* d_tw = nullptr;
  void* d_shift = nullptr;
  void* d_perm = nullptr;
  bool build(int N);  // host tables, device upload and launch shape; false on a CUDA error
  void release();
  size_t smem_bytes() const;
  // synthesis (analysis = false): g (F x (4N-1) x 2N) -> f (F x 2N x (4N-1));
  // analysis: f -> g.  Complex FP64 interleaved.
  cudaError_t launch(const double* in, double* out, int F, bool analysis, cudaStream_t st) const;
};

}  // namespace sht
