// Dense ALT with the Legendre recurrence run on the fly (internal; see
// alt_direct.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace sht {

// Pbar_k^{|m|} at the N positive nodes on the device (the recurrence of the
// on-the-fly transform, on its own): nodes, sqrt(1 - x^2) and the sectoral
// constants of a plan.
struct LegendreDev {
  int N = 0;
  double* d_x = nullptr;
  double* d_s = nullptr;
  double* d_cm = nullptr;
  cudaError_t build(int N, const double* x);  // x: the 2N-point rule, ascending
  void release();
  // out[t * N + i] = Pbar_{am+t}^{am}(x_{N+i}), t < 2N - am, i < N; coef: 2(2N)
  // doubles of scratch.  Asynchronous on st.
  cudaError_t table(int am, double* out, double* coef, cudaStream_t st) const;
};

struct DirectPlan {
  int N = 0, F_max = 0, R_max = 0, grid = 0;
  size_t per_cta = 0;               // scratch doubles per CTA
  double* d_x = nullptr;            // positive nodes x_{N+i}, i < N
  double* d_s = nullptr;            // sqrt(1 - x^2) at those nodes
  double* d_w = nullptr;            // their weights w_{N+i}
  double* d_cm = nullptr;           // Pbar_a^a(x) / (1 - x^2)^{a/2}, a < 2N
  double* d_scratch = nullptr;      // grid * per_cta doubles
  unsigned int* d_counter = nullptr;
  // nodes x and weights w: the 2N-point rule, ascending; F_max fields per call
  cudaError_t build(int N, int F_max, const double* x, const double* w, int sms);
  void release();
  // forward: beta (F x 4N^2 complex) -> g (F x (4N-1) x 2N complex);
  // inverse: g -> beta.  F <= F_max.
  cudaError_t launch(bool fwd, const double* in, double* out, int F, cudaStream_t st) const;
};

}  // namespace sht
