// Many-field FP32 apply (internal interface between apply.cu and apply_f32.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "program.hpp"

namespace sht {

// Right-hand sides per work item: 8 fields x (Re, Im) x (+m, -m).
constexpr int kF32Fields = 8;
constexpr int kF32RT = 4 * kF32Fields;

struct F32Plan {
  const Unit* units;
  const Op* ops;
  const int32_t* phase_tab;
  const int32_t* order;
  const float* fac;   // FP32 copy of the factor store (same offsets)
  const double* w;    // 2N Gauss-Legendre weights
  float* ws;          // per-CTA scratch: max_rows x kF32RT floats each
  unsigned int* counter;
  int N;
  int nunits;
  int max_rows;
};

// Forward (fwd) or inverse ALT of F fields in FP32 arithmetic with FP64 I/O.
// single != 0: one order m with compact per-order arrays (see alt_forward_m).
cudaError_t launch_f32(const F32Plan& p, bool fwd, const double* in, double* out, int F, int single, int m,
                       int grid, cudaStream_t st);

// Resident CTAs per SM of the FP32 kernels.
int f32_ctas_per_sm();

}  // namespace sht
