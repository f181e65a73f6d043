// Tensor-core (tcgen05) many-field apply: internal interface.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "program.hpp"

namespace sht {

constexpr int kTcFields = 32;            // fields per work item
constexpr int kTcR = 4 * kTcFields;      // 128 right-hand sides = MMA M
constexpr int kTcNT = 128;               // N tile (rows of one block product)
constexpr int kTcKC = 32;                // K chunk per pipeline stage
constexpr int kTcThreads = 512;          // 3 producer, 1 MMA, 4 epilogue and 8 I/O warps
constexpr int kTcRowBytes = 3 * kTcR * 2;  // scratch row: 3 BF16 pieces x 128 (or 128 FP32)

struct TcPlan {
  const Unit* units;
  const Op* ops;
  const int32_t* phase_tab;
  const int32_t* order;
  const uint16_t* img;      // split-BF16 operand images of every op
  const int64_t* img_off;   // per op: [forward image, transposed image] element offsets
  const double* w;
  unsigned char* ws;        // per-CTA scratch: max_rows rows of kTcRowBytes
  unsigned int* counter;
  int* err;                 // set to 1 when a bounded wait gives up
  int N;
  int nunits;
  int max_rows;
};

// Elements of the split-BF16 image of an NN x KK block (3 pieces, padded).
size_t tc_image_elems(int NN, int KK);

// Build the forward (NN = mo, KK = ni) and transposed (NN = ni, KK = mo)
// images of every op from the FP64 factor store.
void tc_build_images(const std::vector<Op>& ops, const std::vector<double>& factors, std::vector<uint16_t>& img,
                     std::vector<int64_t>& off);

cudaError_t launch_tc(const TcPlan& p, bool fwd, const double* in, double* out, int F, int single, int m, int grid,
                      cudaStream_t st);

size_t tc_smem_bytes();
int tc_ctas_per_sm();

}  // namespace sht
