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

// One op as the tensor-core kernel reads it: a single 64-byte record with the
// offsets of its operand images, so that walking a unit's ops is one load per
// op (the next one prefetched while the current one runs).
struct alignas(16) TcOp {
  int64_t img[2];                    // forward / transposed image (element offsets)
  int32_t mo, ni;
  int32_t in_off[2], in_len[2];
  int32_t out_off[2], out_len[2];
  int32_t flags, phase;
};
static_assert(sizeof(TcOp) == 64, "TcOp layout");

struct TcPlan {
  const Unit* units;
  const TcOp* ops;          // the program's ops, same order
  const int32_t* tiles;     // per unit: [forward, inverse] number of N tiles of all its ops
  const int32_t* order;
  const uint16_t* img;      // split-BF16 operand images of every op
  const double* w;
  unsigned char* ws;        // per-CTA scratch: max_rows rows of kTcRowBytes
  // Accumulated rows of every work item (forward: Y_e, Y_o; inverse: X), FP32,
  // kTcR values per row, kTcAccRows(N) rows per item; item (group g, order
  // |m|) at (g * nunits + |m|) * kTcAccRows(N) rows.  Zero before a launch.
  float* acc;
  int gmax;                 // field groups the accumulation buffer holds
  unsigned int* counter;
  int* err;                 // set to 1 when a bounded wait gives up
  int N;
  int nunits;
  int max_rows;
};

// Rows of one work item's accumulation region: the 2N outputs forward, the
// 2N - |m| <= 2N inputs of the transposed apply.
__host__ __device__ inline int kTcAccRows(int N) { return 2 * N; }

// Elements of the split-BF16 image of an NN x KK block (3 pieces, padded).
size_t tc_image_elems(int NN, int KK);

// Build the forward (NN = mo, KK = ni) and transposed (NN = ni, KK = mo)
// images of every op from the FP64 factor store, the kernel's op records and
// the per-unit tile counts.
void tc_build_images(const std::vector<Unit>& units, const std::vector<Op>& ops, const std::vector<double>& factors,
                     std::vector<uint16_t>& img, std::vector<TcOp>& tops, std::vector<int32_t>& tiles);

// One apply: clear the accumulation rows, run the persistent tensor-core
// kernel (gather, block products), then the output kernel (parity fold to g,
// or scatter to beta).  F <= kTcFields * p.gmax.
// ev (optional, three events): recorded before the tensor-core kernel, between
// it and the output kernel, and after the output kernel.
cudaError_t launch_tc(const TcPlan& p, bool fwd, const double* in, double* out, int F, int single, int m, int grid,
                      cudaStream_t st, cudaEvent_t* ev = nullptr);

size_t tc_smem_bytes();
int tc_ctas_per_sm();

}  // namespace sht
