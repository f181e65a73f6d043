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
constexpr int kTcThreads = 512;          // producer, 2 spare, MMA, 4 epilogue and 8 I/O warps
constexpr int kTcRowBytes = 3 * kTcR * 2;  // one scratch row: 3 BF16 pieces x 128 values
// The scratch stores rows in groups of 8 in the tensor cores' MN-major core
// matrix layout, so that a run of whole groups is the A operand of a K chunk
// as it sits in shared memory and moves with one bulk copy:
//   group g = row / 8, piece p, 8-value chunk m8 of the 128 right-hand sides,
//   row-in-group e = row % 8:  byte (g * 3 + p) * 2048 + m8 * 128 + e * 16.
constexpr int kTcGrpRows = 8;
constexpr int kTcGrpBytes = kTcGrpRows * kTcRowBytes;  // 6144

// Bytes of one work item's vector space (max_rows rows, whole groups, plus a
// spare group so that a padded K chunk never reads past the slot).
__host__ __device__ inline size_t tc_slot_bytes(int max_rows) {
  return ((size_t)(max_rows + kTcGrpRows - 1) / kTcGrpRows + 1) * kTcGrpBytes;
}

// K side of one block product in a given direction: its input rows are the
// two row segments (off0, len0), (off1, len1) of the vector space.  They are
// widened to whole groups: K position 8 j + e is row 8 G(j) + e with
// G(j) = gs0 + j for the first ng0 slots and gs1 + j - ng0 after; rows outside
// the segments get zero columns in the operand image.  K chunks are 4 groups
// (32), the last one rounded up to a pair of groups (the MMA K step of 16).
struct TcKGeom {
  int gs0, ng0, gs1, ng1, ngt, nK, kp_tot;
};
__host__ __device__ inline TcKGeom tc_kgeom(int off0, int len0, int off1, int len1) {
  TcKGeom g;
  g.gs0 = off0 / kTcGrpRows;
  g.ng0 = len0 > 0 ? (off0 + len0 + kTcGrpRows - 1) / kTcGrpRows - g.gs0 : 0;
  g.gs1 = off1 / kTcGrpRows;
  g.ng1 = len1 > 0 ? (off1 + len1 + kTcGrpRows - 1) / kTcGrpRows - g.gs1 : 0;
  g.ngt = g.ng0 + g.ng1;
  g.nK = (g.ngt + 3) / 4;
  g.kp_tot = g.nK > 0 ? 32 * (g.nK - 1) + 16 * ((g.ngt - 4 * (g.nK - 1) + 1) / 2) : 0;
  return g;
}

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
  unsigned char* ws;        // per-CTA scratch: two vector spaces of tc_slot_bytes(max_rows)
  // Accumulated rows of every work item (forward: Y_e, Y_o; inverse: X), FP32,
  // kTcR values per row, kTcAccRows(N) rows per item; item (group g, order
  // |m|) at (g * nunits + |m|) * kTcAccRows(N) rows.  The kernel zeroes an item's
  // rows when it gathers the item.
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

// One launch of the tensor-core kernel: up to kTcMaxPlans plans (orders N of
// their own), each with its own batch of fields.  The work items are
// (plan, order |m|, field group); they share one work counter, the per-CTA
// scratch slots (sized for the largest plan) and the error flag.
constexpr int kTcMaxPlans = 8;
struct TcLaunch {
  TcPlan plan[kTcMaxPlans];
  const double* in[kTcMaxPlans];  // per plan: its F fields of beta (forward) or g (inverse)
  double* out[kTcMaxPlans];       // per plan: its F fields of g (forward) or beta (inverse)
  int F[kTcMaxPlans];
  int nplans;
  // Work items in processing order as (plan, |m|, field group, 0); null for
  // one plan, whose items are then its orders in cost order x its field groups
  const int4* items;
  int nitems;
  int single, msingle;            // one order msingle of plan 0 (alt_*_m)
  unsigned char* ws;              // per-CTA scratch: two slots of tc_slot_bytes(max_rows)
  int max_rows;
  unsigned int* counter;          // zero before the launch
  int* err;
  // Self-test of the bounded waits: the I/O warps publish no item, so every
  // other role's wait for its first item runs out and the launch reports a
  // timeout through err.
  int stall;
};

// Elements of the split-BF16 image of a block with NN rows and K side kg
// (3 pieces, padded).
size_t tc_image_elems(int NN, const TcKGeom& kg);

// The split-BF16 image of one op in one direction (forward: B, transposed:
// B^T), exactly as tc_build_images lays it out for the kernel.
void tc_op_image(const Op& op, const double* factors, bool transposed, std::vector<uint16_t>& out);

// Build the forward (NN = mo, KK = ni) and transposed (NN = ni, KK = mo)
// images of every op from the FP64 factor store, the kernel's op records and
// the per-unit tile counts.
using TcImages = std::vector<uint16_t, UninitAlloc<uint16_t>>;
void tc_build_images(const std::vector<Unit>& units, const std::vector<Op>& ops, const double* factors,
                     TcImages& img, std::vector<TcOp>& tops, std::vector<int32_t>& tiles);

// One apply: run the persistent tensor-core
// kernel (gather, block products), then the output kernel (parity fold to g,
// or scatter to beta).  F <= kTcFields * p.gmax.
// ev (optional, three events): recorded before the tensor-core kernel, between
// it and the output kernel, and after the output kernel.
cudaError_t launch_tc(const TcPlan& p, bool fwd, const double* in, double* out, int F, int single, int m, int grid,
                      cudaStream_t st, cudaEvent_t* ev = nullptr);

// The same for a batch of plans in one launch of the tensor-core kernel (the
// launch's items, scratch and counter set up by the caller), followed by one
// output kernel per plan.  L.counter must be zero on the stream.
cudaError_t launch_tc_batch(const TcLaunch& L, bool fwd, int grid, cudaStream_t st, cudaEvent_t* ev = nullptr);

// The bounded-wait self-test on plan p (see TcLaunch::stall).
cudaError_t launch_tc_stall(const TcPlan& p, int grid, cudaStream_t st);

size_t tc_smem_bytes();
int tc_ctas_per_sm();

}  // namespace sht
