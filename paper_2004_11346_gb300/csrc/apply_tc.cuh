// Tensor-core (tcgen05) many-field apply: internal interface.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <functional>
#include <vector>

#include "program.hpp"

namespace sht {

constexpr int kTcFields = 32;            // fields per work item
constexpr int kTcR = 4 * kTcFields;      // 128 right-hand sides = MMA M
constexpr int kTcNT = 128;               // N tile (rows of one block product per MMA)
constexpr int kTcKC = 32;                // K chunk per pipeline stage
constexpr int kTcThreads = 512;          // producer, MMA, 2 item, 8 epilogue and 4 output warps
constexpr int kTcRowBytes = 3 * kTcR * 2;  // one scratch row: 3 BF16 pieces x 128 values
// The scratch stores rows in groups of 8 in the tensor cores' K-major core
// matrix layout, so that a run of whole groups is the A operand of a K chunk
// as it sits in shared memory and moves with one bulk copy, and so that one
// thread holding eight consecutive rows of one right-hand side writes them as
// one 16-byte store per piece:
//   group g = row / 8, piece p, right-hand side j, row-in-group e = row % 8:
//   byte (g * 3 + p) * 2048 + j * 16 + e * 2.
constexpr int kTcGrpRows = 8;
constexpr int kTcGrpBytes = kTcGrpRows * kTcRowBytes;  // 6144

__host__ __device__ inline int tc_r8(int v) { return (v + 7) & ~7; }

// Scratch rows of one order's vector space.  The logical layout of a unit is
// X_e (nce rows), X_o (nco), Y_e (N), Y_o (N), then the intermediate segments,
// each of which starts on a multiple of 8.  The tensor-core path moves X_o, Y_e
// and Y_o to group boundaries too, so that every group holds rows of one
// region only: a group of X_e is 8 even degrees, a group of Y_e 8 nodes.  The
// intermediates keep their alignment (shifted by a multiple of 8).
struct TcRows {
  int xo, ye, yo;  // scratch rows of X_o, Y_e, Y_o (X_e starts at 0)
  int shift;       // intermediate row r (logical) -> r + shift
};
__host__ __device__ inline TcRows tc_rows(int nce, int nco, int N) {
  TcRows t;
  t.xo = tc_r8(nce);
  t.ye = tc_r8(t.xo + nco);
  t.yo = t.ye + tc_r8(N);
  t.shift = tc_r8(t.yo + N) - tc_r8(nce + nco + 2 * N);
  return t;
}
// Scratch row of the first row of a logical segment at `off` (each segment
// lies inside one region).
__host__ __device__ inline int tc_seg_row(int off, int nce, int nco, int N, const TcRows& t) {
  if (off < nce) return off;
  if (off < nce + nco) return off - nce + t.xo;
  if (off < nce + nco + N) return off - (nce + nco) + t.ye;
  if (off < nce + nco + 2 * N) return off - (nce + nco + N) + t.yo;
  return off + t.shift;
}
// Rows of an order's scratch vector space.
__host__ __device__ inline int tc_nrows(int nrows, int nce, int nco, int N) {
  const TcRows t = tc_rows(nce, nco, N);
  return nrows + t.shift > t.yo + N ? nrows + t.shift : t.yo + N;
}

// Bytes of one work item's vector space (max_rows scratch rows, whole groups,
// plus a spare group so that a padded K chunk never reads past the slot).
__host__ __device__ inline size_t tc_slot_bytes(int max_rows) {
  return ((size_t)(max_rows + kTcGrpRows - 1) / kTcGrpRows + 1) * kTcGrpBytes;
}

// Accumulated FP32 rows of one work item (kTcR values per row): forward, Y_e
// at rows 0..N-1 and Y_o at r8(N)..; transposed, X_e at 0.. and X_o at
// r8(nce)..
__host__ __device__ inline int tc_acc_rows(int N) { return 2 * N + 8; }
// Row groups of one item's pre-gathered inputs: at most 2 r8(N) rows, both
// for the forward's X_e, X_o (nce, nco <= N) and the transposed Y_e, Y_o
// (rows ye .. yo + N, yo = ye + r8(N)).
__host__ __device__ inline int tc_pre_groups(int N) { return 2 * tc_r8(N) / kTcGrpRows; }

// One side of a block product, widened to whole row groups: its rows are the
// two row segments (off0, len0), (off1, len1) of the scratch vector space, and
// position 8 j + e stands for row 8 G(j) + e with G(j) = gs0 + j for the first
// ng0 groups and gs1 + j - ng0 after; rows outside the segments stand for
// nothing (zero in the operand image).  On the K side, chunks are 4 groups
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
// Group of the scratch behind widened position group j.
__host__ __device__ inline int tc_group(const TcKGeom& g, int j) { return j < g.ng0 ? g.gs0 + j : g.gs1 + j - g.ng0; }

// One op as the tensor-core kernel reads it: a single 64-byte record with the
// offsets of its operand images and its segments in scratch rows.  Besides
// the program's flags, an accumulating op is marked to store (not add) in a
// direction when none of its output rows was written by an earlier op of the
// order in that direction's processing order: it is their first writer, and
// those rows need no zeroing beforehand.
constexpr int32_t kTcFwdStore = 1 << 8;
constexpr int32_t kTcBwdStore = 1 << 9;
struct alignas(16) TcOp {
  int64_t img[2];                    // forward / transposed image (element offsets)
  int32_t mo, ni;
  int32_t in_off[2], in_len[2];
  int32_t out_off[2], out_len[2];
  int32_t flags, phase;
};
static_assert(sizeof(TcOp) == 64, "TcOp layout");

// The shape of one op in one direction (forward: out = B in; transposed:
// in = B^T out).  The N side is the output: rows that accumulate into the
// FP32 rows of the item (Y forward, X transposed) are N positions one to one;
// every other output (intermediate rows, each with a single writer) is
// widened to whole groups like the K side, so that its epilogue writes whole
// groups.  N tiles of kTcNT positions, the last padded to 16.
struct TcDir {
  int NN;       // N positions
  int nT;       // N tiles
  int KK;       // unwidened K side
  int accum;    // outputs accumulate in FP32
  int store;    // ... and this op is their first writer: plain stores
  TcKGeom ng;   // widened output side (when !accum)
  TcKGeom kg;   // widened input side
};
__host__ __device__ inline TcDir tc_dir(const TcOp& op, bool fwd) {
  const int32_t* io = fwd ? op.in_off : op.out_off;
  const int32_t* il = fwd ? op.in_len : op.out_len;
  const int32_t* oo = fwd ? op.out_off : op.in_off;
  const int32_t* ol = fwd ? op.out_len : op.in_len;
  TcDir d;
  d.accum = (op.flags & (fwd ? OP_FWD_ACCUM : OP_BWD_ACCUM)) != 0;
  d.store = d.accum && (op.flags & (fwd ? kTcFwdStore : kTcBwdStore)) != 0;
  d.KK = fwd ? op.ni : op.mo;
  d.kg = tc_kgeom(io[0], il[0], io[1], il[1]);
  if (d.KK <= 0) d.kg.nK = d.kg.ngt = d.kg.kp_tot = 0;
  d.ng = tc_kgeom(oo[0], ol[0], oo[1], ol[1]);
  d.NN = d.accum ? (fwd ? op.mo : op.ni) : kTcGrpRows * d.ng.ngt;
  d.nT = (d.NN + kTcNT - 1) / kTcNT;
  return d;
}

// Elements of the split-BF16 image of one direction (3 pieces, padded); 0
// when the op has no K side.
__host__ __device__ inline size_t tc_image_elems(const TcDir& d) {
  if (d.NN <= 0 || d.kg.kp_tot <= 0) return 0;
  const size_t np_tot = (size_t)kTcNT * (d.nT - 1) + ((d.NN - kTcNT * (d.nT - 1) + 15) & ~15);
  return 3 * np_tot * (size_t)d.kg.kp_tot;
}

// The op with its segments moved to scratch rows (unit u of order N).
TcOp tc_op_of(const Op& op, const Unit& u, int N);

struct TcPlan {
  const Unit* units;
  const TcOp* ops;          // the program's ops, same order, in scratch rows
  const int32_t* tiles;     // per unit: [forward, transposed] number of N tiles of all its ops
  const int32_t* order;
  // The kernel's processing order of each unit's ops, per direction: op
  // indices for positions op_begin .. op_end - 1 (tc_proc_order)
  const int32_t* ford;
  const int32_t* tord;
  const uint16_t* img;      // split-BF16 operand images of every op
  // Accumulation rows that no storing op writes first, as (first row, rows)
  // ranges: order u in direction d (0 forward, 1 transposed) owns ranges
  // zr[zri[2u + d] .. zri[2u + d + 1]).  Only these are zeroed per item.
  const int32_t* zr;
  const int32_t* zri;
  // Per unit: the node rows i < live of Y_e and Y_o that some op writes
  // forward (reads transposed), a multiple of 8 (tc_live_rows); the others
  // hold zero forward and are not gathered transposed
  const int32_t* live;
  const float* w32;          // w_{N+i} rounded to FP32, i < N
  // Accumulated rows of every work item (forward: Y_e, Y_o; transposed: X),
  // item (field group g, order |m|) at (g * nunits + |m|) * tc_acc_rows(N)
  // rows.  The kernel's item warps zero an item's rows (those no op stores
  // first) when they take the item; the output step reads them.
  float* acc;
  // Inputs gathered ahead by tc_in_kernel, the row groups of every item at
  // (g * nunits + |m|) * tc_pre_groups(N) groups: forward, X_e and X_o as
  // they sit from scratch group 0; transposed, the W-weighted parity fold of g
  // as Y_e, Y_o from scratch group ye / 8.  Required: the kernel gathers
  // no inputs itself
  unsigned char* pre;
  int gmax;                 // field groups the accumulation buffer holds
  int N;
  int nunits;
  int max_rows;             // scratch rows of the largest order
};

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
  // The output warps write each finished item's outputs (the output kernel
  // then does not run); otherwise the output kernel runs after the launch.
  int fuse_out;
  // Self-test of the bounded waits: the item warps publish no item, so every
  // other role's wait for its first item runs out and the launch reports a
  // timeout through err.
  int stall;
};

// The split-BF16 image of one op in one direction (forward: B, transposed:
// B^T), exactly as tc_build_images lays it out for the kernel; `top` is the
// op in scratch rows (tc_op_of).
void tc_op_image(const Op& op, const TcOp& top, const double* factors, bool transposed, std::vector<uint16_t>& out);

// Build the forward and transposed images of every op from the FP64 factor
// store, the kernel's op records (with the store marks) and the per-unit tile
// counts; max_rows gets the scratch rows of the largest order.
using TcImages = std::vector<uint16_t, UninitAlloc<uint16_t>>;
void tc_build_images(int N, const std::vector<Unit>& units, const std::vector<Op>& ops, const double* factors,
                     TcImages& img, std::vector<TcOp>& tops, std::vector<int32_t>& tiles, int& max_rows);
// The same in parts, so that a large store need not sit on the host whole:
// the layout (op records, tile counts, total elements), then the images of
// ops [i0, i1) packed at dst[offset - base], and a driver that packs windows
// of consecutive ops spanning at most `window` elements (more for one op that
// is larger) into a reusable buffer and hands each to `sink` as (first
// element, data, elements); a false return from `sink` stops it.
size_t tc_image_layout(int N, const std::vector<Unit>& units, const std::vector<Op>& ops, std::vector<TcOp>& tops,
                       std::vector<int32_t>& tiles, int& max_rows);
void tc_pack_ops(const std::vector<Op>& ops, const std::vector<TcOp>& tops, const double* factors, size_t i0,
                 size_t i1, uint16_t* dst, size_t base);
void tc_pack_windows(const std::vector<Op>& ops, const std::vector<TcOp>& tops, const double* factors, size_t tot,
                     size_t window, const std::function<bool(size_t, const uint16_t*, size_t)>& sink);

// The store marks of the ops (in tops) and the zero ranges (zr, zri as in
// TcPlan) of every order, from the op records in scratch rows.
// The processing order of every unit's ops in each direction: forward,
// ascending phases; transposed, descending phases; within a phase the ops
// sorted by the first scratch row of the side they read (forward: the input
// rows, transposed: the output rows), so that products reading the same rows
// (the blocks of one column or row strip) run one after another and find them
// in L2.  ford / tord hold global op indices at the units' op positions.
void tc_proc_order(const std::vector<Unit>& units, const std::vector<TcOp>& tops, std::vector<int32_t>& ford,
                   std::vector<int32_t>& tord);
// Node rows that some op of each unit reaches: the Y_e and Y_o rows written
// forward (read transposed), counted from the first positive node and
// rounded up to whole groups.  The nodes past them, near the poles beyond
// every degree's turning point (Sec. 3.2), have g = 0 and are never read.
void tc_live_rows(int N, const std::vector<Unit>& units, const std::vector<TcOp>& tops, std::vector<int32_t>& live);
// First writers, in the processing order of ford / tord; the zeroed ranges
// leave out the node rows past live (the output step takes them as zero).
void tc_first_writers(int N, const std::vector<Unit>& units, std::vector<TcOp>& tops, const std::vector<int32_t>& ford,
                      const std::vector<int32_t>& tord, const std::vector<int32_t>& live, std::vector<int32_t>& zr,
                      std::vector<int32_t>& zri);

// One apply: the pre-gather of the inputs, then the persistent tensor-core
// kernel (block products into the accumulation rows), and the output step:
// forward, the parity fold to g by the output kernel after the launch;
// transposed, the scatter to beta by the tensor-core kernel's item warps as
// each item finishes.  F <= kTcFields * p.gmax.  ws holds grid CTAs' two
// scratch slots.  ev (optional, three events): recorded before the pre-gather,
// after the tensor-core kernel and after the output kernel (an empty interval
// when the output step ran inside the tensor-core kernel).
cudaError_t launch_tc(const TcPlan& p, bool fwd, const double* in, double* out, int F, int single, int m, int grid,
                      unsigned char* ws, unsigned int* counter, int* err, cudaStream_t st, cudaEvent_t* ev = nullptr);

// The same for a batch of plans in one launch of the tensor-core kernel (the
// launch's items, scratch and counter set up by the caller), after one
// pre-gather launch per plan; forward, one output kernel per plan after it.
// L.counter must be zero on the stream.
cudaError_t launch_tc_batch(const TcLaunch& L, bool fwd, int grid, cudaStream_t st, cudaEvent_t* ev = nullptr);

// The bounded-wait self-test on plan p (see TcLaunch::stall).
cudaError_t launch_tc_stall(const TcPlan& p, unsigned char* ws, unsigned int* counter, int* err, cudaStream_t st);

size_t tc_smem_bytes();
int tc_ctas_per_sm();

}  // namespace sht
