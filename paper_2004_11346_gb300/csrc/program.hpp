// The apply program: what the plan builder hands to the CUDA kernels.
//
// For every order |m| (a "unit") the forward ALT applies the even and odd
// parity matrices of Sec. 3.1.2.  Each matrix is partitioned into blocks
// (Sec. 3.2) and every block is reduced to a short chain of dense block
// products (Sec. 3.3): one product for a trimmed turning-point block, two for
// a low-rank block (V^T then U Sigma), and L+3 for an IDBF block
// U^L ... U^h S^h V^h ... V^L (column-side levels, the middle S, row-side
// levels).  Every product ("op") maps up to two contiguous row segments of
// the unit's vector space to up to two contiguous row segments:
//
//     out[seg0 ; seg1] (+)= B * in[seg0 ; seg1]
//
// with B dense, column-major, leading dimension ld.  The vector space of a
// unit holds, in rows of R right-hand sides, the even and odd inputs X_e, X_o
// (coefficients by degree), the outputs Y_e, Y_o (values at the N positive
// Gauss-Legendre nodes) and the intermediate butterfly vectors Z.  Ops carry
// a phase: all inputs of an op are written in earlier phases.  The inverse
// ALT runs the same ops transposed in reverse phase order (B = A^T W).
#pragma once

#include <cstdint>
#include <memory>
#include <new>
#include <utility>
#include <vector>

namespace sht {

enum OpFlags : int32_t {
  OP_FWD_ACCUM = 1,   // forward output rows are shared with other ops: add
  OP_BWD_ACCUM = 2,   // forward input rows are shared: transposed output adds
};

struct Op {
  int64_t b_off;      // element offset of B in the factor store
  int32_t mo, ni;     // B is mo x ni
  int32_t ld;         // leading dimension of B (>= mo)
  int32_t flags;
  int32_t in_off[2], in_len[2];    // input segments (rows); in_len[0]+in_len[1] = ni
  int32_t out_off[2], out_len[2];  // output segments; out_len[0]+out_len[1] = mo
  int32_t phase;
  int32_t pad;
};
static_assert(sizeof(Op) == 64, "Op layout");

struct Unit {
  int32_t am;             // |m|
  int32_t op_begin;       // ops [op_begin, op_end) sorted by phase
  int32_t op_end;
  int32_t ph_begin;       // phase table entries [ph_begin, ph_begin + nphase + 1)
  int32_t nphase;
  int32_t nrows;          // rows of the vector space
  int32_t xe, xo, ye, yo; // row offsets of X_e, X_o, Y_e, Y_o
  int32_t nce, nco;       // number of even / odd degrees
  int32_t pad;
  float cost;             // estimated flops per right-hand side
};
static_assert(sizeof(Unit) == 56, "Unit layout");

// Allocator whose argument-less construction leaves an element uninitialised,
// so that resizing a store of many GB does not have one thread zero it (and
// touch every page) before the threads that fill it run.  Every element of a
// container using it must be written before it is read.
template <class T>
struct UninitAlloc : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = UninitAlloc<U>;
  };
  UninitAlloc() = default;
  template <class U>
  UninitAlloc(const UninitAlloc<U>&) noexcept {}
  template <class U>
  void construct(U* p) noexcept {
    ::new (static_cast<void*>(p)) U;
  }
  template <class U, class... A>
  void construct(U* p, A&&... a) {
    ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
  }
};

// The FP64 factor store of a program: packed blocks, column-major.
using FactorStore = std::vector<double, UninitAlloc<double>>;

}  // namespace sht
