// Many-field apply of the IDBF-factored ALT on the 5th-generation tensor
// cores (tcgen05, sm_103a), split-BF16 products with FP32 accumulation.
//
// One work item is one order |m| for 32 fields: 128 real right-hand sides.
// Every block product of the apply program, out (+)= B in, is computed
// transposed, out^T = in^T B^T, so that the 128 right-hand sides fill the MMA
// M dimension and the block's rows are N (tiles of <= 128, padded to 16):
//   A operand = in^T (128 x K, MN-major): the op's input rows, kept in the
//               scratch as three BF16 pieces a0 + a1 + a2 (8 bits each) of
//               every value, in groups of 8 rows laid out exactly as the
//               operand sits in shared memory, so that staging one K chunk
//               is one or two bulk copies of whole groups;
//   B operand = B (N x K, K-major): precomputed split-BF16 image b0 + b1 + b2,
//               with zero columns where the K side was widened to whole groups;
//   D         = 128 x N FP32 accumulator in tensor memory.
// The CTA is warp-specialised and persistent (one per SM): one producer
// thread streams (op, tile, 32-wide K chunk) operand stages into a 4-deep
// shared memory ring with bulk copies; an MMA thread issues the tensor-core
// products into two double-buffered TMEM accumulator pairs; four epilogue
// warps drain the accumulators and split the results into BF16 pieces for the
// next level (or add them in FP32 into the shared output rows); the I/O warps
// gather the next item's inputs.  Ops of one phase read only rows written by
// earlier phases: the producer starts a phase after the epilogue has counted
// every earlier tile.
// Per 16-wide K step six MMAs accumulate a_p b_q for p + q <= 2, which keeps
// every product to about 2^-24 relative error (FP32 quality); a0 b0 and the
// five smaller cross products go to two separate accumulators that the
// epilogue adds in FP32.  Operands sit in shared memory in the canonical
// no-swizzle layouts (8 x 16-byte core matrices; LBO = stride between core
// matrices along K, SBO = along M/N).
// All waits are bounded: a wait that runs out sets an error flag, every role
// stops, and the host reports SHT_ERR_TIMEOUT.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "apply_tc.cuh"
#include "f64_bits.cuh"

namespace sht {

// ---------------------------------------------------------------- host image build
static inline int r16(int v) { return (v + 15) & ~15; }

static inline uint16_t bf16_rn(float f) {
  uint32_t b;
  std::memcpy(&b, &f, 4);
  b += 0x7FFFu + ((b >> 16) & 1u);
  return (uint16_t)(b >> 16);
}
static inline double bf16_to_d(uint16_t h) {
  uint32_t b = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &b, 4);
  return (double)f;
}

size_t tc_image_elems(int NN, const TcKGeom& kg) {
  if (NN <= 0 || kg.kp_tot <= 0) return 0;
  const int nT = (NN + kTcNT - 1) / kTcNT;
  const size_t np_tot = (size_t)kTcNT * (nT - 1) + r16(NN - kTcNT * (nT - 1));
  return 3 * np_tot * (size_t)kg.kp_tot;
}

// Layout (matching the kernel): tiles t, chunks c, pieces p, then core
// matrices (ki, mi) in K-outer order, 8 rows x 8 elements each.  elem(n, k)
// is the block entry for row n and K index k of the unwidened K side; K
// positions that fall outside both segments (group widening, padding) are 0.
// Piece p of a value v is the BF16 rounding of what pieces 0..p-1 leave of v.
// Each (tile, chunk) is first gathered into a small buffer, walking the source
// along its contiguous direction (k_contig: consecutive K indices adjacent),
// and the three pieces of every value are computed in one pass.
template <class E>
static void tc_pack(int NN, const TcKGeom& kg, int off0, int len0, int off1, int len1, E elem, bool k_contig,
                    uint16_t* dst) {
  const int nT = (NN + kTcNT - 1) / kTcNT;
  auto korig = [&](int kp) -> int {  // widened K position -> K index, or -1
    const int j = kp / kTcGrpRows, e = kp % kTcGrpRows;
    if (j < kg.ng0) {
      const int r = (kg.gs0 + j) * kTcGrpRows + e;
      return r >= off0 && r < off0 + len0 ? r - off0 : -1;
    }
    if (j < kg.ngt) {
      const int r = (kg.gs1 + j - kg.ng0) * kTcGrpRows + e;
      return r >= off1 && r < off1 + len1 ? len0 + r - off1 : -1;
    }
    return -1;
  };
  std::vector<double> buf((size_t)kTcNT * kTcKC);
  size_t o = 0;
  for (int t = 0; t < nT; ++t) {
    const int Nv = std::min(kTcNT, NN - kTcNT * t);  // valid rows of the tile
    const int Np = r16(Nv);
    for (int c = 0; c < kg.nK; ++c) {
      const int Kp = std::min(kTcKC, kg.kp_tot - kTcKC * c);
      int ko[kTcKC];
      for (int kk = 0; kk < Kp; ++kk) ko[kk] = korig(kTcKC * c + kk);
      // buf[n * Kp + kk] = entry (tile row n, chunk column kk), zero outside
      std::fill(buf.begin(), buf.begin() + (size_t)Np * Kp, 0.0);
      if (k_contig) {
        for (int n = 0; n < Nv; ++n)
          for (int kk = 0; kk < Kp; ++kk)
            if (ko[kk] >= 0) buf[(size_t)n * Kp + kk] = elem(kTcNT * t + n, ko[kk]);
      } else {
        for (int kk = 0; kk < Kp; ++kk)
          if (ko[kk] >= 0)
            for (int n = 0; n < Nv; ++n) buf[(size_t)n * Kp + kk] = elem(kTcNT * t + n, ko[kk]);
      }
      const size_t piece = (size_t)Np * Kp;
      for (int n = 0; n < Np; ++n) {
        const int mi = n / 8, rr = n % 8;
        for (int kk = 0; kk < Kp; ++kk) {
          const int ki = kk / 8;
          const size_t at = o + ((size_t)ki * (Np / 8) + mi) * 64 + rr * 8 + kk % 8;
          double v = buf[(size_t)n * Kp + kk];
          for (int p = 0; p < 3; ++p) {
            const uint16_t h = bf16_rn((float)v);
            v -= bf16_to_d(h);
            dst[at + p * piece] = h;
          }
        }
      }
      o += 3 * piece;
    }
  }
}

void tc_op_image(const Op& op, const double* factors, bool transposed, std::vector<uint16_t>& out) {
  out.clear();
  if (op.ni <= 0) return;
  const double* B = factors + op.b_off;
  const int ld = op.ld;
  if (!transposed) {
    const TcKGeom kg = tc_kgeom(op.in_off[0], op.in_len[0], op.in_off[1], op.in_len[1]);
    out.assign(tc_image_elems(op.mo, kg), 0);
    tc_pack(op.mo, kg, op.in_off[0], op.in_len[0], op.in_off[1], op.in_len[1],
            [&](int r, int k) { return B[(size_t)k * ld + r]; }, false, out.data());
  } else {
    const TcKGeom kg = tc_kgeom(op.out_off[0], op.out_len[0], op.out_off[1], op.out_len[1]);
    out.assign(tc_image_elems(op.ni, kg), 0);
    tc_pack(op.ni, kg, op.out_off[0], op.out_len[0], op.out_off[1], op.out_len[1],
            [&](int r, int k) { return B[(size_t)r * ld + k]; }, true, out.data());
  }
}

void tc_build_images(const std::vector<Unit>& units, const std::vector<Op>& ops, const double* factors,
                     TcImages& img, std::vector<TcOp>& tops, std::vector<int32_t>& tiles) {
  const size_t n = ops.size();
  tops.assign(n, TcOp{});
  size_t tot = 0;
  for (size_t i = 0; i < n; ++i) {
    const Op& op = ops[i];
    TcOp& t = tops[i];
    t.img[0] = (int64_t)tot;
    tot += tc_image_elems(op.mo, tc_kgeom(op.in_off[0], op.in_len[0], op.in_off[1], op.in_len[1]));
    t.img[1] = (int64_t)tot;
    tot += tc_image_elems(op.ni, tc_kgeom(op.out_off[0], op.out_len[0], op.out_off[1], op.out_len[1]));
    t.mo = op.mo;
    t.ni = op.ni;
    for (int s = 0; s < 2; ++s) {
      t.in_off[s] = op.in_off[s];
      t.in_len[s] = op.in_len[s];
      t.out_off[s] = op.out_off[s];
      t.out_len[s] = op.out_len[s];
    }
    t.flags = op.flags;
    t.phase = op.phase;
  }
  tiles.assign(2 * units.size(), 0);
  for (size_t u = 0; u < units.size(); ++u)
    for (int oi = units[u].op_begin; oi < units[u].op_end; ++oi) {
      tiles[2 * u] += (ops[oi].mo + kTcNT - 1) / kTcNT;
      tiles[2 * u + 1] += (ops[oi].ni + kTcNT - 1) / kTcNT;
    }
  // tc_pack writes every element of an op's two images (padding included),
  // so only the minimum-size tail of an empty store needs zeroing here
  img.resize(std::max<size_t>(tot, 8));
  std::fill(img.begin() + tot, img.end(), (uint16_t)0);
#pragma omp parallel for schedule(dynamic, 64)
  for (long i = 0; i < (long)n; ++i) {
    const Op& op = ops[i];
    const double* B = factors + op.b_off;
    const int ld = op.ld;
    if (op.ni > 0) {
      const TcKGeom kf = tc_kgeom(op.in_off[0], op.in_len[0], op.in_off[1], op.in_len[1]);
      const TcKGeom kb = tc_kgeom(op.out_off[0], op.out_len[0], op.out_off[1], op.out_len[1]);
      tc_pack(op.mo, kf, op.in_off[0], op.in_len[0], op.in_off[1], op.in_len[1],
              [&](int r, int k) { return B[(size_t)k * ld + r]; }, false, img.data() + tops[i].img[0]);
      tc_pack(op.ni, kb, op.out_off[0], op.out_len[0], op.out_off[1], op.out_len[1],
              [&](int r, int k) { return B[(size_t)r * ld + k]; }, true, img.data() + tops[i].img[1]);
    }
  }
}

// ---------------------------------------------------------------- device side
namespace {

constexpr int kStages = 4;
constexpr int kProdWarps = 3;                 // warp 0 stages operands (one thread); warps 1-2 are spare
constexpr int kMmaWarp = kProdWarps;          // the MMA-issuing warp
constexpr int kEpiWarp0 = kProdWarps + 1;     // first epilogue warp
constexpr int kEpiWarps = 4;                  // one warpgroup drains the accumulators
constexpr int kIoWarp0 = kEpiWarp0 + kEpiWarps;  // the remaining warps gather the next item's inputs
constexpr int kIoWarps = kTcThreads / 32 - kIoWarp0;
constexpr int kTrStride = 33;                 // padded 32 x 32 transpose tile (floats)
constexpr int kStageA = (kTcKC / kTcGrpRows) * kTcGrpBytes;  // 4 row groups: 24 KB
constexpr int kStageB = 3 * kTcNT * kTcKC * 2; // 24 KB (largest N tile)
constexpr int kStageBytes = kStageA + kStageB;
constexpr int kTmemCols = 512;                 // 2 accumulator pairs (hi, lo) x 128 columns
constexpr long kWaitLimit = 1L << 22;   // try_wait polls per bounded wait

struct Ctl {
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t accf[2];
  uint64_t acce[2];
  uint32_t taddr;
  int abort;
  int gathered;    // items whose gather is complete (or found the queue empty)
  int done_tiles;  // tiles whose epilogue is complete (all items so far)
  int ring[4];     // item index of this CTA's item iseq at ring[iseq % 4]; -1 = no more
};
constexpr size_t kTrBytes = (size_t)kEpiWarps * 32 * kTrStride * 4;
// I/O transpose tile: 32 rows x 128 FP32 columns (row stride padded to 132
// floats: 16-byte aligned rows, conflict-free 8-row column reads)
constexpr int kIoStride = 132;
constexpr size_t kIoBytes = (size_t)32 * kIoStride * 4;
constexpr int kPairsPerIo = 2 * kTcFields / kIoWarps;  // (field, sign) pairs per I/O warp
static_assert(kPairsPerIo * kIoWarps == 2 * kTcFields, "I/O warps split the pairs evenly");
constexpr size_t kSmemTotal = (size_t)kStages * kStageBytes + kTrBytes + kIoBytes + sizeof(Ctl) + 1024;
static_assert(kSmemTotal <= 232448, "fits the 227 KB of shared memory one CTA may use");

__device__ __forceinline__ uint32_t s32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t addr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(addr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s32(bar)) : "memory");
}
// Bounded wait for the phase with the given parity; on running out, flag an abort.
__device__ __forceinline__ bool mbar_wait(Ctl* ctl, uint64_t* bar, uint32_t parity) {
  for (long it = 0; it < kWaitLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(s32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 255) == 255 && *((volatile int*)&ctl->abort)) return false;
  }
  *((volatile int*)&ctl->abort) = 1;
  return false;
}
// Bounded wait for a bulk copy still in flight after an abort: the CTA must
// not exit while a copy can still write its shared memory.
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
  for (long it = 0; it < kWaitLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(s32(bar)), "r"(parity)
        : "memory");
    if (ok) return;
  }
}
// Bounded wait until a shared counter reaches `target`.
__device__ __forceinline__ bool counter_wait(Ctl* ctl, int* ctr, int target) {
  for (long it = 0; it < kWaitLimit; ++it) {
    if (*((volatile int*)ctr) >= target) {
      __threadfence_block();
      return true;
    }
    if (*((volatile int*)&ctl->abort)) return false;
    __nanosleep(256);
  }
  *((volatile int*)&ctl->abort) = 1;
  return false;
}

// This CTA's item number iseq as the I/O warps published it, once its inputs
// are gathered; -1 when the work counter ran out.
__device__ __forceinline__ int next_item(Ctl* ctl, int iseq, bool& ok) {
  ok = counter_wait(ctl, &ctl->gathered, iseq + 1);
  return ok ? *((volatile int*)&ctl->ring[iseq & 3]) : -1;
}

__device__ __forceinline__ void bulk_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(s32(bar))
      : "memory");
}
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
__device__ __forceinline__ void io_bar() { asm volatile("bar.sync 2, %0;" ::"n"(32 * kIoWarps) : "memory"); }
// The named barriers with an AND over the group: every warp of the group takes
// the same decision after a bounded wait, so none is left at a barrier alone.
__device__ __forceinline__ bool epi_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred q, r;\n setp.ne.u32 q, %1, 0;\n bar.red.and.pred r, 1, 128, q;\n selp.u32 %0, 1, 0, r;\n}"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ bool io_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred q, r;\n setp.ne.u32 q, %1, 0;\n bar.red.and.pred r, 2, %2, q;\n selp.u32 %0, 1, 0, r;\n}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(32 * kIoWarps)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ long coef_offset(long N, long m) {
  long a = m < 0 ? -m : m;
  if (a == 0) return 0;
  long pos = 2 * N * (2 * a - 1) - a * (a - 1);
  return m > 0 ? pos : pos + (2 * N - a);
}
__device__ __forceinline__ long order_slot(long m) { return m == 0 ? 0 : (m > 0 ? 2 * m - 1 : -2 * m); }
// Two row segments held in registers: position t -> row.
struct Segs {
  int off0, len0, off1;
};
__device__ __forceinline__ Segs in_segs(const TcOp& op, bool fwd) {
  return fwd ? Segs{op.in_off[0], op.in_len[0], op.in_off[1]} : Segs{op.out_off[0], op.out_len[0], op.out_off[1]};
}
__device__ __forceinline__ Segs out_segs(const TcOp& op, bool fwd) { return in_segs(op, !fwd); }
__device__ __forceinline__ int seg_row(int t, const Segs& g) { return t < g.len0 ? g.off0 + t : g.off1 + (t - g.len0); }
__device__ __forceinline__ const double* coef_base(const double* beta, int N, int am, int f, int s, int F,
                                                   int single, int msingle) {
  if (f >= F || (s == 1 && am == 0)) return nullptr;
  if (single) {
    if ((s == 0 ? am : -am) != msingle) return nullptr;
    return beta + 2L * f * (2 * N - am);
  }
  return beta + 2 * ((long)f * 4L * N * N + coef_offset(N, s == 0 ? am : -am));
}
__device__ __forceinline__ const double* value_base(const double* g, int N, int am, int f, int s, int F, int single,
                                                    int msingle) {
  if (f >= F || (s == 1 && am == 0)) return nullptr;
  if (single) {
    if ((s == 0 ? am : -am) != msingle) return nullptr;
    return g + 2L * f * 2 * N;
  }
  return g + 2 * ((long)f * (4L * N - 1) * 2 * N + order_slot(s == 0 ? am : -am) * 2 * N);
}




// Byte offset of (row, piece, column) in a vector space (the group layout).
__device__ __forceinline__ size_t grp_off(int row, int pc, int col) {
  return (size_t)(row / kTcGrpRows) * kTcGrpBytes + pc * 2048 + (col >> 3) * 128 + (row % kTcGrpRows) * 16 +
         (col & 7) * 2;
}

// eight consecutive values (columns 8 m8 .. 8 m8 + 7) of row `row` -> three
// BF16 pieces, one 16-byte store per piece
__device__ __forceinline__ void put_pieces8(unsigned char* vec, int row, int m8, float4 xa, float4 xb) {
  float a[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
  uint32_t h[3][4];
#pragma unroll
  for (int jj = 0; jj < 8; jj += 2) {
    float a0 = a[jj], a1 = a[jj + 1];
#pragma unroll
    for (int pc = 0; pc < 3; ++pc) {
      const __nv_bfloat162 hb = __floats2bfloat162_rn(a0, a1);
      const float2 hf = __bfloat1622float2(hb);
      a0 -= hf.x;
      a1 -= hf.y;
      h[pc][jj >> 1] = *reinterpret_cast<const uint32_t*>(&hb);
    }
  }
#pragma unroll
  for (int pc = 0; pc < 3; ++pc)
    __stcg(reinterpret_cast<uint4*>(vec + grp_off(row, pc, 8 * m8)), make_uint4(h[pc][0], h[pc][1], h[pc][2], h[pc][3]));
}

// Shape of one op in the requested direction.
struct OpShape {
  int NN, KK, nT;
  TcKGeom kg;  // the K side widened to whole row groups (nK chunks, kp_tot columns)
};
__device__ __forceinline__ OpShape op_shape(const TcOp& op, bool fwd) {
  OpShape s;
  s.NN = fwd ? op.mo : op.ni;
  s.KK = fwd ? op.ni : op.mo;
  s.nT = (s.NN + kTcNT - 1) / kTcNT;
  s.kg = fwd ? tc_kgeom(op.in_off[0], op.in_len[0], op.in_off[1], op.in_len[1])
             : tc_kgeom(op.out_off[0], op.out_len[0], op.out_off[1], op.out_len[1]);
  if (s.KK <= 0) s.kg.nK = s.kg.ngt = s.kg.kp_tot = 0;
  return s;
}

struct Item {
  int plan, grp, am;
};
__device__ __forceinline__ Item item_of(const TcLaunch& L, int it) {
  Item r;
  if (L.items) {
    const int4 v = L.items[it];
    r.plan = v.x;
    r.am = v.y;
    r.grp = v.z;
    return r;
  }
  const int G = (L.F[0] + kTcFields - 1) / kTcFields;
  r.plan = 0;
  r.grp = it % G;
  r.am = L.single ? (L.msingle < 0 ? -L.msingle : L.msingle) : L.plan[0].order[it / G];
  return r;
}

// The k-th op of a unit in processing order: ascending phases forward,
// descending phases for the transposed (inverse) apply.
__device__ __forceinline__ int op_at(const Unit& u, int k, bool fwd) { return fwd ? u.op_begin + k : u.op_end - 1 - k; }

__global__ void __launch_bounds__(kTcThreads, 1) alt_tc_kernel(const __grid_constant__ TcLaunch L, int fwd) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* trbuf = reinterpret_cast<float*>(base + (size_t)kStages * kStageBytes);
  float* iobuf = reinterpret_cast<float*>(base + (size_t)kStages * kStageBytes + kTrBytes);
  Ctl* ctl = reinterpret_cast<Ctl*>(base + (size_t)kStages * kStageBytes + kTrBytes + kIoBytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&ctl->full[s], 1);  // the producer's expect_tx; the bulk copies complete the bytes
      mbar_init(&ctl->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ctl->accf[b], 1);
      mbar_init(&ctl->acce[b], kEpiWarps);
    }
    ctl->abort = 0;
    ctl->gathered = 0;
    ctl->done_tiles = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // Stage memory starts at zero: the MMA of a padded last K step reads one row
  // group that no copy fills (its operand-image columns are zero), which must
  // hold finite values.  Afterwards stages only ever hold copied activations.
  for (int i = tid; i < kStages * kStageBytes / 16; i += kTcThreads)
    reinterpret_cast<uint4*>(base)[i] = make_uint4(0u, 0u, 0u, 0u);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the bulk copies and MMAs
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s32(&ctl->taddr)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = ctl->taddr;

  const int nitems = L.nitems;
  const size_t slot_bytes = tc_slot_bytes(L.max_rows);
  unsigned char* slots = L.ws + (size_t)blockIdx.x * 2 * slot_bytes;  // two vector spaces, alternating by item
  const uint32_t stage0 = s32(base);

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    // One thread streams the stages: per (op, N tile, K chunk) the chunk's
    // operand-image piece block and its input row groups (at most one run of
    // whole groups per segment), all as bulk copies whose bytes the stage's
    // full barrier expects.
    long jp = 0;
    int tiles_before = 0;  // tiles of all earlier phases (all items so far)
    bool ok = true;
    for (int iseq = 0; ok; ++iseq) {
      // the item and its gathered inputs (the I/O warps publish both)
      int it = -1;
      if (lane == 0) it = next_item(ctl, iseq, ok);
      it = __shfl_sync(0xffffffffu, it, 0);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok || it < 0) break;
      const Item itm = item_of(L, it);
      const TcPlan& p = L.plan[itm.plan];
      const Unit u = p.units[itm.am];
      const unsigned char* vec = slots + (size_t)(iseq & 1) * slot_bytes;
      const int nops = u.op_end - u.op_begin;
      TcOp nxt = nops > 0 ? p.ops[op_at(u, 0, fwd)] : TcOp{};
      int cur_phase = -1, tiles_here = 0;
      for (int q = 0; q < nops && ok; ++q) {
        const TcOp op = nxt;
        if (q + 1 < nops) nxt = p.ops[op_at(u, q + 1, fwd)];
        if (op.phase != cur_phase) {
          // a phase reads rows that earlier phases of this item wrote: wait for
          // their tiles (the item's first phase reads only gathered rows)
          tiles_before += tiles_here;
          tiles_here = 0;
          if (cur_phase >= 0 && lane == 0) ok = counter_wait(ctl, &ctl->done_tiles, tiles_before);
          ok = __shfl_sync(0xffffffffu, ok, 0);
          cur_phase = op.phase;
        }
        const OpShape sh = op_shape(op, fwd);
        const TcKGeom& kg = sh.kg;
        const uint16_t* img = p.img + (fwd ? op.img[0] : op.img[1]);
        for (int t = 0; t < sh.nT && ok; ++t) {
          const int Np = (min(kTcNT, sh.NN - kTcNT * t) + 15) & ~15;
          for (int c = 0; c < kg.nK && ok; ++c) {
            if (lane == 0) {
              const int s = (int)(jp % kStages);
              const uint32_t use = (uint32_t)(jp / kStages);
              ok = mbar_wait(ctl, &ctl->empty[s], (use & 1u) ^ 1u);
              if (ok) {
                const int Kp = min(kTcKC, kg.kp_tot - kTcKC * c);
                const uint32_t sA = stage0 + (uint32_t)s * kStageBytes, sB = sA + kStageA;
                // slots [j0, j1) of this chunk: [j0, ja) in segment 0, [ja, j1) in segment 1
                const int j0 = 4 * c, j1 = min(4 * c + 4, kg.ngt);
                const int ja = max(j0, min(j1, kg.ng0));
                const uint32_t bbytes = (uint32_t)(3 * Np * Kp * 2);
                bulk_expect(&ctl->full[s], bbytes + (uint32_t)(j1 - j0) * kTcGrpBytes);
                bulk_copy(sB, img + (size_t)t * 384 * kg.kp_tot + (size_t)Np * (96 * c), bbytes, &ctl->full[s]);
                if (ja > j0)
                  bulk_copy(sA, vec + (size_t)(kg.gs0 + j0) * kTcGrpBytes, (uint32_t)(ja - j0) * kTcGrpBytes,
                            &ctl->full[s]);
                if (j1 > ja)
                  bulk_copy(sA + (uint32_t)(ja - j0) * kTcGrpBytes,
                            vec + (size_t)(kg.gs1 + ja - kg.ng0) * kTcGrpBytes, (uint32_t)(j1 - ja) * kTcGrpBytes,
                            &ctl->full[s]);
              }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (ok) ++jp;  // stages issued so far
          }
          ++tiles_here;
        }
      }
      tiles_before += tiles_here;
    }
    // after an abort, let the copies of the last issued stages land before leaving
    if (!ok && lane == 0)
      for (long j = max(0L, jp - kStages); j < jp; ++j) mbar_drain(&ctl->full[j % kStages], (uint32_t)(j / kStages) & 1u);
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      long jm = 0, tm = 0;
      bool ok = true;
      for (int iseq = 0; ok; ++iseq) {
        const int it = next_item(ctl, iseq, ok);
        if (!ok || it < 0) break;
        const Item itm = item_of(L, it);
        const TcPlan& p = L.plan[itm.plan];
        const Unit u = p.units[itm.am];
        const int nops = u.op_end - u.op_begin;
        TcOp nxt = nops > 0 ? p.ops[op_at(u, 0, fwd)] : TcOp{};
        for (int q = 0; q < nops && ok; ++q) {
          {
            const TcOp op = nxt;
            if (q + 1 < nops) nxt = p.ops[op_at(u, q + 1, fwd)];
            const OpShape sh = op_shape(op, fwd);
            for (int t = 0; t < sh.nT && ok; ++t, ++tm) {
              const int b = (int)(tm & 1);
              const uint32_t v = (uint32_t)(tm >> 1);
              ok = mbar_wait(ctl, &ctl->acce[b], (v & 1u) ^ 1u);
              if (!ok) break;
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
              const int Np = (min(kTcNT, sh.NN - kTcNT * t) + 15) & ~15;
              const uint32_t idesc =
                  (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | ((uint32_t)(Np >> 3) << 17) | (8u << 24);
              const uint32_t dhi = taddr + (uint32_t)(b * 256), dlo = dhi + 128;
              // descriptors of stage 0 for this tile; a stage, a K step or a piece
              // moves the start address, i.e. adds (byte offset / 16) to the descriptor
              const uint32_t bK = (uint32_t)(Np / 8) * 128;
              const uint64_t a_desc0 = sdesc(stage0, kTcGrpBytes, 128);
              const uint64_t b_desc0 = sdesc(stage0 + kStageA, bK, 128);
              for (int c = 0; c < sh.kg.nK && ok; ++c, ++jm) {
                const int s = (int)(jm % kStages);
                const uint32_t use = (uint32_t)(jm / kStages);
                ok = mbar_wait(ctl, &ctl->full[s], use & 1u);
                if (!ok) break;
                // the stage was filled by bulk copies (async proxy), which the
                // MMAs read through the same proxy: the barrier orders them
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int Kp = min(kTcKC, sh.kg.kp_tot - kTcKC * c);
                const uint64_t stg = (uint64_t)((s * kStageBytes) >> 4);
                const uint64_t ad0 = a_desc0 + stg, bd0 = b_desc0 + stg;
                const uint64_t bpc = (uint64_t)((Np * Kp * 2) >> 4), bks = (uint64_t)(2 * bK >> 4);
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                  if (ks * 16 >= Kp) break;
                  // A MN-major: core (k8, m8) of piece pa at (k8 * 3 + pa) * 2048 + m8 * 128
                  // (K stride one row group, M stride 128); B K-major, pieces bpc apart
                  const uint64_t ak = ad0 + (uint64_t)((ks * 2 * kTcGrpBytes) >> 4), bk = bd0 + ks * bks;
                  const uint32_t first = (c > 0 || ks > 0) ? 1u : 0u;
                  mma_bf16(dhi, ak, bk, idesc, first);                           // a0 b0
                  mma_bf16(dlo, ak, bk + bpc, idesc, first);                     // a0 b1
                  mma_bf16(dlo, ak + (2048 >> 4), bk, idesc, 1u);                // a1 b0
                  mma_bf16(dlo, ak, bk + 2 * bpc, idesc, 1u);                    // a0 b2
                  mma_bf16(dlo, ak + (2048 >> 4), bk + bpc, idesc, 1u);          // a1 b1
                  mma_bf16(dlo, ak + (4096 >> 4), bk, idesc, 1u);                // a2 b0
                }
                mma_commit(&ctl->empty[s]);
              }
              if (ok) mma_commit(&ctl->accf[b]);
            }
          }
        }
      }
    }
    __syncwarp();
  } else if (warp >= kEpiWarp0 && warp < kIoWarp0) {
    // accumulators -> rows: warp ew owns TMEM lane quadrant ew (right-hand sides 32 ew ..)
    const int ew = warp - kEpiWarp0;
    const int e = tid - 32 * kEpiWarp0;
    float* T = trbuf + (size_t)ew * 32 * kTrStride;
    long te = 0;
    int done = 0;
    bool ok = true;
    for (int iseq = 0; ok; ++iseq) {
      const int it = next_item(ctl, iseq, ok);
      ok = epi_and(ok);
      if (!ok || it < 0) break;
      const Item itm = item_of(L, it);
      const TcPlan& p = L.plan[itm.plan];
      const Unit u = p.units[itm.am];
      unsigned char* vec = slots + (size_t)(iseq & 1) * slot_bytes;
      const int nops = u.op_end - u.op_begin;
      // accumulated rows (Y forward, X inverse) live in the item's accumulation region
      float* acc_item = p.acc + ((size_t)itm.grp * p.nunits + itm.am) * (size_t)kTcAccRows(p.N) * kTcR;
      const int acc0 = fwd ? u.ye : 0;
      TcOp nxt = nops > 0 ? p.ops[op_at(u, 0, fwd)] : TcOp{};
      for (int q = 0; q < nops && ok; ++q) {
        {
          const TcOp op = nxt;
          if (q + 1 < nops) nxt = p.ops[op_at(u, q + 1, fwd)];
          const OpShape sh = op_shape(op, fwd);
          const Segs osg = out_segs(op, fwd);
          const bool accum = (op.flags & (fwd ? OP_FWD_ACCUM : OP_BWD_ACCUM)) != 0;
          for (int t = 0; t < sh.nT && ok; ++t, ++te) {
            const int b = (int)(te & 1);
            const uint32_t v = (uint32_t)(te >> 1);
            ok = epi_and(mbar_wait(ctl, &ctl->accf[b], v & 1u));
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int Nt = min(kTcNT, sh.NN - kTcNT * t);
            if (sh.KK > 0 || !accum) {
              for (int c0 = 0; c0 < Nt; c0 += 32) {
                if (sh.KK > 0) {
                  uint32_t hv[32], lv[32];
                  const uint32_t lanes = (uint32_t)(32 * ew) << 16;
                  tmem_ld32(taddr + lanes + (uint32_t)(b * 256 + c0), hv);
                  tmem_ld32(taddr + lanes + (uint32_t)(b * 256 + 128 + c0), lv);
                  tmem_wait_ld();
#pragma unroll
                  for (int q = 0; q < 32; ++q) T[q * kTrStride + lane] = __uint_as_float(hv[q]) + __uint_as_float(lv[q]);
                } else {
#pragma unroll
                  for (int q = 0; q < 32; ++q) T[q * kTrStride + lane] = 0.f;
                }
                __syncwarp();
                const int oc = lane & 3;
#pragma unroll
                for (int kq = 0; kq < 4; ++kq) {
                  const int rl = (lane >> 2) + 8 * kq, i = c0 + rl;
                  if (i < Nt) {
                    float x[8];
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) x[jj] = T[rl * kTrStride + 8 * oc + jj];
                    const int r = seg_row(kTcNT * t + i, osg);
                    const int c8 = 32 * ew + 8 * oc;
                    if (accum) {
                      float* dst = acc_item + (size_t)(r - acc0) * kTcR + c8;
                      asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(x[0]),
                                   "f"(x[1]), "f"(x[2]), "f"(x[3])
                                   : "memory");
                      asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst + 4), "f"(x[4]),
                                   "f"(x[5]), "f"(x[6]), "f"(x[7])
                                   : "memory");
                    } else {
                      uint32_t h[3][4];
#pragma unroll
                      for (int jj = 0; jj < 8; jj += 2) {
                        float a0 = x[jj], a1 = x[jj + 1];
#pragma unroll
                        for (int pc = 0; pc < 3; ++pc) {
                          const __nv_bfloat162 hb = __floats2bfloat162_rn(a0, a1);
                          const float2 hf = __bfloat1622float2(hb);
                          a0 -= hf.x;
                          a1 -= hf.y;
                          h[pc][jj >> 1] = *reinterpret_cast<const uint32_t*>(&hb);
                        }
                      }
#pragma unroll
                      for (int pc = 0; pc < 3; ++pc)
                        __stcg(reinterpret_cast<uint4*>(vec + grp_off(r, pc, c8)),
                               make_uint4(h[pc][0], h[pc][1], h[pc][2], h[pc][3]));
                    }
                  }
                }
                __syncwarp();
              }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl->acce[b]);
            // the rows written above are read next by bulk copies (async proxy)
            asm volatile("fence.proxy.async.global;" ::: "memory");
            __threadfence_block();
            epi_bar();
            ++done;
            if (e == 0) *((volatile int*)&ctl->done_tiles) = done;
          }
        }
      }
    }
  } else if (warp >= kIoWarp0) {
    // I/O warps.  They take this CTA's items from the launch's work counter
    // (decreasing cost: orders by cost, field groups inside an order), publish
    // each in ctl->ring for the other roles, and gather item i into slot i % 2
    // once item i - 2 (the slot's previous user) has finished all of its tiles.
    // The outputs go to the accumulation buffer and leave through the output
    // kernel.  Global data moves through a 32 x 128 shared tile: every load
    // instruction reads contiguous 512-byte runs of one (field, sign) pair, each
    // warp keeps its 8 pairs' loads in flight together, and every store writes
    // whole 16-byte pieces of 8 consecutive columns, 8 rows of a group at a time.
    // Column c = 4 field + 2 sign + {re, im}.
    const int iw = warp - kIoWarp0;  // 0 .. kIoWarps - 1
    float* T = iobuf;
    const int e = tid - 32 * kIoWarp0;
    int t_m2 = 0, t_m1 = 0;  // tiles of all items up to i-2, up to i-1
    bool ok = L.stall == 0;
    for (int iseq = 0; ok; ++iseq) {
      ok = io_and(counter_wait(ctl, &ctl->done_tiles, t_m2));
      if (!ok) break;
      if (e == 0) {
        const unsigned int w = atomicAdd(L.counter, 1u);
        ctl->ring[iseq & 3] = w < (unsigned int)nitems ? (int)w : -1;
      }
      io_bar();
      const int it = *((volatile int*)&ctl->ring[iseq & 3]);
      if (it < 0) {
        __threadfence_block();
        if (e == 0) *((volatile int*)&ctl->gathered) = iseq + 1;
        break;
      }
      const Item itm = item_of(L, it);
      const TcPlan& p = L.plan[itm.plan];
      const int am = itm.am, grp = itm.grp, N = p.N, F = L.F[itm.plan];
      const double* in = L.in[itm.plan];
      const int single = L.single, msingle = L.msingle;
      const Unit u = p.units[am];
      unsigned char* vec = slots + (size_t)(iseq & 1) * slot_bytes;
      const int nx = u.nce + u.nco;
      if (fwd) {
        // X rows from beta: degree k = am + d; d even -> row d/2 (X_e), d odd ->
        // row nce + d/2 (X_o).  Tile row dl = degree d0 + dl.
        for (int d0 = 0; d0 < nx; d0 += 32) {
          const int d = d0 + lane;
          double2 v[kPairsPerIo];
#pragma unroll
          for (int k = 0; k < kPairsPerIo; ++k) {
            const int pr = iw + kIoWarps * k;
            const double* bsrc = coef_base(in, N, am, grp * kTcFields + (pr >> 1), pr & 1, F, single, msingle);
            v[k] = (bsrc && d < nx) ? __ldg(reinterpret_cast<const double2*>(bsrc) + d) : make_double2(0.0, 0.0);
          }
#pragma unroll
          for (int k = 0; k < kPairsPerIo; ++k) {
            const int pr = iw + kIoWarps * k;
            *reinterpret_cast<float2*>(T + lane * kIoStride + 2 * pr) =
                make_float2(f64_to_f32_bits(v[k].x), f64_to_f32_bits(v[k].y));
          }
          io_bar();
          // warp iw: 8 rows of one parity (block iw % 4) x 8 of the 16 column
          // chunks (half iw / 4); lane = (row, chunk)
          const int blk = iw & 3, par = blk >> 1;
          const int j = (blk & 1) * 8 + (lane & 7);  // row of this parity within the chunk
          const int dd = 2 * j + par;                // its tile row
          if (d0 + dd < nx) {
            const int row = (par ? u.nce : 0) + (d0 >> 1) + j;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              const int m8 = (iw >> 2) * 8 + q * 4 + (lane >> 3);
              put_pieces8(vec, row, m8, *reinterpret_cast<const float4*>(T + dd * kIoStride + 8 * m8),
                          *reinterpret_cast<const float4*>(T + dd * kIoStride + 8 * m8 + 4));
            }
          }
          io_bar();
        }
      } else {
        // weighted parity fold of g into Y_e, Y_o (Sec. 3.1.1 with the W of
        // B = A^T W), 16 nodes i0 .. i0 + 15 at a time: lanes 0-15 read
        // g(theta_{N+i}), lanes 16-31 g(theta_{N-1-i}) of the same node; tile
        // rows 0-15 take u_e = w (a + b), rows 16-31 u_o = w (a - b).
        const int hl = lane & 15, hi = lane >> 4;
        for (int i0 = 0; i0 < N; i0 += 16) {
          const int i = i0 + hl;
          const float wi = i < N ? f64_to_f32_bits(__ldg(p.w + N + i)) : 0.f;
          double2 v[kPairsPerIo];
#pragma unroll
          for (int k = 0; k < kPairsPerIo; ++k) {
            const int pr = iw + kIoWarps * k;
            const double* gb = value_base(in, N, am, grp * kTcFields + (pr >> 1), pr & 1, F, single, msingle);
            v[k] = (gb && i < N) ? __ldg(reinterpret_cast<const double2*>(gb) + (hi ? N - 1 - i : N + i))
                                 : make_double2(0.0, 0.0);
          }
#pragma unroll
          for (int k = 0; k < kPairsPerIo; ++k) {
            const int pr = iw + kIoWarps * k;
            const float x = f64_to_f32_bits(v[k].x), y = f64_to_f32_bits(v[k].y);
            const float ox = __shfl_xor_sync(0xffffffffu, x, 16), oy = __shfl_xor_sync(0xffffffffu, y, 16);
            // lane < 16 holds a, its partner b; lane >= 16 holds b, its partner a
            const float2 r = hi ? make_float2(wi * (ox - x), wi * (oy - y)) : make_float2(wi * (x + ox), wi * (y + oy));
            *reinterpret_cast<float2*>(T + lane * kIoStride + 2 * pr) = r;
          }
          io_bar();
          // warp iw: tile rows 8 (iw % 4) .. + 7 x 8 of the 16 column chunks (half iw / 4)
          const int tr = (iw & 3) * 8 + (lane & 7);
          const int ii = i0 + (tr & 15);
          if (ii < N) {
            const int row = (tr < 16 ? u.ye : u.yo) + ii;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              const int m8 = (iw >> 2) * 8 + q * 4 + (lane >> 3);
              put_pieces8(vec, row, m8, *reinterpret_cast<const float4*>(T + tr * kIoStride + 8 * m8),
                          *reinterpret_cast<const float4*>(T + tr * kIoStride + 8 * m8 + 4));
            }
          }
          io_bar();
        }
      }
      // the item's accumulation rows start at zero: the epilogue adds into them
      // (forward: the 2N node rows; inverse: the nx degree rows).  Zeroing them
      // here keeps the lines in L2 for those additions.
      {
        float4* acc4 = reinterpret_cast<float4*>(p.acc + ((size_t)grp * p.nunits + am) * (size_t)kTcAccRows(N) * kTcR);
        const int n4 = (fwd ? 2 * N : nx) * (kTcR / 4);
        for (int k = e; k < n4; k += 32 * kIoWarps) __stcg(acc4 + k, make_float4(0.f, 0.f, 0.f, 0.f));
      }
      asm volatile("fence.proxy.async.global;" ::: "memory");  // the rows are read by bulk copies
      __threadfence();
      io_bar();
      if (e == 0) *((volatile int*)&ctl->gathered) = iseq + 1;
      const int t_cur = t_m1 + p.tiles[2 * am + (fwd ? 0 : 1)];
      t_m2 = t_m1;
      t_m1 = t_cur;
    }
  }
  if (*((volatile int*)&ctl->abort) && tid == 0) atomicExch(L.err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kMmaWarp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTmemCols) : "memory");
}

// Output side of the apply: the accumulated rows of every work item (FP32,
// kTcR right-hand sides per row) to g (forward: the parity fold of Sec. 3.1.2,
// g(theta_{N+i}) = y_e + y_o, g(theta_{N-1-i}) = y_e - y_o) or to beta
// (inverse: X rows back to degrees).  A streaming kernel with many warps per
// SM, so that this part of the I/O runs at HBM bandwidth.  One CTA step is
// one item and 32 nodes (or degrees), transposed through shared memory so
// that reads are whole rows and writes are 512-byte runs per (field, sign).
constexpr int kOutThreads = 256;
__global__ void __launch_bounds__(kOutThreads) tc_out_kernel(TcPlan p, double* __restrict__ out, int F, int single,
                                                            int msingle, int fwd) {
  __shared__ __align__(16) float Te[32 * kIoStride];
  __shared__ __align__(16) float To[32 * kIoStride];
  const int N = p.N, lane = threadIdx.x & 31, iw = threadIdx.x >> 5;
  const int G = (F + kTcFields - 1) / kTcFields;
  const int nitems = single ? G : p.nunits * G;
  const int cpi = fwd ? (N + 31) / 32 : (2 * N + 31) / 32;  // chunks per item
  const long total = (long)nitems * cpi;
  for (long w = blockIdx.x; w < total; w += gridDim.x) {
    const int item = (int)(w / cpi), chunk = (int)(w % cpi);
    const int grp = item % G;
    const int am = single ? (msingle < 0 ? -msingle : msingle) : item / G;
    const Unit u = p.units[am];
    const float* acc_item = p.acc + ((size_t)grp * p.nunits + am) * (size_t)kTcAccRows(N) * kTcR;
    if (fwd) {
      const int i0 = 32 * chunk;
      for (int r = iw; r < 32; r += kOutThreads / 32) {
        if (i0 + r < N) {
          *reinterpret_cast<float4*>(Te + r * kIoStride + 4 * lane) =
              __ldcs(reinterpret_cast<const float4*>(acc_item + (size_t)(i0 + r) * kTcR) + lane);
          *reinterpret_cast<float4*>(To + r * kIoStride + 4 * lane) =
              __ldcs(reinterpret_cast<const float4*>(acc_item + (size_t)(N + i0 + r) * kTcR) + lane);
        }
      }
      __syncthreads();
      const int i = i0 + lane;
      for (int pr = iw; pr < 2 * kTcFields; pr += kOutThreads / 32) {
        const int fl = pr >> 1, sgn = pr & 1;
        const double* gb = value_base(out, N, am, grp * kTcFields + fl, sgn, F, single, msingle);
        if (gb && i < N) {
          const float2 ev = *reinterpret_cast<const float2*>(Te + lane * kIoStride + 4 * fl + 2 * sgn);
          const float2 ov = *reinterpret_cast<const float2*>(To + lane * kIoStride + 4 * fl + 2 * sgn);
          double2* gp = reinterpret_cast<double2*>(const_cast<double*>(gb));
          __stcs(gp + N + i, make_double2(f32_to_f64_bits(ev.x + ov.x), f32_to_f64_bits(ev.y + ov.y)));
          __stcs(gp + N - 1 - i, make_double2(f32_to_f64_bits(ev.x - ov.x), f32_to_f64_bits(ev.y - ov.y)));
        }
      }
      __syncthreads();
    } else {
      const int nx = u.nce + u.nco, d0 = 32 * chunk;
      if (d0 >= nx) continue;  // uniform over the CTA
      for (int dl = iw; dl < 32; dl += kOutThreads / 32) {
        const int d = d0 + dl;
        if (d < nx) {
          const int t = (d & 1) ? u.nce + (d >> 1) : (d >> 1);
          *reinterpret_cast<float4*>(Te + dl * kIoStride + 4 * lane) =
              __ldcs(reinterpret_cast<const float4*>(acc_item + (size_t)t * kTcR) + lane);
        }
      }
      __syncthreads();
      const int d = d0 + lane;
      for (int pr = iw; pr < 2 * kTcFields; pr += kOutThreads / 32) {
        const int fl = pr >> 1, sgn = pr & 1;
        const double* bdst = coef_base(out, N, am, grp * kTcFields + fl, sgn, F, single, msingle);
        if (bdst && d < nx) {
          const float2 v = *reinterpret_cast<const float2*>(Te + lane * kIoStride + 4 * fl + 2 * sgn);
          __stcs(reinterpret_cast<double2*>(const_cast<double*>(bdst)) + d,
                 make_double2(f32_to_f64_bits(v.x), f32_to_f64_bits(v.y)));
        }
      }
      __syncthreads();
    }
  }
}

}  // namespace

size_t tc_smem_bytes() { return kSmemTotal; }

int tc_ctas_per_sm() { return 1; }  // the kernel holds all 512 tensor-memory columns

static int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

static cudaError_t launch_out(const TcPlan& p, bool fwd, double* out, int F, int single, int m, int sms, cudaStream_t st) {
  const int G = (F + kTcFields - 1) / kTcFields;
  const long items = (long)(single ? 1 : p.nunits) * G;
  const long chunks = items * (fwd ? (p.N + 31) / 32 : (2 * p.N + 31) / 32);
  const int out_grid = (int)std::max(1L, std::min(chunks, (long)sms * 6));
  tc_out_kernel<<<out_grid, kOutThreads, 0, st>>>(p, out, F, single, m, fwd ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_tc(const TcPlan& p, bool fwd, const double* in, double* out, int F, int single, int m, int grid,
                      cudaStream_t st, cudaEvent_t* ev) {
  const int G = (F + kTcFields - 1) / kTcFields;
  if (G > p.gmax) return cudaErrorInvalidValue;
  TcLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.plan[0] = p;
  L.in[0] = in;
  L.out[0] = out;
  L.F[0] = F;
  L.nplans = 1;
  L.items = nullptr;
  L.nitems = single ? G : p.nunits * G;
  L.single = single;
  L.msingle = m;
  L.ws = p.ws;
  L.max_rows = p.max_rows;
  L.counter = p.counter;
  L.err = p.err;
  // (the kernel zeroes each item's accumulation rows itself when it gathers the item)
  cudaError_t e = cudaFuncSetAttribute(alt_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTotal);
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
  alt_tc_kernel<<<grid, kTcThreads, kSmemTotal, st>>>(L, fwd ? 1 : 0);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[1], st)) != cudaSuccess) return e;
  e = launch_out(p, fwd, out, F, single, m, sm_count(), st);
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], st);
  return e;
}

cudaError_t launch_tc_stall(const TcPlan& p, int grid, cudaStream_t st) {
  TcLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.plan[0] = p;
  L.F[0] = 1;
  L.nplans = 1;
  L.nitems = 1;
  L.ws = p.ws;
  L.max_rows = p.max_rows;
  L.counter = p.counter;
  L.err = p.err;
  L.stall = 1;
  cudaError_t e = cudaFuncSetAttribute(alt_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTotal);
  if (e != cudaSuccess) return e;
  alt_tc_kernel<<<grid, kTcThreads, kSmemTotal, st>>>(L, 1);
  return cudaGetLastError();
}

cudaError_t launch_tc_batch(const TcLaunch& L, bool fwd, int grid, cudaStream_t st, cudaEvent_t* ev) {
  if (L.nplans < 1 || L.nplans > kTcMaxPlans || !L.items) return cudaErrorInvalidValue;
  for (int q = 0; q < L.nplans; ++q)
    if ((L.F[q] + kTcFields - 1) / kTcFields > L.plan[q].gmax) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(alt_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTotal);
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
  alt_tc_kernel<<<grid, kTcThreads, kSmemTotal, st>>>(L, fwd ? 1 : 0);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[1], st)) != cudaSuccess) return e;
  const int sms = sm_count();
  for (int q = 0; q < L.nplans && e == cudaSuccess; ++q)
    if (L.F[q] > 0) e = launch_out(L.plan[q], fwd, L.out[q], L.F[q], 0, 0, sms, st);
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], st);
  return e;
}

}  // namespace sht
