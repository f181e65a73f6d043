// Many-field apply of the IDBF-factored ALT on the 5th-generation tensor
// cores (tcgen05, sm_103a), split-BF16 products with FP32 accumulation.
//
// One work item is one order |m| for 32 fields: 128 real right-hand sides.
// Every block product of the apply program, out (+)= B in, is computed
// transposed, out^T = in^T B^T, so that the 128 right-hand sides fill the MMA
// M dimension and the block's rows are N (tiles of <= 128, padded to 16):
//   A operand = in^T (128 x K, K-major): the op's input rows, kept in the
//               scratch as three BF16 pieces a0 + a1 + a2 (8 bits each) of
//               every value, in groups of 8 rows laid out exactly as the
//               operand sits in shared memory, so that staging one K chunk
//               is one or two bulk copies of whole groups;
//   B operand = B (N x K, K-major): precomputed split-BF16 image b0 + b1 + b2,
//               with zero columns where the K side was widened to whole groups
//               (and zero rows where an intermediate output side was);
//   D         = 128 x N FP32 accumulators in tensor memory.
// The CTA is warp-specialised and persistent (one per SM): one producer
// thread streams (op, tile, 32-wide K chunk) operand stages into a 4-deep
// shared memory ring with bulk copies; the MMA warp issues the tensor-core
// products (one elected lane) into two alternating TMEM accumulator pairs;
// two teams of four epilogue warps drain them, each thread one right-hand
// side, and either split the results into BF16 pieces for the next level
// (eight rows per 16-byte store) or add them in FP32 into the item's
// accumulation rows; two item warps take the items and zero their
// accumulation rows.  The inputs (forward: beta into X rows; transposed: the
// W-weighted parity fold of g into Y rows) are gathered ahead of the launch by
// a streaming kernel, tc_in_kernel, whose per-item row groups the producer's
// bulk copies read.  Ops of one phase read only rows written by earlier
// phases: the producer starts a phase after the epilogue has counted every
// earlier tile.  Forward, a streaming output kernel then writes g (the parity
// fold of Sec. 3.1.2) from the accumulation rows; transposed, four output
// warps scatter each finished item's rows to beta inside this kernel.
// Per 16-wide K step six MMAs accumulate a_p b_q for p + q <= 2, which keeps
// every product to about 2^-24 relative error (FP32 quality); a0 b0 and the
// five smaller cross products go to two separate accumulators that the
// epilogue adds in FP32 (the tensor cores' FP32 accumulation is not rounded to
// nearest: summing the small terms into the large accumulator measured 8x the
// error at N = 1024).  Operands sit in
// shared memory in the canonical no-swizzle K-major layout (8 x 16-byte core
// matrices; LBO = stride between core matrices along K, SBO = along M/N).
// All waits are bounded: a wait that runs out sets an error flag, every role
// stops, and the host reports SHT_ERR_TIMEOUT.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <functional>

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

TcOp tc_op_of(const Op& op, const Unit& u, int N) {
  const TcRows tr = tc_rows(u.nce, u.nco, N);
  TcOp t{};
  t.mo = op.mo;
  t.ni = op.ni;
  for (int s = 0; s < 2; ++s) {
    t.in_len[s] = op.in_len[s];
    t.out_len[s] = op.out_len[s];
    t.in_off[s] = op.in_len[s] > 0 ? tc_seg_row(op.in_off[s], u.nce, u.nco, N, tr) : 0;
    t.out_off[s] = op.out_len[s] > 0 ? tc_seg_row(op.out_off[s], u.nce, u.nco, N, tr) : 0;
  }
  t.flags = op.flags;
  t.phase = op.phase;
  return t;
}

// Widened position -> index into the unwidened side (0 .. len0 + len1 - 1),
// or -1 where the position only pads.
static inline int widened_index(const TcKGeom& g, int off0, int len0, int off1, int len1, int pos) {
  const int j = pos / kTcGrpRows, e = pos % kTcGrpRows;
  if (j < g.ng0) {
    const int r = (g.gs0 + j) * kTcGrpRows + e;
    return r >= off0 && r < off0 + len0 ? r - off0 : -1;
  }
  if (j < g.ngt) {
    const int r = (g.gs1 + j - g.ng0) * kTcGrpRows + e;
    return r >= off1 && r < off1 + len1 ? len0 + r - off1 : -1;
  }
  return -1;
}

// Layout (matching the kernel): tiles t of kTcNT positions, chunks c, pieces
// p, then core matrices (ki, mi) in K-outer order, 8 positions x 8 elements
// each.  elem(n, k) is the block entry for output index n and input index k
// of the unwidened sides; positions that stand for no row (widening, padding)
// are 0.  Piece p of a value v is the BF16 rounding of what pieces 0..p-1
// leave of v.  Each (tile, chunk) is first gathered into a small buffer,
// walking the source along its contiguous direction (k_contig: consecutive K
// indices adjacent), and the three pieces of every value are computed in one
// pass.
template <class E>
static void tc_pack(const TcDir& d, const int* no, const int* nl, const int* ko, const int* kl, E elem, bool k_contig,
                    uint16_t* dst) {
  const TcKGeom& kg = d.kg;
  std::vector<double> buf((size_t)kTcNT * kTcKC);
  std::vector<int> nidx(kTcNT);
  size_t o = 0;
  for (int t = 0; t < d.nT; ++t) {
    const int Nv = std::min(kTcNT, d.NN - kTcNT * t);  // positions of the tile
    const int Np = r16(Nv);
    for (int n = 0; n < Np; ++n) {
      const int pos = kTcNT * t + n;
      nidx[n] = n >= Nv ? -1 : d.accum ? pos : widened_index(d.ng, no[0], nl[0], no[1], nl[1], pos);
    }
    for (int c = 0; c < kg.nK; ++c) {
      const int Kp = std::min(kTcKC, kg.kp_tot - kTcKC * c);
      int kx[kTcKC];
      for (int kk = 0; kk < Kp; ++kk) kx[kk] = widened_index(kg, ko[0], kl[0], ko[1], kl[1], kTcKC * c + kk);
      // buf[n * Kp + kk] = entry (tile position n, chunk column kk), zero outside
      std::fill(buf.begin(), buf.begin() + (size_t)Np * Kp, 0.0);
      if (k_contig) {
        for (int n = 0; n < Np; ++n)
          if (nidx[n] >= 0)
            for (int kk = 0; kk < Kp; ++kk)
              if (kx[kk] >= 0) buf[(size_t)n * Kp + kk] = elem(nidx[n], kx[kk]);
      } else {
        for (int kk = 0; kk < Kp; ++kk)
          if (kx[kk] >= 0)
            for (int n = 0; n < Np; ++n)
              if (nidx[n] >= 0) buf[(size_t)n * Kp + kk] = elem(nidx[n], kx[kk]);
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

static void pack_dir(const Op& op, const TcOp& top, const double* factors, bool transposed, uint16_t* dst) {
  const double* B = factors + op.b_off;
  const int ld = op.ld;
  const TcDir d = tc_dir(top, !transposed);
  if (tc_image_elems(d) == 0) return;
  if (!transposed)
    tc_pack(d, top.out_off, top.out_len, top.in_off, top.in_len, [&](int r, int k) { return B[(size_t)k * ld + r]; },
            false, dst);
  else
    tc_pack(d, top.in_off, top.in_len, top.out_off, top.out_len, [&](int r, int k) { return B[(size_t)r * ld + k]; },
            true, dst);
}

void tc_op_image(const Op& op, const TcOp& top, const double* factors, bool transposed, std::vector<uint16_t>& out) {
  out.assign(tc_image_elems(tc_dir(top, !transposed)), 0);
  pack_dir(op, top, factors, transposed, out.data());
}

size_t tc_image_layout(int N, const std::vector<Unit>& units, const std::vector<Op>& ops, std::vector<TcOp>& tops,
                       std::vector<int32_t>& tiles, int& max_rows) {
  const size_t n = ops.size();
  tops.assign(n, TcOp{});
  tiles.assign(2 * units.size(), 0);
  max_rows = 0;
  size_t tot = 0;
  for (size_t u = 0; u < units.size(); ++u) {
    const Unit& un = units[u];
    max_rows = std::max(max_rows, tc_nrows(un.nrows, un.nce, un.nco, N));
    for (int oi = un.op_begin; oi < un.op_end; ++oi) {
      TcOp& t = tops[(size_t)oi];
      t = tc_op_of(ops[(size_t)oi], un, N);
      const TcDir df = tc_dir(t, true), db = tc_dir(t, false);
      t.img[0] = (int64_t)tot;
      tot += tc_image_elems(df);
      t.img[1] = (int64_t)tot;
      tot += tc_image_elems(db);
      tiles[2 * u] += df.nT;
      tiles[2 * u + 1] += db.nT;
    }
  }
  return tot;
}

void tc_pack_ops(const std::vector<Op>& ops, const std::vector<TcOp>& tops, const double* factors, size_t i0,
                 size_t i1, uint16_t* dst, size_t base) {
#pragma omp parallel for schedule(dynamic, 64)
  for (long i = (long)i0; i < (long)i1; ++i) {
    pack_dir(ops[(size_t)i], tops[(size_t)i], factors, false, dst + ((size_t)tops[(size_t)i].img[0] - base));
    pack_dir(ops[(size_t)i], tops[(size_t)i], factors, true, dst + ((size_t)tops[(size_t)i].img[1] - base));
  }
}

void tc_pack_windows(const std::vector<Op>& ops, const std::vector<TcOp>& tops, const double* factors, size_t tot,
                     size_t window, const std::function<bool(size_t, const uint16_t*, size_t)>& sink) {
  const size_t n = ops.size();
  // the images of op i occupy [tops[i].img[0], end(i)), op after op
  auto end_of = [&](size_t i) { return i + 1 < n ? (size_t)tops[i + 1].img[0] : tot; };
  TcImages buf;
  for (size_t i0 = 0; i0 < n;) {
    const size_t begin = (size_t)tops[i0].img[0];
    size_t i1 = i0 + 1;
    while (i1 < n && end_of(i1) - begin <= window) ++i1;
    const size_t span = end_of(i1 - 1) - begin;
    if (buf.size() < span) buf.resize(span);
    tc_pack_ops(ops, tops, factors, i0, i1, buf.data(), begin);
    if (!sink(begin, buf.data(), span)) return;
    i0 = i1;
  }
}

void tc_build_images(int N, const std::vector<Unit>& units, const std::vector<Op>& ops, const double* factors,
                     TcImages& img, std::vector<TcOp>& tops, std::vector<int32_t>& tiles, int& max_rows) {
  const size_t tot = tc_image_layout(N, units, ops, tops, tiles, max_rows);
  // pack_dir writes every element of an op's two images (padding included),
  // so only the minimum-size tail of an empty store needs zeroing here
  img.resize(std::max<size_t>(tot, 8));
  std::fill(img.begin() + tot, img.end(), (uint16_t)0);
  tc_pack_ops(ops, tops, factors, 0, ops.size(), img.data(), 0);
}

void tc_proc_order(const std::vector<Unit>& units, const std::vector<TcOp>& tops, std::vector<int32_t>& ford,
                   std::vector<int32_t>& tord) {
  ford.resize(tops.size());
  tord.resize(tops.size());
  for (const Unit& un : units) {
    const int b = un.op_begin, e = un.op_end;
    for (int d = 0; d < 2; ++d) {
      const bool fwd = d == 0;
      std::vector<int32_t>& o = fwd ? ford : tord;
      for (int i = b; i < e; ++i) o[(size_t)i] = i;
      auto key = [&](int32_t i) {
        const TcOp& t = tops[(size_t)i];
        const int32_t* off = fwd ? t.in_off : t.out_off;
        const int32_t* len = fwd ? t.in_len : t.out_len;
        return len[0] > 0 ? off[0] : off[1];
      };
      std::stable_sort(o.begin() + b, o.begin() + e, [&](int32_t x, int32_t y) {
        const int px = tops[(size_t)x].phase, py = tops[(size_t)y].phase;
        if (px != py) return fwd ? px < py : px > py;
        return key(x) < key(y);
      });
    }
  }
}

void tc_live_rows(int N, const std::vector<Unit>& units, const std::vector<TcOp>& tops, std::vector<int32_t>& live) {
  live.assign(units.size(), 0);
  for (size_t u = 0; u < units.size(); ++u) {
    const Unit& un = units[u];
    const TcRows tr = tc_rows(un.nce, un.nco, N);
    int lv = 0;
    for (int q = un.op_begin; q < un.op_end; ++q) {
      const TcOp& t = tops[(size_t)q];
      for (int sg = 0; sg < 2; ++sg) {
        if (t.out_len[sg] <= 0) continue;
        const int off = t.out_off[sg], end = off + t.out_len[sg];
        if (off >= tr.ye && off < tr.yo)
          lv = std::max(lv, tc_r8(end - tr.ye));
        else if (off >= tr.yo && off < tr.yo + tc_r8(N))
          lv = std::max(lv, tc_r8(end - tr.yo));
      }
    }
    live[u] = std::min(lv, tc_r8(N));
  }
}

void tc_first_writers(int N, const std::vector<Unit>& units, std::vector<TcOp>& tops, const std::vector<int32_t>& ford,
                      const std::vector<int32_t>& tord, const std::vector<int32_t>& live, std::vector<int32_t>& zr,
                      std::vector<int32_t>& zri) {
  zr.clear();
  zri.assign(2 * units.size() + 1, 0);
  const int R = tc_acc_rows(N);
  std::vector<char> written(R), stored(R);
  for (size_t u = 0; u < units.size(); ++u) {
    const Unit& un = units[u];
    const TcRows tr = tc_rows(un.nce, un.nco, N);
    for (int d = 0; d < 2; ++d) {
      const bool fwd = d == 0;
      std::fill(written.begin(), written.end(), 0);
      std::fill(stored.begin(), stored.end(), 0);
      const int acc0 = fwd ? tr.ye : 0;
      const int nops = un.op_end - un.op_begin;
      for (int q = 0; q < nops; ++q) {  // the kernel's processing order
        TcOp& t = tops[(size_t)(fwd ? ford : tord)[(size_t)(un.op_begin + q)]];
        t.flags &= ~(fwd ? kTcFwdStore : kTcBwdStore);
        if (!(t.flags & (fwd ? OP_FWD_ACCUM : OP_BWD_ACCUM))) continue;
        const int32_t* oo = fwd ? t.out_off : t.in_off;
        const int32_t* ol = fwd ? t.out_len : t.in_len;
        bool fresh = true;
        for (int sg = 0; sg < 2; ++sg)
          for (int r = 0; r < ol[sg]; ++r) fresh = fresh && !written[oo[sg] + r - acc0];
        if (fresh) t.flags |= fwd ? kTcFwdStore : kTcBwdStore;
        for (int sg = 0; sg < 2; ++sg)
          for (int r = 0; r < ol[sg]; ++r) {
            written[oo[sg] + r - acc0] = 1;
            if (fresh) stored[oo[sg] + r - acc0] = 1;
          }
      }
      // rows the output step reads that no store writes first: zeroed per item
      // (forward, only the live node rows: the output step reads no others)
      const int nl = std::min(N, live[u]);
      const int ranges[2][2] = {{0, fwd ? nl : un.nce}, {fwd ? tr.yo - tr.ye : tr.xo, fwd ? nl : un.nco}};
      for (const auto& rg : ranges)
        for (int r = rg[0]; r < rg[0] + rg[1];) {
          if (stored[r]) {
            ++r;
            continue;
          }
          int e = r;
          while (e < rg[0] + rg[1] && !stored[e]) ++e;
          zr.push_back(r);
          zr.push_back(e - r);
          r = e;
        }
      zri[2 * u + d + 1] = (int32_t)(zr.size() / 2);
    }
  }
}

// ---------------------------------------------------------------- device side
namespace {

constexpr int kStages = 4;
constexpr int kProdWarp = 0;                  // one thread stages operands
constexpr int kMmaWarp = 1;                   // one thread issues the MMAs; the warp owns TMEM
constexpr int kEpiWarp0 = 4;                  // warps 4-11: two teams of four, TMEM lane quadrant warp % 4
constexpr int kEpiWarps = 8;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kIoWarp0 = 2;                   // warps 2-3 take the items and zero their rows
constexpr int kIoThreads = 64;
constexpr int kOutWarp0 = 12;                 // warps 12-15 write finished items' outputs
constexpr int kOutTeam = kTcThreads - 32 * kOutWarp0;
constexpr int kRing = 16;                     // published items a CTA keeps for its roles
// The input gathers (tc_in_kernel's CTAs): 8 warps
constexpr int kGatherWarps = 8;
constexpr int kGatherThreads = 32 * kGatherWarps;
constexpr int kPairs = 2 * kTcFields;         // (field, sign) pairs of an item: right-hand sides 2 pr, 2 pr + 1
static_assert(kPairs % kGatherWarps == 0, "the gather's warps split the pairs evenly");
static_assert(kGatherThreads == 4 * kPairs, "four gather threads per (field, sign) pair write the row groups");
static_assert(kEpiWarp0 % 4 == 0 && kEpiWarps == 8, "each epilogue team covers the four TMEM lane quadrants");
constexpr int kIoStride = 132;           // floats per I/O tile row (16-byte aligned rows)
constexpr int kIoTile = 32 * kIoStride;  // the gather's 32-row tile
constexpr int kStageA = (kTcKC / kTcGrpRows) * kTcGrpBytes;  // 4 row groups: 24 KB
constexpr int kStageB = 3 * kTcNT * kTcKC * 2;               // 24 KB (largest N tile)
constexpr int kStageBytes = kStageA + kStageB;
constexpr int kAccCols = 2 * kTcNT;             // an accumulator pair (hi, lo) of N columns each
constexpr int kTmemCols = 2 * kAccCols;         // two pairs, alternating by tile
constexpr long kWaitLimit = 1L << 22;           // try_wait polls per bounded wait

struct Ctl {
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t accf[2];
  uint64_t acce[2];
  uint32_t taddr;
  int abort;
  int gathered;    // items whose gather is complete (or found the queue empty)
  int done_tiles;  // tiles whose epilogue is complete (all items so far)
  int out_next;    // items whose index the output warps have taken from the ring
  int ring[kRing];  // item index of this CTA's item iseq at ring[iseq % kRing]; -1 = no more
};
constexpr size_t kSmemTotal = (size_t)kStages * kStageBytes + sizeof(Ctl) + 1024;
static_assert(kSmemTotal <= 232448, "fits the 227 KB of shared memory one CTA may use");

__device__ __forceinline__ uint32_t s32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// One MMA and one commit, issued by a single lane elected from the converged
// MMA warp: every lane computes the same operands, so they stay warp-uniform
// (issuing from a lane-0 branch instead took the forward call from 7.54 to
// 7.77 ms).
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
      " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
      " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}" ::"r"(s32(bar))
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

// This CTA's item number iseq as the item warps published it, once its rows
// are zeroed; -1 when the work counter ran out.
__device__ __forceinline__ int next_item(Ctl* ctl, int iseq, bool& ok) {
  ok = counter_wait(ctl, &ctl->gathered, iseq + 1);
  return ok ? *((volatile int*)&ctl->ring[iseq % kRing]) : -1;
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
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory"); }
__device__ __forceinline__ void io_bar() { asm volatile("bar.sync 2, %0;" ::"n"(kIoThreads) : "memory"); }
__device__ __forceinline__ void out_bar() { asm volatile("bar.sync 3, %0;" ::"n"(kOutTeam) : "memory"); }
__device__ __forceinline__ void gather_bar() { asm volatile("bar.sync 2, %0;" ::"n"(kGatherThreads) : "memory"); }
// The named barriers with an AND over the group: every warp of the group takes
// the same decision after a bounded wait, so none is left at a barrier alone.
__device__ __forceinline__ bool epi_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred q, r;\n setp.ne.u32 q, %1, 0;\n bar.red.and.pred r, 1, %2, q;\n selp.u32 %0, 1, 0, r;\n}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kEpiThreads)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ bool io_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred q, r;\n setp.ne.u32 q, %1, 0;\n bar.red.and.pred r, 2, %2, q;\n selp.u32 %0, 1, 0, r;\n}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kIoThreads)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ bool out_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred q, r;\n setp.ne.u32 q, %1, 0;\n bar.red.and.pred r, 3, %2, q;\n selp.u32 %0, 1, 0, r;\n}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kOutTeam)
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

// Eight consecutive rows (one group) of one right-hand side -> three BF16
// pieces, one 16-byte store per piece.
__device__ __forceinline__ void put_group(unsigned char* vec, int grp, int rhs, const float (&x)[8]) {
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
    __stcg(reinterpret_cast<uint4*>(vec + ((size_t)grp * 3 + pc) * 2048 + (size_t)rhs * 16),
           make_uint4(h[pc][0], h[pc][1], h[pc][2], h[pc][3]));
}

__device__ __forceinline__ void red_add4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
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

// The k-th op of a unit in processing order (tc_proc_order): ascending
// phases forward, descending phases for the transposed (inverse) apply.
__device__ __forceinline__ int op_at(const TcPlan& p, const Unit& u, int k, bool fwd) {
  return __ldg((fwd ? p.ford : p.tord) + u.op_begin + k);
}

// Scratch row of N position n of an accumulating output (plain segments).
__device__ __forceinline__ int acc_pos_row(int n, const int32_t* off, const int32_t* len) {
  return n < len[0] ? off[0] + n : off[1] + (n - len[0]);
}

// ------------------------------------------------------------------ input gathers
// All global traffic of the pre-gather moves through a 32-row shared tile so
// that every warp access is a run of 32 consecutive complex values (512 bytes)
// of one (field, sign) pair: lanes walk degrees or nodes when loading from or
// storing to beta and g, and walk right-hand sides when writing row groups.
// Thread e (0 .. kGatherThreads - 1) is lane e % 32 of gather warp e / 32; for the
// row-group writes it is pair e % kPairs, quarter e / kPairs.

// Every loop below is software-pipelined: the loads of window w + 1 are
// issued into registers before window w is taken out of the tile, so that
// their latency overlaps the previous window's stores.

// Forward gather: a window of 32 degrees |m| + d0 .. is two X_e groups (even
// degrees, Sec. 3.1.2) and two X_o groups (odd degrees).
__device__ void gather_forward(const TcLaunch& L, const Item& itm, const Unit& u, unsigned char* vec, float* T,
                               int e) {
  const TcPlan& p = L.plan[itm.plan];
  const int N = p.N, nx = u.nce + u.nco, iw = e >> 5, lane = e & 31;
  const TcRows tr = tc_rows(u.nce, u.nco, N);
  const int pr = e % kPairs, q = e / kPairs, par = q >> 1, half = q & 1;
  constexpr int kP = kPairs / kGatherWarps;  // pairs each lane loads per window
  const double2* src[kP];
#pragma unroll
  for (int k = 0; k < kP; ++k) {
    const int pk = iw + kGatherWarps * k;
    src[k] = reinterpret_cast<const double2*>(coef_base(L.in[itm.plan], N, itm.am, itm.grp * kTcFields + (pk >> 1),
                                                        pk & 1, L.F[itm.plan], L.single, L.msingle));
  }
  double2 v[kP];
  auto load = [&](int d0) {
#pragma unroll
    for (int k = 0; k < kP; ++k) {
      const int d = d0 + lane;
      v[k] = (src[k] && d < nx) ? __ldg(src[k] + d) : make_double2(0.0, 0.0);
    }
  };
  load(0);
  for (int d0 = 0; d0 < nx; d0 += 32) {
#pragma unroll
    for (int k = 0; k < kP; ++k)
      *reinterpret_cast<float2*>(T + lane * kIoStride + 2 * (iw + kGatherWarps * k)) =
          make_float2(f64_to_f32_bits(v[k].x), f64_to_f32_bits(v[k].y));
    gather_bar();
    if (d0 + 32 < nx) load(d0 + 32);
    const int j = d0 / 16 + half;  // group of X_e (par 0) or X_o (par 1)
    if (kTcGrpRows * j < (par ? u.nco : u.nce)) {
      float re[8], im[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float2 x = *reinterpret_cast<const float2*>(T + (16 * half + 2 * k + par) * kIoStride + 2 * pr);
        re[k] = x.x;
        im[k] = x.y;
      }
      const int G = (par ? tr.xo / kTcGrpRows : 0) + j;
      put_group(vec, G, 2 * pr, re);
      put_group(vec, G, 2 * pr + 1, im);
    }
    gather_bar();
  }
}

// Transposed gather: the W-weighted parity fold of g (Sec. 3.1.1 with the W
// of B = A^T W): Y_e[i] = w_{N+i} (g(theta_{N+i}) + g(theta_{N-1-i})),
// Y_o[i] = w_{N+i} (g(theta_{N+i}) - g(theta_{N-1-i})).  A window is 16
// nodes: lanes 0-15 load g(theta_{N+i}) into tile rows 0-15, lanes 16-31
// g(theta_{N-1-i}) into rows 16-31; it makes two groups of each of Y_e, Y_o.
// Groups are written at their scratch-row group index minus gbase.
__device__ void gather_inverse(const TcLaunch& L, const Item& itm, const Unit& u, unsigned char* vec, float* T,
                               int e, int gbase) {
  const TcPlan& p = L.plan[itm.plan];
  const int N = p.N, iw = e >> 5, lane = e & 31;
  const TcRows tr = tc_rows(u.nce, u.nco, N);
  const int pr = e % kPairs, q = e / kPairs, grp8 = q & 1, par = q >> 1;
  constexpr int kP = kPairs / kGatherWarps;
  const double2* src[kP];
#pragma unroll
  for (int k = 0; k < kP; ++k) {
    const int pk = iw + kGatherWarps * k;
    src[k] = reinterpret_cast<const double2*>(value_base(L.in[itm.plan], N, itm.am, itm.grp * kTcFields + (pk >> 1),
                                                         pk & 1, L.F[itm.plan], L.single, L.msingle));
  }
  const int hl = lane & 15, hi = lane >> 4;
  // node rows that some op reads (whole groups); the rest are never read
  const int lv = __ldg(p.live + itm.am), nl = min(N, lv);
  double2 v[kP];
  auto load = [&](int i0) {
    const int i = i0 + hl;
#pragma unroll
    for (int k = 0; k < kP; ++k)
      v[k] = (src[k] && i < nl) ? __ldg(src[k] + (hi ? N - 1 - i : N + i)) : make_double2(0.0, 0.0);
  };
  load(0);
  for (int i0 = 0; i0 < lv; i0 += 16) {
#pragma unroll
    for (int k = 0; k < kP; ++k)
      *reinterpret_cast<float2*>(T + lane * kIoStride + 2 * (iw + kGatherWarps * k)) =
          make_float2(f64_to_f32_bits(v[k].x), f64_to_f32_bits(v[k].y));
    gather_bar();
    if (i0 + 16 < lv) load(i0 + 16);
    if (i0 + kTcGrpRows * grp8 < lv) {
      float xr[8], xi[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int r = kTcGrpRows * grp8 + k, i = i0 + r;
        const float wi = i < nl ? __ldg(p.w32 + i) : 0.f;
        const float2 a = *reinterpret_cast<const float2*>(T + r * kIoStride + 2 * pr);
        const float2 b = *reinterpret_cast<const float2*>(T + (16 + r) * kIoStride + 2 * pr);
        xr[k] = par ? wi * (a.x - b.x) : wi * (a.x + b.x);
        xi[k] = par ? wi * (a.y - b.y) : wi * (a.y + b.y);
      }
      const int G = (par ? tr.yo : tr.ye) / kTcGrpRows + i0 / kTcGrpRows + grp8 - gbase;
      put_group(vec, G, 2 * pr, xr);
      put_group(vec, G, 2 * pr + 1, xi);
    }
    gather_bar();
  }
}

// The call's inputs ahead of the apply, one item per CTA iteration: the
// gathers above, into the item's block of plan 0's pre-gathered
// buffer (forward: X_e, X_o from group 0; transposed: Y_e, Y_o), by many CTAs
// per SM.
__global__ void __launch_bounds__(kGatherThreads) tc_in_kernel(const __grid_constant__ TcLaunch L, int fwd) {
  __shared__ __align__(16) float T[kIoTile];
  const TcPlan& p = L.plan[0];
  const int npg = tc_pre_groups(p.N);
  for (int it = blockIdx.x; it < L.nitems; it += gridDim.x) {
    const Item itm = item_of(L, it);
    const Unit u = p.units[itm.am];
    unsigned char* dst = p.pre + ((size_t)itm.grp * p.nunits + itm.am) * npg * kTcGrpBytes;
    if (fwd)
      gather_forward(L, itm, u, dst, T, threadIdx.x);
    else
      gather_inverse(L, itm, u, dst, T, threadIdx.x, tc_rows(u.nce, u.nco, p.N).ye / kTcGrpRows);
  }
}

// Output side of one finished item, by the persistent kernel's output warps
// while the tensor cores work on later items: the item's accumulated rows
// (FP32, kTcR right-hand sides per row) to g (forward: the parity fold of
// Sec. 3.1.2, g(theta_{N+i}) = y_e + y_o, g(theta_{N-1-i}) = y_e - y_o) or to
// beta (transposed: X rows back to degrees, even degrees from X_e, odd from
// X_o).  A warp's unit is 16 rows and 8 fields: lanes 2k, 2k + 1 read one 32-byte
// sector of row k (the (+m, -m) values of two fields each), so every load
// takes whole sectors, and every store instruction writes two 256-byte runs
// (16 consecutive nodes or degrees of two fields).  The rows were written by
// this CTA's epilogue and are read past L1.  The loads of U units are issued
// before any of their stores, so that each warp keeps U units in flight.
template <bool FWD, int U>
__device__ void item_out_t(const TcLaunch& L, const Item& itm, int e, int nthreads) {
  const TcPlan& p = L.plan[itm.plan];
  const Unit u = p.units[itm.am];
  const int N = p.N, lane = e & 31, k = lane >> 1, h = lane & 1, nw = nthreads >> 5;
  double* out = L.out[itm.plan];
  const int F = L.F[itm.plan];
  const float* acc = p.acc + ((size_t)itm.grp * p.nunits + itm.am) * (size_t)tc_acc_rows(N) * kTcR;
  const int nrow = FWD ? N : u.nce + u.nco;
  const int yo = tc_r8(N), xo = tc_r8(u.nce);
  const int nlive = FWD ? __ldg(p.live + itm.am) : nrow;  // rows past it are zero (never written)
  constexpr int kUF = kTcFields / 8;  // units per 16 rows
  const int units = ((nrow + 15) >> 4) * kUF;
  for (int q0 = e >> 5; q0 < units; q0 += U * nw) {
    float4 a[U][4], b[FWD ? U : 1][4];
#pragma unroll
    for (int v = 0; v < U; ++v) {
      const int q = q0 + v * nw, r = 16 * (q / kUF) + k, fb = 8 * (q % kUF);
      if (q < units && r < nrow && r < nlive) {
        const int row = FWD ? r : ((r & 1) ? xo + (r >> 1) : (r >> 1));
        const float4* src = reinterpret_cast<const float4*>(acc + (size_t)row * kTcR + 4 * fb) + h;
#pragma unroll
        for (int j = 0; j < 4; ++j) a[v][j] = __ldcg(src + 2 * j);
        if (FWD) {
          const float4* so = reinterpret_cast<const float4*>(acc + (size_t)(yo + r) * kTcR + 4 * fb) + h;
#pragma unroll
          for (int j = 0; j < 4; ++j) b[FWD ? v : 0][j] = __ldcg(so + 2 * j);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          a[v][j] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (FWD) b[FWD ? v : 0][j] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
    }
#pragma unroll
    for (int v = 0; v < U; ++v) {
      const int q = q0 + v * nw, r = 16 * (q / kUF) + k, fb = 8 * (q % kUF);
      if (q >= units || r >= nrow) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int f = itm.grp * kTcFields + fb + 2 * j + h;  // this lane's field; float4 = (+m re, im, -m re, im)
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const float xr = s ? a[v][j].z : a[v][j].x, xi = s ? a[v][j].w : a[v][j].y;
          if (FWD) {
            const double* gb = value_base(out, N, itm.am, f, s, F, L.single, L.msingle);
            if (gb) {
              const float4 y = b[FWD ? v : 0][j];
              const float yr = s ? y.z : y.x, yi = s ? y.w : y.y;
              double2* gp = reinterpret_cast<double2*>(const_cast<double*>(gb));
              __stcs(gp + N + r, make_double2(f32_to_f64_bits(xr + yr), f32_to_f64_bits(xi + yi)));
              __stcs(gp + N - 1 - r, make_double2(f32_to_f64_bits(xr - yr), f32_to_f64_bits(xi - yi)));
            }
          } else {
            const double* bdst = coef_base(out, N, itm.am, f, s, F, L.single, L.msingle);
            if (bdst)
              __stcs(reinterpret_cast<double2*>(const_cast<double*>(bdst)) + r,
                     make_double2(f32_to_f64_bits(xr), f32_to_f64_bits(xi)));
          }
        }
      }
    }
  }
}
__device__ __forceinline__ void item_out(const TcLaunch& L, const Item& itm, bool fwd, int e, int nthreads) {
  if (fwd)
    item_out_t<true, 1>(L, itm, e, nthreads);
  else
    item_out_t<false, 4>(L, itm, e, nthreads);
}

__global__ void __launch_bounds__(kTcThreads, 1) alt_tc_kernel(const __grid_constant__ TcLaunch L, int fwd) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  Ctl* ctl = reinterpret_cast<Ctl*>(base + (size_t)kStages * kStageBytes);
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
    ctl->out_next = 0;
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

  const size_t slot_bytes = tc_slot_bytes(L.max_rows);
  unsigned char* slots = L.ws + (size_t)blockIdx.x * 2 * slot_bytes;  // two vector spaces, alternating by item
  const uint32_t stage0 = s32(base);

  if (warp == kProdWarp) {
    // ------------------------------------------------------------ producer
    // One thread streams the stages: per (op, N tile, K chunk) the chunk's
    // operand-image piece block and its input row groups (at most one run of
    // whole groups per segment), all as bulk copies whose bytes the stage's
    // full barrier expects.
    long jp = 0;
    int tiles_before = 0;  // tiles of all earlier phases (all items so far)
    bool ok = true;
    for (int iseq = 0; ok; ++iseq) {
      int it = -1;
      if (lane == 0) it = next_item(ctl, iseq, ok);
      it = __shfl_sync(0xffffffffu, it, 0);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok || it < 0) break;
      const Item itm = item_of(L, it);
      const TcPlan& p = L.plan[itm.plan];
      const Unit u = p.units[itm.am];
      const unsigned char* vec = slots + (size_t)(iseq & 1) * slot_bytes;
      // transposed inputs gathered ahead: the groups of Y_e, Y_o come from
      // the item's block of the pre-gathered buffer
      // inputs gathered ahead: forward, the X_e, X_o groups (from group 0);
      // transposed, the Y_e, Y_o groups (from group ye / 8), each from the
      // item's block of the pre-gathered buffer
      const TcRows trp = tc_rows(u.nce, u.nco, p.N);
      const int pg0 = fwd ? 0 : trp.ye / kTcGrpRows;
      const int png = fwd ? (trp.xo + tc_r8(u.nco)) / kTcGrpRows : tc_pre_groups(p.N);
      const unsigned char* pre =
          p.pre ? p.pre + ((size_t)itm.grp * p.nunits + itm.am) * tc_pre_groups(p.N) * kTcGrpBytes : nullptr;
      auto grp_src = [&](int g) -> const unsigned char* {
        return (pre && g >= pg0 && g < pg0 + png) ? pre + (size_t)(g - pg0) * kTcGrpBytes
                                                  : vec + (size_t)g * kTcGrpBytes;
      };
      const int nops = u.op_end - u.op_begin;
      TcOp nxt = nops > 0 ? p.ops[op_at(p, u, 0, fwd)] : TcOp{};
      int cur_phase = -1, tiles_here = 0;
      for (int q = 0; q < nops && ok; ++q) {
        const TcOp op = nxt;
        if (q + 1 < nops) nxt = p.ops[op_at(p, u, q + 1, fwd)];
        if (op.phase != cur_phase) {
          // a phase reads rows that earlier phases of this item wrote: wait for
          // their tiles (the item's first phase reads only gathered rows)
          tiles_before += tiles_here;
          tiles_here = 0;
          if (cur_phase >= 0 && lane == 0) ok = counter_wait(ctl, &ctl->done_tiles, tiles_before);
          ok = __shfl_sync(0xffffffffu, ok, 0);
          cur_phase = op.phase;
        }
        const TcDir d = tc_dir(op, fwd);
        const TcKGeom& kg = d.kg;
        const uint16_t* img = p.img + (fwd ? op.img[0] : op.img[1]);
        for (int t = 0; t < d.nT && ok; ++t) {
          const int Np = (min(kTcNT, d.NN - kTcNT * t) + 15) & ~15;
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
                bulk_copy(sB, img + (size_t)t * (3 * kTcNT) * kg.kp_tot + (size_t)Np * (3 * kTcKC * c), bbytes,
                          &ctl->full[s]);
                if (ja > j0)
                  bulk_copy(sA, grp_src(kg.gs0 + j0), (uint32_t)(ja - j0) * kTcGrpBytes, &ctl->full[s]);
                if (j1 > ja)
                  bulk_copy(sA + (uint32_t)(ja - j0) * kTcGrpBytes, grp_src(kg.gs1 + ja - kg.ng0),
                            (uint32_t)(j1 - ja) * kTcGrpBytes, &ctl->full[s]);
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
    // The whole warp runs the loop with warp-uniform values (broadcast from
    // lane 0), and one elected lane issues each MMA and commit.
    long jm = 0, tm = 0;
    bool ok = true;
    for (int iseq = 0; ok; ++iseq) {
      int it = next_item(ctl, iseq, ok);
      ok = __all_sync(0xffffffffu, ok);
      it = __shfl_sync(0xffffffffu, it, 0);
      if (!ok || it < 0) break;
      const Item itm = item_of(L, it);
      const TcPlan& p = L.plan[itm.plan];
      const Unit u = p.units[itm.am];
      const int nops = __shfl_sync(0xffffffffu, u.op_end - u.op_begin, 0);
      TcOp nxt = nops > 0 ? p.ops[op_at(p, u, 0, fwd)] : TcOp{};
      for (int q = 0; q < nops && ok; ++q) {
        const TcOp op = nxt;
        if (q + 1 < nops) nxt = p.ops[op_at(p, u, q + 1, fwd)];
        const TcDir d = tc_dir(op, fwd);
        const int nT = __shfl_sync(0xffffffffu, d.nT, 0), NN = __shfl_sync(0xffffffffu, d.NN, 0);
        const int nK = __shfl_sync(0xffffffffu, d.kg.nK, 0), kp_tot = __shfl_sync(0xffffffffu, d.kg.kp_tot, 0);
        for (int t = 0; t < nT && ok; ++t, ++tm) {
          const int b = (int)(tm & 1);
          const uint32_t v = (uint32_t)(tm >> 1);
          ok = __all_sync(0xffffffffu, mbar_wait(ctl, &ctl->acce[b], (v & 1u) ^ 1u));
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const int Np = (min(kTcNT, NN - kTcNT * t) + 15) & ~15;
          // BF16 A and B, FP32 D, both operands K-major, N = Np, M = 128
          const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(Np >> 3) << 17) | (8u << 24);
          const uint32_t dhi = taddr + (uint32_t)(b * kAccCols), dlo = dhi + kTcNT;
          // descriptors of stage 0 for this tile; a stage, a K step or a piece
          // moves the start address, i.e. adds (byte offset / 16) to the descriptor
          const uint32_t bK = (uint32_t)(Np / 8) * 128;
          const uint64_t a_desc0 = sdesc(stage0, kTcGrpBytes, 128);
          const uint64_t b_desc0 = sdesc(stage0 + kStageA, bK, 128);
          for (int c = 0; c < nK && ok; ++c, ++jm) {
            const int s = (int)(jm % kStages);
            const uint32_t use = (uint32_t)(jm / kStages);
            ok = __all_sync(0xffffffffu, mbar_wait(ctl, &ctl->full[s], use & 1u));
            if (!ok) break;
            // the stage was filled by bulk copies (async proxy), which the
            // MMAs read through the same proxy: the barrier orders them
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int Kp = min(kTcKC, kp_tot - kTcKC * c);
            const uint64_t stg = (uint64_t)((s * kStageBytes) >> 4);
            const uint64_t ad0 = a_desc0 + stg, bd0 = b_desc0 + stg;
            const uint64_t bpc = (uint64_t)((Np * Kp * 2) >> 4), bks = (uint64_t)(2 * bK >> 4);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
              if (ks * 16 >= Kp) break;
              // A K-major: core (m8, k8) of piece pa at (k8 * 3 + pa) * 2048 + m8 * 128
              // (K stride one row group, M stride 128); B K-major, pieces bpc apart
              const uint64_t ak = ad0 + (uint64_t)((ks * 2 * kTcGrpBytes) >> 4), bk = bd0 + ks * bks;
              const uint32_t first = (c > 0 || ks > 0) ? 1u : 0u;
              mma_bf16(dhi, ak, bk, idesc, first);                          // a0 b0
              mma_bf16(dlo, ak, bk + bpc, idesc, first);                    // a0 b1
              mma_bf16(dlo, ak + (2048 >> 4), bk, idesc, 1u);               // a1 b0
              mma_bf16(dlo, ak, bk + 2 * bpc, idesc, 1u);                   // a0 b2
              mma_bf16(dlo, ak + (2048 >> 4), bk + bpc, idesc, 1u);         // a1 b1
              mma_bf16(dlo, ak + (4096 >> 4), bk, idesc, 1u);               // a2 b0
            }
            mma_commit(&ctl->empty[s]);
          }
          if (ok) mma_commit(&ctl->accf[b]);
        }
      }
    }
    __syncwarp();
  } else if (warp >= kEpiWarp0 && warp < kEpiWarp0 + kEpiWarps) {
    // ------------------------------------------------------------ epilogue
    // accumulator -> rows: two teams of four warps; warp w owns TMEM lane
    // quadrant ew = w % 4, thread = one right-hand side (32 ew + lane); team
    // t takes the 32-position chunks t, t + 2, ... of every tile
    const int ew = warp % 4, team = (warp - kEpiWarp0) / 4;
    const int e = tid - 32 * kEpiWarp0;
    const int rhs = 32 * ew + lane;
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
      float* acc = p.acc + ((size_t)itm.grp * p.nunits + itm.am) * (size_t)tc_acc_rows(p.N) * kTcR;
      const TcRows tr = tc_rows(u.nce, u.nco, p.N);
      const int acc0 = fwd ? tr.ye : 0;  // accumulated rows: Y forward, X transposed
      const int nops = u.op_end - u.op_begin;
      TcOp nxt = nops > 0 ? p.ops[op_at(p, u, 0, fwd)] : TcOp{};
      for (int q = 0; q < nops && ok; ++q) {
        const TcOp op = nxt;
        if (q + 1 < nops) nxt = p.ops[op_at(p, u, q + 1, fwd)];
        const TcDir d = tc_dir(op, fwd);
        const int32_t* oo = fwd ? op.out_off : op.in_off;
        const int32_t* ol = fwd ? op.out_len : op.in_len;
        for (int t = 0; t < d.nT && ok; ++t, ++te) {
          const int b = (int)(te & 1);
          const uint32_t v = (uint32_t)(te >> 1);
          ok = epi_and(mbar_wait(ctl, &ctl->accf[b], v & 1u));
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const int Nt = min(kTcNT, d.NN - kTcNT * t);
          if (32 * team >= Nt) {
            // no chunk of this tile for this team: its share of the accumulator is free
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl->acce[b]);
          }
          for (int c0 = 32 * team; c0 < Nt; c0 += 64) {
            uint32_t hv[32];
            if (d.KK > 0) {
              uint32_t lv[32];
              const uint32_t ta = taddr + ((uint32_t)(32 * ew) << 16) + (uint32_t)(b * kAccCols + c0);
              tmem_ld32(ta, hv);
              tmem_ld32(ta + kTcNT, lv);
              tmem_wait_ld();
#pragma unroll
              for (int k = 0; k < 32; ++k) hv[k] = __float_as_uint(__uint_as_float(hv[k]) + __uint_as_float(lv[k]));
            } else {
#pragma unroll
              for (int k = 0; k < 32; ++k) hv[k] = 0u;
            }
            if (c0 + 64 >= Nt) {
              // the team's last columns of the tile are in registers: its share
              // of the accumulator pair is free for the MMAs of tile te + 2
              asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
              __syncwarp();
              if (lane == 0) mbar_arrive(&ctl->acce[b]);
            }
            const int n0 = kTcNT * t + c0;  // N position of hv[0]
            if (d.accum) {
              // 4 x 4 transposes within each quad of lanes (right-hand sides
              // 4 q .. 4 q + 3): afterwards lane 4 q + k holds row 4 j + k of
              // all four, added with one 16-byte reduction
              const int k4 = lane & 3;
              const bool b0 = (k4 & 1) != 0, b1 = (k4 & 2) != 0;
              float* arow = acc + (32 * ew + (lane & ~3));
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                float x0 = __uint_as_float(hv[4 * j]), x1 = __uint_as_float(hv[4 * j + 1]);
                float x2 = __uint_as_float(hv[4 * j + 2]), x3 = __uint_as_float(hv[4 * j + 3]);
                float r0 = __shfl_xor_sync(0xffffffffu, b1 ? x0 : x2, 2);
                float r1 = __shfl_xor_sync(0xffffffffu, b1 ? x1 : x3, 2);
                if (b1) {
                  x0 = r0;
                  x1 = r1;
                } else {
                  x2 = r0;
                  x3 = r1;
                }
                r0 = __shfl_xor_sync(0xffffffffu, b0 ? x0 : x1, 1);
                r1 = __shfl_xor_sync(0xffffffffu, b0 ? x2 : x3, 1);
                if (b0) {
                  x0 = r0;
                  x2 = r1;
                } else {
                  x1 = r0;
                  x3 = r1;
                }
                if (c0 + 4 * j + k4 < Nt) {
                  const int r = acc_pos_row(n0 + 4 * j + k4, oo, ol) - acc0;
                  if (d.store)  // the rows' first writer
                    __stcg(reinterpret_cast<float4*>(arow + (size_t)r * kTcR), make_float4(x0, x1, x2, x3));
                  else
                    red_add4(arow + (size_t)r * kTcR, x0, x1, x2, x3);
                }
              }
            } else {
#pragma unroll
              for (int jj = 0; jj < 4; ++jj)
                if (c0 + 8 * jj < Nt) {
                  float x[8];
#pragma unroll
                  for (int k = 0; k < 8; ++k) x[k] = __uint_as_float(hv[8 * jj + k]);
                  put_group(vec, tc_group(d.ng, n0 / 8 + jj), rhs, x);
                }
            }
          }
          // rows written above are read next by bulk copies (async proxy); the
          // accumulated rows, after the item's last tile, by the item warps'
          // output step, which reads them from L2: there every epilogue
          // thread's stores and reductions are made visible at GPU scope
          if (!d.accum) asm volatile("fence.proxy.async.global;" ::: "memory");
          if (L.fuse_out && q + 1 == nops && t + 1 == d.nT)
            __threadfence();
          else
            __threadfence_block();
          epi_bar();
          ++done;
          if (e == 0) *((volatile int*)&ctl->done_tiles) = done;
        }
      }
    }
  } else if (warp >= kIoWarp0 && warp < kIoWarp0 + kIoThreads / 32) {
    // ------------------------------------------------------------ item warps
    // They take this CTA's items from the launch's work counter (decreasing
    // cost) once item i - 2 has finished all of its tiles (slot i % 2 of the
    // intermediate rows is item i - 2's) and, when the kernel writes the
    // outputs, the output warps have taken item i - kRing from the ring; zero
    // the item's accumulation rows that no op stores first, and publish it in
    // ctl->ring for the other roles.  Its inputs were gathered ahead by
    // tc_in_kernel.
    const int e = tid - 32 * kIoWarp0;
    int t_m2 = 0, t_m1 = 0;  // tiles of all items up to i-2, up to i-1
    bool ok = L.stall == 0;
    for (int iseq = 0; ok; ++iseq) {
      ok = counter_wait(ctl, &ctl->done_tiles, t_m2);
      if (ok && L.fuse_out) ok = counter_wait(ctl, &ctl->out_next, iseq - kRing + 1);
      ok = io_and(ok);
      if (!ok) break;
      if (e == 0) {
        const unsigned int w = atomicAdd(L.counter, 1u);
        ctl->ring[iseq % kRing] = w < (unsigned int)L.nitems ? (int)w : -1;
      }
      io_bar();
      const int it = *((volatile int*)&ctl->ring[iseq % kRing]);
      if (it < 0) {
        __threadfence_block();
        if (e == 0) *((volatile int*)&ctl->gathered) = iseq + 1;
        break;
      }
      const Item itm = item_of(L, it);
      const TcPlan& p = L.plan[itm.plan];
      // accumulation rows that no op stores first start at zero (the
      // epilogue adds into them; the output step reads every row)
      {
        float4* a4 = reinterpret_cast<float4*>(p.acc + ((size_t)itm.grp * p.nunits + itm.am) *
                                                           (size_t)tc_acc_rows(p.N) * kTcR);
        const int z1 = p.zri[2 * itm.am + (fwd ? 1 : 2)];
        for (int z = p.zri[2 * itm.am + (fwd ? 0 : 1)]; z < z1; ++z) {
          float4* a = a4 + (size_t)p.zr[2 * z] * (kTcR / 4);
          const int n4 = p.zr[2 * z + 1] * (kTcR / 4);
          for (int k = e; k < n4; k += kIoThreads) __stcg(a + k, make_float4(0.f, 0.f, 0.f, 0.f));
        }
      }
      __threadfence();
      io_bar();
      if (e == 0) *((volatile int*)&ctl->gathered) = iseq + 1;
      const int t_cur = t_m1 + p.tiles[2 * itm.am + (fwd ? 0 : 1)];
      t_m2 = t_m1;
      t_m1 = t_cur;
    }
  } else if (warp >= kOutWarp0 && L.fuse_out) {
    // ------------------------------------------------------------ output warps
    // Each published item in turn, once its last tile is done: its outputs
    // from its finished rows (item_out), while the tensor cores work on the
    // items after it.  They run behind the other roles by as many items as
    // the outputs take, up to kRing - 1.
    const int e = tid - 32 * kOutWarp0;
    int t_acc = 0;  // tiles of all items up to this one
    bool ok = true;
    for (int j = 0; ok; ++j) {
      ok = out_and(counter_wait(ctl, &ctl->gathered, j + 1));
      if (!ok) break;
      const int it = *((volatile int*)&ctl->ring[j % kRing]);
      out_bar();
      if (e == 0) *((volatile int*)&ctl->out_next) = j + 1;
      if (it < 0) break;
      const Item itm = item_of(L, it);
      t_acc += L.plan[itm.plan].tiles[2 * itm.am + (fwd ? 0 : 1)];
      ok = out_and(counter_wait(ctl, &ctl->done_tiles, t_acc));
      if (!ok) break;
      item_out(L, itm, fwd, e, kOutTeam);
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
// (transposed: X rows back to degrees).  A streaming kernel with many warps per
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
  const int yo = tc_r8(N);  // Y_o's first accumulation row
  for (long w = blockIdx.x; w < total; w += gridDim.x) {
    const int item = (int)(w / cpi), chunk = (int)(w % cpi);
    const int grp = item % G;
    const int am = single ? (msingle < 0 ? -msingle : msingle) : item / G;
    const Unit u = p.units[am];
    const float* acc_item = p.acc + ((size_t)grp * p.nunits + am) * (size_t)tc_acc_rows(N) * kTcR;
    if (fwd) {
      const int i0 = 32 * chunk;
      const int nl = __ldg(p.live + am);  // node rows past it are zero (never written)
      for (int r = iw; r < 32; r += kOutThreads / 32) {
        if (i0 + r < N && i0 + r < nl) {
          *reinterpret_cast<float4*>(Te + r * kIoStride + 4 * lane) =
              __ldcs(reinterpret_cast<const float4*>(acc_item + (size_t)(i0 + r) * kTcR) + lane);
          *reinterpret_cast<float4*>(To + r * kIoStride + 4 * lane) =
              __ldcs(reinterpret_cast<const float4*>(acc_item + (size_t)(yo + i0 + r) * kTcR) + lane);
        } else if (i0 + r < N) {
          *reinterpret_cast<float4*>(Te + r * kIoStride + 4 * lane) = make_float4(0.f, 0.f, 0.f, 0.f);
          *reinterpret_cast<float4*>(To + r * kIoStride + 4 * lane) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      __syncthreads();
      const int i = i0 + lane;
      for (int pr = iw; pr < kPairs; pr += kOutThreads / 32) {
        const double* gb = value_base(out, N, am, grp * kTcFields + (pr >> 1), pr & 1, F, single, msingle);
        if (gb && i < N) {
          const float2 ev = *reinterpret_cast<const float2*>(Te + lane * kIoStride + 2 * pr);
          const float2 ov = *reinterpret_cast<const float2*>(To + lane * kIoStride + 2 * pr);
          double2* gp = reinterpret_cast<double2*>(const_cast<double*>(gb));
          __stcs(gp + N + i, make_double2(f32_to_f64_bits(ev.x + ov.x), f32_to_f64_bits(ev.y + ov.y)));
          __stcs(gp + N - 1 - i, make_double2(f32_to_f64_bits(ev.x - ov.x), f32_to_f64_bits(ev.y - ov.y)));
        }
      }
      __syncthreads();
    } else {
      const int nx = u.nce + u.nco, d0 = 32 * chunk, xo = tc_r8(u.nce);
      if (d0 >= nx) continue;  // uniform over the CTA
      for (int dl = iw; dl < 32; dl += kOutThreads / 32) {
        const int d = d0 + dl;
        if (d < nx) {
          const int t = (d & 1) ? xo + (d >> 1) : (d >> 1);
          *reinterpret_cast<float4*>(Te + dl * kIoStride + 4 * lane) =
              __ldcs(reinterpret_cast<const float4*>(acc_item + (size_t)t * kTcR) + lane);
        }
      }
      __syncthreads();
      const int d = d0 + lane;
      for (int pr = iw; pr < kPairs; pr += kOutThreads / 32) {
        const double* bdst = coef_base(out, N, am, grp * kTcFields + (pr >> 1), pr & 1, F, single, msingle);
        if (bdst && d < nx) {
          const float2 v = *reinterpret_cast<const float2*>(Te + lane * kIoStride + 2 * pr);
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
                      unsigned char* ws, unsigned int* counter, int* err, cudaStream_t st, cudaEvent_t* ev) {
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
  L.ws = ws;
  L.max_rows = p.max_rows;
  L.counter = counter;
  L.err = err;
  L.fuse_out = fwd ? 0 : 1;
  cudaError_t e = cudaFuncSetAttribute(alt_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTotal);
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
  if (!p.pre) return cudaErrorInvalidValue;  // the inputs are always gathered ahead
  {
    tc_in_kernel<<<std::max(1, std::min(L.nitems, 8 * sm_count())), kGatherThreads, 0, st>>>(L, fwd ? 1 : 0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  alt_tc_kernel<<<grid, kTcThreads, kSmemTotal, st>>>(L, fwd ? 1 : 0);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[1], st)) != cudaSuccess) return e;
  if (!L.fuse_out) e = launch_out(p, fwd, out, F, single, m, sm_count(), st);
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], st);
  return e;
}

cudaError_t launch_tc_stall(const TcPlan& p, unsigned char* ws, unsigned int* counter, int* err, cudaStream_t st) {
  TcLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.plan[0] = p;
  L.F[0] = 1;
  L.nplans = 1;
  L.nitems = 1;
  L.ws = ws;
  L.max_rows = p.max_rows;
  L.counter = counter;
  L.err = err;
  L.stall = 1;
  cudaError_t e = cudaFuncSetAttribute(alt_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTotal);
  if (e != cudaSuccess) return e;
  alt_tc_kernel<<<1, kTcThreads, kSmemTotal, st>>>(L, 1);
  return cudaGetLastError();
}

cudaError_t launch_tc_batch(const TcLaunch& L, bool fwd, int grid, cudaStream_t st, cudaEvent_t* ev) {
  if (L.nplans < 1 || L.nplans > kTcMaxPlans || !L.items) return cudaErrorInvalidValue;
  for (int q = 0; q < L.nplans; ++q)
    if ((L.F[q] + kTcFields - 1) / kTcFields > L.plan[q].gmax) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(alt_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTotal);
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
  {
    // each plan's inputs gathered ahead, one launch per plan
    for (int q = 0; q < L.nplans; ++q) {
      if (L.F[q] <= 0) continue;
      if (!L.plan[q].pre) return cudaErrorInvalidValue;
      TcLaunch Lq;
      std::memset(&Lq, 0, sizeof(Lq));
      Lq.plan[0] = L.plan[q];
      Lq.in[0] = L.in[q];
      Lq.out[0] = L.out[q];
      Lq.F[0] = L.F[q];
      Lq.nplans = 1;
      Lq.nitems = L.plan[q].nunits * ((L.F[q] + kTcFields - 1) / kTcFields);
      tc_in_kernel<<<std::max(1, std::min(Lq.nitems, 8 * sm_count())), kGatherThreads, 0, st>>>(Lq, fwd ? 1 : 0);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  TcLaunch Lk = L;
  Lk.fuse_out = fwd ? 0 : 1;
  alt_tc_kernel<<<grid, kTcThreads, kSmemTotal, st>>>(Lk, fwd ? 1 : 0);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[1], st)) != cudaSuccess) return e;
  const int sms = sm_count();
  for (int q = 0; q < L.nplans && e == cudaSuccess && !Lk.fuse_out; ++q)
    if (L.F[q] > 0) e = launch_out(L.plan[q], fwd, L.out[q], L.F[q], 0, 0, sms, st);
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], st);
  return e;
}

}  // namespace sht
