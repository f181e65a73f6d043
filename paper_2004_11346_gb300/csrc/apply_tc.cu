// Many-field apply of the IDBF-factored ALT on the 5th-generation tensor
// cores (tcgen05, sm_103a), split-BF16 products with FP32 accumulation.
//
// One work item is one order |m| for 32 fields: 128 real right-hand sides.
// Every block product of the apply program, out (+)= B in, is computed
// transposed, out^T = in^T B^T, so that the 128 right-hand sides fill the MMA
// M dimension and the block's rows are N (tiles of <= 128, padded to 16):
//   A operand = in^T (128 x K, MN-major): the op's input rows, kept in the
//               scratch as three BF16 pieces a0 + a1 + a2 (8 bits each) of
//               every value, so staging is a plain asynchronous copy;
//   B operand = B (N x K, K-major): precomputed split-BF16 image b0 + b1 + b2;
//   D         = 128 x N FP32 accumulator in tensor memory.
// The CTA is warp-specialised and persistent (one per SM): a producer warp
// streams (op, tile, 32-wide K chunk) operand stages into a 4-deep shared
// memory ring with cp.async; an MMA warp issues the tensor-core products into
// two double-buffered TMEM accumulator pairs; four epilogue warps drain the
// accumulators, split the results into BF16 pieces for the next level (or add
// them in FP32 into the shared output rows), and run the gather and the
// parity fold.  Ops of one phase read only rows written by earlier phases: the
// producer starts a phase after the epilogue has counted every earlier tile.
// Per 16-wide K step six MMAs accumulate a_p b_q for p + q <= 2, which keeps
// every product to about 2^-24 relative error (FP32 quality); a0 b0 and the
// five smaller cross products go to two separate accumulators that the
// epilogue adds in FP32.  Operands sit
// in shared memory in the canonical no-swizzle K-major layout (8 x 16-byte
// core matrices; LBO = stride between core matrices along K, SBO = along M/N).
// All waits are bounded: a wait that runs out sets an error flag, every role
// stops, and the host reports SHT_ERR_TIMEOUT.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "apply_tc.cuh"

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

size_t tc_image_elems(int NN, int KK) {
  if (NN <= 0 || KK <= 0) return 0;
  const int nK = (KK + kTcKC - 1) / kTcKC;
  const size_t kp_tot = (size_t)kTcKC * (nK - 1) + r16(KK - kTcKC * (nK - 1));
  const int nT = (NN + kTcNT - 1) / kTcNT;
  const size_t np_tot = (size_t)kTcNT * (nT - 1) + r16(NN - kTcNT * (nT - 1));
  return 3 * np_tot * kp_tot;
}

// Layout (matching the kernel): tiles t, chunks c, pieces p, then core
// matrices (ki, mi) in K-outer order, 8 rows x 8 elements each.
template <class E>
static void tc_pack(int NN, int KK, E elem, uint16_t* dst) {
  const int nT = (NN + kTcNT - 1) / kTcNT, nK = (KK + kTcKC - 1) / kTcKC;
  size_t o = 0;
  for (int t = 0; t < nT; ++t) {
    const int Np = r16(std::min(kTcNT, NN - kTcNT * t));
    for (int c = 0; c < nK; ++c) {
      const int Kp = r16(std::min(kTcKC, KK - kTcKC * c));
      // pieces of every element of the chunk
      for (int p = 0; p < 3; ++p)
        for (int ki = 0; ki < Kp / 8; ++ki)
          for (int mi = 0; mi < Np / 8; ++mi)
            for (int rr = 0; rr < 8; ++rr)
              for (int kk = 0; kk < 8; ++kk) {
                const int n = kTcNT * t + mi * 8 + rr, k = kTcKC * c + ki * 8 + kk;
                double v = (n < NN && k < KK) ? elem(n, k) : 0.0;
                uint16_t h = 0;
                for (int q = 0; q <= p; ++q) {  // piece q of v: bf16 of the remainder
                  h = bf16_rn((float)v);
                  v -= bf16_to_d(h);
                }
                dst[o++] = h;
              }
    }
  }
}

void tc_build_images(const std::vector<Op>& ops, const std::vector<double>& factors, std::vector<uint16_t>& img,
                     std::vector<int64_t>& off) {
  const size_t n = ops.size();
  off.assign(2 * n, 0);
  size_t tot = 0;
  for (size_t i = 0; i < n; ++i) {
    off[2 * i] = (int64_t)tot;
    tot += tc_image_elems(ops[i].mo, ops[i].ni);
    off[2 * i + 1] = (int64_t)tot;
    tot += tc_image_elems(ops[i].ni, ops[i].mo);
  }
  img.assign(std::max<size_t>(tot, 8), 0);
#pragma omp parallel for schedule(dynamic, 64)
  for (long i = 0; i < (long)n; ++i) {
    const Op& op = ops[i];
    const double* B = factors.data() + op.b_off;
    const int ld = op.ld;
    if (op.ni > 0) {
      tc_pack(op.mo, op.ni, [&](int r, int k) { return B[(size_t)k * ld + r]; }, img.data() + off[2 * i]);
      tc_pack(op.ni, op.mo, [&](int r, int k) { return B[(size_t)r * ld + k]; }, img.data() + off[2 * i + 1]);
    }
  }
}

// ---------------------------------------------------------------- device side
namespace {

constexpr int kStages = 3;
constexpr int kProdWarps = 3;                 // warps staging operands
constexpr int kMmaWarp = kProdWarps;          // the MMA-issuing warp
constexpr int kEpiWarp0 = kProdWarps + 1;     // first epilogue warp
constexpr int kEpiWarps = 4;                  // one warpgroup drains the accumulators
constexpr int kIoWarp0 = kEpiWarp0 + kEpiWarps;  // 8 I/O warps: gather, parity fold / scatter
constexpr int kTrStride = 33;                 // padded 32 x 32 transpose tile (floats)
constexpr int kPieceA = kTcR * kTcKC * 2;      // bytes of one A piece in a stage (8 KB)
constexpr int kStageA = 3 * kPieceA;           // 24 KB
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
  int gathered;    // items whose gather is complete
  int done_tiles;  // tiles whose epilogue is complete (all items so far)
};
constexpr size_t kTrBytes = (size_t)kEpiWarps * 32 * kTrStride * 4;
constexpr size_t kSmemTotal = (size_t)kStages * kStageBytes + kTrBytes + sizeof(Ctl) + 1024;

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

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
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
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(s32(bar)) : "memory");
}

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
__device__ __forceinline__ void io_bar() { asm volatile("bar.sync 2, 256;" ::: "memory"); }

__device__ __forceinline__ long coef_offset(long N, long m) {
  long a = m < 0 ? -m : m;
  if (a == 0) return 0;
  long pos = 2 * N * (2 * a - 1) - a * (a - 1);
  return m > 0 ? pos : pos + (2 * N - a);
}
__device__ __forceinline__ long order_slot(long m) { return m == 0 ? 0 : (m > 0 ? 2 * m - 1 : -2 * m); }
__device__ __forceinline__ int seg_row(int t, const int32_t off[2], const int32_t len[2]) {
  return t < len[0] ? off[0] + t : off[1] + (t - len[0]);
}
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

__device__ __forceinline__ uint16_t f2bf(float f) { return __bfloat16_as_ushort(__float2bfloat16_rn(f)); }
__device__ __forceinline__ float bf2f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

// value -> three BF16 pieces at column `col` of a scratch row
__device__ __forceinline__ void put_pieces(unsigned char* row, int col, float v) {
  unsigned short* p = reinterpret_cast<unsigned short*>(row) + col;
  const uint16_t h0 = f2bf(v);
  v -= bf2f(h0);
  const uint16_t h1 = f2bf(v);
  v -= bf2f(h1);
  const uint16_t h2 = f2bf(v);
  __stcg(p, (unsigned short)h0);
  __stcg(p + kTcR, (unsigned short)h1);
  __stcg(p + 2 * kTcR, (unsigned short)h2);
}
__device__ __forceinline__ float* fp32_at(unsigned char* row, int col) { return reinterpret_cast<float*>(row) + col; }

// Shape of one op in the requested direction.
struct OpShape {
  int NN, KK, nT, nK, kp_tot;
};
__device__ __forceinline__ OpShape op_shape(const Op& op, bool fwd) {
  OpShape s;
  s.NN = fwd ? op.mo : op.ni;
  s.KK = fwd ? op.ni : op.mo;
  s.nT = (s.NN + kTcNT - 1) / kTcNT;
  s.nK = s.KK > 0 ? (s.KK + kTcKC - 1) / kTcKC : 0;
  s.kp_tot = s.KK > 0 ? kTcKC * (s.nK - 1) + ((s.KK - kTcKC * (s.nK - 1) + 15) & ~15) : 0;
  return s;
}

struct Item {
  int grp, am;
};
__device__ __forceinline__ int row_kk(const Unit& u, int t) { return t < u.nce ? 2 * t : 2 * (t - u.nce) + 1; }
__device__ __forceinline__ Item item_of(const TcPlan& p, int it, int G, int single, int msingle) {
  Item r;
  r.grp = it % G;
  r.am = single ? (msingle < 0 ? -msingle : msingle) : p.order[it / G];
  return r;
}

// Tiles (epilogue units) of one work item.
__device__ int item_tiles(const TcPlan& p, const Unit& u, bool fwd) {
  int n = 0;
  for (int oi = u.op_begin; oi < u.op_end; ++oi) n += op_shape(p.ops[oi], fwd).nT;
  return n;
}

__global__ void __launch_bounds__(kTcThreads, 1) alt_tc_kernel(TcPlan p, const double* __restrict__ in,
                                                               double* __restrict__ out, int F, int single,
                                                               int msingle, int fwd) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* trbuf = reinterpret_cast<float*>(base + (size_t)kStages * kStageBytes);
  Ctl* ctl = reinterpret_cast<Ctl*>(base + (size_t)kStages * kStageBytes + kTrBytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&ctl->full[s], 32 * kProdWarps + 1);  // cp.async arrivals + the bulk copy's expect_tx
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

  const int N = p.N;
  const int G = (F + kTcFields - 1) / kTcFields;
  const int nitems = single ? G : p.nunits * G;
  const size_t slot_bytes = (size_t)p.max_rows * kTcRowBytes;
  unsigned char* slots = p.ws + (size_t)blockIdx.x * 2 * slot_bytes;  // two vector spaces, alternating by item
  const uint32_t stage0 = s32(base);

  if (warp < kProdWarps) {
    // ------------------------------------------------------------ producers
    long jp = 0;
    int tiles_before = 0;
    bool ok = true;
    for (int it = blockIdx.x, iseq = 0; it < nitems && ok; it += gridDim.x, ++iseq) {
      const Item itm = item_of(p, it, G, single, msingle);
      const Unit u = p.units[itm.am];
      unsigned char* vec = slots + (size_t)(iseq & 1) * slot_bytes;
      ok = counter_wait(ctl, &ctl->gathered, iseq + 1);
      for (int k = 0; k < u.nphase && ok; ++k) {
        const int ph = fwd ? k : u.nphase - 1 - k;
        ok = counter_wait(ctl, &ctl->done_tiles, tiles_before);
        int tiles_here = 0;
        for (int oi = p.phase_tab[u.ph_begin + ph]; oi < p.phase_tab[u.ph_begin + ph + 1] && ok; ++oi) {
          const Op op = p.ops[oi];
          const OpShape sh = op_shape(op, fwd);
          const int32_t* ioff = fwd ? op.in_off : op.out_off;
          const int32_t* ilen = fwd ? op.in_len : op.out_len;
          const uint16_t* img = p.img + p.img_off[2 * oi + (fwd ? 0 : 1)];
          for (int t = 0; t < sh.nT && ok; ++t) {
            const int Np = (min(kTcNT, sh.NN - kTcNT * t) + 15) & ~15;
            for (int c = 0; c < sh.nK && ok; ++c, ++jp) {
              const int s = (int)(jp % kStages);
              const uint32_t use = (uint32_t)(jp / kStages);
              ok = mbar_wait(ctl, &ctl->empty[s], (use & 1u) ^ 1u);
              if (!ok) break;
              const int Kp = (min(kTcKC, sh.KK - kTcKC * c) + 15) & ~15;
              const uint32_t sA = stage0 + (uint32_t)s * kStageBytes, sB = sA + kStageA;
              // B: the image chunk (3 pieces, contiguous) in one bulk copy whose
              // bytes the full barrier expects
              if (warp == 0 && lane == 0) {
                const uint16_t* src = img + (size_t)t * 384 * sh.kp_tot + (size_t)Np * (96 * c);
                const uint32_t bytes = (uint32_t)(3 * Np * Kp * 2);
                bulk_expect(&ctl->full[s], bytes);
                bulk_copy(sB, src, bytes, &ctl->full[s]);
              }
              // A: Kp input rows x 3 pieces x 16 chunks of 8 right-hand sides
              // (MN-major cores).  Lane l owns the row pointer of row l and the
              // (piece, 8-column chunk) pairs l and l + 32 of every row.
              {
                const int j = kTcKC * c + lane;
                const bool valid = lane < Kp && j < sh.KK;
                const unsigned char* myrow = valid ? vec + (size_t)seg_row(j, ioff, ilen) * kTcRowBytes : vec;
                const int pc0 = lane >> 4, m80 = lane & 15;           // pair lane
                const int pc1 = (lane + 32) >> 4, m81 = (lane + 32) & 15;  // pair lane + 32 (lanes < 16)
                const uint32_t d0 = sA + pc0 * kPieceA + m80 * 128, d1 = sA + pc1 * kPieceA + m81 * 128;
                const uint32_t o0 = pc0 * (kTcR * 2) + m80 * 16, o1 = pc1 * (kTcR * 2) + m81 * 16;
                for (int kj = warp; kj < Kp; kj += kProdWarps) {
                  const unsigned char* row =
                      reinterpret_cast<const unsigned char*>(__shfl_sync(0xffffffffu, reinterpret_cast<uintptr_t>(myrow), kj));
                  const uint32_t ok_src = __shfl_sync(0xffffffffu, valid ? 16u : 0u, kj);
                  const uint32_t kofs = (uint32_t)((kj >> 3) * 2048 + (kj & 7) * 16);
                  cp_async16(d0 + kofs, row + o0, ok_src);
                  if (lane < 16) cp_async16(d1 + kofs, row + o1, ok_src);
                }
              }
              cp_async_arrive(&ctl->full[s]);
            }
            ++tiles_here;
          }
        }
        tiles_before += tiles_here;
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      long jm = 0, tm = 0;
      bool ok = true;
      for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
        const Item itm = item_of(p, it, G, single, msingle);
        const Unit u = p.units[itm.am];
        for (int k = 0; k < u.nphase && ok; ++k) {
          const int ph = fwd ? k : u.nphase - 1 - k;
          for (int oi = p.phase_tab[u.ph_begin + ph]; oi < p.phase_tab[u.ph_begin + ph + 1] && ok; ++oi) {
            const Op op = p.ops[oi];
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
              for (int c = 0; c < sh.nK && ok; ++c, ++jm) {
                const int s = (int)(jm % kStages);
                const uint32_t use = (uint32_t)(jm / kStages);
                ok = mbar_wait(ctl, &ctl->full[s], use & 1u);
                if (!ok) break;
                // the stage was written by cp.async (generic proxy); the MMAs read it
                // through the async proxy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int Kp = (min(kTcKC, sh.KK - kTcKC * c) + 15) & ~15;
                const uint32_t sA = stage0 + (uint32_t)s * kStageBytes, sB = sA + kStageA;
                const uint32_t bPiece = (uint32_t)Np * Kp * 2, bK = (uint32_t)(Np / 8) * 128;
                for (int ks = 0; ks < Kp / 16; ++ks) {
                  int lo = 0;
#pragma unroll
                  for (int pa = 0; pa < 3; ++pa)
#pragma unroll
                    for (int pb = 0; pb < 3; ++pb) {
                      if (pa + pb > 2) continue;
                      // A MN-major: cores (k8, m8) at (k8 * 16 + m8) * 128 B: K stride 2048, M stride 128
                      const uint64_t ad = sdesc(sA + pa * kPieceA + ks * 2 * 2048, 2048, 128);
                      const uint64_t bd = sdesc(sB + pb * bPiece + ks * 2 * bK, bK, 128);
                      if (pa + pb == 0) {
                        mma_bf16(dhi, ad, bd, idesc, (c > 0 || ks > 0) ? 1u : 0u);
                      } else {
                        mma_bf16(dlo, ad, bd, idesc, (c > 0 || ks > 0 || lo > 0) ? 1u : 0u);
                        ++lo;
                      }
                    }
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
  } else if (warp < kIoWarp0) {
    // accumulators -> rows: warp ew owns TMEM lane quadrant ew (right-hand sides 32 ew ..)
    const int ew = warp - kEpiWarp0;
    const int e = tid - 32 * kEpiWarp0;
    float* T = trbuf + (size_t)ew * 32 * kTrStride;
    long te = 0;
    int done = 0;
    bool ok = true;
    for (int it = blockIdx.x, iseq = 0; it < nitems && ok; it += gridDim.x, ++iseq) {
      const Item itm = item_of(p, it, G, single, msingle);
      const Unit u = p.units[itm.am];
      unsigned char* vec = slots + (size_t)(iseq & 1) * slot_bytes;
      for (int k = 0; k < u.nphase && ok; ++k) {
        const int ph = fwd ? k : u.nphase - 1 - k;
        for (int oi = p.phase_tab[u.ph_begin + ph]; oi < p.phase_tab[u.ph_begin + ph + 1] && ok; ++oi) {
          const Op op = p.ops[oi];
          const OpShape sh = op_shape(op, fwd);
          const int32_t* ooff = fwd ? op.out_off : op.in_off;
          const int32_t* olen = fwd ? op.out_len : op.in_len;
          const bool accum = (op.flags & (fwd ? OP_FWD_ACCUM : OP_BWD_ACCUM)) != 0;
          for (int t = 0; t < sh.nT && ok; ++t, ++te) {
            const int b = (int)(te & 1);
            const uint32_t v = (uint32_t)(te >> 1);
            ok = mbar_wait(ctl, &ctl->accf[b], v & 1u);
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
                    unsigned char* row = vec + (size_t)seg_row(kTcNT * t + i, ooff, olen) * kTcRowBytes;
                    const int c8 = 32 * ew + 8 * oc;
                    if (accum) {
                      float* dst = fp32_at(row, c8);
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
                        __stcg(reinterpret_cast<uint4*>(row + pc * (kTcR * 2) + c8 * 2),
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
            __threadfence_block();
            epi_bar();
            ++done;
            if (e == 0) *((volatile int*)&ctl->done_tiles) = done;
          }
        }
      }
    }
  } else if (warp >= kIoWarp0) {
    // I/O warps: gather of item i into slot i % 2 (after the fold of item i-2 from that
    // slot), parity fold / scatter of item i once its tiles are done
    const int e = tid - 32 * kIoWarp0;  // 0..255
    const int col = e & 127, half = e >> 7;  // column (right-hand side); row half
    const int fl = col >> 2, sg = (col >> 1) & 1, cc = col & 1;
    int tiles_through = 0;
    bool ok = true;
    int prev_it = -1, prev_iseq = -1;
    for (int it = blockIdx.x, iseq = 0; ok; it += gridDim.x, ++iseq) {
      const bool have = it < nitems;
      // 1. gather item `it` into slot iseq % 2 (its previous user, item iseq-2, is folded)
      if (have) {
        const Item itm = item_of(p, it, G, single, msingle);
        const int am = itm.am, grp = itm.grp;
        const Unit u = p.units[am];
        unsigned char* vec = slots + (size_t)(iseq & 1) * slot_bytes;
        const int nx = u.nce + u.nco;
        if (fwd) {
          const double* bsrc = coef_base(in, N, am, grp * kTcFields + fl, sg, F, single, msingle);
          for (int t0 = 16 * half; t0 < nx; t0 += 32) {
            float v[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              const int t = t0 + q;
              v[q] = (bsrc && t < nx) ? (float)__ldg(bsrc + 2 * row_kk(u, t) + cc) : 0.f;
            }
#pragma unroll
            for (int q = 0; q < 16; ++q)
              if (t0 + q < nx) put_pieces(vec + (size_t)(t0 + q) * kTcRowBytes, col, v[q]);
          }
          for (int i = half; i < 2 * N; i += 2) __stcg(fp32_at(vec + (size_t)(u.ye + i) * kTcRowBytes, col), 0.f);
        } else {
          const double* gb = value_base(in, N, am, grp * kTcFields + fl, sg, F, single, msingle);
          for (int i0 = 8 * half; i0 < N; i0 += 16) {
            double a[8], b[8], wi[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int i = i0 + q;
              const bool in_range = gb && i < N;
              a[q] = in_range ? __ldg(gb + 2 * (N + i) + cc) : 0.0;
              b[q] = in_range ? __ldg(gb + 2 * (N - 1 - i) + cc) : 0.0;
              wi[q] = i < N ? __ldg(p.w + N + i) : 0.0;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int i = i0 + q;
              if (i < N) {
                put_pieces(vec + (size_t)(u.ye + i) * kTcRowBytes, col, (float)(wi[q] * (a[q] + b[q])));
                put_pieces(vec + (size_t)(u.yo + i) * kTcRowBytes, col, (float)(wi[q] * (a[q] - b[q])));
              }
            }
          }
          for (int t = half; t < nx; t += 2) __stcg(fp32_at(vec + (size_t)t * kTcRowBytes, col), 0.f);
        }
        __threadfence_block();
        io_bar();
        if (e == 0) *((volatile int*)&ctl->gathered) = iseq + 1;
      }
      // 2. fold / scatter the previous item once all of its tiles are done
      if (prev_it >= 0) {
        const Item itm = item_of(p, prev_it, G, single, msingle);
        const int am = itm.am, grp = itm.grp;
        const Unit u = p.units[am];
        unsigned char* vec = slots + (size_t)(prev_iseq & 1) * slot_bytes;
        tiles_through += item_tiles(p, u, fwd != 0);
        ok = counter_wait(ctl, &ctl->done_tiles, tiles_through);
        if (!ok) break;
        const int nx = u.nce + u.nco;
        if (fwd) {
          const int total = N * 2 * kTcFields;
          for (int idx0 = e; idx0 < total; idx0 += 256 * 8) {
            float2 ev[8], ov[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int idx = idx0 + 256 * q;
              ev[q] = make_float2(0.f, 0.f);
              ov[q] = make_float2(0.f, 0.f);
              if (idx < total) {
                const int i = idx % N, fs = idx / N, cl = 4 * (fs >> 1) + 2 * (fs & 1);
                ev[q] = __ldcg(reinterpret_cast<const float2*>(fp32_at(vec + (size_t)(u.ye + i) * kTcRowBytes, cl)));
                ov[q] = __ldcg(reinterpret_cast<const float2*>(fp32_at(vec + (size_t)(u.yo + i) * kTcRowBytes, cl)));
              }
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int idx = idx0 + 256 * q;
              if (idx >= total) continue;
              const int i = idx % N, fs = idx / N;
              const double* gb = value_base(out, N, am, grp * kTcFields + (fs >> 1), fs & 1, F, single, msingle);
              if (!gb) continue;
              double2* gp = reinterpret_cast<double2*>(const_cast<double*>(gb));
              gp[N + i] = make_double2((double)ev[q].x + (double)ov[q].x, (double)ev[q].y + (double)ov[q].y);
              gp[N - 1 - i] = make_double2((double)ev[q].x - (double)ov[q].x, (double)ev[q].y - (double)ov[q].y);
            }
          }
        } else {
          const double* bdst = coef_base(out, N, am, grp * kTcFields + fl, sg, F, single, msingle);
          if (bdst)
            for (int t0 = 16 * half; t0 < nx; t0 += 32) {
              float v[16];
#pragma unroll
              for (int q = 0; q < 16; ++q)
                v[q] = t0 + q < nx ? __ldcg(fp32_at(vec + (size_t)(t0 + q) * kTcRowBytes, col)) : 0.f;
#pragma unroll
              for (int q = 0; q < 16; ++q) {
                const int t = t0 + q;
                if (t < nx) const_cast<double*>(bdst)[2 * row_kk(u, t) + cc] = (double)v[q];
              }
            }
        }
        __threadfence_block();
        io_bar();
      }
      if (!have) break;
      prev_it = it;
      prev_iseq = iseq;
    }
  }
  if (*((volatile int*)&ctl->abort) && tid == 0) atomicExch(p.err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kMmaWarp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTmemCols) : "memory");
}

}  // namespace

size_t tc_smem_bytes() { return kSmemTotal; }

int tc_ctas_per_sm() { return 1; }  // the kernel holds all 512 tensor-memory columns

cudaError_t launch_tc(const TcPlan& p, bool fwd, const double* in, double* out, int F, int single, int m, int grid,
                      cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(alt_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTotal);
  if (e != cudaSuccess) return e;
  alt_tc_kernel<<<grid, kTcThreads, kSmemTotal, st>>>(p, in, out, F, single, m, fwd ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace sht
