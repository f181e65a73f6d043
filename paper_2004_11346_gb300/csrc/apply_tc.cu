// Many-field apply of the IDBF-factored ALT on the 5th-generation tensor
// cores (tcgen05, sm_103a), split-BF16 products with FP32 accumulation.
//
// One work item is one order |m| for 32 fields: 128 real right-hand sides.
// Every block product of the apply program, out (+)= B in, is computed
// transposed, out^T = in^T B^T, so that the 128 right-hand sides fill the MMA
// M dimension and the block's rows are N (tiles of <= 128, padded to 16):
//   A operand = in^T (128 x K): staged from the FP32 vector rows, each value
//               split into three BF16 pieces a0 + a1 + a2 (8 bits each);
//   B operand = B (N x K, K-major): precomputed split-BF16 image b0 + b1 + b2;
//   D         = 128 x N FP32 accumulator in tensor memory.
// Per 16-wide K step six MMAs accumulate a_p b_q for p + q <= 2, which keeps
// every product to about 2^-24 relative error (FP32 quality); a0 b0 and the
// five smaller cross products go to two separate accumulators that the
// epilogue adds in FP32.  Operands sit
// in shared memory in the canonical no-swizzle K-major layout (8 x 16-byte
// core matrices; LBO = stride between core matrices along K, SBO = along M/N).
// One thread issues the MMAs and commits them to an mbarrier; all waits are
// bounded and report an error status instead of hanging.  The epilogue reads
// D with tcgen05.ld (warp w owns right-hand sides 32w..32w+31), so every
// output row is written by 32 lanes as one coalesced 128-byte segment.
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

constexpr int kPieceA = kTcR * kTcKC;    // elements per A piece (16 KB)
constexpr int kPieceB = kTcNT * kTcKC;   // elements per B piece, largest
constexpr size_t kSmemA = 3 * kPieceA * 2;
constexpr size_t kSmemB = 3 * kPieceB * 2;
constexpr size_t kSmemTotal = kSmemA + kSmemB + 1024 /*alignment*/ + 64;
constexpr long kWaitLimit = 1L << 24;
constexpr int kTmemCols = 2 * kTcNT;     // hi and lo accumulators, 128 x 128 FP32 each

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

__device__ __forceinline__ void tmem_ld32(uint32_t addr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Bounded wait for mbarrier phase `parity`; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long it = 0; it < kWaitLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(s32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

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

__device__ __forceinline__ uint16_t f2bf(float f) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(f));
}
__device__ __forceinline__ float bf2f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

struct Smem {
  uint16_t* A;
  uint16_t* B;
  uint64_t* bar;
  uint32_t* taddr;
  int* flag;
};

// One block product, transposed onto the tensor cores.  Returns false when a
// wait gave up (the caller stops).
__device__ bool tc_op(const TcPlan& p, const Smem& sm, uint32_t taddr, uint32_t& phase, const Op& op, bool fwd,
                      const uint16_t* img, float* vec) {
  const int tid = threadIdx.x, warp = tid >> 5;
  const int NN = fwd ? op.mo : op.ni, KK = fwd ? op.ni : op.mo;
  const int32_t* ooff = fwd ? op.out_off : op.in_off;
  const int32_t* olen = fwd ? op.out_len : op.in_len;
  const bool accum = (op.flags & (fwd ? OP_FWD_ACCUM : OP_BWD_ACCUM)) != 0;
  if (KK == 0) {  // empty product: the outputs are zero
    if (!accum)
      for (int i = 0; i < NN; ++i) __stcg(vec + (size_t)seg_row(i, ooff, olen) * kTcR + tid, 0.f);
    return true;
  }
  const int32_t* ioff = fwd ? op.in_off : op.out_off;
  const int32_t* ilen = fwd ? op.in_len : op.out_len;
  const int nT = (NN + kTcNT - 1) / kTcNT, nK = (KK + kTcKC - 1) / kTcKC;
  const int kp_tot = kTcKC * (nK - 1) + ((KK - kTcKC * (nK - 1) + 15) & ~15);
  const uint32_t aBase = s32(sm.A), bBase = s32(sm.B);
  for (int t = 0; t < nT; ++t) {
    const int Nt = min(kTcNT, NN - kTcNT * t), Np = (Nt + 15) & ~15;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(Np >> 3) << 17) | (8u << 24);
    for (int c = 0; c < nK; ++c) {
      const int Kc = min(kTcKC, KK - kTcKC * c), Kp = (Kc + 15) & ~15;
      // stage B first (asynchronous 16-byte copies of the contiguous image chunk)
      {
        const uint16_t* src = img + (size_t)t * 384 * kp_tot + (size_t)Np * (192 * c);
        const int n16 = 3 * Np * Kp / 8;
        const uint32_t dB = bBase;
        for (int q = tid; q < n16; q += kTcThreads)
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dB + 16u * q), "l"(src + 8 * q)
                       : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
      }
      // stage A = in^T: thread owns right-hand side r = tid; all of its K values
      // of the chunk are loaded before any is used, so the loads overlap
      {
        float xv[kTcKC];
#pragma unroll
        for (int kk = 0; kk < kTcKC; ++kk) {
          const int j = kTcKC * c + kk;
          xv[kk] = (kk < Kp && j < KK) ? __ldcg(vec + (size_t)seg_row(j, ioff, ilen) * kTcR + tid) : 0.f;
        }
#pragma unroll
        for (int k8 = 0; k8 < kTcKC / 8; ++k8) {
          if (k8 < Kp / 8) {
            uint32_t h[3][4];
#pragma unroll
            for (int kk = 0; kk < 8; kk += 2) {
              uint16_t q0[2], q1[2], q2[2];
#pragma unroll
              for (int e = 0; e < 2; ++e) {
                float v = xv[8 * k8 + kk + e];
                q0[e] = f2bf(v);
                v -= bf2f(q0[e]);
                q1[e] = f2bf(v);
                v -= bf2f(q1[e]);
                q2[e] = f2bf(v);
              }
              h[0][kk / 2] = (uint32_t)q0[0] | ((uint32_t)q0[1] << 16);
              h[1][kk / 2] = (uint32_t)q1[0] | ((uint32_t)q1[1] << 16);
              h[2][kk / 2] = (uint32_t)q2[0] | ((uint32_t)q2[1] << 16);
            }
            const int o = ((k8 * (kTcR / 8) + (tid >> 3)) * 64 + (tid & 7) * 8);
#pragma unroll
            for (int pc = 0; pc < 3; ++pc)
              *reinterpret_cast<uint4*>(sm.A + pc * kPieceA + o) =
                  make_uint4(h[pc][0], h[pc][1], h[pc][2], h[pc][3]);
          }
        }
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t bPiece = (uint32_t)Np * Kp * 2;
        const uint32_t bK = (uint32_t)(Np / 8) * 128;
        for (int s = 0; s < Kp / 16; ++s) {
          // a0 b0 into the "hi" accumulator, the five small cross products
          // (p + q = 1, 2) into the "lo" accumulator: the lo sum is ~2^-8 of
          // the hi sum, so its accumulation rounding stays negligible
          int lo = 0;
#pragma unroll
          for (int pa = 0; pa < 3; ++pa)
#pragma unroll
            for (int pb = 0; pb < 3; ++pb) {
              if (pa + pb > 2) continue;
              const uint64_t ad = sdesc(aBase + pa * (kPieceA * 2) + s * 2 * 2048, 2048, 128);
              const uint64_t bd = sdesc(bBase + pb * bPiece + s * 2 * bK, bK, 128);
              if (pa + pb == 0) {
                mma_bf16(taddr, ad, bd, idesc, (c > 0 || s > 0) ? 1u : 0u);
              } else {
                mma_bf16(taddr + kTcNT, ad, bd, idesc, (c > 0 || s > 0 || lo > 0) ? 1u : 0u);
                ++lo;
              }
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         s32(sm.bar))
                     : "memory");
      }
      const bool ok = mbar_wait(sm.bar, phase);
      phase ^= 1u;
      if (!ok) *sm.flag = 1;
      __syncthreads();
      if (*sm.flag) return false;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: D[r][n] -> out row n, right-hand side r = 32 warp + lane
    for (int c0 = 0; c0 < Nt; c0 += 32) {
      uint32_t v[32], w[32];
      tmem_ld32(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
      tmem_ld32(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)(kTcNT + c0), w);
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int i = c0 + q;
        if (i < Nt) {
          float* dst = vec + (size_t)seg_row(kTcNT * t + i, ooff, olen) * kTcR + tid;
          const float val = __uint_as_float(v[q]) + __uint_as_float(w[q]);
          if (accum) atomicAdd(dst, val);
          else __stcg(dst, val);
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  return true;
}

__device__ __forceinline__ int next_item(unsigned int* counter, int* s_item) {
  __syncthreads();
  if (threadIdx.x == 0) *s_item = (int)atomicAdd(counter, 1u);
  __syncthreads();
  return *s_item;
}

__global__ void __launch_bounds__(kTcThreads, 1) alt_tc_kernel(TcPlan p, const double* __restrict__ in,
                                                               double* __restrict__ out, int F, int single,
                                                               int msingle, int fwd) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  Smem sm;
  sm.A = reinterpret_cast<uint16_t*>(base);
  sm.B = reinterpret_cast<uint16_t*>(base + kSmemA);
  sm.bar = reinterpret_cast<uint64_t*>(base + kSmemA + kSmemB);
  sm.taddr = reinterpret_cast<uint32_t*>(base + kSmemA + kSmemB + 8);
  sm.flag = reinterpret_cast<int*>(base + kSmemA + kSmemB + 16);
  int* s_item = reinterpret_cast<int*>(base + kSmemA + kSmemB + 24);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s32(sm.taddr)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s32(sm.bar)), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *sm.flag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = *sm.taddr;
  uint32_t phase = 0;

  const int N = p.N;
  const int G = (F + kTcFields - 1) / kTcFields;
  float* vec = p.ws + (size_t)blockIdx.x * p.max_rows * kTcR;
  const int nitems = single ? G : p.nunits * G;
  bool alive = true;
  while (alive) {
    const int item = next_item(p.counter, s_item);
    if (item >= nitems) break;
    const int grp = item % G;
    const int am = single ? (msingle < 0 ? -msingle : msingle) : p.order[item / G];
    const Unit u = p.units[am];
    const int nx = u.nce + u.nco;
    if (fwd) {
      // gather X: row t, column 4 fl + 2 s + c; zero Y
      {
        // column tid of every X row: field fl, sign s, Re/Im cc are fixed per thread
        const int fl = tid >> 2, s = (tid >> 1) & 1, cc = tid & 1;
        const double* b = coef_base(in, N, am, grp * kTcFields + fl, s, F, single, msingle);
        for (int t0 = 0; t0 < nx; t0 += 8) {
          float v[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int t = t0 + e;
            const int kk = t < u.nce ? 2 * t : 2 * (t - u.nce) + 1;
            v[e] = (b && t < nx) ? (float)__ldg(b + 2 * kk + cc) : 0.f;
          }
#pragma unroll
          for (int e = 0; e < 8; ++e)
            if (t0 + e < nx) __stcg(vec + (size_t)(t0 + e) * kTcR + tid, v[e]);
        }
      }
      for (int idx = tid; idx < 2 * N * kTcR; idx += kTcThreads) __stcg(vec + (size_t)u.ye * kTcR + idx, 0.f);
    } else {
      for (int idx = tid; idx < N * 2 * kTcFields; idx += kTcThreads) {
        const int i = idx % N, fs = idx / N, fl = fs >> 1, s = fs & 1;
        const double* gb = value_base(in, N, am, grp * kTcFields + fl, s, F, single, msingle);
        double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
        if (gb) {
          a = __ldg(reinterpret_cast<const double2*>(gb) + N + i);
          b = __ldg(reinterpret_cast<const double2*>(gb) + N - 1 - i);
        }
        const double wi = __ldg(p.w + N + i);
        const int col = 4 * fl + 2 * s;
        float* ye = vec + (size_t)(u.ye + i) * kTcR + col;
        float* yo = vec + (size_t)(u.yo + i) * kTcR + col;
        __stcg(ye, (float)(wi * (a.x + b.x)));
        __stcg(ye + 1, (float)(wi * (a.y + b.y)));
        __stcg(yo, (float)(wi * (a.x - b.x)));
        __stcg(yo + 1, (float)(wi * (a.y - b.y)));
      }
      for (int idx = tid; idx < nx * kTcR; idx += kTcThreads) __stcg(vec + idx, 0.f);
    }
    __syncthreads();
    for (int k = 0; k < u.nphase && alive; ++k) {
      const int ph = fwd ? k : u.nphase - 1 - k;
      for (int oi = p.phase_tab[u.ph_begin + ph]; oi < p.phase_tab[u.ph_begin + ph + 1]; ++oi) {
        const Op op = p.ops[oi];
        if (!tc_op(p, sm, taddr, phase, op, fwd != 0, p.img + p.img_off[2 * oi + (fwd ? 0 : 1)], vec)) {
          alive = false;
          break;
        }
      }
      __syncthreads();
    }
    if (!alive) break;
    if (fwd) {
      for (int idx = tid; idx < N * 2 * kTcFields; idx += kTcThreads) {
        const int i = idx % N, fs = idx / N, fl = fs >> 1, s = fs & 1;
        const double* gb = value_base(out, N, am, grp * kTcFields + fl, s, F, single, msingle);
        if (!gb) continue;
        const int col = 4 * fl + 2 * s;
        const float er = __ldcg(vec + (size_t)(u.ye + i) * kTcR + col);
        const float ei = __ldcg(vec + (size_t)(u.ye + i) * kTcR + col + 1);
        const float orr = __ldcg(vec + (size_t)(u.yo + i) * kTcR + col);
        const float oi = __ldcg(vec + (size_t)(u.yo + i) * kTcR + col + 1);
        double2* gp = reinterpret_cast<double2*>(const_cast<double*>(gb));
        gp[N + i] = make_double2((double)er + (double)orr, (double)ei + (double)oi);
        gp[N - 1 - i] = make_double2((double)er - (double)orr, (double)ei - (double)oi);
      }
    } else {
      for (int idx = tid; idx < nx * kTcR; idx += kTcThreads) {
        const int t = idx / kTcR, col = idx % kTcR;
        const int fl = col >> 2, s = (col >> 1) & 1, cc = col & 1;
        const double* b = coef_base(out, N, am, grp * kTcFields + fl, s, F, single, msingle);
        if (!b) continue;
        const int kk = t < u.nce ? 2 * t : 2 * (t - u.nce) + 1;
        const_cast<double*>(b)[2 * kk + cc] = (double)__ldcg(vec + (size_t)t * kTcR + col);
      }
    }
  }
  if (!alive && tid == 0) atomicExch(p.err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTmemCols) : "memory");
}

}  // namespace

size_t tc_smem_bytes() { return kSmemTotal; }

int tc_ctas_per_sm() {
  // resident CTAs per SM from the three limits: shared memory (with the
  // driver's 1 KB per CTA), registers, and the 512 tensor-memory columns
  int dev = 0, smem_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaFuncAttributes fa;
  int regs = 255;
  if (cudaFuncGetAttributes(&fa, alt_tc_kernel) == cudaSuccess) regs = fa.numRegs;
  const int by_smem = (int)(smem_sm / (kSmemTotal + 1024));
  const int by_regs = 65536 / (((regs + 7) & ~7) * kTcThreads);
  const int by_tmem = 512 / kTmemCols;
  return std::max(1, std::min(std::min(by_smem, by_regs), by_tmem));
}

cudaError_t launch_tc(const TcPlan& p, bool fwd, const double* in, double* out, int F, int single, int m, int grid,
                      cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(alt_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTotal);
  if (e != cudaSuccess) return e;
  alt_tc_kernel<<<grid, kTcThreads, kSmemTotal, st>>>(p, in, out, F, single, m, fwd ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace sht
