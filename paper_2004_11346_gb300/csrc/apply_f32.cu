// Many-field apply of the IDBF-factored ALT in FP32 arithmetic (sm_103a).
//
// Same apply program as the FP64 path (program.hpp), but one work item is one
// order |m| for a group of 8 fields: 32 real right-hand sides (Re/Im of +m
// and -m per field), one per warp lane.  Each block product runs as a warp:
// the lanes walk the columns of B together, every lane multiplying the same
// (broadcast) B entries into its own right-hand side, 16 output rows at a
// time in registers.  Factors are the FP32 copy of the plan's store; inputs
// and outputs stay FP64 (converted in the gather and the fold).  Items are
// ordered order-major, group-minor, so the groups of one order run side by
// side and share its factor blocks through L2.
#include <cuda_runtime.h>

#include "apply_f32.cuh"

namespace sht {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int RT = kF32RT;   // 32
constexpr int TI = 16;       // output rows per register tile (forward)
constexpr int TJ = 8;        // output columns per register tile (transposed)

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
__device__ __forceinline__ int next_item(unsigned int* counter) {
  __shared__ int s_item;
  __syncthreads();
  if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
  __syncthreads();
  return s_item;
}

// y[out rows] (+)= B x[in rows], lane = right-hand side.
__device__ void ops_forward(const F32Plan& p, int begin, int end, float* vec) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int oi = begin + warp; oi < end; oi += kWarps) {
    const Op op = p.ops[oi];
    const float* B = p.fac + op.b_off;
    for (int i0 = 0; i0 < op.mo; i0 += TI) {
      const int nq = min(TI / 4, (op.ld - i0) >> 2);  // float4 chunks of this tile inside the column
      float acc[TI];
#pragma unroll
      for (int t = 0; t < TI; ++t) acc[t] = 0.f;
      if (nq == TI / 4) {
        for (int j = 0; j < op.ni; ++j) {
          const float xv = __ldcg(vec + (size_t)seg_row(j, op.in_off, op.in_len) * RT + lane);
          const float4* bc = reinterpret_cast<const float4*>(B + (size_t)j * op.ld + i0);
#pragma unroll
          for (int q = 0; q < TI / 4; ++q) {
            const float4 b = __ldg(bc + q);
            acc[4 * q + 0] = fmaf(b.x, xv, acc[4 * q + 0]);
            acc[4 * q + 1] = fmaf(b.y, xv, acc[4 * q + 1]);
            acc[4 * q + 2] = fmaf(b.z, xv, acc[4 * q + 2]);
            acc[4 * q + 3] = fmaf(b.w, xv, acc[4 * q + 3]);
          }
        }
      } else {
        for (int j = 0; j < op.ni; ++j) {
          const float xv = __ldcg(vec + (size_t)seg_row(j, op.in_off, op.in_len) * RT + lane);
          const float4* bc = reinterpret_cast<const float4*>(B + (size_t)j * op.ld + i0);
#pragma unroll
          for (int q = 0; q < TI / 4; ++q) {
            if (q < nq) {
              const float4 b = __ldg(bc + q);
              acc[4 * q + 0] = fmaf(b.x, xv, acc[4 * q + 0]);
              acc[4 * q + 1] = fmaf(b.y, xv, acc[4 * q + 1]);
              acc[4 * q + 2] = fmaf(b.z, xv, acc[4 * q + 2]);
              acc[4 * q + 3] = fmaf(b.w, xv, acc[4 * q + 3]);
            }
          }
        }
      }
      const bool accum = (op.flags & OP_FWD_ACCUM) != 0;
#pragma unroll
      for (int t = 0; t < TI; ++t) {
        const int i = i0 + t;
        if (i < op.mo) {
          float* y = vec + (size_t)seg_row(i, op.out_off, op.out_len) * RT + lane;
          if (accum) atomicAdd(y, acc[t]);
          else __stcg(y, acc[t]);
        }
      }
    }
  }
}

// x[in rows] (+)= B^T y[out rows], lane = right-hand side.
__device__ void ops_transpose(const F32Plan& p, int begin, int end, float* vec) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int oi = begin + warp; oi < end; oi += kWarps) {
    const Op op = p.ops[oi];
    const float* B = p.fac + op.b_off;
    for (int j0 = 0; j0 < op.ni; j0 += TJ) {
      const int nj = min(TJ, op.ni - j0);
      float acc[TJ];
#pragma unroll
      for (int t = 0; t < TJ; ++t) acc[t] = 0.f;
      for (int i = 0; i < op.mo; i += 4) {  // rows i..i+3 lie inside the column (ld % 4 == 0)
        float y[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          y[q] = (i + q < op.mo) ? __ldcg(vec + (size_t)seg_row(i + q, op.out_off, op.out_len) * RT + lane) : 0.f;
#pragma unroll
        for (int t = 0; t < TJ; ++t) {
          if (t < nj) {
            const float4 b = __ldg(reinterpret_cast<const float4*>(B + (size_t)(j0 + t) * op.ld + i));
            acc[t] = fmaf(b.x, y[0], fmaf(b.y, y[1], fmaf(b.z, y[2], fmaf(b.w, y[3], acc[t]))));
          }
        }
      }
      const bool accum = (op.flags & OP_BWD_ACCUM) != 0;
#pragma unroll
      for (int t = 0; t < TJ; ++t) {
        if (t < nj) {
          float* x = vec + (size_t)seg_row(j0 + t, op.in_off, op.in_len) * RT + lane;
          if (accum) atomicAdd(x, acc[t]);
          else __stcg(x, acc[t]);
        }
      }
    }
  }
}

struct ItemCtx {
  int am, grp;
};

// Coefficient array of field f and sign s (0: +m, 1: -m), or nullptr.
__device__ __forceinline__ const double* coef_base(const double* beta, int N, int am, int f, int s, int F,
                                                   int single, int msingle) {
  if (f >= F || (s == 1 && am == 0)) return nullptr;
  const int K = 2 * N;
  if (single) {
    const int m = s == 0 ? am : -am;
    if (m != msingle) return nullptr;
    return beta + 2L * f * (K - am);
  }
  return beta + 2 * ((long)f * 4L * N * N + coef_offset(N, s == 0 ? am : -am));
}

__device__ __forceinline__ const double* value_base(const double* g, int N, int am, int f, int s, int F, int single,
                                                    int msingle) {
  if (f >= F || (s == 1 && am == 0)) return nullptr;
  const int K = 2 * N;
  if (single) {
    const int m = s == 0 ? am : -am;
    if (m != msingle) return nullptr;
    return g + 2L * f * K;
  }
  return g + 2 * ((long)f * (4L * N - 1) * K + order_slot(s == 0 ? am : -am) * K);
}

__global__ void __launch_bounds__(kThreads) alt_forward_f32_kernel(F32Plan p, const double* __restrict__ beta,
                                                                   double* __restrict__ g, int F, int single,
                                                                   int msingle) {
  const int N = p.N;
  const int G = (F + kF32Fields - 1) / kF32Fields;
  float* vec = p.ws + (size_t)blockIdx.x * p.max_rows * RT;
  const int nitems = single ? G : p.nunits * G;
  for (;;) {
    const int item = next_item(p.counter);
    if (item >= nitems) break;
    const int grp = item % G;
    const int am = single ? (msingle < 0 ? -msingle : msingle) : p.order[item / G];
    const Unit u = p.units[am];
    const int nx = u.nce + u.nco;
    // gather: X row t, column 4 fl + 2 s + c
    for (int idx = threadIdx.x; idx < nx * RT; idx += kThreads) {
      const int t = idx / RT, col = idx % RT;
      const int fl = col >> 2, s = (col >> 1) & 1, c = col & 1;
      const double* b = coef_base(beta, N, am, grp * kF32Fields + fl, s, F, single, msingle);
      const int kk = t < u.nce ? 2 * t : 2 * (t - u.nce) + 1;
      __stcg(vec + (size_t)t * RT + col, b ? (float)__ldg(b + 2 * kk + c) : 0.f);
    }
    for (int idx = threadIdx.x; idx < 2 * N * RT; idx += kThreads) __stcg(vec + (size_t)u.ye * RT + idx, 0.f);
    __syncthreads();
    for (int ph = 0; ph < u.nphase; ++ph) {
      ops_forward(p, p.phase_tab[u.ph_begin + ph], p.phase_tab[u.ph_begin + ph + 1], vec);
      __syncthreads();
    }
    // parity fold
    for (int idx = threadIdx.x; idx < N * 2 * kF32Fields; idx += kThreads) {
      const int i = idx % N, fs = idx / N, fl = fs >> 1, s = fs & 1;
      const double* gb = value_base(g, N, am, grp * kF32Fields + fl, s, F, single, msingle);
      if (!gb) continue;
      const int col = 4 * fl + 2 * s;
      const float er = __ldcg(vec + (size_t)(u.ye + i) * RT + col), ei = __ldcg(vec + (size_t)(u.ye + i) * RT + col + 1);
      const float orr = __ldcg(vec + (size_t)(u.yo + i) * RT + col), oi = __ldcg(vec + (size_t)(u.yo + i) * RT + col + 1);
      double2* gp = reinterpret_cast<double2*>(const_cast<double*>(gb));
      gp[N + i] = make_double2((double)er + (double)orr, (double)ei + (double)oi);
      gp[N - 1 - i] = make_double2((double)er - (double)orr, (double)ei - (double)oi);
    }
  }
}

__global__ void __launch_bounds__(kThreads) alt_inverse_f32_kernel(F32Plan p, const double* __restrict__ g,
                                                                   double* __restrict__ beta, int F, int single,
                                                                   int msingle) {
  const int N = p.N;
  const int G = (F + kF32Fields - 1) / kF32Fields;
  float* vec = p.ws + (size_t)blockIdx.x * p.max_rows * RT;
  const int nitems = single ? G : p.nunits * G;
  for (;;) {
    const int item = next_item(p.counter);
    if (item >= nitems) break;
    const int grp = item % G;
    const int am = single ? (msingle < 0 ? -msingle : msingle) : p.order[item / G];
    const Unit u = p.units[am];
    const int nx = u.nce + u.nco;
    // W-weighted parity fold of g into Y_e, Y_o
    for (int idx = threadIdx.x; idx < N * 2 * kF32Fields; idx += kThreads) {
      const int i = idx % N, fs = idx / N, fl = fs >> 1, s = fs & 1;
      const double* gb = value_base(g, N, am, grp * kF32Fields + fl, s, F, single, msingle);
      double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
      if (gb) {
        a = __ldg(reinterpret_cast<const double2*>(gb) + N + i);
        b = __ldg(reinterpret_cast<const double2*>(gb) + N - 1 - i);
      }
      const double wi = __ldg(p.w + N + i);
      const int col = 4 * fl + 2 * s;
      float* ye = vec + (size_t)(u.ye + i) * RT + col;
      float* yo = vec + (size_t)(u.yo + i) * RT + col;
      __stcg(ye, (float)(wi * (a.x + b.x)));
      __stcg(ye + 1, (float)(wi * (a.y + b.y)));
      __stcg(yo, (float)(wi * (a.x - b.x)));
      __stcg(yo + 1, (float)(wi * (a.y - b.y)));
    }
    for (int idx = threadIdx.x; idx < nx * RT; idx += kThreads) __stcg(vec + idx, 0.f);
    __syncthreads();
    for (int ph = u.nphase - 1; ph >= 0; --ph) {
      ops_transpose(p, p.phase_tab[u.ph_begin + ph], p.phase_tab[u.ph_begin + ph + 1], vec);
      __syncthreads();
    }
    // scatter X into beta
    for (int idx = threadIdx.x; idx < nx * RT; idx += kThreads) {
      const int t = idx / RT, col = idx % RT;
      const int fl = col >> 2, s = (col >> 1) & 1, c = col & 1;
      const double* b = coef_base(beta, N, am, grp * kF32Fields + fl, s, F, single, msingle);
      if (!b) continue;
      const int kk = t < u.nce ? 2 * t : 2 * (t - u.nce) + 1;
      const_cast<double*>(b)[2 * kk + c] = (double)__ldcg(vec + (size_t)t * RT + col);
    }
  }
}

}  // namespace

cudaError_t launch_f32(const F32Plan& p, bool fwd, const double* in, double* out, int F, int single, int m,
                       int grid, cudaStream_t st) {
  if (fwd)
    alt_forward_f32_kernel<<<grid, kThreads, 0, st>>>(p, in, out, F, single, m);
  else
    alt_inverse_f32_kernel<<<grid, kThreads, 0, st>>>(p, in, out, F, single, m);
  return cudaGetLastError();
}

int f32_ctas_per_sm() {
  int a = 0, b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, alt_forward_f32_kernel, kThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, alt_inverse_f32_kernel, kThreads, 0);
  int r = a < b ? a : b;
  return r < 1 ? 1 : r;
}

}  // namespace sht
