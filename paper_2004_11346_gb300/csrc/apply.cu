// CUDA apply of the IDBF-factored associated Legendre transform (sm_103a).
//
// One work item = one order |m| (both parity matrices of Sec. 3.1.2) for one
// field.  A CTA takes items from an atomic counter in decreasing-cost order
// (the program's schedule), and for each item:
//   1. gathers beta_{k,+m}, beta_{k,-m} into the even/odd input rows X_e, X_o
//      (4 real right-hand sides: Re/Im of +m and -m share Pbar^{|m|});
//   2. runs the item's dense block products phase by phase (Sec. 3.3: IDBF
//      levels, low-rank factors, trimmed turning-point blocks), one warp per
//      product, each lane owning output rows;
//   3. folds the parity outputs into g at all 2N nodes (Sec. 3.1.2):
//      g(theta_{N+i}) = g_e + g_o, g(theta_{N-1-i}) = g_e - g_o.
// The inverse runs the transposed products in reverse phase order after the
// W-weighted fold (Sec. 3.1.1, B = A^T W) and scatters X back into beta.
#include <cuda_runtime.h>
#include <omp.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <string>

#include "alt_direct.cuh"
#include "dense.hpp"
#include "apply_f32.cuh"
#include "apply_tc.cuh"
#include "f64_bits.cuh"
#include "phi_dft.cuh"
#include "plan.hpp"

using namespace sht;

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRT = 4;  // real right-hand sides per item: Re/Im of +m and -m

struct DevPlan {
  const Unit* units;
  const Op* ops;
  const int32_t* phase_tab;
  const int32_t* order;
  const double* fac;
  const double* w;  // all 2N weights
  double* ws;       // per-CTA scratch: max_rows x kRT doubles each
  unsigned int* counter;
  int N;
  int nunits;
  int max_rows;
};

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

// Fetch the next work item (item index in schedule order) for this CTA.
__device__ __forceinline__ int next_item(unsigned int* counter) {
  __shared__ int s_item;
  __syncthreads();
  if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
  __syncthreads();
  return s_item;
}

// Forward products of one phase range: y = B x, warp per op, lane per row.
__device__ void run_ops_forward(const DevPlan& p, const Op* ops, int begin, int end, double* vec) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int oi = begin + warp; oi < end; oi += kWarps) {
    const Op op = ops[oi];
    const double* B = p.fac + op.b_off;
    for (int i0 = 0; i0 < op.mo; i0 += 32) {
      const int i = i0 + lane;
      if (i >= op.mo) break;
      double acc[kRT] = {0.0, 0.0, 0.0, 0.0};
      for (int j = 0; j < op.ni; ++j) {
        const int row = seg_row(j, op.in_off, op.in_len);
        const double b = __ldg(B + (size_t)j * op.ld + i);
        const double2* xr = reinterpret_cast<const double2*>(vec + (size_t)row * kRT);
        const double2 x01 = __ldcg(xr), x23 = __ldcg(xr + 1);
        acc[0] = fma(b, x01.x, acc[0]);
        acc[1] = fma(b, x01.y, acc[1]);
        acc[2] = fma(b, x23.x, acc[2]);
        acc[3] = fma(b, x23.y, acc[3]);
      }
      const int orow = seg_row(i, op.out_off, op.out_len);
      double* yr = vec + (size_t)orow * kRT;
      if (op.flags & OP_FWD_ACCUM) {
#pragma unroll
        for (int r = 0; r < kRT; ++r) atomicAdd(yr + r, acc[r]);
      } else {
        __stcg(reinterpret_cast<double2*>(yr), make_double2(acc[0], acc[1]));
        __stcg(reinterpret_cast<double2*>(yr) + 1, make_double2(acc[2], acc[3]));
      }
    }
  }
}

// Transposed products: x_in = B^T y_out, warp per op, lane per output (column of B).
__device__ void run_ops_transpose(const DevPlan& p, const Op* ops, int begin, int end, double* vec) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int oi = begin + warp; oi < end; oi += kWarps) {
    const Op op = ops[oi];
    const double* B = p.fac + op.b_off;
    for (int j0 = 0; j0 < op.ni; j0 += 32) {
      const int j = j0 + lane;
      if (j >= op.ni) break;
      const double* Bc = B + (size_t)j * op.ld;
      double acc[kRT] = {0.0, 0.0, 0.0, 0.0};
      for (int i = 0; i < op.mo; ++i) {
        const int row = seg_row(i, op.out_off, op.out_len);
        const double b = __ldg(Bc + i);
        const double2* xr = reinterpret_cast<const double2*>(vec + (size_t)row * kRT);
        const double2 x01 = __ldcg(xr), x23 = __ldcg(xr + 1);
        acc[0] = fma(b, x01.x, acc[0]);
        acc[1] = fma(b, x01.y, acc[1]);
        acc[2] = fma(b, x23.x, acc[2]);
        acc[3] = fma(b, x23.y, acc[3]);
      }
      const int orow = seg_row(j, op.in_off, op.in_len);
      double* yr = vec + (size_t)orow * kRT;
      if (op.flags & OP_BWD_ACCUM) {
#pragma unroll
        for (int r = 0; r < kRT; ++r) atomicAdd(yr + r, acc[r]);
      } else {
        __stcg(reinterpret_cast<double2*>(yr), make_double2(acc[0], acc[1]));
        __stcg(reinterpret_cast<double2*>(yr) + 1, make_double2(acc[2], acc[3]));
      }
    }
  }
}

// single != 0: one order `msingle` with compact per-order arrays (F fields of
// 2N-|m| coefficients / 2N values); otherwise all orders, full layouts.
__global__ void __launch_bounds__(kThreads) alt_forward_f64_kernel(DevPlan p, const double* __restrict__ beta,
                                                                   double* __restrict__ g, int F, int single,
                                                                   int msingle) {
  const int N = p.N, K = 2 * N;
  double* vec = p.ws + (size_t)blockIdx.x * p.max_rows * kRT;
  const long ncoef = 4L * N * N, nval = (4L * N - 1) * K;
  const int nitems = single ? F : p.nunits * F;
  for (;;) {
    const int item = next_item(p.counter);
    if (item >= nitems) break;
    const int f = single ? item : item % F;
    const int am = single ? (msingle < 0 ? -msingle : msingle) : p.order[item / F];
    const Unit u = p.units[am];
    // 1. gather
    const double* bp;
    const double* bn;
    if (single) {
      bp = msingle >= 0 ? beta + 2L * f * (K - am) : nullptr;
      bn = msingle < 0 ? beta + 2L * f * (K - am) : nullptr;
    } else {
      bp = beta + 2 * (f * ncoef + coef_offset(N, am));
      bn = am > 0 ? beta + 2 * (f * ncoef + coef_offset(N, -am)) : nullptr;
    }
    for (int t = threadIdx.x; t < u.nce + u.nco; t += kThreads) {
      const int kk = t < u.nce ? 2 * t : 2 * (t - u.nce) + 1;  // k - |m|
      double2 pv = bp ? __ldg(reinterpret_cast<const double2*>(bp) + kk) : make_double2(0.0, 0.0);
      double2 nv = bn ? __ldg(reinterpret_cast<const double2*>(bn) + kk) : make_double2(0.0, 0.0);
      double2* xr = reinterpret_cast<double2*>(vec + (size_t)t * kRT);  // xe = 0, xo = nce
      __stcg(xr, pv);
      __stcg(xr + 1, nv);
    }
    for (int t = threadIdx.x; t < 2 * N; t += kThreads) {
      double2* yr = reinterpret_cast<double2*>(vec + (size_t)(u.ye + t) * kRT);  // ye, yo contiguous
      __stcg(yr, make_double2(0.0, 0.0));
      __stcg(yr + 1, make_double2(0.0, 0.0));
    }
    __syncthreads();
    // 2. phases
    for (int ph = 0; ph < u.nphase; ++ph) {
      run_ops_forward(p, p.ops, p.phase_tab[u.ph_begin + ph], p.phase_tab[u.ph_begin + ph + 1], vec);
      __syncthreads();
    }
    // 3. parity fold into g
    for (int i = threadIdx.x; i < N; i += kThreads) {
      const double2* ye = reinterpret_cast<const double2*>(vec + (size_t)(u.ye + i) * kRT);
      const double2* yo = reinterpret_cast<const double2*>(vec + (size_t)(u.yo + i) * kRT);
      const double2 e0 = __ldcg(ye), e1 = __ldcg(ye + 1), o0 = __ldcg(yo), o1 = __ldcg(yo + 1);
      for (int s = 0; s < 2; ++s) {
        const long m = s == 0 ? am : -am;
        if (s == 1 && am == 0) break;
        double2* gp;
        if (single) {
          if (m != msingle) continue;
          gp = reinterpret_cast<double2*>(g + 2L * f * K);
        } else {
          gp = reinterpret_cast<double2*>(g + 2 * (f * nval + order_slot(m) * K));
        }
        const double2 e = s == 0 ? e0 : e1, o = s == 0 ? o0 : o1;
        gp[N + i] = make_double2(e.x + o.x, e.y + o.y);
        gp[N - 1 - i] = make_double2(e.x - o.x, e.y - o.y);
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads) alt_inverse_f64_kernel(DevPlan p, const double* __restrict__ g,
                                                                   double* __restrict__ beta, int F, int single,
                                                                   int msingle) {
  const int N = p.N, K = 2 * N;
  double* vec = p.ws + (size_t)blockIdx.x * p.max_rows * kRT;
  const long ncoef = 4L * N * N, nval = (4L * N - 1) * K;
  const int nitems = single ? F : p.nunits * F;
  for (;;) {
    const int item = next_item(p.counter);
    if (item >= nitems) break;
    const int f = single ? item : item % F;
    const int am = single ? (msingle < 0 ? -msingle : msingle) : p.order[item / F];
    const Unit u = p.units[am];
    // 1. W-weighted parity fold of g into Y_e, Y_o; zero X
    for (int i = threadIdx.x; i < N; i += kThreads) {
      double2 ev[2], ov[2];
      const double wi = __ldg(p.w + N + i);
      for (int s = 0; s < 2; ++s) {
        const long m = s == 0 ? am : -am;
        const double2* gp = nullptr;
        if (single) {
          if (m == msingle && !(s == 1 && am == 0)) gp = reinterpret_cast<const double2*>(g + 2L * f * K);
        } else if (!(s == 1 && am == 0)) {
          gp = reinterpret_cast<const double2*>(g + 2 * (f * nval + order_slot(m) * K));
        }
        double2 a = gp ? __ldg(gp + N + i) : make_double2(0.0, 0.0);
        double2 b = gp ? __ldg(gp + N - 1 - i) : make_double2(0.0, 0.0);
        ev[s] = make_double2(wi * (a.x + b.x), wi * (a.y + b.y));
        ov[s] = make_double2(wi * (a.x - b.x), wi * (a.y - b.y));
      }
      double2* ye = reinterpret_cast<double2*>(vec + (size_t)(u.ye + i) * kRT);
      double2* yo = reinterpret_cast<double2*>(vec + (size_t)(u.yo + i) * kRT);
      __stcg(ye, ev[0]);
      __stcg(ye + 1, ev[1]);
      __stcg(yo, ov[0]);
      __stcg(yo + 1, ov[1]);
    }
    for (int t = threadIdx.x; t < u.nce + u.nco; t += kThreads) {
      double2* xr = reinterpret_cast<double2*>(vec + (size_t)t * kRT);
      __stcg(xr, make_double2(0.0, 0.0));
      __stcg(xr + 1, make_double2(0.0, 0.0));
    }
    __syncthreads();
    // 2. transposed phases, last first
    for (int ph = u.nphase - 1; ph >= 0; --ph) {
      run_ops_transpose(p, p.ops, p.phase_tab[u.ph_begin + ph], p.phase_tab[u.ph_begin + ph + 1], vec);
      __syncthreads();
    }
    // 3. scatter X into beta
    double* bp;
    double* bn;
    if (single) {
      bp = msingle >= 0 ? beta + 2L * f * (K - am) : nullptr;
      bn = msingle < 0 ? beta + 2L * f * (K - am) : nullptr;
    } else {
      bp = beta + 2 * (f * ncoef + coef_offset(N, am));
      bn = am > 0 ? beta + 2 * (f * ncoef + coef_offset(N, -am)) : nullptr;
    }
    for (int t = threadIdx.x; t < u.nce + u.nco; t += kThreads) {
      const int kk = t < u.nce ? 2 * t : 2 * (t - u.nce) + 1;
      const double2* xr = reinterpret_cast<const double2*>(vec + (size_t)t * kRT);
      if (bp) reinterpret_cast<double2*>(bp)[kk] = __ldcg(xr);
      if (bn) reinterpret_cast<double2*>(bn)[kk] = __ldcg(xr + 1);
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Scratch of the forward single-order ALT without any allocation
// (alt_forward_m_noalloc, at the end of this file).
//
// Some callers cannot allocate device memory: code that runs inside a
// memory-pool or arena that owns the whole device, real-time loops where a
// cudaMalloc/cudaFree would synchronise the device and stall other streams,
// and embedders whose allocator is not CUDA's.  For them that entry point runs
// the same forward kernel as alt_forward_m, but with its per-CTA vector
// scratch and its work counter taken from the fixed array below instead of
// the plan's workspace.  It calls no cudaMalloc, cudaFree or allocating
// library routine.
//
// The array lives in the library's device image: every GPU that loads
// libsht.so holds kNoAllocScratchBytes of it until the process exits.  Host
// code must not pass the array's name to a kernel (on the host it is only a
// stand-in symbol); its device address is looked up with cudaGetSymbolAddress
// when a plan is created, with the plan's device current, and kept in the
// plan, so the entry point itself does no set-up.  All calls share the one
// array, so calls that may overlap on the GPU (different streams, or several
// plans at once) race on it: serialise them.
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // 8 MiB
constexpr size_t kNoAllocCounterBytes = 256;              // work counter, padded

static __device__ __align__(256) unsigned char noalloc_scratch[kNoAllocScratchBytes];

}  // namespace

// ---------------------------------------------------------------------------
// Plan object and C ABI

struct sht_plan_s {
  HostProgram prog;
  int device = 0;
  int nslots = 0;
  Unit* d_units = nullptr;
  Op* d_ops = nullptr;
  int32_t* d_phase = nullptr;
  int32_t* d_order = nullptr;
  double* d_fac = nullptr;
  double* d_w = nullptr;
  double* d_ws = nullptr;
  unsigned int* d_counter = nullptr;
  sht_status latched = SHT_OK;
  bool host_only = false;
  bool direct = false;  // SHT_FLAG_DIRECT: no ALT program; dense ALT by the recurrence on the fly
  DirectPlan dplan;
  LegendreDev leg;               // Pbar on the device (sht_legendre)
  double* d_legcoef = nullptr;   // its recurrence coefficients, 4N doubles
  // FP32 many-field path (precision SHT_FP32 / SHT_MIXED)
  float* d_fac32 = nullptr;
  float* d_ws32 = nullptr;
  int nslots32 = 0;
  // phi-direction DFT (FP64 tables for FP64 plans, FP32 otherwise) and the
  // ALT-value workspace of sht_forward / sht_inverse (max_fields fields)
  PhiTables<double> phi64;
  PhiTables<float> phi32;
  int phi_grid = 0;
  double* d_gws = nullptr;
  // tensor-core path (precision SHT_MIXED): split-BF16 operand images
  uint16_t* d_img = nullptr;
  TcOp* d_tcops = nullptr;
  int32_t* d_tctiles = nullptr;
  int32_t* d_tczr = nullptr;   // accumulation row ranges to zero per order and direction
  int32_t* d_tczri = nullptr;
  int32_t* d_tclive = nullptr;  // per order: node rows that some op reaches (tc_live_rows)
  unsigned char* d_wstc = nullptr;
  float* d_acc = nullptr;  // accumulated rows of every work item (tc_gmax field groups)
  unsigned char* d_pre = nullptr;  // transposed inputs gathered ahead (tc_gmax field groups)
  float* d_w32 = nullptr;          // the weights of the positive nodes, rounded to FP32
  int32_t* d_tcford = nullptr;     // the tensor-core kernel's op processing order, forward
  int32_t* d_tctord = nullptr;     // and transposed
  int tc_gmax = 0;
  int tc_max_rows = 0;     // scratch rows of the largest order (tensor-core layout)
  int* d_err = nullptr;
  int nslots_tc = 0;
  // device address of noalloc_scratch in this plan's context (looked up at
  // creation; used only by alt_forward_m_noalloc)
  unsigned char* d_noalloc = nullptr;
  // SHT_FLAG_TIMING: three events per recorded launch (before, between, after
  // the kernels), a ring of kTimingSlots launches
  std::vector<cudaEvent_t> tev;
  int64_t tev_count = 0, tev_base = 0;
  bool timing_on = true;  // sht_plan_set_timing
};

namespace {

// Host-side fault injection for tests: with SHT_FAIL_ALLOC=k in the
// environment, the k-th device allocation of a plan or batch creation fails as
// if the device were out of memory, so that the error path (everything
// allocated so far released, SHT_ERR_OOM) can be exercised without a real
// shortage.  The count restarts with every creation; not for concurrent use.
int g_alloc_fail_at = 0;
int g_alloc_seen = 0;

void alloc_hook_reset() {
  const char* v = std::getenv("SHT_FAIL_ALLOC");
  g_alloc_fail_at = v ? std::atoi(v) : 0;
  g_alloc_seen = 0;
}

// Tensor-core image sets up to this size are packed whole on the host before
// one copy; larger ones in windows of about kImageWindow bytes.
constexpr size_t kImagesWhole = (size_t)32 << 30;
constexpr size_t kImageWindow = (size_t)1 << 30;

cudaError_t plan_malloc(void** ptr, size_t bytes) {
  if (g_alloc_fail_at > 0 && ++g_alloc_seen == g_alloc_fail_at) {
    *ptr = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(ptr, bytes);
}

template <class T, class A>
cudaError_t upload(T** dst, const std::vector<T, A>& v) {
  size_t bytes = std::max<size_t>(sizeof(T), v.size() * sizeof(T));
  cudaError_t e = plan_malloc(reinterpret_cast<void**>(dst), bytes);
  if (e != cudaSuccess) return e;
  if (!v.empty()) e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

constexpr int kTimingSlots = 256;

// Events of the next recorded launch (nullptr without SHT_FLAG_TIMING).
cudaEvent_t* timing_slot(sht_plan_s* p) {
  if (p->tev.empty() || !p->timing_on) return nullptr;
  cudaEvent_t* ev = p->tev.data() + 3 * (p->tev_count % kTimingSlots);
  ++p->tev_count;
  return ev;
}

void free_device(sht_plan_s* p) {
  for (cudaEvent_t ev : p->tev) cudaEventDestroy(ev);
  p->tev.clear();
  cudaFree(p->d_units);
  cudaFree(p->d_ops);
  cudaFree(p->d_phase);
  cudaFree(p->d_order);
  cudaFree(p->d_fac);
  cudaFree(p->d_w);
  cudaFree(p->d_ws);
  cudaFree(p->d_counter);
  cudaFree(p->d_fac32);
  cudaFree(p->d_ws32);
  cudaFree(p->d_gws);
  cudaFree(p->d_img);
  cudaFree(p->d_tcops);
  cudaFree(p->d_tctiles);
  cudaFree(p->d_tczr);
  cudaFree(p->d_tczri);
  cudaFree(p->d_tclive);
  cudaFree(p->d_wstc);
  cudaFree(p->d_acc);
  cudaFree(p->d_pre);
  cudaFree(p->d_w32);
  cudaFree(p->d_tcford);
  cudaFree(p->d_tctord);
  cudaFree(p->d_err);
  p->phi64.release();
  p->phi32.release();
  p->dplan.release();
  p->leg.release();
  cudaFree(p->d_legcoef);
  p->d_legcoef = nullptr;
}

// The device's Legendre table for this plan (kept when the builder made it).
cudaError_t attach_legendre(sht_plan_s* p) {
  cudaError_t e = p->leg.d_x ? cudaSuccess : p->leg.build(p->prog.N, p->prog.x.data());
  if (e == cudaSuccess && !p->d_legcoef) e = cudaMalloc(&p->d_legcoef, 4 * (size_t)p->prog.N * sizeof(double));
  return e;
}

DevPlan dev_plan(const sht_plan_s* p) {
  DevPlan d;
  d.units = p->d_units;
  d.ops = p->d_ops;
  d.phase_tab = p->d_phase;
  d.order = p->d_order;
  d.fac = p->d_fac;
  d.w = p->d_w;
  d.ws = p->d_ws;
  d.counter = p->d_counter;
  d.N = p->prog.N;
  d.nunits = 2 * p->prog.N;
  d.max_rows = p->prog.max_rows;
  return d;
}

// The tensor-core kernel's view of a SHT_MIXED plan.
TcPlan tc_plan_of(const sht_plan_s* p) {
  TcPlan t;
  t.units = p->d_units;
  t.ops = p->d_tcops;
  t.tiles = p->d_tctiles;
  t.order = p->d_order;
  t.img = p->d_img;
  t.zr = p->d_tczr;
  t.zri = p->d_tczri;
  t.live = p->d_tclive;
  t.w32 = p->d_w32;
  t.acc = p->d_acc;
  t.pre = p->d_pre;
  t.ford = p->d_tcford;
  t.tord = p->d_tctord;
  t.gmax = p->tc_gmax;
  t.N = p->prog.N;
  t.nunits = 2 * p->prog.N;
  t.max_rows = p->tc_max_rows;
  return t;
}

sht_status launch(sht_plan_s* p, bool fwd, const double* in, double* out, int F, int single, int m,
                  cudaStream_t st) {
  if (p->host_only) return SHT_ERR_UNSUPPORTED;
  // complex values are moved as 16-byte pairs
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15u) return SHT_ERR_ARG;
  if ((int64_t)F * 2 * p->prog.N > (int64_t)1 << 30) return SHT_ERR_ARG;
  if (p->latched != SHT_OK) {
    sht_status s = p->latched;
    p->latched = SHT_OK;
    return s;
  }
  if (p->direct) {
    // the dense recurrence on the fly, all orders, max_fields fields per launch
    if (single) return SHT_ERR_UNSUPPORTED;
    const int N = p->prog.N;
    const int64_t nb = 2L * 4L * N * N, ng = 2L * (4L * N - 1) * 2 * N;  // doubles per field
    const int64_t in_stride = fwd ? nb : ng, out_stride = fwd ? ng : nb;
    cudaEvent_t* ev = timing_slot(p);
    if (ev && cudaEventRecord(ev[0], st) != cudaSuccess) return SHT_ERR_CUDA;
    for (int f0 = 0; f0 < F; f0 += p->dplan.F_max) {
      const int Fb = std::min(p->dplan.F_max, F - f0);
      if (p->dplan.launch(fwd, in + f0 * in_stride, out + f0 * out_stride, Fb, st) != cudaSuccess)
        return SHT_ERR_CUDA;
    }
    if (ev && (cudaEventRecord(ev[1], st) != cudaSuccess || cudaEventRecord(ev[2], st) != cudaSuccess))
      return SHT_ERR_CUDA;
    return SHT_OK;
  }
  if (cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned int), st) != cudaSuccess) return SHT_ERR_CUDA;
  if (p->prog.opts.precision == SHT_MIXED) {
    const TcPlan t = tc_plan_of(p);
    // the accumulation buffer holds tc_gmax groups of kTcFields fields: larger
    // batches run as several launches on consecutive fields
    const int N = p->prog.N;
    const int64_t nb = 2L * (single ? 2 * N - (m < 0 ? -m : m) : 4L * N * N);  // doubles per field of beta
    const int64_t ng = 2L * (single ? 2 * N : (4L * N - 1) * 2 * N);           // doubles per field of g
    const int64_t in_stride = fwd ? nb : ng, out_stride = fwd ? ng : nb;
    const int fb = kTcFields * p->tc_gmax;
    for (int f0 = 0; f0 < F; f0 += fb) {
      const int Fb = std::min(fb, F - f0);
      if (f0 > 0 && cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned int), st) != cudaSuccess) return SHT_ERR_CUDA;
      const int groups = (Fb + kTcFields - 1) / kTcFields;
      const int items = (single ? 1 : 2 * N) * groups;
      const int grid_tc = std::min(p->nslots_tc, std::max(1, items));
      if (launch_tc(t, fwd, in + f0 * in_stride, out + f0 * out_stride, Fb, single, m, grid_tc, p->d_wstc,
                    p->d_counter, p->d_err, st, timing_slot(p)) != cudaSuccess)
        return SHT_ERR_CUDA;
    }
    return SHT_OK;
  }
  if (p->prog.opts.precision == SHT_FP32) {
    F32Plan f;
    f.units = p->d_units;
    f.ops = p->d_ops;
    f.phase_tab = p->d_phase;
    f.order = p->d_order;
    f.fac = p->d_fac32;
    f.w = p->d_w;
    f.ws = p->d_ws32;
    f.counter = p->d_counter;
    f.N = p->prog.N;
    f.nunits = 2 * p->prog.N;
    f.max_rows = p->prog.max_rows;
    const int groups = (F + kF32Fields - 1) / kF32Fields;
    const int items32 = (single ? 1 : 2 * p->prog.N) * groups;
    const int grid32 = std::min(p->nslots32, std::max(1, items32));
    cudaEvent_t* ev = timing_slot(p);
    if (ev && cudaEventRecord(ev[0], st) != cudaSuccess) return SHT_ERR_CUDA;
    if (launch_f32(f, fwd, in, out, F, single, m, grid32, st) != cudaSuccess) return SHT_ERR_CUDA;
    if (ev && (cudaEventRecord(ev[1], st) != cudaSuccess || cudaEventRecord(ev[2], st) != cudaSuccess))
      return SHT_ERR_CUDA;
    return SHT_OK;
  }
  const int items = single ? F : 2 * p->prog.N * F;
  const int grid = std::min(p->nslots, std::max(1, items));
  DevPlan d = dev_plan(p);
  cudaEvent_t* ev = timing_slot(p);
  if (ev && cudaEventRecord(ev[0], st) != cudaSuccess) return SHT_ERR_CUDA;
  if (fwd)
    alt_forward_f64_kernel<<<grid, kThreads, 0, st>>>(d, in, out, F, single, m);
  else
    alt_inverse_f64_kernel<<<grid, kThreads, 0, st>>>(d, in, out, F, single, m);
  if (cudaGetLastError() != cudaSuccess) return SHT_ERR_CUDA;
  if (ev && (cudaEventRecord(ev[1], st) != cudaSuccess || cudaEventRecord(ev[2], st) != cudaSuccess))
    return SHT_ERR_CUDA;
  return SHT_OK;
}

// The conversion helpers over an array (sht_selftest_convert).
__global__ void convert_selftest_kernel(const double* __restrict__ f64, float* __restrict__ f32,
                                        double* __restrict__ back, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = f64_to_f32_bits(f64[i]);
    f32[i] = v;
    back[i] = f32_to_f64_bits(v);
  }
}

sht_status launch_phi(sht_plan_s* p, const double* in, double* out, int F, bool analysis, cudaStream_t st) {
  if (p->host_only) return SHT_ERR_UNSUPPORTED;
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15u) return SHT_ERR_ARG;
  if ((int64_t)F * 2 * p->prog.N > (int64_t)1 << 30) return SHT_ERR_ARG;
  if (p->phi_grid < 1) return SHT_ERR_UNSUPPORTED;
  cudaError_t e = p->prog.opts.precision == SHT_FP64 ? p->phi64.launch(in, out, F, analysis, st)
                                                     : p->phi32.launch(in, out, F, analysis, st);
  return e == cudaSuccess ? SHT_OK : SHT_ERR_CUDA;
}

}  // namespace

extern "C" {

void sht_opts_default(int N, double eps, sht_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->eps = eps;
  o->n0 = N >= 2048 ? 512 : std::max(16, N / 4);
  o->n_leaf = N >= 1024 ? 64 : std::max(8, N / 16);
  o->r_k = 150;
  o->oversample = 2.0;
  o->rsvd_r = 30;
  o->rsvd_q = 2;
  o->trim_delta = std::max(1e-3 * eps, 0x1p-52);
  o->sampling = 0;
  o->precision = SHT_FP64;
  o->max_fields = 1;
  o->flags = 0;
  o->seed = 0x5eed2004u;
}

namespace {

// Device side of a plan: upload the program and factors, build the operand
// images of the precision's kernel, size the workspaces and the phi tables.
// On failure everything allocated here is released again.
sht_status attach_device(sht_plan_s* p) {
  alloc_hook_reset();
  const int N = p->prog.N;
  const sht_opts& o = p->prog.opts;
  auto t0 = std::chrono::steady_clock::now();
  cudaGetDevice(&p->device);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, alt_forward_f64_kernel, kThreads, 0);
  p->nslots = std::max(1, sms * std::max(1, per_sm));
  const HostProgram& P = p->prog;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = upload(&p->d_units, P.units);
  if (e == cudaSuccess) e = upload(&p->d_ops, P.ops);
  if (e == cudaSuccess) e = upload(&p->d_phase, P.phase_tab);
  if (e == cudaSuccess) e = upload(&p->d_order, P.order);
  // the FP64 factor store is read only by the FP64 kernels; the other precisions
  // upload their own representation below
  if (e == cudaSuccess && o.precision == SHT_FP64) e = upload(&p->d_fac, P.factors);
  if (e == cudaSuccess) e = upload(&p->d_w, P.w);
  size_t ws = o.precision == SHT_FP64 ? (size_t)p->nslots * P.max_rows * kRT * sizeof(double) : 0;
  if (e == cudaSuccess) e = plan_malloc(reinterpret_cast<void**>(&p->d_ws), std::max<size_t>(ws, 8));
  if (e == cudaSuccess) e = plan_malloc(reinterpret_cast<void**>(&p->d_counter), sizeof(unsigned int));
  if (e == cudaSuccess && o.precision == SHT_FP64) {
    void* na = nullptr;
    e = cudaGetSymbolAddress(&na, noalloc_scratch);
    if (e == cudaSuccess && !na) e = cudaErrorInvalidSymbol;
    p->d_noalloc = static_cast<unsigned char*>(na);
  }
  size_t ws32 = 0;
  if (e == cudaSuccess && o.precision == SHT_MIXED) {
    std::vector<TcOp> tops;
    std::vector<int32_t> tiles;
    const size_t img_elems = tc_image_layout(N, P.units, P.ops, tops, tiles, p->tc_max_rows);
    const size_t img_alloc = std::max<size_t>(img_elems, 8);
    std::vector<int32_t> zr, zri;
    std::vector<int32_t> ford, tord;
    tc_proc_order(P.units, tops, ford, tord);
    std::vector<int32_t> live;
    tc_live_rows(N, P.units, tops, live);
    tc_first_writers(N, P.units, tops, ford, tord, live, zr, zri);
    if (img_alloc * sizeof(uint16_t) <= kImagesWhole) {
      // packed whole on the host, one copy
      TcImages img(img_alloc);
      std::fill(img.begin() + img_elems, img.end(), (uint16_t)0);
      tc_pack_ops(P.ops, tops, P.factors.data(), 0, P.ops.size(), img.data(), 0);
      e = upload(&p->d_img, img);
    } else {
      // a store larger than that (N around 2048 and up) is packed in windows
      // of consecutive ops, each copied to its place, so that the host holds
      // one window beside the FP64 factor store instead of the whole image set
      e = plan_malloc(reinterpret_cast<void**>(&p->d_img), img_alloc * sizeof(uint16_t));
      if (e == cudaSuccess)
        tc_pack_windows(P.ops, tops, P.factors.data(), img_elems, kImageWindow / sizeof(uint16_t),
                        [&](size_t first, const uint16_t* data, size_t n) {
                          e = cudaMemcpy(p->d_img + first, data, n * sizeof(uint16_t), cudaMemcpyHostToDevice);
                          return e == cudaSuccess;
                        });
    }
    {
      // round to nearest, as the kernels' FP64 -> FP32 conversions do
      std::vector<float> w32((size_t)N);
      for (int i = 0; i < N; ++i) w32[(size_t)i] = (float)P.w[(size_t)(N + i)];
      if (e == cudaSuccess) e = upload(&p->d_w32, w32);
    }
    if (e == cudaSuccess) e = upload(&p->d_tcops, tops);
    if (e == cudaSuccess) e = upload(&p->d_tczr, zr);
    if (e == cudaSuccess) e = upload(&p->d_tczri, zri);
    if (e == cudaSuccess) e = upload(&p->d_tclive, live);
    if (e == cudaSuccess) e = upload(&p->d_tcford, ford);
    if (e == cudaSuccess) e = upload(&p->d_tctord, tord);
    if (e == cudaSuccess) e = upload(&p->d_tctiles, tiles);
    p->nslots_tc = std::max(1, sms * tc_ctas_per_sm());
    ws32 = (size_t)p->nslots_tc * 2 * tc_slot_bytes(p->tc_max_rows);  // two vector spaces per CTA
    if (e == cudaSuccess) e = plan_malloc(reinterpret_cast<void**>(&p->d_wstc), std::max<size_t>(ws32, 8));
    // rows that widened K chunks read but no op writes must hold finite values
    if (e == cudaSuccess) e = cudaMemset(p->d_wstc, 0, std::max<size_t>(ws32, 8));
    p->tc_gmax = (o.max_fields + kTcFields - 1) / kTcFields;
    const size_t acc = (size_t)p->tc_gmax * 2 * N * tc_acc_rows(N) * kTcR * sizeof(float);
    if (e == cudaSuccess) e = plan_malloc(reinterpret_cast<void**>(&p->d_acc), acc);
    const size_t pre = (size_t)p->tc_gmax * 2 * N * tc_pre_groups(N) * kTcGrpBytes;
    if (e == cudaSuccess) e = plan_malloc(reinterpret_cast<void**>(&p->d_pre), pre);
    ws32 += pre;
    ws32 += acc;
    if (e == cudaSuccess) e = plan_malloc(reinterpret_cast<void**>(&p->d_err), sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(int));
    p->prog.info.factor_bytes = (int64_t)(img_alloc * sizeof(uint16_t));
  }
  if (e == cudaSuccess && o.precision == SHT_FP32) {
    std::vector<float, UninitAlloc<float>> f32(P.factors.size());
#pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)f32.size(); ++i) f32[(size_t)i] = (float)P.factors[(size_t)i];
    e = upload(&p->d_fac32, f32);
    p->nslots32 = std::max(1, sms * f32_ctas_per_sm());
    ws32 = (size_t)p->nslots32 * P.max_rows * kF32RT * sizeof(float);
    if (e == cudaSuccess) e = plan_malloc(reinterpret_cast<void**>(&p->d_ws32), std::max<size_t>(ws32, 8));
  }
  size_t gws = 0;
  if (e == cudaSuccess) {
    const bool ok = o.precision == SHT_FP64 ? p->phi64.build(N) : p->phi32.build(N);
    if (!ok) e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = attach_legendre(p);
    // co-resident clusters of the transform's launch shape; 0: one row does
    // not fit the shared memory of a cluster
    p->phi_grid = o.precision == SHT_FP64 ? p->phi64.max_clusters : p->phi32.max_clusters;
  }
  if (e == cudaSuccess) {
    gws = (size_t)o.max_fields * (4 * (size_t)N - 1) * 2 * N * 2 * sizeof(double);
    e = plan_malloc(reinterpret_cast<void**>(&p->d_gws), gws);
  }
  if (e == cudaSuccess && (o.flags & SHT_FLAG_TIMING)) {
    p->tev.assign(3 * kTimingSlots, nullptr);
    for (cudaEvent_t& ev : p->tev)
      if (e == cudaSuccess) e = cudaEventCreate(&ev);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_device(p);
    return e == cudaErrorMemoryAllocation ? SHT_ERR_OOM : SHT_ERR_CUDA;
  }
  p->prog.info.workspace_bytes = (int64_t)(ws + ws32 + gws);
  if (o.precision != SHT_MIXED)
    p->prog.info.factor_bytes =
        (int64_t)(P.factors.size() * (o.precision == SHT_FP64 ? sizeof(double) : sizeof(float)));
  p->prog.info.t_upload_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return SHT_OK;
}


// The options a plan of order N is built with (the defaults when opts is
// NULL, the tolerance always eps); false when N, eps or an option is out of
// range.
bool resolve_opts(int N, double eps, const sht_opts* opts, sht_opts& o) {
  if (N < 1 || N > (1 << 14) || !(eps > 0.0 && eps < 1.0)) return false;
  if (opts) {
    o = *opts;
    o.eps = eps;
  } else {
    sht_opts_default(N, eps, &o);
  }
  return o.n0 >= 1 && o.n_leaf >= 1 && o.r_k >= 1 && o.rsvd_r >= 1 && o.rsvd_q >= 1 && o.oversample >= 1.0 &&
         o.trim_delta >= 0.0 && o.max_fields >= 1;
}

// Device side of a direct plan: the phi-direction tables and the dense
// on-the-fly ALT (nodes, weights and per-CTA scratch for max_fields fields).
sht_status attach_direct(sht_plan_s* p) {
  alloc_hook_reset();
  const int N = p->prog.N;
  const sht_opts& o = p->prog.opts;
  cudaGetDevice(&p->device);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  const bool fp64 = o.precision == SHT_FP64;
  const bool ok = fp64 ? p->phi64.build(N) : p->phi32.build(N);
  cudaError_t e = ok ? cudaSuccess : cudaErrorMemoryAllocation;
  if (e == cudaSuccess) e = p->dplan.build(N, o.max_fields, p->prog.x.data(), p->prog.w.data(), std::max(1, sms));
  if (e == cudaSuccess) e = attach_legendre(p);
  if (e == cudaSuccess) {
    const size_t gws = (size_t)o.max_fields * (4 * (size_t)N - 1) * 2 * N * 2 * sizeof(double);
    e = plan_malloc(reinterpret_cast<void**>(&p->d_gws), gws);
    p->prog.info.workspace_bytes =
        (int64_t)(gws + (size_t)p->dplan.grid * p->dplan.per_cta * sizeof(double));
  }
  if (e == cudaSuccess && (o.flags & SHT_FLAG_TIMING)) {
    p->tev.assign(3 * kTimingSlots, nullptr);
    for (cudaEvent_t& ev : p->tev)
      if (e == cudaSuccess) e = cudaEventCreate(&ev);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_device(p);
    return e == cudaErrorMemoryAllocation ? SHT_ERR_OOM : SHT_ERR_CUDA;
  }
  p->phi_grid = fp64 ? p->phi64.max_clusters : p->phi32.max_clusters;
  return SHT_OK;
}

// The plan builder's Legendre matrices from the device (SHT_FLAG_GPU_LEGENDRE):
// each host thread has its own stream, device table and pinned host copy;
// the table of one order is computed, copied back and split by parity.
class DeviceLegendreSource final : public LegendreSource {
 public:
  DeviceLegendreSource(const LegendreDev& leg, int N) : leg_(leg), N_(N), slots_((size_t)omp_get_max_threads()) {}
  ~DeviceLegendreSource() override {
    for (Slot& s : slots_) {
      if (s.st) cudaStreamDestroy(s.st);
      cudaFree(s.d_out);
      cudaFree(s.d_coef);
      cudaFreeHost(s.h_out);
    }
  }
  bool parity_matrices(int N, int am, const double* /*xp*/, Mat& E, Mat& O) override {
    const int tid = omp_get_thread_num();
    if (N != N_ || tid < 0 || tid >= (int)slots_.size()) return false;
    Slot& s = slots_[(size_t)tid];
    const size_t full = 2 * (size_t)N * N;
    if (!s.st) {
      if (cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess ||
          cudaMalloc(&s.d_out, full * sizeof(double)) != cudaSuccess ||
          cudaMalloc(&s.d_coef, 4 * (size_t)N * sizeof(double)) != cudaSuccess ||
          cudaMallocHost(&s.h_out, full * sizeof(double)) != cudaSuccess)
        return false;
    }
    const int K = 2 * N - am;
    if (leg_.table(am, s.d_out, s.d_coef, s.st) != cudaSuccess) return false;
    if (cudaMemcpyAsync(s.h_out, s.d_out, (size_t)K * N * sizeof(double), cudaMemcpyDeviceToHost, s.st) !=
            cudaSuccess ||
        cudaStreamSynchronize(s.st) != cudaSuccess)
      return false;
    E = Mat(N, (K + 1) / 2);
    O = Mat(N, K / 2);
    for (int t = 0; t < K; ++t)
      std::memcpy((t & 1) ? O.col(t >> 1) : E.col(t >> 1), s.h_out + (size_t)t * N, sizeof(double) * (size_t)N);
    return true;
  }

 private:
  struct Slot {
    cudaStream_t st = nullptr;
    double* d_out = nullptr;
    double* d_coef = nullptr;
    double* h_out = nullptr;
  };
  const LegendreDev& leg_;
  int N_;
  std::vector<Slot> slots_;
};

}  // namespace

sht_status sht_plan_create(int N, double eps, const sht_opts* opts, sht_plan_t* out) {
  if (!out) return SHT_ERR_ARG;
  *out = nullptr;
  sht_opts o;
  if (!resolve_opts(N, eps, opts, o)) return SHT_ERR_ARG;
  const bool host_only = (o.flags & SHT_FLAG_HOST_ONLY) != 0;
  const bool direct = (o.flags & SHT_FLAG_DIRECT) != 0;
  if (host_only && direct) return SHT_ERR_ARG;  // nothing to build
  if (host_only && (o.flags & SHT_FLAG_GPU_LEGENDRE)) return SHT_ERR_ARG;  // the builder would need a device
  int ndev = 0;
  if (!host_only && (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1)) return SHT_ERR_CUDA;
  sht_plan_s* p = new (std::nothrow) sht_plan_s();
  if (!p) return SHT_ERR_OOM;
  if (direct) {
    p->direct = true;
    p->prog.N = N;
    p->prog.opts = o;
    p->prog.info.N = N;
    p->prog.info.eps = o.eps;
    sht_status s = SHT_OK;
    try {
      gauss_legendre(2 * N, p->prog.x, p->prog.w);
    } catch (const std::bad_alloc&) {
      s = SHT_ERR_OOM;
    }
    if (s == SHT_OK) s = attach_direct(p);
    if (s != SHT_OK) {
      delete p;
      return s;
    }
    *out = p;
    return SHT_OK;
  }
  std::string err;
  sht_status s;
  try {
    if (o.flags & SHT_FLAG_GPU_LEGENDRE) {
      // the builder's Legendre matrices from the device; the table stays with the plan
      std::vector<double> x, w;
      gauss_legendre(2 * N, x, w);
      if (p->leg.build(N, x.data()) != cudaSuccess) {
        p->leg.release();
        delete p;
        return SHT_ERR_CUDA;
      }
      DeviceLegendreSource src(p->leg, N);
      s = build_program(N, o, p->prog, err, &src);
    } else {
      s = build_program(N, o, p->prog, err);
    }
  } catch (const std::bad_alloc&) {
    s = SHT_ERR_OOM;
  }
  if (s != SHT_OK) {
    p->leg.release();
    delete p;
    return s;
  }
  if (host_only) {
    p->host_only = true;
    *out = p;
    return SHT_OK;
  }
  s = attach_device(p);
  if (s != SHT_OK) {
    delete p;
    return s;
  }
  *out = p;
  return SHT_OK;
}

sht_status sht_plan_destroy(sht_plan_t p) {
  if (!p) return SHT_ERR_ARG;
  if (!p->host_only) free_device(p);
  delete p;
  return SHT_OK;
}

sht_status sht_plan_stats(sht_plan_t p, sht_plan_info* out) {
  if (!p || !out) return SHT_ERR_ARG;
  *out = p->prog.info;
  return SHT_OK;
}

sht_status sht_order_stats(int N, double eps, const sht_opts* opts, int count, const int* m, sht_order_info* out) {
  sht_opts o;
  if (!resolve_opts(N, eps, opts, o) || count < 0 || (count > 0 && (!m || !out))) return SHT_ERR_ARG;
  std::vector<int> am((size_t)count);
  for (int i = 0; i < count; ++i) {
    if (m[i] <= -2 * N || m[i] >= 2 * N) return SHT_ERR_ARG;
    am[(size_t)i] = std::abs(m[i]);
  }
  std::vector<OrderBuild> b;
  try {
    const sht_status s = build_orders(N, o, count, am.data(), b);
    if (s != SHT_OK) return s;
  } catch (const std::bad_alloc&) {
    return SHT_ERR_OOM;
  }
  for (int i = 0; i < count; ++i) {
    const OrderBuild& r = b[(size_t)i];
    sht_order_info& q = out[i];
    std::memset(&q, 0, sizeof(q));
    q.N = N;
    q.am = am[(size_t)i];
    q.cols_even = r.unit.nce;
    q.cols_odd = r.unit.nco;
    q.n_blocks_idbf = r.n_idbf;
    q.n_blocks_lowrank = r.n_low;
    q.n_blocks_dense = r.n_dense;
    q.n_blocks_dropped = r.n_drop;
    q.entries_idbf = r.e_idbf;
    q.entries_lowrank = r.e_low;
    q.entries_dense = r.e_dense;
    q.entries_total = r.e_idbf + r.e_low + r.e_dense;
    q.entries_matrix = (int64_t)N * (r.unit.nce + r.unit.nco);
    q.factor_doubles = r.n_factors;
    for (const Op& op : r.ops) {
      const TcOp top = tc_op_of(op, r.unit, N);
      const TcDir df = tc_dir(top, true);
      const int64_t fwd = (int64_t)tc_image_elems(df);
      q.image_elems += fwd + (int64_t)tc_image_elems(tc_dir(top, false));
      if (op.ni <= 0) continue;
      q.tc_stages += (int64_t)df.nT * df.kg.nK;
      q.tc_tiles += df.nT;
      q.tc_image_fwd_bytes += 2 * fwd;
      q.tc_act_bytes += (int64_t)df.nT * df.kg.ngt * (int64_t)kTcGrpBytes;
    }
    q.max_rank = r.max_rank;
    q.n_ops = (int64_t)r.ops.size();
    q.n_phases = r.unit.nphase;
    q.rows = r.unit.nrows;
    q.flops_per_rhs = r.unit.cost;
    q.t_mat_s = r.t_mat_s;
    q.t_fac_s = r.t_fac_s;
  }
  return SHT_OK;
}

sht_status sht_plan_export(sht_plan_t p, int what, void* dst, size_t* bytes) {
  if (!p || !bytes) return SHT_ERR_ARG;
  const void* src = nullptr;
  size_t n = 0;
  const HostProgram& P = p->prog;
  switch (what) {
    case SHT_EXPORT_UNITS: src = P.units.data(); n = P.units.size() * sizeof(Unit); break;
    case SHT_EXPORT_OPS: src = P.ops.data(); n = P.ops.size() * sizeof(Op); break;
    case SHT_EXPORT_PHASES: src = P.phase_tab.data(); n = P.phase_tab.size() * sizeof(int32_t); break;
    case SHT_EXPORT_FACTORS: src = P.factors.data(); n = P.factors.size() * sizeof(double); break;
    case SHT_EXPORT_ORDER: src = P.order.data(); n = P.order.size() * sizeof(int32_t); break;
    case SHT_EXPORT_OPTS: src = &P.opts; n = sizeof(sht_opts); break;
    case SHT_EXPORT_UNIT_BLOCKS: src = P.unit_blocks.data(); n = P.unit_blocks.size() * sizeof(int32_t); break;
    default: return SHT_ERR_ARG;
  }
  if (!dst) {
    *bytes = n;
    return SHT_OK;
  }
  if (*bytes < n) return SHT_ERR_ARG;
  if (n) std::memcpy(dst, src, n);
  *bytes = n;
  return SHT_OK;
}

sht_status sht_plan_op_image(sht_plan_t p, int64_t op, int transposed, uint16_t* dst, size_t* count) {
  if (!p || !count || op < 0 || op >= (int64_t)p->prog.ops.size()) return SHT_ERR_ARG;
  // the order the op belongs to fixes its scratch rows
  const Unit* un = nullptr;
  for (const Unit& u : p->prog.units)
    if (op >= u.op_begin && op < u.op_end) un = &u;
  if (!un) return SHT_ERR_ARG;
  std::vector<uint16_t> img;
  try {
    const Op& o = p->prog.ops[(size_t)op];
    tc_op_image(o, tc_op_of(o, *un, p->prog.N), p->prog.factors.data(), transposed != 0, img);
  } catch (const std::bad_alloc&) {
    return SHT_ERR_OOM;
  }
  if (!dst) {
    *count = img.size();
    return SHT_OK;
  }
  if (*count < img.size()) return SHT_ERR_ARG;
  if (!img.empty()) std::memcpy(dst, img.data(), img.size() * sizeof(uint16_t));
  *count = img.size();
  return SHT_OK;
}

// ---------------------------------------------------------------------------
// Plan files.  Layout (native byte order; both supported hosts are
// little-endian):
//   "SHTPLAN\0", u32 version, u32 sizeof(Op), sizeof(Unit), sizeof(sht_opts),
//   sizeof(sht_plan_info), i32 N, i32 max_rows, sht_opts, sht_plan_info,
//   then x, w, units, ops, phase table, factors, schedule as (u64 count,
//   elements), then the 64-bit FNV-1a hash of every byte before it.

}  // extern "C"

namespace {

constexpr char kPlanMagic[8] = {'S', 'H', 'T', 'P', 'L', 'A', 'N', '\0'};
constexpr uint32_t kPlanVersion = 2;  // 2: intermediate segments start on 8-row boundaries

struct PlanWriter {
  std::FILE* f;
  uint64_t h = 0xcbf29ce484222325ull;
  bool ok = true;
  void put(const void* src, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(src);
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 0x100000001b3ull;
    if (n && std::fwrite(src, 1, n, f) != n) ok = false;
  }
  template <class T, class A>
  void vec(const std::vector<T, A>& v) {
    const uint64_t n = v.size();
    put(&n, sizeof n);
    put(v.data(), v.size() * sizeof(T));
  }
};

struct PlanReader {
  std::FILE* f;
  uint64_t left;  // bytes of the file not read yet
  uint64_t h = 0xcbf29ce484222325ull;
  bool ok = true;
  void get(void* dst, size_t n) {
    if (!ok || n > left || (n && std::fread(dst, 1, n, f) != n)) {
      ok = false;
      return;
    }
    left -= n;
    const unsigned char* b = static_cast<const unsigned char*>(dst);
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 0x100000001b3ull;
  }
  template <class T, class A>
  void vec(std::vector<T, A>& v, uint64_t max_elems) {
    uint64_t n = 0;
    get(&n, sizeof n);
    // a count the rest of the file cannot hold is refused before any allocation
    if (!ok || n > max_elems || n > left / sizeof(T)) {
      ok = false;
      return;
    }
    v.resize((size_t)n);
    get(v.data(), v.size() * sizeof(T));
  }
};

}  // namespace

extern "C" {

sht_status sht_plan_save(sht_plan_t p, const char* path) {
  if (!p || !path) return SHT_ERR_ARG;
  if (p->direct) return SHT_ERR_UNSUPPORTED;  // no program to save
  std::FILE* f = std::fopen(path, "wb");
  if (!f) return SHT_ERR_IO;
  const HostProgram& P = p->prog;
  PlanWriter w{f};
  const uint32_t hdr[5] = {kPlanVersion, (uint32_t)sizeof(Op), (uint32_t)sizeof(Unit), (uint32_t)sizeof(sht_opts),
                           (uint32_t)sizeof(sht_plan_info)};
  w.put(kPlanMagic, sizeof kPlanMagic);
  w.put(hdr, sizeof hdr);
  const int32_t nm[2] = {P.N, P.max_rows};
  w.put(nm, sizeof nm);
  w.put(&P.opts, sizeof P.opts);
  w.put(&P.info, sizeof P.info);
  w.vec(P.x);
  w.vec(P.w);
  w.vec(P.units);
  w.vec(P.ops);
  w.vec(P.phase_tab);
  w.vec(P.factors);
  w.vec(P.order);
  const uint64_t h = w.h;
  if (std::fwrite(&h, sizeof h, 1, f) != 1) w.ok = false;
  if (std::fclose(f) != 0) w.ok = false;
  return w.ok ? SHT_OK : SHT_ERR_IO;
}

sht_status sht_plan_load(const char* path, sht_plan_t* out) {
  if (!path || !out) return SHT_ERR_ARG;
  *out = nullptr;
  std::FILE* f = std::fopen(path, "rb");
  if (!f) return SHT_ERR_IO;
  sht_plan_s* p = new (std::nothrow) sht_plan_s();
  if (!p) {
    std::fclose(f);
    return SHT_ERR_OOM;
  }
  HostProgram& P = p->prog;
  uint64_t file_bytes = 0;
  if (std::fseek(f, 0, SEEK_END) == 0) {
    const long end = std::ftell(f);
    file_bytes = end > 0 ? (uint64_t)end : 0;
  }
  std::rewind(f);
  PlanReader r{f, file_bytes};
  char magic[8];
  uint32_t hdr[5];
  int32_t nm[2];
  r.get(magic, sizeof magic);
  r.get(hdr, sizeof hdr);
  r.get(nm, sizeof nm);
  bool ok = r.ok && std::memcmp(magic, kPlanMagic, sizeof magic) == 0 && hdr[0] == kPlanVersion &&
            hdr[1] == sizeof(Op) && hdr[2] == sizeof(Unit) && hdr[3] == sizeof(sht_opts) &&
            hdr[4] == sizeof(sht_plan_info) && nm[0] >= 1 && nm[0] <= (1 << 14) && nm[1] >= 0;
  sht_status s = SHT_OK;
  try {
    if (ok) {
      P.N = nm[0];
      P.max_rows = nm[1];
      r.get(&P.opts, sizeof P.opts);
      r.get(&P.info, sizeof P.info);
      // element-count limits keep a damaged header from requesting absurd allocations
      const uint64_t K = 2 * (uint64_t)P.N, big = (uint64_t)1 << 40;
      r.vec(P.x, K);
      r.vec(P.w, K);
      r.vec(P.units, K);
      r.vec(P.ops, big);
      r.vec(P.phase_tab, big);
      r.vec(P.factors, big);
      r.vec(P.order, K);
      uint64_t h = 0;
      const uint64_t expect = r.h;
      ok = r.ok && std::fread(&h, sizeof h, 1, f) == 1 && h == expect;
    }
  } catch (const std::bad_alloc&) {
    s = SHT_ERR_OOM;
  }
  std::fclose(f);
  if (s == SHT_OK && !ok) s = SHT_ERR_IO;
  std::string err;
  if (s == SHT_OK && (P.opts.max_fields < 1 || !(P.opts.eps > 0.0 && P.opts.eps < 1.0) ||
                      (P.opts.precision != SHT_FP64 && P.opts.precision != SHT_FP32 &&
                       P.opts.precision != SHT_MIXED) ||
                      !validate_program(P, err)))
    s = SHT_ERR_IO;
  // the statistics' identity fields must describe this program: callers size
  // their buffers from sht_plan_stats().N
  if (s == SHT_OK && (P.info.N != P.N || P.info.n_units != 2 * (int64_t)P.N ||
                      P.info.n_ops != (int64_t)P.ops.size() || !(P.info.eps == P.opts.eps)))
    s = SHT_ERR_IO;
  if (s == SHT_OK) {
    if (P.opts.flags & SHT_FLAG_HOST_ONLY) {
      p->host_only = true;
    } else {
      int ndev = 0;
      s = (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) ? SHT_ERR_CUDA : attach_device(p);
    }
  }
  if (s != SHT_OK) {
    delete p;
    return s;
  }
  *out = p;
  return SHT_OK;
}

sht_status sht_plan_nodes(sht_plan_t p, double* x, double* w) {
  if (!p || !x || !w) return SHT_ERR_ARG;
  std::memcpy(x, p->prog.x.data(), sizeof(double) * p->prog.x.size());
  std::memcpy(w, p->prog.w.data(), sizeof(double) * p->prog.w.size());
  return SHT_OK;
}

sht_status alt_forward(sht_plan_t p, const double* beta, double* g, int F, void* stream) {
  if (!p || F < 0) return SHT_ERR_ARG;
  if (F == 0) return SHT_OK;  // nothing to do: the pointers may be NULL
  if (!beta || !g) return SHT_ERR_ARG;
  return launch(p, true, beta, g, F, 0, 0, static_cast<cudaStream_t>(stream));
}

sht_status alt_inverse(sht_plan_t p, const double* g, double* beta, int F, void* stream) {
  if (!p || F < 0) return SHT_ERR_ARG;
  if (F == 0) return SHT_OK;
  if (!beta || !g) return SHT_ERR_ARG;
  return launch(p, false, g, beta, F, 0, 0, static_cast<cudaStream_t>(stream));
}

sht_status alt_forward_m(sht_plan_t p, int m, const double* beta_m, double* g_m, int F, void* stream) {
  if (!p || F < 0) return SHT_ERR_ARG;
  if (m <= -2 * p->prog.N || m >= 2 * p->prog.N) return SHT_ERR_ARG;
  if (F == 0) return SHT_OK;
  if (!beta_m || !g_m) return SHT_ERR_ARG;
  return launch(p, true, beta_m, g_m, F, 1, m, static_cast<cudaStream_t>(stream));
}

sht_status alt_inverse_m(sht_plan_t p, int m, const double* g_m, double* beta_m, int F, void* stream) {
  if (!p || F < 0) return SHT_ERR_ARG;
  if (m <= -2 * p->prog.N || m >= 2 * p->prog.N) return SHT_ERR_ARG;
  if (F == 0) return SHT_OK;
  if (!beta_m || !g_m) return SHT_ERR_ARG;
  return launch(p, false, g_m, beta_m, F, 1, m, static_cast<cudaStream_t>(stream));
}

sht_status sht_phi_synthesis(sht_plan_t p, const double* g, double* f, int F, void* stream) {
  if (!p || F < 0) return SHT_ERR_ARG;
  if (F == 0) return SHT_OK;
  if (!g || !f) return SHT_ERR_ARG;
  return launch_phi(p, g, f, F, false, static_cast<cudaStream_t>(stream));
}

sht_status sht_phi_analysis(sht_plan_t p, const double* f, double* g, int F, void* stream) {
  if (!p || F < 0) return SHT_ERR_ARG;
  if (F == 0) return SHT_OK;
  if (!g || !f) return SHT_ERR_ARG;
  return launch_phi(p, f, g, F, true, static_cast<cudaStream_t>(stream));
}

sht_status sht_forward(sht_plan_t p, const double* beta, double* f, int F, void* stream) {
  if (!p || F < 0) return SHT_ERR_ARG;
  if (F == 0) return SHT_OK;
  if (!beta || !f) return SHT_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t N = p->prog.N, ncoef = 4 * N * N * 2, nval = (4 * N - 1) * 2 * N * 2;
  for (int f0 = 0; f0 < F; f0 += p->prog.opts.max_fields) {
    const int n = std::min(F - f0, p->prog.opts.max_fields);
    sht_status s = launch(p, true, beta + f0 * ncoef, p->d_gws, n, 0, 0, st);
    if (s == SHT_OK) s = launch_phi(p, p->d_gws, f + f0 * nval, n, false, st);
    if (s != SHT_OK) return s;
  }
  return SHT_OK;
}

sht_status sht_inverse(sht_plan_t p, const double* f, double* beta, int F, void* stream) {
  if (!p || F < 0) return SHT_ERR_ARG;
  if (F == 0) return SHT_OK;
  if (!beta || !f) return SHT_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t N = p->prog.N, ncoef = 4 * N * N * 2, nval = (4 * N - 1) * 2 * N * 2;
  for (int f0 = 0; f0 < F; f0 += p->prog.opts.max_fields) {
    const int n = std::min(F - f0, p->prog.opts.max_fields);
    sht_status s = launch_phi(p, f + f0 * nval, p->d_gws, n, true, st);
    if (s == SHT_OK) s = launch(p, false, p->d_gws, beta + f0 * ncoef, n, 0, 0, st);
    if (s != SHT_OK) return s;
  }
  return SHT_OK;
}

sht_status sht_plan_kernel_time(sht_plan_t p, int reset, double* apply_ms, double* output_ms, int64_t* launches) {
  if (!p || !apply_ms || !output_ms || !launches) return SHT_ERR_ARG;
  if (p->tev.empty()) return SHT_ERR_UNSUPPORTED;
  const int64_t first = std::max(p->tev_base, p->tev_count - kTimingSlots);
  double a = 0.0, o = 0.0;
  for (int64_t k = first; k < p->tev_count; ++k) {
    cudaEvent_t* ev = p->tev.data() + 3 * (k % kTimingSlots);
    float t0 = 0.f, t1 = 0.f;
    if (cudaEventSynchronize(ev[2]) != cudaSuccess || cudaEventElapsedTime(&t0, ev[0], ev[1]) != cudaSuccess ||
        cudaEventElapsedTime(&t1, ev[1], ev[2]) != cudaSuccess)
      return SHT_ERR_CUDA;
    a += t0;
    o += p->prog.opts.precision == SHT_MIXED ? t1 : 0.0;  // only the tensor-core path has an output kernel
  }
  *apply_ms = a;
  *output_ms = o;
  *launches = p->tev_count - first;
  if (reset) p->tev_base = p->tev_count;
  return SHT_OK;
}

sht_status sht_plan_set_timing(sht_plan_t p, int enable) {
  if (!p) return SHT_ERR_ARG;
  if (p->tev.empty()) return SHT_ERR_UNSUPPORTED;
  p->timing_on = enable != 0;
  return SHT_OK;
}

sht_status sht_sync(sht_plan_t p, void* stream) {
  if (!p) return SHT_ERR_ARG;
  if (p->host_only) return SHT_ERR_UNSUPPORTED;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return SHT_ERR_CUDA;
  if (p->d_err) {
    int h = 0;
    if (cudaMemcpy(&h, p->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SHT_ERR_CUDA;
    if (h) {
      cudaMemset(p->d_err, 0, sizeof(int));
      return SHT_ERR_TIMEOUT;
    }
  }
  sht_status s = p->latched;
  p->latched = SHT_OK;
  return s;
}

const char* sht_status_str(sht_status s) {
  switch (s) {
    case SHT_OK: return "ok";
    case SHT_ERR_ARG: return "invalid argument";
    case SHT_ERR_OOM: return "out of memory";
    case SHT_ERR_CUDA: return "CUDA error or no device";
    case SHT_ERR_TIMEOUT: return "device wait timed out";
    case SHT_ERR_NUMERIC: return "precomputation did not reach the tolerance";
    case SHT_ERR_IO: return "plan file error";
    case SHT_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches of plans: several orders N, each with its own fields, in one launch
// of the tensor-core kernel.  The work items of all plans, (plan, |m|, field
// group), form one queue in decreasing order of estimated cost, so that the
// persistent kernel balances uneven transforms across the SMs.

struct sht_batch_s {
  int device = 0;
  int nplans = 0;
  sht_plan_s* plans[kTcMaxPlans] = {};
  int F[kTcMaxPlans] = {};
  int4* d_items = nullptr;
  int nitems = 0;
  unsigned char* d_ws = nullptr;
  int max_rows = 0;        // scratch rows of the largest order of all plans
  unsigned int* d_counter = nullptr;
  int* d_err = nullptr;
  int grid = 0;
};

namespace {

void free_batch(sht_batch_s* b) {
  cudaFree(b->d_items);
  cudaFree(b->d_ws);
  cudaFree(b->d_counter);
  cudaFree(b->d_err);
}

sht_status launch_batch(sht_batch_s* b, bool fwd, const double* const* in, double* const* out, cudaStream_t st) {
  TcLaunch L;
  std::memset(&L, 0, sizeof(L));
  for (int q = 0; q < b->nplans; ++q) {
    sht_plan_s* p = b->plans[q];
    if (b->F[q] > 0) {
      if (!in[q] || !out[q]) return SHT_ERR_ARG;
      if ((reinterpret_cast<uintptr_t>(in[q]) | reinterpret_cast<uintptr_t>(out[q])) & 15u) return SHT_ERR_ARG;
    }
    if (p->latched != SHT_OK) {
      sht_status s = p->latched;
      p->latched = SHT_OK;
      return s;
    }
    L.plan[q] = tc_plan_of(p);
    L.in[q] = in[q];
    L.out[q] = out[q];
    L.F[q] = b->F[q];
  }
  if (b->nitems == 0) return SHT_OK;
  L.nplans = b->nplans;
  L.items = b->d_items;
  L.nitems = b->nitems;
  L.ws = b->d_ws;
  L.max_rows = b->max_rows;
  L.counter = b->d_counter;
  L.err = b->d_err;
  if (cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned int), st) != cudaSuccess) return SHT_ERR_CUDA;
  if (launch_tc_batch(L, fwd, std::min(b->grid, b->nitems), st) != cudaSuccess) return SHT_ERR_CUDA;
  return SHT_OK;
}

}  // namespace

extern "C" {

sht_status sht_batch_create(int P, const sht_plan_t* plans, const int* fields, sht_batch_t* out) {
  if (!out || !plans || !fields || P < 1 || P > kTcMaxPlans) return SHT_ERR_ARG;
  *out = nullptr;
  int dev = 0;
  for (int q = 0; q < P; ++q) {
    if (!plans[q] || fields[q] < 0) return SHT_ERR_ARG;
    for (int r = 0; r < q; ++r)
      if (plans[r] == plans[q]) return SHT_ERR_ARG;  // each plan's accumulation rows serve one batch slot
    if (plans[q]->host_only || plans[q]->direct || plans[q]->prog.opts.precision != SHT_MIXED)
      return SHT_ERR_UNSUPPORTED;
    if (fields[q] > plans[q]->prog.opts.max_fields) return SHT_ERR_ARG;
    if ((int64_t)fields[q] * 2 * plans[q]->prog.N > (int64_t)1 << 30) return SHT_ERR_ARG;
  }
  if (cudaGetDevice(&dev) != cudaSuccess) return SHT_ERR_CUDA;
  for (int q = 0; q < P; ++q)
    if (plans[q]->device != dev) return SHT_ERR_ARG;
  sht_batch_s* b = new (std::nothrow) sht_batch_s();
  if (!b) return SHT_ERR_OOM;
  alloc_hook_reset();
  b->device = dev;
  b->nplans = P;
  // the queue: every (plan, |m|, field group), in decreasing estimated cost
  // (flops per right-hand side of the order), ties by plan, order and group
  struct Entry {
    float cost;
    int4 it;
  };
  std::vector<Entry> q;
  for (int k = 0; k < P; ++k) {
    const sht_plan_s* p = plans[k];
    b->plans[k] = plans[k];
    b->F[k] = fields[k];
    b->max_rows = std::max(b->max_rows, p->tc_max_rows);
    const int G = (fields[k] + kTcFields - 1) / kTcFields;
    for (const Unit& u : p->prog.units)
      for (int g = 0; g < G; ++g) q.push_back({u.cost, make_int4(k, u.am, g, 0)});
  }
  std::stable_sort(q.begin(), q.end(), [](const Entry& a, const Entry& c) { return a.cost > c.cost; });
  std::vector<int4> items(q.size());
  for (size_t i = 0; i < q.size(); ++i) items[i] = q[i].it;
  b->nitems = (int)items.size();
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->grid = std::max(1, sms * tc_ctas_per_sm());
  const size_t ws = (size_t)b->grid * 2 * tc_slot_bytes(b->max_rows);
  cudaError_t e = plan_malloc(reinterpret_cast<void**>(&b->d_items), std::max<size_t>(items.size(), 1) * sizeof(int4));
  if (e == cudaSuccess && !items.empty())
    e = cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = plan_malloc(reinterpret_cast<void**>(&b->d_ws), ws);
  // rows that widened K chunks read but no op writes must hold finite values
  if (e == cudaSuccess) e = cudaMemset(b->d_ws, 0, ws);
  if (e == cudaSuccess) e = plan_malloc(reinterpret_cast<void**>(&b->d_counter), sizeof(unsigned int));
  if (e == cudaSuccess) e = plan_malloc(reinterpret_cast<void**>(&b->d_err), sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_batch(b);
    delete b;
    return e == cudaErrorMemoryAllocation ? SHT_ERR_OOM : SHT_ERR_CUDA;
  }
  *out = b;
  return SHT_OK;
}

sht_status sht_batch_destroy(sht_batch_t b) {
  if (!b) return SHT_ERR_ARG;
  cudaSetDevice(b->device);
  free_batch(b);
  delete b;
  return SHT_OK;
}

sht_status alt_forward_batch(sht_batch_t b, const double* const* beta, double* const* g, void* stream) {
  if (!b || !beta || !g) return SHT_ERR_ARG;
  return launch_batch(b, true, beta, g, static_cast<cudaStream_t>(stream));
}

sht_status alt_inverse_batch(sht_batch_t b, const double* const* g, double* const* beta, void* stream) {
  if (!b || !g || !beta) return SHT_ERR_ARG;
  return launch_batch(b, false, g, beta, static_cast<cudaStream_t>(stream));
}

sht_status sht_forward_batch(sht_batch_t b, const double* const* beta, double* const* f, void* stream) {
  if (!b || !beta || !f) return SHT_ERR_ARG;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the ALT values of every plan's fields pass through that plan's workspace
  double* gws[kTcMaxPlans] = {};
  for (int q = 0; q < b->nplans; ++q) gws[q] = b->plans[q]->d_gws;
  sht_status s = launch_batch(b, true, beta, gws, st);
  for (int q = 0; q < b->nplans && s == SHT_OK; ++q)
    if (b->F[q] > 0) {
      if (!f[q] || (reinterpret_cast<uintptr_t>(f[q]) & 15u)) return SHT_ERR_ARG;
      s = launch_phi(b->plans[q], gws[q], f[q], b->F[q], false, st);
    }
  return s;
}

sht_status sht_inverse_batch(sht_batch_t b, const double* const* f, double* const* beta, void* stream) {
  if (!b || !f || !beta) return SHT_ERR_ARG;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double* gws[kTcMaxPlans] = {};
  for (int q = 0; q < b->nplans; ++q) {
    gws[q] = b->plans[q]->d_gws;
    if (b->F[q] > 0) {
      if (!f[q] || (reinterpret_cast<uintptr_t>(f[q]) & 15u)) return SHT_ERR_ARG;
      const sht_status s = launch_phi(b->plans[q], f[q], b->plans[q]->d_gws, b->F[q], true, st);
      if (s != SHT_OK) return s;
    }
  }
  return launch_batch(b, false, gws, beta, st);
}

sht_status sht_selftest_timeout(sht_plan_t p, void* stream) {
  if (!p) return SHT_ERR_ARG;
  if (p->host_only || p->direct || p->prog.opts.precision != SHT_MIXED) return SHT_ERR_UNSUPPORTED;
  return launch_tc_stall(tc_plan_of(p), p->d_wstc, p->d_counter, p->d_err,
                         static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? SHT_OK
             : SHT_ERR_CUDA;
}

sht_status sht_legendre(sht_plan_t p, int am, double* out, void* stream) {
  if (!p || !out || am < 0 || am >= 2 * p->prog.N) return SHT_ERR_ARG;
  if (p->host_only || !p->leg.d_x || !p->d_legcoef) return SHT_ERR_UNSUPPORTED;
  return p->leg.table(am, out, p->d_legcoef, static_cast<cudaStream_t>(stream)) == cudaSuccess ? SHT_OK
                                                                                                 : SHT_ERR_CUDA;
}

sht_status sht_plan_set_order(sht_plan_t p, const int32_t* order, int n) {
  if (!p || !order || n != 2 * p->prog.N) return SHT_ERR_ARG;
  if (p->direct) return SHT_ERR_UNSUPPORTED;
  std::vector<char> seen((size_t)n, 0);
  for (int q = 0; q < n; ++q) {
    if (order[q] < 0 || order[q] >= n || seen[(size_t)order[q]]) return SHT_ERR_ARG;
    seen[(size_t)order[q]] = 1;
  }
  if (!p->host_only) {
    if (cudaDeviceSynchronize() != cudaSuccess) return SHT_ERR_CUDA;
    if (cudaMemcpy(p->d_order, order, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess)
      return SHT_ERR_CUDA;
  }
  std::copy(order, order + n, p->prog.order.begin());
  return SHT_OK;
}

sht_status sht_selftest_convert(const double* f64, float* f32, double* back, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!f64 || !f32 || !back))) return SHT_ERR_ARG;
  if (n == 0) return SHT_OK;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  convert_selftest_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(f64, f32, back, n);
  return cudaGetLastError() == cudaSuccess ? SHT_OK : SHT_ERR_CUDA;
}

sht_status sht_batch_sync(sht_batch_t b, void* stream) {
  if (!b) return SHT_ERR_ARG;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return SHT_ERR_CUDA;
  int h = 0;
  if (cudaMemcpy(&h, b->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SHT_ERR_CUDA;
  if (h) {
    cudaMemset(b->d_err, 0, sizeof(int));
    return SHT_ERR_TIMEOUT;
  }
  return SHT_OK;
}

}  // extern "C"

extern "C" sht_status alt_forward_m_noalloc(sht_plan_t p, int m, const double* beta_m, double* g_m, int F,
                                            void* stream) {
  if (!p || F < 0) return SHT_ERR_ARG;
  if (m <= -2 * p->prog.N || m >= 2 * p->prog.N) return SHT_ERR_ARG;
  if (F == 0) return SHT_OK;
  if (!beta_m || !g_m) return SHT_ERR_ARG;
  if (p->host_only || !p->d_fac) return SHT_ERR_UNSUPPORTED;  // runs the FP64 kernels: FP64 plans only
  if ((reinterpret_cast<uintptr_t>(beta_m) | reinterpret_cast<uintptr_t>(g_m)) & 15u) return SHT_ERR_ARG;
  if ((int64_t)F * 2 * p->prog.N > (int64_t)1 << 30) return SHT_ERR_ARG;
  // one CTA's vector space must fit next to the counter
  const size_t slot = (size_t)p->prog.max_rows * kRT * sizeof(double);
  if (slot == 0 || slot > kNoAllocScratchBytes - kNoAllocCounterBytes) return SHT_ERR_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return SHT_ERR_ARG;
  unsigned char* base = p->d_noalloc;  // looked up when the plan was created
  if (!base) return SHT_ERR_CUDA;
  if (p->latched != SHT_OK) {
    const sht_status s = p->latched;
    p->latched = SHT_OK;
    return s;
  }
  const int slots = (int)((kNoAllocScratchBytes - kNoAllocCounterBytes) / slot);
  const int grid = std::max(1, std::min(std::min(slots, p->nslots), F));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DevPlan d = dev_plan(p);
  d.counter = reinterpret_cast<unsigned int*>(base);  // must start at zero: cleared below
  d.ws = reinterpret_cast<double*>(base + kNoAllocCounterBytes);
  if (cudaMemsetAsync(d.counter, 0, sizeof(unsigned int), st) != cudaSuccess) return SHT_ERR_CUDA;
  cudaEvent_t* ev = timing_slot(p);  // SHT_FLAG_TIMING plans: counted like every other apply launch
  if (ev && cudaEventRecord(ev[0], st) != cudaSuccess) return SHT_ERR_CUDA;
  alt_forward_f64_kernel<<<grid, kThreads, 0, st>>>(d, beta_m, g_m, F, 1, m);
  if (cudaGetLastError() != cudaSuccess) return SHT_ERR_CUDA;
  if (ev && (cudaEventRecord(ev[1], st) != cudaSuccess || cudaEventRecord(ev[2], st) != cudaSuccess))
    return SHT_ERR_CUDA;
  return SHT_OK;
}
