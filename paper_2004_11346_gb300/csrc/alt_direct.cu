// Dense ALT with the Legendre recurrence run on the fly: the O(N^3) baseline
// that stores nothing between calls, so that it serves any N the nodes fit.
//
//   forward (Eq. sht_lt): g(m, theta_l) = sum_{k=|m|}^{2N-1} beta_{k,m} Pbar_k^{|m|}(x_l)
//   inverse (Sec. 3.1.1): beta_{k,m} = sum_l w_l Pbar_k^{|m|}(x_l) g(m, theta_l)
//
// in FP64.  Both orders +a and -a share Pbar^a, and the parity
// Pbar_k^a(-x) = (-1)^{k-a} Pbar_k^a(x) (Sec. 3.1.2) lets every product run
// over the N positive nodes x_{N+i} only: with S_e, S_o the sums over the
// degrees of even and odd k - a, g(x_{N+i}) = S_e + S_o and
// g(x_{N-1-i}) = S_e - S_o; for the inverse, the even degrees contract with
// u_e(i) = w_{N+i} (g(x_{N+i}) + g(x_{N-1-i})) and the odd ones with
// u_o(i) = w_{N+i} (g(x_{N+i}) - g(x_{N-1-i})).
//
// A persistent CTA takes orders a = 0, 1, ... (decreasing work 2N - a) from
// an atomic counter and, for each, in its own global scratch:
//   1. the recurrence coefficients of the order (one per degree);
//   2. Pbar_k^a(x_{N+i}) for every degree and positive node (one thread per
//      node, sequential in k): the normalised three-term recurrence from
//      Pbar_a^a = c_a (1 - x^2)^{a/2}, carried as mantissa and binary
//      exponent while the values are below the FP64 range (they grow
//      monotonically until the turning point); values still below 2^-760
//      are stored as zero, which changes no sum by more than that;
//   3. the right-hand sides packed per degree (forward: beta_{k,+-a} of every
//      field, real and imaginary parts) or per node (inverse: u_e, u_o);
//   4. the products, as 64 x 64 output tiles of a shared-memory FP64 GEMM.
// Nothing waits on another CTA.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "alt_direct.cuh"

namespace sht {

namespace {

constexpr int kDThreads = 256;
constexpr int kDTile = 64;   // output tile (rows x right-hand sides)
constexpr int kDChunk = 16;  // reduction step staged in shared memory
constexpr int kDScaleBits = 200;
constexpr int kDPlainExp = -960;  // binary exponent at which values become plain doubles

__device__ __forceinline__ long order_slot(long m) { return m == 0 ? 0 : (m > 0 ? 2 * m - 1 : -2 * m); }
// first coefficient of order m: orders before it hold 2N - |m'| degrees each
__device__ __forceinline__ long coef_offset(long N, long m) {
  const long a = m < 0 ? -m : m;
  if (a == 0) return 0;
  const long pos = 2 * N * (2 * a - 1) - a * (a - 1);
  return m > 0 ? pos : pos + (2 * N - a);
}

struct DirectArgs {
  int N, F, R, fwd;
  const double* in;
  double* out;
  const double *x, *s, *w, *cm;
  double* scratch;
  size_t per_cta;
  unsigned int* counter;
};

// Right-hand side j of order a: field j / 4, order +a (bit 1 clear) or -a,
// real (bit 0 clear) or imaginary part; order -0 does not exist.
__device__ __forceinline__ bool rhs_valid(int j, int a, int F) { return j < 4 * F && (a > 0 || (j & 2) == 0); }

// s^a as mantissa * 2^e, by squaring with the exponent kept apart
__device__ void pow_ext(double s, int a, double& mant, int& e) {
  int eb;
  double b = frexp(s, &eb);
  mant = 1.0;
  e = 0;
  while (a) {
    int t;
    if (a & 1) {
      mant = frexp(mant * b, &t);
      e += eb + t;
    }
    a >>= 1;
    if (a) {
      b = frexp(b * b, &t);
      eb = 2 * eb + t;
    }
  }
}

// The recurrence coefficients of order a for degrees a + t, t in [t0, K),
// stepping by `stride` from t0: coef[2t] = sqrt((4k^2 - 1) / (k^2 - a^2)),
// coef[2t + 1] = sqrt((2k + 1)(k - 1 - a)(k - 1 + a) / ((2k - 3)(k^2 - a^2))),
// k = a + t, t >= 1 (0 for t = 1, where Pbar_{a-1}^a does not exist).
__device__ __forceinline__ void legendre_coefs(int a, int K, int t0, int stride, double* coef) {
  for (int t = t0; t < K; t += stride) {
    if (t < 1) continue;
    const double k = (double)(a + t), aa = (double)a;
    const double d = k * k - aa * aa;
    coef[2 * t] = sqrt((4.0 * k * k - 1.0) / d);
    coef[2 * t + 1] = t >= 2 ? sqrt((2.0 * k + 1.0) * (k - 1.0 - aa) * (k - 1.0 + aa) / ((2.0 * k - 3.0) * d)) : 0.0;
  }
}

// Pbar_{a+t}^a(x) for t < K into P[t * ld], one node: from
// Pbar_a^a = c_a s^a (s = sqrt(1 - x^2)), carried as mantissa and binary
// exponent while below the FP64 range, plain doubles from exponent -960 on;
// values still below that are stored as 0 (they are below 2^-760).
__device__ __forceinline__ void legendre_node(double x, double s, double ca, int a, int K, const double* coef,
                                              double* P, size_t ld) {
  double cur;
  int e;
  pow_ext(s, a, cur, e);
  cur *= ca;
  double prev = 0.0;
  bool plain = e >= kDPlainExp;
  if (plain) cur = ldexp(cur, e);
  for (int t = 0; t < K; ++t) {
    P[(size_t)t * ld] = plain ? cur : 0.0;
    if (t + 1 < K) {
      const double nx = coef[2 * (t + 1)] * x * cur - coef[2 * (t + 1) + 1] * prev;
      prev = cur;
      cur = nx;
      if (!plain && fabs(cur) > 0x1p200) {
        cur = ldexp(cur, -kDScaleBits);
        prev = ldexp(prev, -kDScaleBits);
        e += kDScaleBits;
        if (e >= kDPlainExp) {
          cur = ldexp(cur, e);
          prev = ldexp(prev, e);
          plain = true;
        }
      }
    }
  }
}

// Steps 1 and 2 for order a: coefficients, then Pbar_{a+t}^a(x_{N+i}) into
// P[t * N + i], t < K = 2N - a.
__device__ void direct_legendre(const DirectArgs& g, int a, double* coef, double* P) {
  const int N = g.N, K = 2 * N - a;
  legendre_coefs(a, K, threadIdx.x, blockDim.x, coef);
  __syncthreads();
  for (int i = threadIdx.x; i < N; i += blockDim.x) legendre_node(g.x[i], g.s[i], g.cm[a], a, K, coef, P + i, N);
}

// The same table for one order as a grid of its own: coefficients first (one
// kernel), then one thread per node.
__global__ void legendre_coef_kernel(int a, int K, double* coef) {
  legendre_coefs(a, K, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, coef);
}
__global__ void legendre_table_kernel(int N, int a, const double* __restrict__ x, const double* __restrict__ s,
                                      const double* __restrict__ cm, const double* __restrict__ coef, double* P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) legendre_node(x[i], s[i], cm[a], a, 2 * N - a, coef, P + i, N);
}

// Step 3, forward: B[t * R + j] = the degree-(a + t) coefficient of right-hand
// side j (zero for the padding columns).
__device__ void direct_pack_forward(const DirectArgs& g, int a, double* B) {
  const int N = g.N, K = 2 * N - a, R = g.R;
  const long ncoef = 4L * N * N;  // complex coefficients per field
  for (long idx = threadIdx.x; idx < (long)R * K; idx += blockDim.x) {
    const int j = (int)(idx / K), t = (int)(idx - (long)j * K);  // degrees fastest: reads follow beta
    double v = 0.0;
    if (rhs_valid(j, a, g.F)) {
      const int f = j >> 2, m = (j & 2) ? -a : a;
      v = g.in[2 * ((long)f * ncoef + coef_offset(N, m) + t) + (j & 1)];
    }
    B[(size_t)t * R + j] = v;
  }
}

// Step 3, inverse: U[(p * N + i) * R + j], p = 0 for u_e, 1 for u_o.
__device__ void direct_pack_inverse(const DirectArgs& g, int a, double* U) {
  const int N = g.N, R = g.R, M = 4 * N - 1;
  for (long idx = threadIdx.x; idx < (long)R * N; idx += blockDim.x) {
    const int j = (int)(idx / N), i = (int)(idx - (long)j * N);  // nodes fastest: reads follow g
    double ue = 0.0, uo = 0.0;
    if (rhs_valid(j, a, g.F)) {
      const int f = j >> 2, m = (j & 2) ? -a : a;
      const double* gv = g.in + 2 * (((long)f * M + order_slot(m)) * 2 * N);
      const double hi = gv[2 * (N + i) + (j & 1)], lo = gv[2 * (N - 1 - i) + (j & 1)];
      ue = g.w[i] * (hi + lo);
      uo = g.w[i] * (hi - lo);
    }
    U[(size_t)i * R + j] = ue;
    U[((size_t)N + i) * R + j] = uo;
  }
}

// Step 4, forward: for nodes i and right-hand sides j, S_e and S_o over the
// degrees, then g at x_{N+i} and x_{N-1-i}.  Thread (tx, ty) of a 16 x 16
// layout holds nodes ty * 4 + r and right-hand sides tx * 4 + c of the tile.
__device__ void direct_gemm_forward(const DirectArgs& g, int a, const double* P, const double* B, double* sm) {
  const int N = g.N, K = 2 * N - a, R = g.R, M = 4 * N - 1;
  double* Ps = sm;                      // [kDChunk][kDTile] node values per degree
  double* Bs = sm + kDChunk * kDTile;   // [kDChunk][kDTile] right-hand sides per degree
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int ntile_i = (N + kDTile - 1) / kDTile, ntile_j = R / kDTile;
  for (int tile = 0; tile < ntile_i * ntile_j; ++tile) {
    const int i0 = (tile / ntile_j) * kDTile, j0 = (tile % ntile_j) * kDTile;
    double se[4][4] = {}, so[4][4] = {};
    for (int t0 = 0; t0 < K; t0 += kDChunk) {
      for (int q = threadIdx.x; q < kDChunk * kDTile; q += blockDim.x) {
        const int kk = q / kDTile, c = q % kDTile, t = t0 + kk, i = i0 + c;
        Ps[q] = (t < K && i < N) ? P[(size_t)t * N + i] : 0.0;
        Bs[q] = t < K ? B[(size_t)t * R + j0 + c] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < kDChunk; ++kk) {
        double pv[4], bv[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) pv[r] = Ps[kk * kDTile + ty * 4 + r];
#pragma unroll
        for (int c = 0; c < 4; ++c) bv[c] = Bs[kk * kDTile + tx * 4 + c];
        // t0 is even: the parity of kk is that of k - a
        if ((kk & 1) == 0) {
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) se[r][c] = fma(pv[r], bv[c], se[r][c]);
        } else {
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) so[r][c] = fma(pv[r], bv[c], so[r][c]);
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + tx * 4 + c;
      if (!rhs_valid(j, a, g.F)) continue;
      const int f = j >> 2, m = (j & 2) ? -a : a;
      double* gv = g.out + 2 * (((long)f * M + order_slot(m)) * 2 * N) + (j & 1);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = i0 + ty * 4 + r;
        if (i < N) {
          gv[2 * (N + i)] = se[r][c] + so[r][c];
          gv[2 * (N - 1 - i)] = se[r][c] - so[r][c];
        }
      }
    }
  }
}

// Step 4, inverse: beta_{a+t} = sum_i P[t][i] U_p(t)[i] over the nodes, p(t)
// the parity of t.  Thread (tx, ty) holds degrees t0 + ty + 16 r (one parity,
// that of ty) and right-hand sides tx * 4 + c of the tile.
__device__ void direct_gemm_inverse(const DirectArgs& g, int a, const double* P, const double* U, double* sm) {
  const int N = g.N, K = 2 * N - a, R = g.R;
  const long ncoef = 4L * N * N;
  constexpr int ld = kDTile + 1;                // padded: the transposing stores hit distinct banks
  double* Ps = sm;                              // [kDChunk nodes][ld] degrees
  double* Ue = sm + kDChunk * ld;               // [kDChunk nodes][kDTile rhs]
  double* Uo = Ue + kDChunk * kDTile;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int ntile_t = (K + kDTile - 1) / kDTile, ntile_j = R / kDTile;
  for (int tile = 0; tile < ntile_t * ntile_j; ++tile) {
    const int t0 = (tile / ntile_j) * kDTile, j0 = (tile % ntile_j) * kDTile;
    double acc[4][4] = {};
    const double* Us = (ty & 1) ? Uo : Ue;
    for (int i0 = 0; i0 < N; i0 += kDChunk) {
      for (int q = threadIdx.x; q < kDChunk * kDTile; q += blockDim.x) {
        // P: degree q / kDChunk, node q % kDChunk (nodes contiguous in P)
        const int dt = q / kDChunk, ii = q % kDChunk, t = t0 + dt, i = i0 + ii;
        Ps[ii * ld + dt] = (t < K && i < N) ? P[(size_t)t * N + i] : 0.0;
        const int kk = q / kDTile, c = q % kDTile, iu = i0 + kk;
        Ue[q] = iu < N ? U[(size_t)iu * R + j0 + c] : 0.0;
        Uo[q] = iu < N ? U[((size_t)N + iu) * R + j0 + c] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int ii = 0; ii < kDChunk; ++ii) {
        double pv[4], uv[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) pv[r] = Ps[ii * ld + ty + 16 * r];
#pragma unroll
        for (int c = 0; c < 4; ++c) uv[c] = Us[ii * kDTile + tx * 4 + c];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = fma(pv[r], uv[c], acc[r][c]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + tx * 4 + c;
      if (!rhs_valid(j, a, g.F)) continue;
      const int f = j >> 2, m = (j & 2) ? -a : a;
      double* bv = g.out + 2 * ((long)f * ncoef + coef_offset(N, m)) + (j & 1);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int t = t0 + ty + 16 * r;
        if (t < K) bv[2 * t] = acc[r][c];
      }
    }
  }
}

__global__ void __launch_bounds__(kDThreads) alt_direct_kernel(DirectArgs g) {
  __shared__ double sm[3 * kDChunk * (kDTile + 1)];
  __shared__ int s_order;
  double* base = g.scratch + (size_t)blockIdx.x * g.per_cta;
  const int N = g.N;
  double* coef = base;                       // 2 * 2N
  double* P = base + 4 * (size_t)N;          // 2N * N
  double* X = P + 2 * (size_t)N * N;         // forward 2N * R, inverse 2 * N * R
  for (;;) {
    if (threadIdx.x == 0) s_order = (int)atomicAdd(g.counter, 1u);
    __syncthreads();
    const int a = s_order;
    __syncthreads();
    if (a >= 2 * N) break;
    direct_legendre(g, a, coef, P);
    if (g.fwd)
      direct_pack_forward(g, a, X);
    else
      direct_pack_inverse(g, a, X);
    __syncthreads();
    if (g.fwd)
      direct_gemm_forward(g, a, P, X, sm);
    else
      direct_gemm_inverse(g, a, P, X, sm);
    __syncthreads();
  }
}

}  // namespace

// c_a = Pbar_a^a(x) / (1 - x^2)^{a/2}: c_0 = 1 / sqrt(2), c_a = c_{a-1} sqrt((2a + 1) / (2a))
static std::vector<double> sectoral_constants(int n) {
  std::vector<double> c(n);
  long double v = 1.0L / std::sqrt(2.0L);
  for (int a = 0; a < n; ++a) {
    if (a > 0) v *= std::sqrt((2.0L * a + 1.0L) / (2.0L * a));
    c[a] = (double)v;
  }
  return c;
}

cudaError_t LegendreDev::build(int N_, const double* x) {
  N = N_;
  std::vector<double> xp(N), sp(N);
  for (int i = 0; i < N; ++i) {
    const long double xi = x[N + i];
    xp[i] = x[N + i];
    sp[i] = (double)std::sqrt((1.0L - xi) * (1.0L + xi));
  }
  const std::vector<double> cm = sectoral_constants(2 * N);
  cudaError_t e = cudaSuccess;
  auto up = [&](double** d, const std::vector<double>& h) {
    if (e == cudaSuccess) e = cudaMalloc(d, h.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(*d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice);
  };
  up(&d_x, xp);
  up(&d_s, sp);
  up(&d_cm, cm);
  return e;
}

void LegendreDev::release() {
  cudaFree(d_x);
  cudaFree(d_s);
  cudaFree(d_cm);
  d_x = d_s = d_cm = nullptr;
}

cudaError_t LegendreDev::table(int am, double* out, double* coef, cudaStream_t st) const {
  if (am < 0 || am >= 2 * N || !d_x) return cudaErrorInvalidValue;
  const int K = 2 * N - am;
  legendre_coef_kernel<<<std::max(1, (K + 255) / 256), 256, 0, st>>>(am, K, coef);
  legendre_table_kernel<<<std::max(1, (N + 127) / 128), 128, 0, st>>>(N, am, d_x, d_s, d_cm, coef, out);
  return cudaGetLastError();
}

cudaError_t DirectPlan::build(int N_, int F_, const double* x, const double* w, int sms) {
  N = N_;
  F_max = F_;
  R_max = (4 * F_max + kDTile - 1) / kDTile * kDTile;
  // coefficients 4N, Pbar 2N x N, right-hand sides max(2N x R, 2 x N x R)
  per_cta = 4 * (size_t)N + 2 * (size_t)N * N + 2 * (size_t)N * R_max;
  std::vector<double> xp(N), sp(N), wp(N);
  for (int i = 0; i < N; ++i) {
    const long double xi = x[N + i];
    xp[i] = x[N + i];
    sp[i] = (double)std::sqrt((1.0L - xi) * (1.0L + xi));
    wp[i] = w[N + i];
  }
  const std::vector<double> cm = sectoral_constants(2 * N);
  cudaError_t e = cudaSuccess;
  auto up = [&](double** d, const std::vector<double>& h) {
    if (e == cudaSuccess) e = cudaMalloc(d, h.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(*d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice);
  };
  up(&d_x, xp);
  up(&d_s, sp);
  up(&d_w, wp);
  up(&d_cm, cm);
  // one CTA per SM while the scratch stays within an eighth of the free memory
  size_t free_b = 0, total_b = 0;
  if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
  if (e == cudaSuccess) {
    const size_t cta_bytes = per_cta * sizeof(double);
    grid = (int)std::max<size_t>(1, std::min<size_t>((size_t)sms, free_b / 8 / cta_bytes));
    e = cudaMalloc(&d_scratch, (size_t)grid * cta_bytes);
  }
  if (e == cudaSuccess) e = cudaMalloc(&d_counter, sizeof(unsigned int));
  return e;
}

void DirectPlan::release() {
  cudaFree(d_x);
  cudaFree(d_s);
  cudaFree(d_w);
  cudaFree(d_cm);
  cudaFree(d_scratch);
  cudaFree(d_counter);
  d_x = d_s = d_w = d_cm = d_scratch = nullptr;
  d_counter = nullptr;
}

cudaError_t DirectPlan::launch(bool fwd, const double* in, double* out, int F, cudaStream_t st) const {
  if (F < 1 || F > F_max || !d_scratch) return cudaErrorInvalidValue;
  DirectArgs g;
  g.N = N;
  g.F = F;
  g.R = (4 * F + kDTile - 1) / kDTile * kDTile;
  g.fwd = fwd ? 1 : 0;
  g.in = in;
  g.out = out;
  g.x = d_x;
  g.s = d_s;
  g.w = d_w;
  g.cm = d_cm;
  g.scratch = d_scratch;
  g.per_cta = per_cta;
  g.counter = d_counter;
  cudaError_t e = cudaMemsetAsync(d_counter, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  alt_direct_kernel<<<grid, kDThreads, 0, st>>>(g);
  return cudaGetLastError();
}

}  // namespace sht
