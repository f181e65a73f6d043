// phi-direction DFT of the SHT (Eq. sht_fft), batched over nodes and fields.
//
//   synthesis: f(theta_l, phi_j) = sum_{m=-(2N-1)}^{2N-1} g(m, theta_l) e^{i m phi_j}
//   analysis:  g(m, theta_l)     = (1/M) sum_{j=0}^{M-1} f(theta_l, phi_j) e^{-i m phi_j}
//
// with M = 4N-1 samples phi_j = 2 pi (j + 1/2) / M.  Writing
// e^{i m phi_j} = e^{i pi m / M} e^{2 pi i m j / M}, synthesis is a length-M
// DFT of c[m mod M] = g(m) e^{i pi m / M}, and analysis is the conjugate
// transform followed by the conjugate shift.  One CTA transforms one
// (node, field) row in shared memory with a self-sorting mixed-radix
// (Stockham) FFT over the factors of M; every pass reads its twiddles from a
// host-built table e^{+2 pi i t / (Ns R)}, t < Ns R.  The shift factors
// e^{i pi m / M} come from a table too.  Arithmetic type T is double or float;
// inputs and outputs are FP64 complex.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "f64_bits.cuh"
#include "phi_dft.cuh"

namespace sht {

template <class T>
struct C2 {
  T x, y;
};

namespace {

// threads per CTA: FP32 rows fit three CTAs per SM; an FP64 row's two buffers
// take most of shared memory, so its single CTA carries more warps
template <class T>
struct PhiThreads {
  static constexpr int value = sizeof(T) == 8 ? 512 : 256;
};

__device__ __forceinline__ long order_slot(long m) { return m == 0 ? 0 : (m > 0 ? 2 * m - 1 : -2 * m); }

// FP64 I/O values to and from the arithmetic type (integer conversions for FP32)
template <class T>
__device__ __forceinline__ T from_f64(double v);
template <>
__device__ __forceinline__ double from_f64<double>(double v) { return v; }
template <>
__device__ __forceinline__ float from_f64<float>(double v) { return f64_to_f32_bits(v); }
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) { return f32_to_f64_bits(v); }

template <class T>
__device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
  return C2<T>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// One Stockham pass of radix R: y[idxD + k Ns] = sum_r x[j + r n/R] w^{r (j%Ns + k Ns)}
// with w = e^{s 2 pi i / (Ns R)} (s = +1 synthesis, -1 analysis via conjugation).
// Generic form (any R): every output re-reads its R inputs; used only for
// radices without a specialised butterfly (prime factors of M above 13).
template <class T>
__device__ void stockham_pass(const C2<T>* __restrict__ x, C2<T>* __restrict__ y, int n, int R, int Ns,
                              const C2<T>* __restrict__ tw, bool conj) {
  const int nb = n / R, NsR = Ns * R;
  for (int o = threadIdx.x; o < n; o += blockDim.x) {
    const int j = o % nb, k = o / nb;  // butterfly j, output k of it
    const int q = j % Ns + k * Ns;     // in [0, Ns R)
    const int idxD = (j / Ns) * NsR + (j % Ns);
    T ax = 0, ay = 0;
    int t = 0;  // (r q) mod Ns R
    for (int r = 0; r < R; ++r) {
      const C2<T> v = x[j + r * nb];
      C2<T> w = tw[t];
      if (conj) w.y = -w.y;
      ax += v.x * w.x - v.y * w.y;
      ay += v.x * w.y + v.y * w.x;
      t += q;
      if (t >= NsR) t -= NsR;
    }
    y[idxD + k * Ns] = C2<T>{ax, ay};
  }
}

// The same pass for a fixed small odd radix.  The phase factor splits as
// w^{r (jn + k Ns)} = w^{r jn} * omega^{r k} (jn = j mod Ns, omega =
// e^{s 2 pi i / R} = w^{Ns}): each thread takes whole butterflies, loads the
// R inputs once and applies the R-1 twiddles w^{r jn} (r jn < Ns R, a table
// entry).  The R-point DFT that remains pairs outputs k and R-k: with
// P_r = v_r + v_{R-r}, Q_r = v_r - v_{R-r} (r = 1..h, h = (R-1)/2),
//   y_k, y_{R-k} = v_0 + sum_r P_r cos(2 pi r k / R) +- i sum_r Q_r s sin(2 pi r k / R),
// about a quarter of the multiplications of the direct R x R product.
template <class T, int R>
__device__ void stockham_pass_r(const C2<T>* __restrict__ x, C2<T>* __restrict__ y, int n, int Ns,
                                const C2<T>* __restrict__ tw, bool conj) {
  static_assert(R % 2 == 1, "odd radix");
  constexpr int h = (R - 1) / 2;
  const int nb = n / R;
  const T sg = conj ? T(-1) : T(1);
  T cs[h + 1], sn[h + 1];  // cos and s*sin of 2 pi t / R, t = 0..h
#pragma unroll
  for (int t = 0; t <= h; ++t) {
    const C2<T> w = tw[t * Ns];
    cs[t] = w.x;
    sn[t] = sg * w.y;
  }
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    const int jn = j % Ns;
    const int idxD = (j - jn) * R + jn;  // (j / Ns) * Ns R + jn
    C2<T> v[R];
    v[0] = x[j];
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = x[j + r * nb];
#pragma unroll
    for (int r = 1; r < R; ++r) {
      C2<T> w = tw[r * jn];
      w.y *= sg;
      v[r] = cmul(v[r], w);
    }
    C2<T> P[h + 1], Q[h + 1];
    T sx = v[0].x, sy = v[0].y;
#pragma unroll
    for (int r = 1; r <= h; ++r) {
      P[r] = C2<T>{v[r].x + v[R - r].x, v[r].y + v[R - r].y};
      Q[r] = C2<T>{v[r].x - v[R - r].x, v[r].y - v[R - r].y};
      sx += P[r].x;
      sy += P[r].y;
    }
    y[idxD] = C2<T>{sx, sy};
#pragma unroll
    for (int k = 1; k <= h; ++k) {
      T ax = v[0].x, ay = v[0].y, bx = 0, by = 0;
#pragma unroll
      for (int r = 1; r <= h; ++r) {
        const int t = (r * k) % R;  // compile-time after unrolling
        const T c = t <= h ? cs[t] : cs[R - t];
        const T sv = t <= h ? sn[t] : -sn[R - t];
        ax += P[r].x * c;
        ay += P[r].y * c;
        bx += Q[r].x * sv;
        by += Q[r].y * sv;
      }
      y[idxD + k * Ns] = C2<T>{ax - by, ay + bx};
      y[idxD + (R - k) * Ns] = C2<T>{ax + by, ay - bx};
    }
  }
}

template <class T>
__device__ __forceinline__ void run_pass(const C2<T>* x, C2<T>* y, int n, int R, int Ns, const C2<T>* tw,
                                         bool conj) {
  switch (R) {
    case 3: stockham_pass_r<T, 3>(x, y, n, Ns, tw, conj); break;
    case 5: stockham_pass_r<T, 5>(x, y, n, Ns, tw, conj); break;
    case 7: stockham_pass_r<T, 7>(x, y, n, Ns, tw, conj); break;
    case 11: stockham_pass_r<T, 11>(x, y, n, Ns, tw, conj); break;
    case 13: stockham_pass_r<T, 13>(x, y, n, Ns, tw, conj); break;
    default: stockham_pass<T>(x, y, n, R, Ns, tw, conj); break;
  }
}

template <class T>
__global__ void __launch_bounds__(PhiThreads<T>::value) phi_kernel(PhiPlanDev<T> p, const double* __restrict__ in,
                                                       double* __restrict__ out, int F, int analysis) {
  extern __shared__ unsigned char smem_raw[];
  C2<T>* buf0 = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* buf1 = buf0 + p.M;
  const int N = p.N, K = 2 * N, M = p.M;
  const long nval = (long)M * K;  // per-field size of g and of f (complex)
  const int rows = K * F;
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {
    const int f = row / K, l = row % K;
    // load
    if (!analysis) {
      // c[m mod M] = g(m, l) e^{i pi m / M}; unrolled so that several strided loads are in flight
#pragma unroll 8
      for (int mm = threadIdx.x; mm < M; mm += blockDim.x) {
        const int m = mm - (K - 1);  // -(K-1) .. K-1
        const double2 v = __ldg(reinterpret_cast<const double2*>(in) + f * nval + order_slot(m) * K + l);
        const C2<T> s = p.shift[mm];
        const C2<T> a{from_f64<T>(v.x), from_f64<T>(v.y)};
        buf0[(m % M + M) % M] = cmul(a, s);
      }
    } else {
#pragma unroll 8
      for (int j = threadIdx.x; j < M; j += blockDim.x) {
        const double2 v = __ldg(reinterpret_cast<const double2*>(in) + f * nval + (long)l * M + j);
        buf0[j] = C2<T>{from_f64<T>(v.x), from_f64<T>(v.y)};
      }
    }
    __syncthreads();
    C2<T>* src = buf0;
    C2<T>* dst = buf1;
    for (int ps = 0; ps < p.npass; ++ps) {
      run_pass<T>(src, dst, M, p.radix[ps], p.ns[ps], p.tw + p.tw_off[ps], analysis != 0);
      __syncthreads();
      C2<T>* t = src;
      src = dst;
      dst = t;
    }
    // store
    if (!analysis) {
      for (int j = threadIdx.x; j < M; j += blockDim.x) {
        const C2<T> v = src[j];
        reinterpret_cast<double2*>(out)[f * nval + (long)l * M + j] = make_double2(to_f64(v.x), to_f64(v.y));
      }
    } else {
      // g(m, l) = (1/M) e^{-i pi m / M} C[m mod M]
      for (int mm = threadIdx.x; mm < M; mm += blockDim.x) {
        const int m = mm - (K - 1);
        C2<T> s = p.shift[mm];
        s.y = -s.y;
        const C2<T> v = cmul(src[(m % M + M) % M], s);
        const T inv = T(1) / (T)M;
        reinterpret_cast<double2*>(out)[f * nval + order_slot(m) * K + l] = make_double2(to_f64(v.x * inv), to_f64(v.y * inv));
      }
    }
    __syncthreads();
  }
}

}  // namespace

// Factor M into radices (small primes first, then any remaining factor).
static std::vector<int> factor_radices(int M) {
  std::vector<int> r;
  int n = M;
  for (int p : {4, 2, 3, 5, 7, 11, 13}) {
    while (n % p == 0) {
      r.push_back(p);
      n /= p;
    }
  }
  for (int p = 17; (long)p * p <= n; p += 2)
    while (n % p == 0) {
      r.push_back(p);
      n /= p;
    }
  if (n > 1) r.push_back(n);
  return r;
}

template <class T>
bool PhiTables<T>::build(int N) {
  M = 4 * N - 1;
  std::vector<int> rad = factor_radices(M);
  if ((int)rad.size() > kMaxPasses) return false;
  npass = (int)rad.size();
  std::vector<C2<T>> tw_h;
  int Ns = 1;
  for (int ps = 0; ps < npass; ++ps) {
    radix[ps] = rad[ps];
    ns[ps] = Ns;
    tw_off[ps] = (int)tw_h.size();
    const int L = Ns * rad[ps];
    for (int t = 0; t < L; ++t) {
      // e^{+2 pi i t / L}, argument reduced exactly (t < L)
      const long double a = 2.0L * 3.141592653589793238462643383279502884L * (long double)t / (long double)L;
      tw_h.push_back(C2<T>{(T)std::cos(a), (T)std::sin(a)});
    }
    Ns *= rad[ps];
  }
  std::vector<C2<T>> sh(M);
  for (int mm = 0; mm < M; ++mm) {
    const long m = mm - (2L * N - 1);
    long r = (m % (2L * M) + 2L * M) % (2L * M);  // e^{i pi m / M} = e^{2 pi i r / (2M)}
    const long double a = 3.141592653589793238462643383279502884L * (long double)r / (long double)M;
    sh[mm] = C2<T>{(T)std::cos(a), (T)std::sin(a)};
  }
  n_tw = (int)tw_h.size();
  if (cudaMalloc(&d_tw, sizeof(C2<T>) * tw_h.size()) != cudaSuccess) return false;
  if (cudaMalloc(&d_shift, sizeof(C2<T>) * sh.size()) != cudaSuccess) return false;
  if (cudaMemcpy(d_tw, tw_h.data(), sizeof(C2<T>) * tw_h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return false;
  if (cudaMemcpy(d_shift, sh.data(), sizeof(C2<T>) * sh.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return false;
  this->N = N;
  return true;
}

template <class T>
void PhiTables<T>::release() {
  cudaFree(d_tw);
  cudaFree(d_shift);
  d_tw = nullptr;
  d_shift = nullptr;
}

template <class T>
cudaError_t PhiTables<T>::launch(const double* in, double* out, int F, bool analysis, int grid,
                                 cudaStream_t st) const {
  PhiPlanDev<T> d;
  d.N = N;
  d.M = M;
  d.npass = npass;
  for (int i = 0; i < kMaxPasses; ++i) {
    d.radix[i] = radix[i];
    d.ns[i] = ns[i];
    d.tw_off[i] = tw_off[i];
  }
  d.tw = static_cast<const C2<T>*>(d_tw);
  d.shift = static_cast<const C2<T>*>(d_shift);
  const size_t smem = 2 * sizeof(C2<T>) * (size_t)M;
  cudaError_t e = cudaFuncSetAttribute(phi_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  phi_kernel<T><<<grid, PhiThreads<T>::value, smem, st>>>(d, in, out, F, analysis ? 1 : 0);
  return cudaGetLastError();
}

template <class T>
size_t PhiTables<T>::smem_bytes() const {
  return 2 * sizeof(C2<T>) * (size_t)M;
}

template struct PhiTables<double>;
template struct PhiTables<float>;

}  // namespace sht
