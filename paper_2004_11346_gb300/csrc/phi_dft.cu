// phi-direction DFT of the SHT (Eq. sht_fft), batched over nodes and fields.
//
//   synthesis: f(theta_l, phi_j) = sum_{m=-(2N-1)}^{2N-1} g(m, theta_l) e^{i m phi_j}
//   analysis:  g(m, theta_l)     = (1/M) sum_{j=0}^{M-1} f(theta_l, phi_j) e^{-i m phi_j}
//
// with M = 4N-1 samples phi_j = 2 pi (j + 1/2) / M.  Writing
// e^{i m phi_j} = e^{i pi m / M} e^{2 pi i m j / M}, synthesis is a length-M
// DFT of c[m mod M] = g(m) e^{i pi m / M}, and analysis is the conjugate
// transform followed by the conjugate shift.
//
// One CTA transforms NT consecutive (node, field) rows in shared memory, one
// buffer of M values per row: an in-place mixed-radix decimation-in-time FFT
// over the factors R_0 .. R_{P-1} of M.  The load places input n at its
// digit-reversed position (n = s_{P-1} + R_{P-1} (s_{P-2} + ...) goes to
// sum_p s_p L_p with L_p = R_0 ... R_{p-1}); pass p then combines blocks of
// length L_p into blocks of length L_p R_p, each butterfly reading and writing
// the same R_p positions, and the result ends in natural order.  Every pass
// reads its twiddles from a host-built table e^{+2 pi i t / (L_p R_p)}; the
// shift factors e^{i pi m / M} come from a table too.  Arithmetic type T is
// double or float; inputs and outputs are FP64 complex.  With NT = 2 the two
// rows are adjacent nodes, so that the strided accesses along the orders of g
// move whole 32-byte sectors.
#include <cuda_runtime.h>

#include <algorithm>
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

template <class T>
struct PhiThreads {
  static constexpr int value = 256;
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

// One DIT pass of radix R over NT rows of M values each, out of place: output
// position b Ns R + q Ns + j (b < M / (Ns R), q < R, j < Ns) is
// X_q = sum_s x_s w^{s j} e^{+-2 pi i s q / R} over the inputs x_s at
// b Ns R + s Ns + j, with w = e^{+-2 pi i / (Ns R)}; w^{s j} e^{2 pi i s q / R}
// is the table entry tw[s (j + q Ns) mod Ns R].  Every output re-reads its R
// inputs: used only for radices without a specialised butterfly (prime
// factors of M above 13), which is why such plans keep a second buffer.
template <class T, int NT>
__device__ void dit_pass_oop(const C2<T>* __restrict__ xin, C2<T>* __restrict__ yout, int M, int R, int Ns,
                             const C2<T>* __restrict__ tw, bool conj) {
  const int NsR = Ns * R;
  const T sg = conj ? T(-1) : T(1);
  for (int o = threadIdx.x; o < NT * M; o += blockDim.x) {
    const int row = o / M, pos = o % M;
    const C2<T>* x = xin + (size_t)row * M;
    const int rem = pos % NsR, q = rem / Ns, j = rem % Ns;
    const int base = pos - rem + j;
    const int step = j + q * Ns;  // < Ns R
    T ax = 0, ay = 0;
    int t = 0;
    for (int s = 0; s < R; ++s) {
      const C2<T> v = x[base + s * Ns];
      C2<T> w = tw[t];
      w.y *= sg;
      ax += v.x * w.x - v.y * w.y;
      ay += v.x * w.y + v.y * w.x;
      t += step;
      if (t >= NsR) t -= NsR;
    }
    yout[(size_t)row * M + pos] = C2<T>{ax, ay};
  }
}

// The same pass for a fixed small odd radix.  The R-point DFT after the
// twiddles pairs outputs q and R-q: with P_r = v_r + v_{R-r},
// Q_r = v_r - v_{R-r} (r = 1..h, h = (R-1)/2),
//   y_q, y_{R-q} = v_0 + sum_r P_r cos(2 pi r q / R) +- i sum_r Q_r s sin(2 pi r q / R),
// about a quarter of the multiplications of the direct R x R product.
template <class T, int R, int NT>
__device__ void dit_pass_r(C2<T>* __restrict__ buf, int M, int Ns, const C2<T>* __restrict__ tw, bool conj) {
  static_assert(R % 2 == 1, "odd radix");
  constexpr int h = (R - 1) / 2;
  const int nb = M / R;
  const T sg = conj ? T(-1) : T(1);
  T cs[h + 1], sn[h + 1];  // cos and s*sin of 2 pi t / R, t = 0..h
#pragma unroll
  for (int t = 0; t <= h; ++t) {
    const C2<T> w = tw[t * Ns];
    cs[t] = w.x;
    sn[t] = sg * w.y;
  }
  for (int o = threadIdx.x; o < NT * nb; o += blockDim.x) {
    const int row = o / nb, bf = o % nb;
    C2<T>* x = buf + (size_t)row * M;
    const int j = bf % Ns, base = (bf / Ns) * Ns * R + j;
    C2<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = x[base + r * Ns];
#pragma unroll
    for (int r = 1; r < R; ++r) {
      C2<T> w = tw[r * j];
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
    x[base] = C2<T>{sx, sy};
#pragma unroll
    for (int q = 1; q <= h; ++q) {
      T ax = v[0].x, ay = v[0].y, bx = 0, by = 0;
#pragma unroll
      for (int r = 1; r <= h; ++r) {
        const int t = (r * q) % R;  // compile-time after unrolling
        const T c = t <= h ? cs[t] : cs[R - t];
        const T sv = t <= h ? sn[t] : -sn[R - t];
        ax += P[r].x * c;
        ay += P[r].y * c;
        bx += Q[r].x * sv;
        by += Q[r].y * sv;
      }
      x[base + q * Ns] = C2<T>{ax - by, ay + bx};
      x[base + (R - q) * Ns] = C2<T>{ax + by, ay - bx};
    }
  }
}

// Radix 2 and 4 (even factors of M never occur: M = 4N - 1 is odd; kept for
// completeness of the factorisation).
template <class T, int NT>
__device__ void dit_pass_2(C2<T>* __restrict__ buf, int M, int Ns, const C2<T>* __restrict__ tw, bool conj) {
  const int nb = M / 2;
  const T sg = conj ? T(-1) : T(1);
  for (int o = threadIdx.x; o < NT * nb; o += blockDim.x) {
    const int row = o / nb, bf = o % nb;
    C2<T>* x = buf + (size_t)row * M;
    const int j = bf % Ns, base = (bf / Ns) * Ns * 2 + j;
    C2<T> w = tw[j];
    w.y *= sg;
    const C2<T> a = x[base], b = cmul(x[base + Ns], w);
    x[base] = C2<T>{a.x + b.x, a.y + b.y};
    x[base + Ns] = C2<T>{a.x - b.x, a.y - b.y};
  }
}

__host__ __device__ __forceinline__ bool in_place_radix(int R) {
  return R == 2 || R == 3 || R == 5 || R == 7 || R == 11 || R == 13;
}

// Pass on the current buffer; an out-of-place pass writes the other one and
// the two swap.
template <class T, int NT>
__device__ __forceinline__ void run_pass(C2<T>*& cur, C2<T>*& oth, int M, int R, int Ns, const C2<T>* tw,
                                         bool conj) {
  switch (R) {
    case 2: dit_pass_2<T, NT>(cur, M, Ns, tw, conj); break;
    case 3: dit_pass_r<T, 3, NT>(cur, M, Ns, tw, conj); break;
    case 5: dit_pass_r<T, 5, NT>(cur, M, Ns, tw, conj); break;
    case 7: dit_pass_r<T, 7, NT>(cur, M, Ns, tw, conj); break;
    case 11: dit_pass_r<T, 11, NT>(cur, M, Ns, tw, conj); break;
    case 13: dit_pass_r<T, 13, NT>(cur, M, Ns, tw, conj); break;
    default: {
      dit_pass_oop<T, NT>(cur, oth, M, R, Ns, tw, conj);
      C2<T>* t = cur;
      cur = oth;
      oth = t;
    }
  }
}

template <class T, int NT>
__global__ void __launch_bounds__(PhiThreads<T>::value) phi_kernel(PhiPlanDev<T> p, const double* __restrict__ in,
                                                       double* __restrict__ out, int F, int analysis) {
  extern __shared__ unsigned char smem_raw[];
  C2<T>* buf0 = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* buf1 = buf0 + (size_t)NT * p.M;  // used by out-of-place passes only
  const int N = p.N, K = 2 * N, M = p.M;
  const long nval = (long)M * K;  // per-field size of g and of f (complex)
  const int groups = K * F / NT;  // NT divides K (even)
  for (int grp = blockIdx.x; grp < groups; grp += gridDim.x) {
    const int row0 = grp * NT, f = row0 / K, l0 = row0 % K;
    // load into digit-reversed positions
    if (!analysis) {
      // c[m mod M] = g(m, l) e^{i pi m / M}; the NT nodes of one order are adjacent
#pragma unroll 4
      for (int idx = threadIdx.x; idx < NT * M; idx += blockDim.x) {
        const int mm = idx / NT, r = idx % NT;
        const int m = mm - (K - 1);  // -(K-1) .. K-1
        const double2 v = __ldg(reinterpret_cast<const double2*>(in) + f * nval + order_slot(m) * K + l0 + r);
        const C2<T> a{from_f64<T>(v.x), from_f64<T>(v.y)};
        buf0[(size_t)r * M + __ldg(p.perm + (m % M + M) % M)] = cmul(a, p.shift[mm]);
      }
    } else {
#pragma unroll 4
      for (int idx = threadIdx.x; idx < NT * M; idx += blockDim.x) {
        const int r = idx / M, j = idx % M;
        const double2 v = __ldg(reinterpret_cast<const double2*>(in) + f * nval + (long)(l0 + r) * M + j);
        buf0[(size_t)r * M + __ldg(p.perm + j)] = C2<T>{from_f64<T>(v.x), from_f64<T>(v.y)};
      }
    }
    __syncthreads();
    C2<T>* cur = buf0;
    C2<T>* oth = buf1;
    for (int ps = 0; ps < p.npass; ++ps) {
      run_pass<T, NT>(cur, oth, M, p.radix[ps], p.ns[ps], p.tw + p.tw_off[ps], analysis != 0);
      __syncthreads();
    }
    // store (natural order)
    if (!analysis) {
      for (int idx = threadIdx.x; idx < NT * M; idx += blockDim.x) {
        const int r = idx / M, j = idx % M;
        const C2<T> v = cur[idx];
        reinterpret_cast<double2*>(out)[f * nval + (long)(l0 + r) * M + j] = make_double2(to_f64(v.x), to_f64(v.y));
      }
    } else {
      // g(m, l) = (1/M) e^{-i pi m / M} C[m mod M]
      const T inv = T(1) / (T)M;
      for (int idx = threadIdx.x; idx < NT * M; idx += blockDim.x) {
        const int mm = idx / NT, r = idx % NT;
        const int m = mm - (K - 1);
        C2<T> sh = p.shift[mm];
        sh.y = -sh.y;
        const C2<T> v = cmul(cur[(size_t)r * M + (m % M + M) % M], sh);
        reinterpret_cast<double2*>(out)[f * nval + order_slot(m) * K + l0 + r] =
            make_double2(to_f64(v.x * inv), to_f64(v.y * inv));
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
  for (int p : {2, 3, 5, 7, 11, 13}) {
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
  two_buf = false;
  std::vector<C2<T>> tw_h;
  int Ns = 1;
  for (int ps = 0; ps < npass; ++ps) {
    radix[ps] = rad[ps];
    ns[ps] = Ns;
    tw_off[ps] = (int)tw_h.size();
    two_buf = two_buf || !in_place_radix(rad[ps]);
    const int L = Ns * rad[ps];
    for (int t = 0; t < L; ++t) {
      // e^{+2 pi i t / L}, argument reduced exactly (t < L)
      const long double a = 2.0L * 3.141592653589793238462643383279502884L * (long double)t / (long double)L;
      tw_h.push_back(C2<T>{(T)std::cos(a), (T)std::sin(a)});
    }
    Ns *= rad[ps];
  }
  // digit-reversed position of input n: with n = s_{P-1} + R_{P-1} (s_{P-2} + ...),
  // position sum_p s_p L_p, L_p = R_0 ... R_{p-1}
  std::vector<int> L(npass + 1, 1);
  for (int ps = 0; ps < npass; ++ps) L[ps + 1] = L[ps] * rad[ps];
  std::vector<int> perm(M);
  for (int n0 = 0; n0 < M; ++n0) {
    int n = n0, pos = 0;
    for (int ps = npass - 1; ps >= 0; --ps) {
      pos += (n % rad[ps]) * L[ps];
      n /= rad[ps];
    }
    perm[n0] = pos;
  }
  std::vector<C2<T>> sh(M);
  for (int mm = 0; mm < M; ++mm) {
    const long m = mm - (2L * N - 1);
    long r = (m % (2L * M) + 2L * M) % (2L * M);  // e^{i pi m / M} = e^{2 pi i r / (2M)}
    const long double a = 3.141592653589793238462643383279502884L * (long double)r / (long double)M;
    sh[mm] = C2<T>{(T)std::cos(a), (T)std::sin(a)};
  }
  // two adjacent rows per CTA while three such CTAs still fit an SM
  nt = (sizeof(T) == 4 && 2 * (two_buf ? 2 : 1) * sizeof(C2<T>) * (size_t)M <= 76 * 1024) ? 2 : 1;
  n_tw = (int)tw_h.size();
  if (cudaMalloc(&d_tw, sizeof(C2<T>) * tw_h.size()) != cudaSuccess) return false;
  if (cudaMalloc(&d_shift, sizeof(C2<T>) * sh.size()) != cudaSuccess) return false;
  if (cudaMalloc(&d_perm, sizeof(int) * perm.size()) != cudaSuccess) return false;
  if (cudaMemcpy(d_tw, tw_h.data(), sizeof(C2<T>) * tw_h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return false;
  if (cudaMemcpy(d_shift, sh.data(), sizeof(C2<T>) * sh.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return false;
  if (cudaMemcpy(d_perm, perm.data(), sizeof(int) * perm.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return false;
  this->N = N;
  return true;
}

template <class T>
void PhiTables<T>::release() {
  cudaFree(d_tw);
  cudaFree(d_shift);
  cudaFree(d_perm);
  d_tw = nullptr;
  d_shift = nullptr;
  d_perm = nullptr;
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
  d.perm = static_cast<const int*>(d_perm);
  const size_t smem = smem_bytes();
  const int groups = std::max(1, 2 * N * F / nt);
  grid = std::max(1, std::min(grid, groups));
  cudaError_t e;
  if (nt == 2) {
    e = cudaFuncSetAttribute(phi_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    phi_kernel<T, 2><<<grid, PhiThreads<T>::value, smem, st>>>(d, in, out, F, analysis ? 1 : 0);
  } else {
    e = cudaFuncSetAttribute(phi_kernel<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    phi_kernel<T, 1><<<grid, PhiThreads<T>::value, smem, st>>>(d, in, out, F, analysis ? 1 : 0);
  }
  return cudaGetLastError();
}

template <class T>
size_t PhiTables<T>::smem_bytes() const {
  return (size_t)nt * (two_buf ? 2 : 1) * sizeof(C2<T>) * (size_t)M;
}

template struct PhiTables<double>;
template struct PhiTables<float>;

}  // namespace sht
