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
// Each row (node, field) is transformed in shared memory by an in-place
// mixed-radix decimation-in-time FFT over the factors R_0 .. R_{P-1} of M.
// The load places input n at its digit-reversed position
// (n = s_{P-1} + R_{P-1} (s_{P-2} + ...) goes to sum_p s_p L_p with
// L_p = R_0 ... R_{p-1}); pass p then combines blocks of length L_p into
// blocks of length L_p R_p, each butterfly reading and writing the same R_p
// positions, and the result ends in natural order.  Every pass reads its
// twiddles from a host-built table e^{+2 pi i t / (L_p R_p)}; the shift
// factors e^{i pi m / M} come from a table too.  Arithmetic type T is double
// or float; inputs and outputs are FP64 complex.
//
// Whole-row mode: each CTA holds NT whole rows (adjacent nodes of one field;
// two in FP32, so that the strided side of g moves whole 32-byte sectors).  Split
// mode, for rows longer than one CTA's shared memory: one row spread over a
// cluster of CL CTAs (thread-block cluster, distributed shared memory),
// positions [c * chunk, (c + 1) * chunk) in CTA c, and every pass works
// through distributed shared memory.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cmath>
#include <vector>

#include "f64_bits.cuh"
#include "phi_dft.cuh"

namespace cg = cooperative_groups;

namespace sht {

template <class T>
struct C2 {
  T x, y;
};

namespace {

constexpr int kPhiThreads = 256;
constexpr int kPhiUnroll = 4;                  // global loads in flight per thread (split mode)
constexpr size_t kPhiSmemTarget = 76 * 1024;  // three CTAs per SM

// CTAs per SM the registers must allow: three in FP32 (the shared-memory
// target); two in FP64, whose radix-13 butterfly needs about 128 registers
template <class T>
struct PhiOcc {
  static constexpr int value = sizeof(T) == 4 ? 3 : 2;
};
// global loads in flight per thread in the whole-row gathers: the strided
// order-major side (synthesis) wants more than the contiguous rows (analysis)
template <class T>
struct PhiLoads {
  static constexpr int strided = sizeof(T) == 4 ? 4 : 2, contiguous = 2;
};

__device__ __forceinline__ long order_slot(long m) { return m == 0 ? 0 : (m > 0 ? 2 * m - 1 : -2 * m); }
__device__ __forceinline__ int mod_m(int m, int M) { return m < 0 ? m + M : m; }  // |m| < M
// floor(n / d) for 0 <= n < 2^31 by a multiply-high with host-computed
// constants (mul = 0 stands for d = 1)
__device__ __forceinline__ int divu(int n, unsigned mul, int shr) {
  return mul ? (int)(__umulhi((unsigned)n, mul) >> shr) : n;
}

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
template <class T>
__device__ __forceinline__ C2<T> from_f64c(double2 v) {
  return C2<T>{from_f64<T>(v.x), from_f64<T>(v.y)};
}

// Rows as the passes see them.  LocalRows: NT rows of M values in this CTA's
// shared memory; a row is a plain pointer.  SplitRow: one row, position pos in
// CTA pos / chunk of the cluster, at the same offset from the buffer in every
// CTA.  row(r) gives the row and el(row, pos) the element.
template <class T>
struct LocalRows {
  C2<T>* b;
  int M;
  __device__ __forceinline__ C2<T>* row(int r) const { return b + r * M; }
  __device__ __forceinline__ C2<T>* at(int r, int pos) const { return b + r * M + pos; }
};
template <class T>
struct SplitRow {
  C2<T>* b;
  int chunk;
  __device__ __forceinline__ SplitRow row(int) const { return *this; }
  __device__ __forceinline__ C2<T>* at(int, int pos) const {
    const int c = pos / chunk;
    return cg::this_cluster().map_shared_rank(b + (pos - c * chunk), c);
  }
};
template <class T>
__device__ __forceinline__ C2<T>& el(C2<T>* row, int pos) {
  return row[pos];
}
template <class T>
__device__ __forceinline__ C2<T>& el(const SplitRow<T>& row, int pos) {
  return *row.at(0, pos);
}

// The work of one pass is shared over the threads [start, start + stride):
// this CTA's threads (whole-row mode) or the cluster's (split mode).
struct Share {
  int start, stride;
};

// One DIT pass of radix R over NR rows of M values each, out of place: output
// position b Ns R + q Ns + j (b < M / (Ns R), q < R, j < Ns) is
// X_q = sum_s x_s w^{s j} e^{+-2 pi i s q / R} over the inputs x_s at
// b Ns R + s Ns + j, with w = e^{+-2 pi i / (Ns R)}; w^{s j} e^{2 pi i s q / R}
// is the table entry tw[s (j + q Ns) mod Ns R].  Every output re-reads its R
// inputs: used only for radices without a specialised butterfly (prime
// factors of M above 13), which is why such plans keep a second buffer.
template <class T, int NR, class Rows>
__device__ __forceinline__ void dit_pass_oop(Rows xin, Rows yout, int M, int R, int Ns, const C2<T>* __restrict__ tw,
                                             bool conj, Share sh) {
  const int NsR = Ns * R;
  const T sg = conj ? T(-1) : T(1);
  for (int o = sh.start; o < NR * M; o += sh.stride) {
    const int row = NR == 1 ? 0 : o / M, pos = NR == 1 ? o : o % M;
    const auto xr = xin.row(row);
    const int rem = pos % NsR, q = rem / Ns, j = rem % Ns;
    const int base = pos - rem + j;
    const int step = j + q * Ns;  // < Ns R
    T ax = 0, ay = 0;
    int t = 0;
    for (int s = 0; s < R; ++s) {
      const C2<T> v = el<T>(xr, base + s * Ns);
      C2<T> w = tw[t];
      w.y *= sg;
      ax += v.x * w.x - v.y * w.y;
      ay += v.x * w.y + v.y * w.x;
      t += step;
      if (t >= NsR) t -= NsR;
    }
    el<T>(yout.row(row), pos) = C2<T>{ax, ay};
  }
}

// cos and sin of 2 pi t / R, t = 0..(R-1)/2, for the specialised radices R = 3,
// 5, 7, 11, 13 (cos values then sin values per radix, from offset
// radix_off(R)), in constant memory: the butterflies take them as constant
// operands instead of holding them in registers.
__constant__ double c_rad64[44];
__constant__ float c_rad32[44];
__host__ __device__ constexpr int radix_off(int R) {
  return R == 3 ? 0 : R == 5 ? 4 : R == 7 ? 10 : R == 11 ? 18 : 30;
}
template <class T>
__device__ __forceinline__ T rad_const(int i);
template <>
__device__ __forceinline__ double rad_const<double>(int i) { return c_rad64[i]; }
template <>
__device__ __forceinline__ float rad_const<float>(int i) { return c_rad32[i]; }

// The same pass for a fixed small odd radix, in place.  The R-point DFT after
// the twiddles pairs outputs q and R-q: with P_r = v_r + v_{R-r},
// Q_r = v_r - v_{R-r} (r = 1..h, h = (R-1)/2),
//   y_q, y_{R-q} = v_0 + sum_r P_r cos(2 pi r q / R) +- i sum_r Q_r s sin(2 pi r q / R),
// about a quarter of the multiplications of the direct R x R product.
template <class T, int R, int NR, class Rows>
__device__ __forceinline__ void dit_pass_r(Rows x, int M, int Ns, unsigned mul, int shr, const C2<T>* __restrict__ tw,
                                           bool conj, Share sh) {
  static_assert(R % 2 == 1, "odd radix");
  constexpr int h = (R - 1) / 2, off = radix_off(R);
  const int nb = M / R;
  const T sg = conj ? T(-1) : T(1);
  for (int o = sh.start; o < NR * nb; o += sh.stride) {
    const int row = NR == 1 ? 0 : (NR == 2 ? (o >= nb ? 1 : 0) : o / nb), bf = o - row * nb;
    const auto xr = x.row(row);
    const int qb = divu(bf, mul, shr), j = bf - qb * Ns, base = bf + qb * Ns * (R - 1);
    C2<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = el<T>(xr, base + r * Ns);
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
    el<T>(xr, base) = C2<T>{sx, sy};
#pragma unroll
    for (int q = 1; q <= h; ++q) {
      T ax = v[0].x, ay = v[0].y, bx = 0, by = 0;
#pragma unroll
      for (int r = 1; r <= h; ++r) {
        const int t = (r * q) % R;  // compile-time after unrolling
        const T c = t <= h ? rad_const<T>(off + t) : rad_const<T>(off + R - t);
        const T sv = t <= h ? rad_const<T>(off + h + 1 + t) : -rad_const<T>(off + h + 1 + R - t);
        ax += P[r].x * c;
        ay += P[r].y * c;
        bx += Q[r].x * sv;
        by += Q[r].y * sv;
      }
      bx *= sg;
      by *= sg;
      el<T>(xr, base + q * Ns) = C2<T>{ax - by, ay + bx};
      el<T>(xr, base + (R - q) * Ns) = C2<T>{ax + by, ay - bx};
    }
  }
}

// Radix 2 (even factors of M never occur: M = 4N - 1 is odd; kept for
// completeness of the factorisation).
template <class T, int NR, class Rows>
__device__ __forceinline__ void dit_pass_2(Rows x, int M, int Ns, unsigned mul, int shr, const C2<T>* __restrict__ tw,
                                           bool conj, Share sh) {
  const int nb = M / 2;
  const T sg = conj ? T(-1) : T(1);
  for (int o = sh.start; o < NR * nb; o += sh.stride) {
    const int row = NR == 1 ? 0 : (NR == 2 ? (o >= nb ? 1 : 0) : o / nb), bf = o - row * nb;
    const auto xr = x.row(row);
    const int qb = divu(bf, mul, shr), j = bf - qb * Ns, base = bf + qb * Ns;
    C2<T> w = tw[j];
    w.y *= sg;
    const C2<T> a = el<T>(xr, base), b = cmul(el<T>(xr, base + Ns), w);
    el<T>(xr, base) = C2<T>{a.x + b.x, a.y + b.y};
    el<T>(xr, base + Ns) = C2<T>{a.x - b.x, a.y - b.y};
  }
}

__host__ __device__ __forceinline__ bool in_place_radix(int R) {
  return R == 2 || R == 3 || R == 5 || R == 7 || R == 11 || R == 13;
}

// Pass on the current rows; an out-of-place pass writes the other buffer and
// the two swap.
template <class T, int NR, class Rows>
__device__ __forceinline__ void run_pass(Rows& cur, Rows& oth, const PhiPlanDev<T>& p, int ps, bool conj, Share sh) {
  const int M = p.M, R = p.radix[ps], Ns = p.ns[ps];
  const unsigned mul = p.ns_mul[ps];
  const int shr = p.ns_shr[ps];
  const C2<T>* tw = p.tw + p.tw_off[ps];
  switch (R) {
    case 2: dit_pass_2<T, NR>(cur, M, Ns, mul, shr, tw, conj, sh); break;
    case 3: dit_pass_r<T, 3, NR>(cur, M, Ns, mul, shr, tw, conj, sh); break;
    case 5: dit_pass_r<T, 5, NR>(cur, M, Ns, mul, shr, tw, conj, sh); break;
    case 7: dit_pass_r<T, 7, NR>(cur, M, Ns, mul, shr, tw, conj, sh); break;
    case 11: dit_pass_r<T, 11, NR>(cur, M, Ns, mul, shr, tw, conj, sh); break;
    case 13: dit_pass_r<T, 13, NR>(cur, M, Ns, mul, shr, tw, conj, sh); break;
    default: {
      dit_pass_oop<T, NR>(cur, oth, M, R, Ns, tw, conj, sh);
      const Rows t = cur;
      cur = oth;
      oth = t;
    }
  }
}

// Whole-row mode: group = NT adjacent nodes of one field, CTA b takes groups
// b, b + grid, ...  The loads of a group go through registers, U (strided
// side) or UC (contiguous rows) per thread in flight; three CTAs share an SM
// in FP32, so that one CTA's loads overlap the others' passes.
template <class T, int NT>
__global__ void __launch_bounds__(kPhiThreads, PhiOcc<T>::value)
    phi_rows_kernel(PhiPlanDev<T> p, const double* __restrict__ in, double* __restrict__ out, int F, int analysis) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int U = PhiLoads<T>::strided, UC = PhiLoads<T>::contiguous;
  const int K = 2 * p.N, M = p.M;
  const long nval = (long)M * K;  // per-field size of g and of f (complex)
  const int gpf = K / NT;         // groups per field (NT divides K = 2N)
  const int groups = gpf * F, nv = NT * M;
  C2<T>* buf0 = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* buf1 = buf0 + (size_t)NT * M;  // used by out-of-place passes only
  const double2* __restrict__ in2 = reinterpret_cast<const double2*>(in);
  double2* __restrict__ out2 = reinterpret_cast<double2*>(out);
  const bool conj = analysis != 0;
  // in the order-major gather thread t takes node r_me = t mod NT of the
  // orders t / NT + k mstep (NT divides the thread count)
  const int r_me = threadIdx.x % NT, mstep = blockDim.x / NT;
  for (int grp = blockIdx.x; grp < groups; grp += gridDim.x) {
    const int f = grp / gpf, l0 = (grp - f * gpf) * NT;
    if (!analysis) {
      // c[m mod M] = g(m, l) e^{i pi m / M} at its digit-reversed position;
      // adjacent threads read the adjacent nodes of one order
      C2<T>* row = buf0 + r_me * M;
      for (int m0 = threadIdx.x / NT; m0 < M; m0 += U * mstep) {
        double2 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int mm = m0 + u * mstep;
          if (mm < M) v[u] = __ldg(in2 + f * nval + order_slot(mm - (K - 1)) * K + l0 + r_me);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int mm = m0 + u * mstep;
          if (mm < M) row[__ldg(p.perm + mod_m(mm - (K - 1), M))] = cmul(from_f64c<T>(v[u]), p.shift[mm]);
        }
      }
    } else {
      // the NT rows are contiguous in f
      const double2* src = in2 + f * nval + (long)l0 * M;
      for (int i0 = threadIdx.x; i0 < nv; i0 += UC * blockDim.x) {
        double2 v[UC];
#pragma unroll
        for (int u = 0; u < UC; ++u) {
          const int idx = i0 + u * blockDim.x;
          if (idx < nv) v[u] = __ldg(src + idx);
        }
#pragma unroll
        for (int u = 0; u < UC; ++u) {
          const int idx = i0 + u * blockDim.x;
          if (idx < nv) {
            const int r = NT == 1 ? 0 : (NT == 2 ? (idx >= M ? 1 : 0) : idx / M), j = idx - r * M;
            buf0[r * M + __ldg(p.perm + j)] = from_f64c<T>(v[u]);
          }
        }
      }
    }
    __syncthreads();
    LocalRows<T> cur{buf0, M}, oth{buf1, M};
    for (int ps = 0; ps < p.npass; ++ps) {
      run_pass<T, NT>(cur, oth, p, ps, conj, Share{(int)threadIdx.x, (int)blockDim.x});
      __syncthreads();
    }
    if (!analysis) {
      // the rows in natural order, contiguous in f
      double2* dst = out2 + f * nval + (long)l0 * M;
      for (int idx = threadIdx.x; idx < nv; idx += blockDim.x) {
        const C2<T> v = cur.b[idx];
        dst[idx] = make_double2(to_f64(v.x), to_f64(v.y));
      }
    } else {
      // g(m, l) = (1/M) e^{-i pi m / M} C[m mod M], the NT nodes of an order adjacent
      const T inv = T(1) / (T)M;
      for (int idx = threadIdx.x; idx < nv; idx += blockDim.x) {
        const int mm = idx / NT, r = idx - mm * NT;
        C2<T> s = p.shift[mm];
        s.y = -s.y;
        const C2<T> v = cmul(cur.b[r * M + mod_m(mm - (K - 1), M)], s);
        out2[f * nval + order_slot(mm - (K - 1)) * K + l0 + r] = make_double2(to_f64(v.x * inv), to_f64(v.y * inv));
      }
    }
    __syncthreads();  // the next group's loads overwrite the rows
  }
}

// Split mode: one row per cluster, cluster c takes rows c, c + clusters, ...
template <class T>
__global__ void __launch_bounds__(kPhiThreads, PhiOcc<T>::value)
    phi_split_kernel(PhiPlanDev<T> p, const double* __restrict__ in, double* __restrict__ out, int F, int analysis) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
  const int cid = blockIdx.x / CL, ncl = gridDim.x / CL;
  const int K = 2 * p.N, M = p.M;
  const long nval = (long)M * K;
  C2<T>* buf0 = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* buf1 = buf0 + p.chunk;
  const Share sh{(int)(rank * blockDim.x + threadIdx.x), (int)(CL * blockDim.x)};
  const double2* __restrict__ in2 = reinterpret_cast<const double2*>(in);
  double2* __restrict__ out2 = reinterpret_cast<double2*>(out);
  const bool conj = analysis != 0;
  const int rows = K * F;
  for (int row = cid; row < rows; row += ncl) {
    const int f = row / K, l = row - f * K;
    SplitRow<T> cur{buf0, p.chunk}, oth{buf1, p.chunk};
    for (int i0 = sh.start; i0 < M; i0 += kPhiUnroll * sh.stride) {
      double2 v[kPhiUnroll];
#pragma unroll
      for (int u = 0; u < kPhiUnroll; ++u) {
        const int idx = i0 + u * sh.stride;
        if (idx < M)
          v[u] = __ldg(in2 + f * nval + (analysis ? (long)l * M + idx : order_slot(idx - (K - 1)) * K + l));
      }
#pragma unroll
      for (int u = 0; u < kPhiUnroll; ++u) {
        const int idx = i0 + u * sh.stride;
        if (idx < M) {
          if (analysis)
            *cur.at(0, __ldg(p.perm + idx)) = from_f64c<T>(v[u]);
          else
            *cur.at(0, __ldg(p.perm + mod_m(idx - (K - 1), M))) = cmul(from_f64c<T>(v[u]), p.shift[idx]);
        }
      }
    }
    cluster.sync();
    for (int ps = 0; ps < p.npass; ++ps) {
      run_pass<T, 1>(cur, oth, p, ps, conj, sh);
      cluster.sync();
    }
    if (!analysis) {
      for (int j = sh.start; j < M; j += sh.stride) {
        const C2<T> v = *cur.at(0, j);
        out2[f * nval + (long)l * M + j] = make_double2(to_f64(v.x), to_f64(v.y));
      }
    } else {
      const T inv = T(1) / (T)M;
      for (int mm = sh.start; mm < M; mm += sh.stride) {
        C2<T> s = p.shift[mm];
        s.y = -s.y;
        const C2<T> v = cmul(*cur.at(0, mod_m(mm - (K - 1), M)), s);
        out2[f * nval + order_slot(mm - (K - 1)) * K + l] = make_double2(to_f64(v.x * inv), to_f64(v.y * inv));
      }
    }
    cluster.sync();  // the row's buffers are free for the next row
  }
}

// The kernel of a launch shape.
template <class T>
const void* phi_kernel_of(bool split, int nt) {
  if (split) return reinterpret_cast<const void*>(phi_split_kernel<T>);
  return nt == 2 ? reinterpret_cast<const void*>(phi_rows_kernel<T, 2>)
                 : reinterpret_cast<const void*>(phi_rows_kernel<T, 1>);
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
  max_clusters = 0;
  if ((int)rad.size() > kMaxPasses) return true;  // unsupported: no launch shape
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
  // division constants of every pass: floor(n / d) = (n * mul) >> (32 + shr)
  // for n < 2^31 with l = ceil(log2 d), mul = ceil(2^(31 + l) / d), shr = l - 1
  // (the rounding error of mul moves n / d by less than 1 / d); checked for
  // every n the pass divides
  for (int ps = 0; ps < npass; ++ps) {
    const uint64_t d = (uint64_t)ns[ps];
    ns_mul[ps] = 0;
    ns_shr[ps] = 0;
    if (d > 1) {
      int l = 0;
      while ((1ull << l) < d) ++l;
      ns_mul[ps] = (unsigned)(((1ull << (31 + l)) + d - 1) / d);
      ns_shr[ps] = l - 1;
      for (uint64_t n = 0; n < (uint64_t)M; ++n)
        if ((((n * ns_mul[ps]) >> 32) >> ns_shr[ps]) != n / d) return false;
    }
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
  // the butterflies' constants (same long-double evaluation as the tables)
  T rc[44];
  for (int R : {3, 5, 7, 11, 13}) {
    const int h = (R - 1) / 2;
    for (int t = 0; t <= h; ++t) {
      const long double a = 2.0L * 3.141592653589793238462643383279502884L * (long double)t / (long double)R;
      rc[radix_off(R) + t] = (T)std::cos(a);
      rc[radix_off(R) + h + 1 + t] = (T)std::sin(a);
    }
  }
  if (cudaMemcpyToSymbol(sizeof(T) == 8 ? (const void*)&c_rad64 : (const void*)&c_rad32, rc, sizeof(rc)) !=
      cudaSuccess)
    return false;
  this->N = N;
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

  // Launch shape: whole rows while one row fits a CTA (two adjacent rows per
  // CTA in FP32 while three such CTAs fit an SM); else the
  // row split over the fewest CTAs (2, 4 or 8) whose share lets three CTAs
  // share an SM, failing that two, failing that one.
  int dev = 0, optin = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
  const size_t nb = two_buf ? 2 : 1, vb = sizeof(C2<T>);
  split = false;
  nt = 1;
  cl = 1;
  chunk = 0;
  if (nb * vb * (size_t)M <= (size_t)optin) {
    nt = (sizeof(T) == 4 && 2 * nb * vb * (size_t)M <= kPhiSmemTarget) ? 2 : 1;
  } else {
    split = true;
    cl = 0;
    for (size_t cap : {kPhiSmemTarget, (size_t)optin / 2, (size_t)optin})
      for (int c : {2, 4, 8})
        if (cl == 0 && nb * vb * (size_t)((M + c - 1) / c) <= cap) {
          cl = c;
          chunk = (M + c - 1) / c;
        }
    if (cl == 0) return true;  // unsupported: the row does not fit 8 CTAs
  }
  const void* kern = phi_kernel_of<T>(split, nt);
  const size_t smem = smem_bytes();
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return false;
  if (!split) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPhiThreads, smem) != cudaSuccess) return false;
    max_clusters = per_sm * sms;
    return true;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)cl, 1, 1);
  cfg.blockDim = dim3(kPhiThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int ncl = 0;
  if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) != cudaSuccess) return false;
  max_clusters = ncl;
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
cudaError_t PhiTables<T>::launch(const double* in, double* out, int F, bool analysis, cudaStream_t st) const {
  if (max_clusters < 1) return cudaErrorInvalidConfiguration;
  PhiPlanDev<T> d;
  d.N = N;
  d.M = M;
  d.npass = npass;
  for (int i = 0; i < kMaxPasses; ++i) {
    d.radix[i] = radix[i];
    d.ns[i] = ns[i];
    d.tw_off[i] = tw_off[i];
    d.ns_mul[i] = ns_mul[i];
    d.ns_shr[i] = ns_shr[i];
  }
  d.chunk = chunk;
  d.tw = static_cast<const C2<T>*>(d_tw);
  d.shift = static_cast<const C2<T>*>(d_shift);
  d.perm = static_cast<const int*>(d_perm);
  const size_t smem = smem_bytes();
  const long units = split ? 2L * N * F : 2L * N * F / nt;
  const int clusters = (int)std::max(1L, std::min<long>(max_clusters, units));
  // the attribute is per kernel and another plan may have set it lower
  cudaError_t e = cudaFuncSetAttribute(phi_kernel_of<T>(split, nt), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(clusters * cl), 1, 1);
  cfg.blockDim = dim3(kPhiThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = split ? 1 : 0;  // whole rows: a plain launch
  const int a = analysis ? 1 : 0;
  if (split) return cudaLaunchKernelEx(&cfg, phi_split_kernel<T>, d, in, out, F, a);
  if (nt == 2) return cudaLaunchKernelEx(&cfg, phi_rows_kernel<T, 2>, d, in, out, F, a);
  return cudaLaunchKernelEx(&cfg, phi_rows_kernel<T, 1>, d, in, out, F, a);
}

template <class T>
size_t PhiTables<T>::smem_bytes() const {
  return (two_buf ? 2 : 1) * sizeof(C2<T>) * (split ? (size_t)chunk : (size_t)nt * (size_t)M);
}

template struct PhiTables<double>;
template struct PhiTables<float>;

}  // namespace sht
