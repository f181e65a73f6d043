// Small dense FP64 linear algebra for the plan builder (host only).
//
// Column-major matrices, Householder QR with column pivoting (the
// rank-revealing factorisation of the interpolative decomposition, Sec. 2.1,
// Eq. pivotedQR), thin QR, triangular solves and a one-sided Jacobi SVD for
// the small core matrix of the randomized-sampling SVD (Sec. 2.3, Alg. 1).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

namespace sht {

struct Mat {
  int r = 0, c = 0;
  std::vector<double> a;
  Mat() = default;
  Mat(int rows, int cols) : r(rows), c(cols), a((size_t)rows * cols, 0.0) {}
  double& operator()(int i, int j) { return a[(size_t)i + (size_t)j * r]; }
  double operator()(int i, int j) const { return a[(size_t)i + (size_t)j * r]; }
  double* col(int j) { return a.data() + (size_t)j * r; }
  const double* col(int j) const { return a.data() + (size_t)j * r; }
};

inline Mat transpose(const Mat& A) {
  Mat T(A.c, A.r);
  for (int j = 0; j < A.c; ++j)
    for (int i = 0; i < A.r; ++i) T(j, i) = A(i, j);
  return T;
}

// C = A * B
inline Mat matmul(const Mat& A, const Mat& B) {
  Mat C(A.r, B.c);
  for (int j = 0; j < B.c; ++j)
    for (int l = 0; l < A.c; ++l) {
      double b = B(l, j);
      if (b == 0.0) continue;
      const double* ac = A.col(l);
      double* cc = C.col(j);
      for (int i = 0; i < A.r; ++i) cc[i] += ac[i] * b;
    }
  return C;
}

// Householder reflector for x (length n): returns tau and overwrites x with v
// (v[0] = 1 implied after scaling); x[0] receives beta = -sign(x0) ||x||.
inline double householder(double* x, int n, double& beta_out) {
  double s = 0.0;
  for (int i = 1; i < n; ++i) s += x[i] * x[i];
  double x0 = x[0];
  if (s == 0.0) { beta_out = x0; return 0.0; }
  double nrm = std::sqrt(x0 * x0 + s);
  double beta = x0 <= 0.0 ? nrm : -nrm;
  double v0 = x0 - beta;
  for (int i = 1; i < n; ++i) x[i] /= v0;
  beta_out = beta;
  return (beta - x0) / beta;  // tau
}

// Apply (I - tau v v^T) from the left to columns [c0, c1) of A, rows [r0, m).
inline void apply_reflector(Mat& A, int r0, const double* v, double tau, int c0, int c1) {
  if (tau == 0.0) return;
  int n = A.r - r0;
  int j = c0;
  // four, then two columns per pass over v: independent sums keep the adder
  // busy, and each column's sum runs in the same order as the one-column loop
  // below, so the results are the same bit for bit
  for (; j + 3 < c1; j += 4) {
    double* a0 = A.col(j) + r0;
    double* a1 = A.col(j + 1) + r0;
    double* a2 = A.col(j + 2) + r0;
    double* a3 = A.col(j + 3) + r0;
    double d0 = a0[0], d1 = a1[0], d2 = a2[0], d3 = a3[0];
    for (int i = 1; i < n; ++i) {
      const double vi = v[i];
      d0 += vi * a0[i];
      d1 += vi * a1[i];
      d2 += vi * a2[i];
      d3 += vi * a3[i];
    }
    d0 *= tau;
    d1 *= tau;
    d2 *= tau;
    d3 *= tau;
    a0[0] -= d0;
    a1[0] -= d1;
    a2[0] -= d2;
    a3[0] -= d3;
    for (int i = 1; i < n; ++i) {
      const double vi = v[i];
      a0[i] -= d0 * vi;
      a1[i] -= d1 * vi;
      a2[i] -= d2 * vi;
      a3[i] -= d3 * vi;
    }
  }
  for (; j + 1 < c1; j += 2) {
    double* a0 = A.col(j) + r0;
    double* a1 = A.col(j + 1) + r0;
    double d0 = a0[0], d1 = a1[0];
    for (int i = 1; i < n; ++i) {
      d0 += v[i] * a0[i];
      d1 += v[i] * a1[i];
    }
    d0 *= tau;
    d1 *= tau;
    a0[0] -= d0;
    a1[0] -= d1;
    for (int i = 1; i < n; ++i) {
      a0[i] -= d0 * v[i];
      a1[i] -= d1 * v[i];
    }
  }
  for (; j < c1; ++j) {
    double* aj = A.col(j) + r0;
    double d = aj[0];
    for (int i = 1; i < n; ++i) d += v[i] * aj[i];
    d *= tau;
    aj[0] -= d;
    for (int i = 1; i < n; ++i) aj[i] -= d * v[i];
  }
}

// Rank-revealing QR with column pivoting of A (m x n), in place.
// Stops when the largest remaining column 2-norm is <= tol or after kmax
// steps.  On return perm[j] is the original column in position j, the upper
// k x n part of A holds R (in permuted column order), and k is returned.
inline int pivoted_qr(Mat& A, double tol, int kmax, std::vector<int>& perm) {
  const int m = A.r, n = A.c;
  perm.resize(n);
  for (int j = 0; j < n; ++j) perm[j] = j;
  // squared trailing column norms, downdated after each step (the reflected
  // row k leaves each column); a column whose downdated value has lost most of
  // its last exact value to cancellation is recomputed exactly (the usual
  // safeguard of column-pivoted QR, threshold sqrt(machine epsilon))
  std::vector<double> norm2(n), exact2(n), v(m);
  for (int j = 0; j < n; ++j) {
    const double* aj = A.col(j);
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += aj[i] * aj[i];
    norm2[j] = exact2[j] = s;
  }
  const double kRecompute = 1.4901161193847656e-08;  // 2^-26
  int kcap = std::min(std::min(m, n), kmax);
  int k = 0;
  for (; k < kcap; ++k) {
    int p = k;
    for (int j = k + 1; j < n; ++j)
      if (norm2[j] > norm2[p]) p = j;
    if (std::sqrt(norm2[p]) <= tol) break;
    if (p != k) {
      std::swap_ranges(A.col(k), A.col(k) + m, A.col(p));
      std::swap(perm[k], perm[p]);
      std::swap(norm2[k], norm2[p]);
      std::swap(exact2[k], exact2[p]);
    }
    double* x = A.col(k) + k;
    double beta;
    double tau = householder(x, m - k, beta);
    v[0] = 1.0;
    for (int i = 1; i < m - k; ++i) v[i] = x[i];
    apply_reflector(A, k, v.data(), tau, k + 1, n);
    x[0] = beta;
    for (int i = 1; i < m - k; ++i) x[i] = 0.0;
    for (int j = k + 1; j < n; ++j) {
      const double a = A(k, j);
      const double t = norm2[j] - a * a;
      if (t <= kRecompute * exact2[j]) {
        const double* aj = A.col(j);
        double s = 0.0;
        for (int i = k + 1; i < m; ++i) s += aj[i] * aj[i];
        norm2[j] = exact2[j] = s;
      } else {
        norm2[j] = t;
      }
    }
  }
  return k;
}

// Solve R11 X = B in place for upper-triangular R11 (k x k, leading part of R).
inline void upper_solve(const Mat& R, int k, Mat& B) {
  for (int j = 0; j < B.c; ++j) {
    double* b = B.col(j);
    for (int i = k - 1; i >= 0; --i) {
      double s = b[i];
      for (int l = i + 1; l < k; ++l) s -= R(i, l) * b[l];
      b[i] = s / R(i, i);
    }
  }
}

// Thin QR without pivoting: returns Q (m x min(m,n)) with orthonormal columns.
inline Mat thin_q(const Mat& A0) {
  Mat A = A0;
  const int m = A.r, n = A.c, k = std::min(m, n);
  std::vector<std::vector<double>> vs(k);
  std::vector<double> taus(k);
  for (int j = 0; j < k; ++j) {
    double* x = A.col(j) + j;
    double beta;
    double tau = householder(x, m - j, beta);
    std::vector<double> v(m - j);
    v[0] = 1.0;
    for (int i = 1; i < m - j; ++i) v[i] = x[i];
    apply_reflector(A, j, v.data(), tau, j + 1, n);
    vs[j] = std::move(v);
    taus[j] = tau;
  }
  Mat Q(m, k);
  for (int j = 0; j < k; ++j) Q(j, j) = 1.0;
  for (int j = k - 1; j >= 0; --j) apply_reflector(Q, j, vs[j].data(), taus[j], 0, k);
  return Q;
}

// One-sided Jacobi SVD: A (m x n, m >= n) = U diag(s) V^T, s descending.
inline void jacobi_svd(const Mat& A0, Mat& U, std::vector<double>& s, Mat& V) {
  Mat A = A0;
  const int m = A.r, n = A.c;
  V = Mat(n, n);
  for (int j = 0; j < n; ++j) V(j, j) = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double* ap = A.col(p);
        double* aq = A.col(q);
        double alpha = 0, beta = 0, gamma = 0;
        for (int i = 0; i < m; ++i) { alpha += ap[i] * ap[i]; beta += aq[i] * aq[i]; gamma += ap[i] * aq[i]; }
        if (gamma == 0.0) continue;
        double rel = std::fabs(gamma) / std::sqrt(alpha * beta);
        off = std::max(off, rel);
        if (rel < 1e-15) continue;
        double zeta = (beta - alpha) / (2.0 * gamma);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        double cs = 1.0 / std::sqrt(1.0 + t * t), sn = cs * t;
        for (int i = 0; i < m; ++i) {
          double x = ap[i], y = aq[i];
          ap[i] = cs * x - sn * y;
          aq[i] = sn * x + cs * y;
        }
        double* vp = V.col(p);
        double* vq = V.col(q);
        for (int i = 0; i < n; ++i) {
          double x = vp[i], y = vq[i];
          vp[i] = cs * x - sn * y;
          vq[i] = sn * x + cs * y;
        }
      }
    if (off < 1e-15) break;
  }
  std::vector<double> sv(n);
  for (int j = 0; j < n; ++j) {
    double t = 0;
    for (int i = 0; i < m; ++i) t += A(i, j) * A(i, j);
    sv[j] = std::sqrt(t);
  }
  std::vector<int> ord(n);
  for (int j = 0; j < n; ++j) ord[j] = j;
  std::sort(ord.begin(), ord.end(), [&](int x, int y) { return sv[x] > sv[y]; });
  U = Mat(m, n);
  Mat V2(n, n);
  s.resize(n);
  for (int jj = 0; jj < n; ++jj) {
    int j = ord[jj];
    s[jj] = sv[j];
    for (int i = 0; i < m; ++i) U(i, jj) = sv[j] > 0 ? A(i, j) / sv[j] : 0.0;
    for (int i = 0; i < n; ++i) V2(i, jj) = V(i, j);
  }
  V = V2;
}

// Moore-Penrose pseudo-inverse via SVD, singular values below rtol*s_max dropped.
inline Mat pinv(const Mat& A, double rtol = 1e-14) {
  bool tall = A.r >= A.c;
  Mat B = tall ? A : transpose(A);
  Mat U, V;
  std::vector<double> s;
  jacobi_svd(B, U, s, V);
  double cut = s.empty() ? 0.0 : rtol * s[0];
  // B^+ = V diag(1/s) U^T  (n x m)
  Mat P(B.c, B.r);
  for (int l = 0; l < (int)s.size(); ++l) {
    if (s[l] <= cut || s[l] == 0.0) continue;
    double inv = 1.0 / s[l];
    for (int j = 0; j < B.r; ++j) {
      double u = U(j, l) * inv;
      if (u == 0.0) continue;
      for (int i = 0; i < B.c; ++i) P(i, j) += V(i, l) * u;
    }
  }
  return tall ? P : transpose(P);
}

// splitmix64: deterministic per-block random streams
struct Rng {
  uint64_t s;
  explicit Rng(uint64_t seed) : s(seed) {}
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  int below(int n) { return (int)(next() % (uint64_t)n); }
};

// r distinct indices from [0, n) in random order (randperm(n)(1:r))
inline std::vector<int> randperm(Rng& g, int n, int r) {
  std::vector<int> p(n);
  for (int i = 0; i < n; ++i) p[i] = i;
  r = std::min(r, n);
  for (int i = 0; i < r; ++i) std::swap(p[i], p[i + g.below(n - i)]);
  p.resize(r);
  return p;
}

}  // namespace sht
