// Plan builder (host, FP64): the precomputation of Sec. 3.2-3.3.
//
//   1. Gauss-Legendre rule on 2N nodes (Sec. 1).
//   2. For every order |m|: the even and odd parity matrices of Sec. 3.1.2,
//      Pbar_k^{|m|}(x) at the N positive nodes, by the three-term recurrence in
//      k started from the sectoral value; a shared binary exponent carried
//      with the pair of recurrence values keeps starts far below the FP64
//      range (e.g. Pbar_700^700(0.9375) ~ 5e-321) exact until they grow back.
//   3. Block partition along the turning-point curve (Eq. new5, Eq. nb).
//   4. Per block (Sec. 3.3): IDBF of oscillatory blocks (Sec. 2.2) built
//      from linear-scaling IDs (Sec. 2.1); trimmed non-oscillatory blocks by
//      the randomized-sampling SVD (Alg. 1); trimmed turning-point blocks kept
//      dense.  Blocks with no entry above the trim threshold are dropped.
//   5. Emission of the apply program (program.hpp) and its schedule.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <numeric>
#include <string>

#ifdef _OPENMP
#include <omp.h>
#endif

#include "dense.hpp"
#include "plan.hpp"

namespace sht {

// ------------------------------------------------------------------------
// Gauss-Legendre rule: Newton's method on P_n from Tricomi's asymptotic
// initial guesses; the positive roots are computed and mirrored.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.141592653589793238462643383279502884;
  const int half = n / 2;
#pragma omp parallel for schedule(dynamic, 32)
  for (int k = 1; k <= (n + 1) / 2; ++k) {  // k-th largest root
    double nn = (double)n;
    double z = (1.0 - (nn - 1.0) / (8.0 * nn * nn * nn)) * std::cos(pi * (4.0 * k - 1.0) / (4.0 * nn + 2.0));
    double pn = 0.0, pn1 = 0.0;
    for (int it = 0; it < 50; ++it) {
      double a = 1.0, b = z;  // P_0, P_1
      for (int j = 2; j <= n; ++j) {
        double c = ((2.0 * j - 1.0) * z * b - (j - 1.0) * a) / j;
        a = b;
        b = c;
      }
      pn = n == 0 ? 1.0 : b;
      pn1 = a;
      double dp = nn * (pn1 - z * pn) / ((1.0 - z) * (1.0 + z));
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) <= 1e-17) break;
    }
    {
      double a = 1.0, b = z;
      for (int j = 2; j <= n; ++j) {
        double c = ((2.0 * j - 1.0) * z * b - (j - 1.0) * a) / j;
        a = b;
        b = c;
      }
      pn = b;
      pn1 = a;
    }
    double dp = nn * (pn1 - z * pn) / ((1.0 - z) * (1.0 + z));
    double wt = 2.0 / ((1.0 - z) * (1.0 + z) * dp * dp);
    int hi = n - k, lo = k - 1;  // ascending: largest root last
    if (n % 2 == 1 && k == (n + 1) / 2) { z = 0.0; }
    x[hi] = z;
    w[hi] = wt;
    x[lo] = -z;
    w[lo] = wt;
  }
  (void)half;
}

// ------------------------------------------------------------------------
// Legendre parity matrices for one order am = |m|: E(i, j) = Pbar_{am+2j}^{am}(xp_i),
// O(i, j) = Pbar_{am+1+2j}^{am}(xp_i), xp = the N positive nodes (ascending).
static void legendre_parity_matrices(int N, int am, const double* xp, Mat& E, Mat& O) {
  const int K = 2 * N;
  const int nce = (K - am + 1) / 2, nco = (K - am) / 2;
  E = Mat(N, nce);
  O = Mat(N, nco);
  std::vector<double> a(K + 1, 0.0), b(K + 1, 0.0);
  for (int k = am + 2; k < K; ++k) {
    double kk = k, mm = am, d = kk * kk - mm * mm;
    a[k] = std::sqrt((4.0 * kk * kk - 1.0) / d);
    b[k] = std::sqrt((2.0 * kk + 1.0) * (kk - 1.0 - mm) * (kk - 1.0 + mm) / ((2.0 * kk - 3.0) * d));
  }
  std::vector<double> sect(am + 1);
  for (int j = 1; j <= am; ++j) sect[j] = std::sqrt((2.0 * j + 1.0) / (2.0 * j));
  const double up = std::ldexp(1.0, 256), dn = std::ldexp(1.0, -256);
  // Nodes in blocks of kNB: the recurrence runs for the block's nodes side by
  // side, so that each degree's values land in kNB consecutive rows of one
  // column (the arithmetic per node is exactly the one-node recurrence).
  constexpr int kNB = 8;
  for (int i0 = 0; i0 < N; i0 += kNB) {
    const int nb = std::min(kNB, N - i0);
    double x[kNB], p0[kNB], p1[kNB];
    int e[kNB];  // value = p * 2^e
    bool scaled = false;
    for (int t = 0; t < nb; ++t) {
      x[t] = xp[i0 + t];
      const double u = std::sqrt((1.0 - x[t]) * (1.0 + x[t]));
      double v = 1.0 / std::sqrt(2.0);
      int ee = 0;
      for (int j = 1; j <= am; ++j) {
        v *= sect[j] * u;
        if (v < dn) { v *= up; ee -= 256; }
      }
      e[t] = ee;
      scaled = scaled || ee != 0;
      p0[t] = v;
      p1[t] = std::sqrt(2.0 * am + 3.0) * x[t] * v;
    }
    auto put = [&](int k, const double* val) {
      const int q = k - am;
      double* col = (q & 1) ? &O(i0, q >> 1) : &E(i0, q >> 1);
      if (!scaled) {
        for (int t = 0; t < nb; ++t) col[t] = val[t];
      } else {
        for (int t = 0; t < nb; ++t) col[t] = e[t] == 0 ? val[t] : std::ldexp(val[t], e[t]);
      }
    };
    put(am, p0);
    if (am + 1 < K) put(am + 1, p1);
    for (int k = am + 2; k < K; ++k) {
      double p2[kNB];
      const double ak = a[k], bk = b[k];
      for (int t = 0; t < nb; ++t) p2[t] = ak * x[t] * p1[t] - bk * p0[t];
      if (scaled) {
        bool any = false;
        for (int t = 0; t < nb; ++t) {
          if (e[t] < 0 && std::fabs(p2[t]) > up) {
            const int sh = std::min(256, -e[t]);
            p1[t] = std::ldexp(p1[t], -sh);
            p2[t] = std::ldexp(p2[t], -sh);
            e[t] += sh;
          }
          any = any || e[t] != 0;
        }
        scaled = any;
      }
      put(k, p2);
      for (int t = 0; t < nb; ++t) {
        p0[t] = p1[t];
        p1[t] = p2[t];
      }
    }
  }
}

// ------------------------------------------------------------------------
// Per-unit program under construction.
struct UnitBuild {
  std::vector<Op> ops;
  std::vector<double> fac;  // local factor store (offsets relative)
  int32_t nrows = 0;        // bump allocator for the vector space
  int64_t n_idbf = 0, n_low = 0, n_dense = 0, n_drop = 0;
  int64_t e_idbf = 0, e_low = 0, e_dense = 0;
  int64_t max_rank = 0;
  int64_t dbg[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // dense area by cause (diagnostics)
  int nphase = 0;
  double cost = 0.0;
  std::string err;
};

// Rows for one intermediate vector segment.  Segments start on a multiple of
// 8 rows: the tensor-core apply stages its inputs in whole groups of 8 rows,
// and the rows that pad a segment to its group end are then never written by
// any op.
int32_t alloc_rows(UnitBuild& ub, int n) {
  ub.nrows = (ub.nrows + 7) & ~7;
  const int32_t at = ub.nrows;
  ub.nrows += n;
  return at;
}

static inline int round4(int v) { return (v + 3) & ~3; }

// Append a dense block (mo x ni, column-major accessor f(i, j)) and return its offset.
template <class F>
static int64_t put_block(UnitBuild& ub, int mo, int ni, F f) {
  int ld = round4(std::max(mo, 1));
  int64_t off = (int64_t)ub.fac.size();
  ub.fac.resize(ub.fac.size() + (size_t)ld * ni, 0.0);
  for (int j = 0; j < ni; ++j)
    for (int i = 0; i < mo; ++i) ub.fac[off + (size_t)j * ld + i] = f(i, j);
  return off;
}

static void add_op(UnitBuild& ub, int phase, int mo, int ni, int64_t b_off, int in0, int inl0, int in1, int inl1,
                   int out0, int outl0, int out1, int outl1, int flags) {
  if (mo == 0) return;
  Op op{};
  op.b_off = b_off;
  op.mo = mo;
  op.ni = ni;
  op.ld = round4(std::max(mo, 1));
  op.flags = flags;
  op.in_off[0] = in0; op.in_len[0] = inl0; op.in_off[1] = in1; op.in_len[1] = inl1;
  op.out_off[0] = out0; op.out_len[0] = outl0; op.out_off[1] = out1; op.out_len[1] = outl1;
  op.phase = phase;
  ub.ops.push_back(op);
  ub.nphase = std::max(ub.nphase, phase + 1);
  ub.cost += (double)mo * ni;
}

// Matrix view of one parity matrix of one order.
struct ParityMatrix {
  const Mat* A;      // N x nc
  int am, parity;
  const double* xp;  // positive nodes
  double scale;      // largest |entry|
  int xbase, ybase;  // row offsets of X and Y in the unit vector space
  bool osc(int i, int j) const {
    if (am == 0) return true;
    double k = am + parity + 2.0 * j;
    double s2 = (1.0 - xp[i]) * (1.0 + xp[i]);
    return s2 * (k + 0.5) * (k + 0.5) > (double)am * am - 0.25;
  }
};

enum BlockClass { B_OSC, B_NONOSC, B_CROSS };

// ------------------------------------------------------------------------
// Interpolative decomposition (Sec. 2.1).  Column ID of K(rows, cand): the
// sampled submatrix is factored by QR with column pivoting,
// A(s,:) Lambda = Q [R1 R2], T = R1^-1 R2, V = [I T] Lambda^T.
struct IDResult {
  std::vector<int> skel;  // positions within cand
  Mat V;                  // k x |cand|
};

static IDResult id_from_sample(const Mat& Ms, double tol) {
  Mat M = Ms;
  std::vector<int> perm;
  int k = pivoted_qr(M, tol, std::min(M.r, M.c), perm);
  IDResult r;
  const int c = M.c;
  r.skel.assign(perm.begin(), perm.begin() + k);
  r.V = Mat(k, c);
  if (k == 0) return r;
  Mat T(k, c - k);
  for (int j = 0; j < c - k; ++j)
    for (int i = 0; i < k; ++i) T(i, j) = M(i, k + j);
  upper_solve(M, k, T);
  for (int j = 0; j < k; ++j) r.V(j, perm[j]) = 1.0;
  for (int j = 0; j < c - k; ++j)
    for (int i = 0; i < k; ++i) r.V(i, perm[k + j]) = T(i, j);
  return r;
}

// Mock-Chebyshev (or random) sample of s distinct indices from [0, n).
static std::vector<int> sample_indices(int n, int s, int sampling, Rng& g) {
  std::vector<int> out;
  if (s >= n) {
    out.resize(n);
    std::iota(out.begin(), out.end(), 0);
    return out;
  }
  if (sampling == 1) {
    out = randperm(g, n, s);
    std::sort(out.begin(), out.end());
    return out;
  }
  const double pi = 3.141592653589793238462643383279502884;
  std::vector<char> used(n, 0);
  for (int j = 0; j < s; ++j) {
    double t = 0.5 * (1.0 - std::cos(pi * (j + 0.5) / s));  // Chebyshev point in (0, 1)
    int p = (int)std::lround(t * (n - 1));
    // nearest unused index, ties to the lower one
    for (int d = 0; d < n; ++d) {
      if (p - d >= 0 && !used[p - d]) { p = p - d; break; }
      if (p + d < n && !used[p + d]) { p = p + d; break; }
    }
    used[p] = 1;
  }
  for (int i = 0; i < n; ++i)
    if (used[i]) out.push_back(i);
  return out;
}

struct BlockCtx {
  const ParityMatrix* P;
  int i0, nr, j0, nc;  // block rows/cols inside the parity matrix
  const sht_opts* o;
  double tol;
  Rng* rng;
  double K(int i, int j) const { return (*P->A)(i0 + i, j0 + j); }
};

// Column ID of the block's K(rows of [rs, re), cand) with adaptive sampling.
static IDResult column_id(const BlockCtx& b, int rs, int re, const std::vector<int>& cand) {
  const int n = re - rs, c = (int)cand.size();
  int s = std::min(n, (int)std::ceil(b.o->oversample * b.o->r_k));
  s = std::max(s, std::min(n, c + 8));
  for (;;) {
    std::vector<int> rows = sample_indices(n, s, b.o->sampling, *b.rng);
    Mat Ms((int)rows.size(), c);
    for (int j = 0; j < c; ++j)
      for (int i = 0; i < (int)rows.size(); ++i) Ms(i, j) = b.K(rs + rows[i], cand[j]);
    IDResult r = id_from_sample(Ms, b.tol);
    const int k = (int)r.skel.size();
    if (s < n && k >= std::min((int)rows.size(), c) && k < c) { s = std::min(n, 2 * s); continue; }
    if (s < n) {
      // check the interpolation on rows outside the sample
      std::vector<char> in(n, 0);
      for (int i : rows) in[i] = 1;
      bool ok = true;
      int checked = 0;
      for (int t = 0; t < 64 && checked < 24; ++t) {
        int i = b.rng->below(n);
        if (in[i]) continue;
        ++checked;
        for (int j = 0; j < c && ok; ++j) {
          double approx = 0.0;
          for (int q = 0; q < k; ++q) approx += b.K(rs + i, cand[r.skel[q]]) * r.V(q, j);
          if (std::fabs(approx - b.K(rs + i, cand[j])) > 10.0 * b.tol) ok = false;
        }
      }
      if (!ok) { s = std::min(n, 2 * s); continue; }
    }
    return r;
  }
}

// Row ID: K(cand rows, cols of [cs, ce)) ~= U K(skel rows, :), U = |cand| x k.
static IDResult row_id(const BlockCtx& b, int cs, int ce, const std::vector<int>& cand) {
  // column ID of the transposed block
  struct TCtx {
    const BlockCtx& b;
  };
  const int n = ce - cs, c = (int)cand.size();
  int s = std::min(n, (int)std::ceil(b.o->oversample * b.o->r_k));
  s = std::max(s, std::min(n, c + 8));
  for (;;) {
    std::vector<int> cols = sample_indices(n, s, b.o->sampling, *b.rng);
    Mat Ms((int)cols.size(), c);
    for (int j = 0; j < c; ++j)
      for (int i = 0; i < (int)cols.size(); ++i) Ms(i, j) = b.K(cand[j], cs + cols[i]);
    IDResult r = id_from_sample(Ms, b.tol);
    const int k = (int)r.skel.size();
    if (s < n && k >= std::min((int)cols.size(), c) && k < c) { s = std::min(n, 2 * s); continue; }
    if (s < n) {
      std::vector<char> in(n, 0);
      for (int i : cols) in[i] = 1;
      bool ok = true;
      int checked = 0;
      for (int t = 0; t < 64 && checked < 24; ++t) {
        int jcol = b.rng->below(n);
        if (in[jcol]) continue;
        ++checked;
        for (int j = 0; j < c && ok; ++j) {
          double approx = 0.0;
          for (int q = 0; q < k; ++q) approx += b.K(cand[r.skel[q]], cs + jcol) * r.V(q, j);
          if (std::fabs(approx - b.K(cand[j], cs + jcol)) > 10.0 * b.tol) ok = false;
        }
      }
      if (!ok) { s = std::min(n, 2 * s); continue; }
    }
    return r;  // U = V^T
  }
}

// ------------------------------------------------------------------------
// IDBF of one oscillatory block (Sec. 2.2): K ~= U^L ... U^h S^h V^h ... V^L.
// Returns false (and emits nothing) when the factorisation would store more
// entries than the dense block, unless forced.
struct Node { int s, e; };
static inline Node node_range(int n, int level, int idx) {
  int cnt = 1 << level;
  return Node{(int)((int64_t)n * idx / cnt), (int)((int64_t)n * (idx + 1) / cnt)};
}

static bool emit_idbf(UnitBuild& ub, const BlockCtx& b, int L, bool force) {
  const int h = L / 2;
  // column side: cskel[l][a * ncol + c], V[l][...]; a in [0, 2^l), c in [0, 2^(L-l))
  std::vector<std::vector<std::vector<int>>> cskel(h + 1);
  std::vector<std::vector<Mat>> Vm(h + 1);
  for (int l = 0; l <= h; ++l) {
    int na = 1 << l, nc = 1 << (L - l);
    cskel[l].resize((size_t)na * nc);
    Vm[l].resize((size_t)na * nc);
    for (int a = 0; a < na; ++a)
      for (int c = 0; c < nc; ++c) {
        std::vector<int> cand;
        if (l == 0) {
          Node cn = node_range(b.nc, L, c);
          for (int j = cn.s; j < cn.e; ++j) cand.push_back(j);
        } else {
          const auto& s1 = cskel[l - 1][(size_t)(a / 2) * (nc * 2) + 2 * c];
          const auto& s2 = cskel[l - 1][(size_t)(a / 2) * (nc * 2) + 2 * c + 1];
          cand = s1;
          cand.insert(cand.end(), s2.begin(), s2.end());
        }
        Node rn = node_range(b.nr, l, a);
        IDResult r = column_id(b, rn.s, rn.e, cand);
        std::vector<int> sk(r.skel.size());
        for (size_t t = 0; t < sk.size(); ++t) sk[t] = cand[r.skel[t]];
        ub.max_rank = std::max<int64_t>(ub.max_rank, (int64_t)sk.size());
        cskel[l][(size_t)a * nc + c] = std::move(sk);
        Vm[l][(size_t)a * nc + c] = std::move(r.V);
      }
  }
  // row side: rskel[l'][c * na + a]; c in [0, 2^l'), a in [0, 2^(L-l'))
  const int LR = L - h;
  std::vector<std::vector<std::vector<int>>> rskel(LR + 1);
  std::vector<std::vector<Mat>> Um(LR + 1);  // |cand| x k
  for (int l = 0; l <= LR; ++l) {
    int nc = 1 << l, na = 1 << (L - l);
    rskel[l].resize((size_t)nc * na);
    Um[l].resize((size_t)nc * na);
    for (int c = 0; c < nc; ++c)
      for (int a = 0; a < na; ++a) {
        std::vector<int> cand;
        if (l == 0) {
          Node rn = node_range(b.nr, L, a);
          for (int i = rn.s; i < rn.e; ++i) cand.push_back(i);
        } else {
          const auto& s1 = rskel[l - 1][(size_t)(c / 2) * (na * 2) + 2 * a];
          const auto& s2 = rskel[l - 1][(size_t)(c / 2) * (na * 2) + 2 * a + 1];
          cand = s1;
          cand.insert(cand.end(), s2.begin(), s2.end());
        }
        Node cn = node_range(b.nc, l, c);
        IDResult r = row_id(b, cn.s, cn.e, cand);
        std::vector<int> sk(r.skel.size());
        for (size_t t = 0; t < sk.size(); ++t) sk[t] = cand[r.skel[t]];
        ub.max_rank = std::max<int64_t>(ub.max_rank, (int64_t)sk.size());
        rskel[l][(size_t)c * na + a] = std::move(sk);
        Um[l][(size_t)c * na + a] = transpose(r.V);
      }
  }
  // storage check
  int64_t entries = 0;
  for (int l = 0; l <= h; ++l)
    for (auto& V : Vm[l]) entries += (int64_t)V.r * V.c;
  for (int l = 0; l <= LR; ++l)
    for (auto& U : Um[l]) entries += (int64_t)U.r * U.c;
  {
    int na = 1 << h, nc = 1 << (L - h);
    for (int a = 0; a < na; ++a)
      for (int c = 0; c < nc; ++c)
        entries += (int64_t)rskel[LR][(size_t)c * na + a].size() * cskel[h][(size_t)a * nc + c].size();
  }
  if (!force && entries >= (int64_t)b.nr * b.nc) return false;

  // ---- emission
  const ParityMatrix& P = *b.P;
  // z offsets, column side level l, layout a-major: index a * nc + c
  std::vector<std::vector<int>> zoff(h + 1);
  for (int l = 0; l <= h; ++l) {
    int na = 1 << l, nc = 1 << (L - l);
    zoff[l].resize((size_t)na * nc);
    for (int a = 0; a < na; ++a)
      for (int c = 0; c < nc; ++c) {
        zoff[l][(size_t)a * nc + c] = alloc_rows(ub, (int)cskel[l][(size_t)a * nc + c].size());
      }
  }
  // w offsets, row side level l', layout c-major: index c * na + a
  std::vector<std::vector<int>> woff(LR + 1);
  for (int l = 0; l <= LR; ++l) {
    int nc = 1 << l, na = 1 << (L - l);
    woff[l].resize((size_t)nc * na);
    for (int c = 0; c < nc; ++c)
      for (int a = 0; a < na; ++a) {
        woff[l][(size_t)c * na + a] = alloc_rows(ub, (int)rskel[l][(size_t)c * na + a].size());
      }
  }
  // column leaves (phase 0): z_0(0, c) = V x_C
  {
    int nc = 1 << L;
    for (int c = 0; c < nc; ++c) {
      Node cn = node_range(b.nc, L, c);
      const Mat& V = Vm[0][c];
      int64_t off = put_block(ub, V.r, V.c, [&](int i, int j) { return V(i, j); });
      add_op(ub, 0, V.r, V.c, off, P.xbase + b.j0 + cn.s, cn.e - cn.s, 0, 0, zoff[0][c], V.r, 0, 0, OP_BWD_ACCUM);
    }
  }
  // column levels 1..h (phase l): [z_l(2ap, c); z_l(2ap+1, c)] = [V_(2ap,c); V_(2ap+1,c)] [z_{l-1}(ap, 2c); z_{l-1}(ap, 2c+1)]
  for (int l = 1; l <= h; ++l) {
    int na = 1 << l, nc = 1 << (L - l), ncp = nc * 2;
    for (int ap = 0; ap < na / 2; ++ap)
      for (int c = 0; c < nc; ++c) {
        const Mat& V1 = Vm[l][(size_t)(2 * ap) * nc + c];
        const Mat& V2 = Vm[l][(size_t)(2 * ap + 1) * nc + c];
        int ni = V1.c;
        int mo = V1.r + V2.r;
        int64_t off = put_block(ub, mo, ni, [&](int i, int j) { return i < V1.r ? V1(i, j) : V2(i - V1.r, j); });
        // the candidates are the two children's skeleton rows, in that order
        // (n0 + n1 == ni by construction of cand above)
        const size_t k0 = (size_t)ap * ncp + 2 * c;
        const int n0 = (int)cskel[l - 1][k0].size(), n1 = (int)cskel[l - 1][k0 + 1].size();
        add_op(ub, l, mo, ni, off, zoff[l - 1][k0], n0, zoff[l - 1][k0 + 1], n1, zoff[l][(size_t)(2 * ap) * nc + c],
               V1.r, zoff[l][(size_t)(2 * ap + 1) * nc + c], V2.r, 0);
      }
  }
  // middle (phase h+1): w_LR(c, a) = S_(a,c) z_h(a, c), S = K(p, q)
  {
    int na = 1 << h, nc = 1 << (L - h);
    for (int a = 0; a < na; ++a)
      for (int c = 0; c < nc; ++c) {
        const auto& q = cskel[h][(size_t)a * nc + c];
        const auto& p = rskel[LR][(size_t)c * na + a];
        int64_t off = put_block(ub, (int)p.size(), (int)q.size(), [&](int i, int j) { return b.K(p[i], q[j]); });
        add_op(ub, h + 1, (int)p.size(), (int)q.size(), off, zoff[h][(size_t)a * nc + c], (int)q.size(), 0, 0,
               woff[LR][(size_t)c * na + a], (int)p.size(), 0, 0, 0);
      }
  }
  // row levels l' = LR..1 (phase h+2+(LR-l')):
  // [w_{l'-1}(cp, 2a); w_{l'-1}(cp, 2a+1)] = [U_(2cp,a) U_(2cp+1,a)] [w_l'(2cp, a); w_l'(2cp+1, a)]
  for (int l = LR; l >= 1; --l) {
    int nc = 1 << l, na = 1 << (L - l), nap = na * 2;
    int phase = h + 2 + (LR - l);
    for (int cp = 0; cp < nc / 2; ++cp)
      for (int a = 0; a < na; ++a) {
        const Mat& U1 = Um[l][(size_t)(2 * cp) * na + a];
        const Mat& U2 = Um[l][(size_t)(2 * cp + 1) * na + a];
        int mo = U1.r;  // |cand|, same for both
        int ni = U1.c + U2.c;
        int64_t off = put_block(ub, mo, ni, [&](int i, int j) { return j < U1.c ? U1(i, j) : U2(i, j - U1.c); });
        // the outputs are the two children's skeleton rows, in that order
        // (n0 + n1 == mo by construction of cand above)
        const size_t k0 = (size_t)cp * nap + 2 * a;
        const int n0 = (int)rskel[l - 1][k0].size(), n1 = (int)rskel[l - 1][k0 + 1].size();
        add_op(ub, phase, mo, ni, off, woff[l][(size_t)(2 * cp) * na + a], U1.c, woff[l][(size_t)(2 * cp + 1) * na + a],
               U2.c, woff[l - 1][k0], n0, woff[l - 1][k0 + 1], n1, 0);
      }
  }
  // row leaves (phase L+2): y_A += U_A w_0(0, a)
  {
    int na = 1 << L;
    for (int a = 0; a < na; ++a) {
      Node rn = node_range(b.nr, L, a);
      const Mat& U = Um[0][a];
      int64_t off = put_block(ub, U.r, U.c, [&](int i, int j) { return U(i, j); });
      add_op(ub, L + 2, U.r, U.c, off, woff[0][a], U.c, 0, 0, P.ybase + b.i0 + rn.s, rn.e - rn.s, 0, 0, OP_FWD_ACCUM);
    }
  }
  ub.n_idbf += 1;
  ub.e_idbf += entries;
  return true;
}

// Dense block: for the SIMT kernels one product per chunk of 64 rows, so that
// a large turning-point block spreads over several warps; for the tensor-core
// path (mixed precision) the whole block as one product, whose N tiles the
// kernel cuts itself: the transposed apply then adds each input row once per
// block instead of once per chunk.  Every chunk accumulates into the shared
// output rows (forward) and input rows (transposed).
static void emit_dense(UnitBuild& ub, const BlockCtx& b) {
  const ParityMatrix& P = *b.P;
  const int kDenseRows = b.o->precision == SHT_MIXED ? std::max(1, b.nr) : 64;
  for (int r0 = 0; r0 < b.nr; r0 += kDenseRows) {
    const int nr = std::min(kDenseRows, b.nr - r0);
    int64_t off = put_block(ub, nr, b.nc, [&](int i, int j) { return b.K(r0 + i, j); });
    add_op(ub, 0, nr, b.nc, off, P.xbase + b.j0, b.nc, 0, 0, P.ybase + b.i0 + r0, nr, 0, 0,
           OP_FWD_ACCUM | OP_BWD_ACCUM);
  }
  ub.n_dense += 1;
  ub.e_dense += (int64_t)b.nr * b.nc;
}

// Randomized-sampling SVD (Sec. 2.3, Alg. 1) with an adaptive rank: start at
// rsvd_r, double while the smallest computed singular value stays above the
// tolerance or the factorisation misses the block by more than 10 tol.
static bool emit_lowrank(UnitBuild& ub, const BlockCtx& b, bool force) {
  const int m = b.nr, n = b.nc;
  int r = std::max(1, b.o->rsvd_r);
  const int q = std::max(1, b.o->rsvd_q);
  for (;;) {
    if (!force && (int64_t)r * (m + n) >= (int64_t)m * n) return false;
    if (r >= std::min(m, n)) return false;
    std::vector<int> R = randperm(*b.rng, m, r * q), C = randperm(*b.rng, n, r * q);
    // Pi_col: pivots of QR(A(R, :))
    Mat AR((int)R.size(), n);
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < (int)R.size(); ++i) AR(i, j) = b.K(R[i], j);
    std::vector<int> pc, pr;
    int kc = pivoted_qr(AR, 0.0, r, pc);
    // Pi_row: pivots of QR(A(:, C)^T)
    Mat AC((int)C.size(), m);
    for (int j = 0; j < m; ++j)
      for (int i = 0; i < (int)C.size(); ++i) AC(i, j) = b.K(j, C[i]);
    int kr = pivoted_qr(AC, 0.0, r, pr);
    int rr = std::min(kc, kr);
    if (rr == 0) return false;
    std::vector<int> Pcol(pc.begin(), pc.begin() + rr), Prow(pr.begin(), pr.begin() + rr);
    Mat Acol(m, rr), Arow(n, rr);
    for (int t = 0; t < rr; ++t) {
      for (int i = 0; i < m; ++i) Acol(i, t) = b.K(i, Pcol[t]);
      for (int j = 0; j < n; ++j) Arow(j, t) = b.K(Prow[t], j);
    }
    Mat Qc = thin_q(Acol), Qr = thin_q(Arow);  // m x rr, n x rr
    std::vector<int> Srow = randperm(*b.rng, m, rr), Scol = randperm(*b.rng, n, rr);
    std::vector<int> I = Prow, J = Pcol;
    I.insert(I.end(), Srow.begin(), Srow.end());
    J.insert(J.end(), Scol.begin(), Scol.end());
    Mat QcI((int)I.size(), rr), QrJ((int)J.size(), rr), AIJ((int)I.size(), (int)J.size());
    for (int t = 0; t < rr; ++t) {
      for (size_t i = 0; i < I.size(); ++i) QcI((int)i, t) = Qc(I[i], t);
      for (size_t j = 0; j < J.size(); ++j) QrJ((int)j, t) = Qr(J[j], t);
    }
    for (size_t j = 0; j < J.size(); ++j)
      for (size_t i = 0; i < I.size(); ++i) AIJ((int)i, (int)j) = b.K(I[i], J[j]);
    // M = pinv(Qc(I,:)) A(I,J) pinv(Qr(J,:)^T)
    Mat M = matmul(matmul(pinv(QcI), AIJ), pinv(transpose(QrJ)));
    Mat UM, VM;
    std::vector<double> s;
    jacobi_svd(M, UM, s, VM);
    int keep = 0;
    while (keep < (int)s.size() && s[keep] > b.tol) ++keep;
    if (keep == (int)s.size() && keep == r && 2 * r < std::min(m, n)) { r *= 2; continue; }
    if (keep == 0) keep = 1;
    Mat Uk = matmul(Qc, UM), Vk = matmul(Qr, VM);  // m x rr, n x rr
    // residual check on the whole block
    double worst = 0.0;
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < m; ++i) {
        double acc = 0.0;
        for (int t = 0; t < keep; ++t) acc += Uk(i, t) * s[t] * Vk(j, t);
        worst = std::max(worst, std::fabs(acc - b.K(i, j)));
      }
    if (worst > 10.0 * b.tol) {
      if (2 * r >= std::min(m, n)) return false;
      r *= 2;
      continue;
    }
    const ParityMatrix& P = *b.P;
    int trow = alloc_rows(ub, keep);
    int64_t o1 = put_block(ub, keep, n, [&](int i, int j) { return Vk(j, i); });
    add_op(ub, 0, keep, n, o1, P.xbase + b.j0, n, 0, 0, trow, keep, 0, 0, OP_BWD_ACCUM);
    int64_t o2 = put_block(ub, m, keep, [&](int i, int j) { return Uk(i, j) * s[j]; });
    add_op(ub, 1, m, keep, o2, trow, keep, 0, 0, P.ybase + b.i0, m, 0, 0, OP_FWD_ACCUM);
    ub.n_low += 1;
    ub.e_low += (int64_t)keep * (m + n);
    ub.max_rank = std::max<int64_t>(ub.max_rank, keep);
    return true;
  }
}

// Smallest sub-block holding every entry with |K| >= delta (Sec. 3.3 trimming).
static bool trim(const BlockCtx& b, double delta, int& i0, int& i1, int& j0, int& j1) {
  i0 = b.nr; i1 = -1; j0 = b.nc; j1 = -1;
  for (int j = 0; j < b.nc; ++j)
    for (int i = 0; i < b.nr; ++i)
      if (std::fabs(b.K(i, j)) >= delta) {
        i0 = std::min(i0, i); i1 = std::max(i1, i);
        j0 = std::min(j0, j); j1 = std::max(j1, j);
      }
  if (i1 < 0) return false;
  ++i1; ++j1;
  return true;
}

static void emit_block(UnitBuild& ub, const ParityMatrix& P, const sht_opts& o, Rng& rng, int i0, int nr, int j0,
                       int nc, BlockClass cls) {
  const bool force = (o.flags & 1) != 0;
  BlockCtx b{&P, i0, nr, j0, nc, &o, o.eps * P.scale, &rng};
  if (cls == B_OSC) {
    int mn = std::min(nr, nc);
    int L = -1;
    while ((mn >> (L + 1)) >= o.n_leaf) ++L;  // largest L with mn / 2^L >= n_leaf
    if (L >= 0 && emit_idbf(ub, b, L, force)) return;
    ub.dbg[L >= 0 ? 0 : 1] += (int64_t)nr * nc;  // osc block kept dense (IDBF not smaller / too small)
    emit_dense(ub, b);
    return;
  }
  int ti0, ti1, tj0, tj1;
  if (!trim(b, o.trim_delta * P.scale, ti0, ti1, tj0, tj1)) { ub.n_drop += 1; return; }
  BlockCtx t{&P, i0 + ti0, ti1 - ti0, j0 + tj0, tj1 - tj0, &o, b.tol, &rng};
  ub.dbg[cls == B_NONOSC ? 4 : 5] += (int64_t)nr * nc;  // area before trimming
  if (cls == B_NONOSC && emit_lowrank(ub, t, force)) return;
  ub.dbg[cls == B_NONOSC ? 2 : 3] += (int64_t)t.nr * t.nc;  // trimmed block kept dense
  emit_dense(ub, t);
}

static BlockClass classify(const ParityMatrix& P, int i0, int i1, int j0, int j1) {
  if (P.osc(i1 - 1, j0)) return B_OSC;       // least oscillatory corner
  if (!P.osc(i0, j1 - 1)) return B_NONOSC;   // most oscillatory corner
  return B_CROSS;
}

static void partition(UnitBuild& ub, const ParityMatrix& P, const sht_opts& o, Rng& rng, int i0, int i1, int j0,
                      int j1) {
  BlockClass c = classify(P, i0, i1, j0, j1);
  if (c == B_CROSS && (i1 - i0) >= o.n0 && (j1 - j0) >= o.n0) {
    int im = i0 + (i1 - i0 + 1) / 2, jm = j0 + (j1 - j0 + 1) / 2;
    partition(ub, P, o, rng, i0, im, j0, jm);
    partition(ub, P, o, rng, i0, im, jm, j1);
    partition(ub, P, o, rng, im, i1, j0, jm);
    partition(ub, P, o, rng, im, i1, jm, j1);
    return;
  }
  emit_block(ub, P, o, rng, i0, i1 - i0, j0, j1 - j0, c);
}

static void build_parity(UnitBuild& ub, const ParityMatrix& P, const sht_opts& o, Rng& rng) {
  const int N = P.A->r, nc = P.A->c;
  if (nc == 0) return;
  if (o.flags & SHT_FLAG_DENSE) {  // the unfactored O(N^3) transform: every entry, no trimming
    BlockCtx b{&P, 0, N, 0, nc, &o, 0.0, &rng};
    emit_dense(ub, b);
    return;
  }
  // Eq. nb: b row blocks of ~N/b rows, each holding all columns (nearly square)
  long b = std::lround((double)N / (double)nc);
  b = std::max(1L, std::min((long)N, b));
  for (long t = 0; t < b; ++t) {
    int r0 = (int)(t * (N / b) + std::min<long>(t, N % b));
    int r1 = (int)((t + 1) * (N / b) + std::min<long>(t + 1, N % b));
    partition(ub, P, o, rng, r0, r1, 0, nc);
  }
}

static void build_unit(int N, int am, const sht_opts& o, const double* xp, UnitBuild& ub, Unit& u,
                       double* t_mat = nullptr, LegendreSource* src = nullptr) {
  Mat E, O;
  const auto t0 = std::chrono::steady_clock::now();
  if (src) {
    if (!src->parity_matrices(N, am, xp, E, O)) {
      ub.err = "device Legendre evaluation failed";
      return;
    }
  } else {
    legendre_parity_matrices(N, am, xp, E, O);
  }
  if (t_mat) *t_mat = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  const int nce = E.c, nco = O.c;
  u = Unit{};
  u.am = am;
  u.nce = nce;
  u.nco = nco;
  u.xe = 0;
  u.xo = nce;
  u.ye = nce + nco;
  u.yo = nce + nco + N;
  ub.nrows = nce + nco + 2 * N;
  // the unit's factors usually take less room than its two dense matrices
  // (rounded to 4 rows): reserving that keeps the store from being copied as
  // it grows block by block.  Capped at 2^21 doubles (16 MB, every unit up to
  // N = 1024), since all units' stores are alive until they are concatenated.
  ub.fac.reserve(std::min<size_t>((size_t)((N + 3) & ~3) * (size_t)(nce + nco), (size_t)1 << 21));
  auto maxabs = [](const Mat& A) {
    double s = 0.0;
    for (double v : A.a) s = std::max(s, std::fabs(v));
    return s;
  };
  ParityMatrix PE{&E, am, 0, xp, maxabs(E), u.xe, u.ye};
  ParityMatrix PO{&O, am, 1, xp, maxabs(O), u.xo, u.yo};
  Rng rng(o.seed ^ (0x51ED27A3ull * (uint64_t)(am + 1)));
  build_parity(ub, PE, o, rng);
  build_parity(ub, PO, o, rng);
  std::stable_sort(ub.ops.begin(), ub.ops.end(), [](const Op& a, const Op& b) { return a.phase < b.phase; });
  u.nrows = ub.nrows;
  u.nphase = ub.nphase;
  u.cost = (float)ub.cost;
}

sht_status build_program(int N, const sht_opts& opts, HostProgram& P, std::string& err, LegendreSource* src) {
  auto t0 = std::chrono::steady_clock::now();
  P = HostProgram{};
  P.N = N;
  P.opts = opts;
  gauss_legendre(2 * N, P.x, P.w);
  const double* xp = P.x.data() + N;
  const int K = 2 * N;
  std::vector<UnitBuild> ub(K);
  std::vector<Unit> units(K);
  int threads = 1;
#ifdef _OPENMP
  threads = omp_get_max_threads();
#endif
  // heavy orders (small |m|) first
#pragma omp parallel for schedule(dynamic, 1)
  for (int am = 0; am < K; ++am) build_unit(N, am, opts, xp, ub[am], units[am], nullptr, src);
  for (int am = 0; am < K; ++am)
    if (ub[am].err == "device Legendre evaluation failed") {
      err = ub[am].err + " at order " + std::to_string(am);
      return SHT_ERR_CUDA;
    }
  const auto t_units = std::chrono::steady_clock::now();

  // concatenate into the global program: offsets first, then every unit's
  // factors and ops copied in parallel to their places
  sht_plan_info& I = P.info;
  std::vector<int64_t> fac_at(K + 1, 0), op_at(K + 1, 0);
  for (int am = 0; am < K; ++am) {
    fac_at[am + 1] = fac_at[am] + (int64_t)ub[am].fac.size();
    op_at[am + 1] = op_at[am] + (int64_t)ub[am].ops.size();
  }
  // the store is left uninitialised here (FactorStore): the copies below
  // write every element, and first touch its pages from all threads
  P.factors.resize((size_t)fac_at[K]);
  P.ops.resize((size_t)op_at[K]);
#pragma omp parallel for schedule(dynamic, 4)
  for (int am = 0; am < K; ++am) {
    UnitBuild& b = ub[am];
    std::copy(b.fac.begin(), b.fac.end(), P.factors.begin() + fac_at[am]);
    for (size_t q = 0; q < b.ops.size(); ++q) {
      Op op = b.ops[q];
      op.b_off += fac_at[am];
      P.ops[(size_t)op_at[am] + q] = op;
    }
    std::vector<double>().swap(b.fac);  // the unit's copy is no longer needed
  }
  const auto t_concat = std::chrono::steady_clock::now();
  P.units = units;
  for (int am = 0; am < K; ++am) {
    UnitBuild& b = ub[am];
    Unit& u = P.units[am];
    u.op_begin = (int32_t)op_at[am];
    u.op_end = (int32_t)op_at[am + 1];
    u.ph_begin = (int32_t)P.phase_tab.size();
    int idx = u.op_begin;
    for (int ph = 0; ph <= u.nphase; ++ph) {
      while (idx < u.op_end && P.ops[idx].phase < ph) ++idx;
      P.phase_tab.push_back(idx);
    }
    P.max_rows = std::max(P.max_rows, u.nrows);
    I.n_blocks_idbf += b.n_idbf;
    I.n_blocks_lowrank += b.n_low;
    I.n_blocks_dense += b.n_dense;
    I.n_blocks_dropped += b.n_drop;
    P.unit_blocks.insert(P.unit_blocks.end(), {(int32_t)b.n_idbf, (int32_t)b.n_low, (int32_t)b.n_dense, (int32_t)b.n_drop});
    I.entries_idbf += b.e_idbf;
    I.entries_lowrank += b.e_low;
    I.entries_dense += b.e_dense;
    I.max_rank = std::max(I.max_rank, b.max_rank);
    I.max_phases = std::max<int64_t>(I.max_phases, u.nphase);
    I.entries_matrix += (int64_t)N * (u.nce + u.nco);
  }
  P.order.resize(K);
  std::iota(P.order.begin(), P.order.end(), 0);
  std::stable_sort(P.order.begin(), P.order.end(),
                   [&](int a, int b) { return P.units[a].cost > P.units[b].cost; });
  if (!validate_program(P, err)) return SHT_ERR_NUMERIC;
  if (std::getenv("SHT_PLAN_DEBUG")) {
    int64_t d[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int am = 0; am < K; ++am)
      for (int t = 0; t < 8; ++t) d[t] += ub[am].dbg[t];
    std::fprintf(stderr,
                 "[plan] dense area: osc(idbf not smaller)=%lld osc(small)=%lld nonosc(trimmed)=%lld "
                 "cross(trimmed)=%lld | untrimmed area nonosc=%lld cross=%lld\n",
                 (long long)d[0], (long long)d[1], (long long)d[2], (long long)d[3], (long long)d[4],
                 (long long)d[5]);
    auto sec = [](std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
      return std::chrono::duration<double>(b - a).count();
    };
    std::fprintf(stderr, "[plan] units %.3f s, concatenation %.3f s, tables and checks %.3f s\n", sec(t0, t_units),
                 sec(t_units, t_concat), sec(t_concat, std::chrono::steady_clock::now()));
  }
  I.N = N;
  I.eps = opts.eps;
  I.n_units = K;
  I.n_ops = (int64_t)P.ops.size();
  I.entries_total = I.entries_idbf + I.entries_lowrank + I.entries_dense;
  I.threads = threads;
  I.t_factor_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return SHT_OK;
}

sht_status build_orders(int N, const sht_opts& opts, int count, const int* am, std::vector<OrderBuild>& out) {
  std::vector<double> x, w;
  gauss_legendre(2 * N, x, w);
  const double* xp = x.data() + N;
  out.assign((size_t)count, OrderBuild{});
  bool oom = false;
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < count; ++i) {
    OrderBuild& r = out[(size_t)i];
    try {
      UnitBuild ub;
      const auto t0 = std::chrono::steady_clock::now();
      build_unit(N, am[i], opts, xp, ub, r.unit, &r.t_mat_s);
      r.t_fac_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() - r.t_mat_s;
      r.unit.op_begin = 0;
      r.unit.op_end = (int32_t)ub.ops.size();
      r.ops = std::move(ub.ops);
      r.n_factors = (int64_t)ub.fac.size();
      r.n_idbf = ub.n_idbf;
      r.n_low = ub.n_low;
      r.n_dense = ub.n_dense;
      r.n_drop = ub.n_drop;
      r.e_idbf = ub.e_idbf;
      r.e_low = ub.e_low;
      r.e_dense = ub.e_dense;
      r.max_rank = ub.max_rank;
    } catch (const std::bad_alloc&) {
#pragma omp atomic write
      oom = true;
    }
  }
  return oom ? SHT_ERR_OOM : SHT_OK;
}

bool validate_program(const HostProgram& P, std::string& err) {
  const int N = P.N;
  const int K = 2 * N;
  auto fail = [&](const char* what, int am) {
    err = std::string(what) + " at order " + std::to_string(am);
    return false;
  };
  if (N < 1 || (int)P.x.size() != K || (int)P.w.size() != K || (int)P.units.size() != K ||
      (int)P.order.size() != K || P.max_rows < 0) {
    err = "program sizes do not match N";
    return false;
  }
  // the schedule is a permutation of the orders
  std::vector<char> seen(K, 0);
  for (int32_t v : P.order) {
    if (v < 0 || v >= K || seen[v]) {
      err = "schedule is not a permutation of the orders";
      return false;
    }
    seen[v] = 1;
  }
  const int64_t nops = (int64_t)P.ops.size(), nfac = (int64_t)P.factors.size();
  const int64_t nph = (int64_t)P.phase_tab.size();
  for (int am = 0; am < K; ++am) {
    const Unit& u = P.units[am];
    // vector-space layout: X_e, X_o, Y_e, Y_o, then the butterfly rows
    const int nce = N - am / 2, nco = 2 * N - am - nce;
    if (u.am != am || u.nce != nce || u.nco != nco || u.xe != 0 || u.xo != nce || u.ye != nce + nco ||
        u.yo != u.ye + N || u.nrows < u.yo + N || u.nrows > P.max_rows)
      return fail("unit layout failed validation", am);
    if (u.op_begin < 0 || u.op_end < u.op_begin || u.op_end > nops || u.nphase < 0 || u.ph_begin < 0 ||
        (int64_t)u.ph_begin + u.nphase + 1 > nph)
      return fail("unit op range failed validation", am);
    const int32_t* ph = P.phase_tab.data() + u.ph_begin;
    if (ph[0] != u.op_begin || ph[u.nphase] != u.op_end) return fail("phase table failed validation", am);
    for (int q = 0; q < u.nphase; ++q) {
      if (ph[q + 1] < ph[q]) return fail("phase table failed validation", am);
      for (int oi = ph[q]; oi < ph[q + 1]; ++oi)
        if (P.ops[oi].phase != q) return fail("phase table failed validation", am);
    }
    // every op stays inside its unit's vector space and the factor store
    for (int oi = u.op_begin; oi < u.op_end; ++oi) {
      const Op& op = P.ops[oi];
      bool ok = op.mo >= 1 && op.ni >= 0 && op.ld >= op.mo && op.ld % 4 == 0 && op.b_off >= 0 &&
                op.b_off % 4 == 0 && op.b_off + (int64_t)op.ld * op.ni <= nfac && op.in_len[0] >= 0 &&
                op.in_len[1] >= 0 && op.in_len[0] + op.in_len[1] == op.ni && op.out_len[0] >= 0 &&
                op.out_len[1] >= 0 && op.out_len[0] + op.out_len[1] == op.mo && op.phase >= 0 &&
                op.phase < u.nphase && (op.flags & ~(OP_FWD_ACCUM | OP_BWD_ACCUM)) == 0;
      for (int s = 0; s < 2 && ok; ++s) {
        ok = ok && op.in_off[s] >= 0 && op.in_off[s] + op.in_len[s] <= u.nrows;
        ok = ok && op.out_off[s] >= 0 && op.out_off[s] + op.out_len[s] <= u.nrows;
      }
      if (!ok) return fail("apply program failed validation", am);
      // intermediate segments (past Y_o) start on 8-row groups: the tensor-core
      // apply copies whole groups and relies on the rows that pad a segment to
      // its group end being written by no op
      for (int s = 0; s < 2 && ok; ++s) {
        if (op.in_len[s] > 0 && op.in_off[s] >= u.yo + N) ok = op.in_off[s] % 8 == 0;
        if (ok && op.out_len[s] > 0 && op.out_off[s] >= u.yo + N) ok = op.out_off[s] % 8 == 0;
      }
      if (!ok) return fail("intermediate segment not on an 8-row boundary", am);
      // shared rows are exactly the accumulated ones: an op writes Y rows (the
      // N-node outputs of both parities) iff it accumulates forward, and reads
      // X rows (the coefficients) iff its transpose accumulates
      for (int s = 0; s < 2 && ok; ++s) {
        if (op.out_len[s] > 0) {
          const bool in_y = op.out_off[s] >= u.ye && op.out_off[s] + op.out_len[s] <= u.ye + 2 * N;
          const bool off_y = op.out_off[s] + op.out_len[s] <= u.ye || op.out_off[s] >= u.ye + 2 * N;
          ok = (op.flags & OP_FWD_ACCUM) ? in_y : off_y;
        }
        if (ok && op.in_len[s] > 0) {
          const bool in_x = op.in_off[s] + op.in_len[s] <= nce + nco;
          const bool off_x = op.in_off[s] >= nce + nco;
          ok = (op.flags & OP_BWD_ACCUM) ? in_x : off_x;
        }
      }
      if (!ok) return fail("accumulated rows failed validation", am);
    }
  }
  return true;
}

}  // namespace sht
