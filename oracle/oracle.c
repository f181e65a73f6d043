/*
 * Dense FP64 CPU oracle for the associated Legendre transform (ALT) and the
 * spherical harmonic transform (SHT) of Bremer, Chen & Yang,
 * "Rapid Application of the Spherical Harmonic Transform via Interpolative
 * Decomposition Butterfly Factorization" (arXiv:2004.11346).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path links,
 * loads or calls this file; only the tests, the smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code with the CUDA path.
 *
 * Everything here is the plain definition of the maps, written out with no
 * blocking, no parity folding and no factorisation:
 *   - Gauss-Legendre rule on 2N nodes (Sec. 1, the grid; Sec. 3.1.1).
 *   - L2-normalised associated Legendre functions by the textbook three-term
 *     recurrence, carried with an extended exponent so that values far below
 *     the FP64 range do not underflow before they grow back (Sec. 1, Eq. sht_re).
 *   - Forward ALT: g(m,theta_l) = sum_{k>=|m|} beta_{k,m} Pbar_k^{|m|}(x_l)
 *     (Eq. sht_lt / Eq. new1).
 *   - Inverse ALT: beta_{k,m} = sum_l w_l Pbar_k^{|m|}(x_l) g(m,theta_l)
 *     (Sec. 3.1.1, B = A^T W).
 *   - phi-direction synthesis f(theta_l,phi_j) = sum_m g(m,theta_l) e^{i m phi_j}
 *     with phi_j = 2 pi (j + 1/2)/(4N-1) (Eq. sht_fft), and its inverse
 *     (1/M) sum_j f e^{-i m phi_j}, M = 4N-1, written as direct sums.
 *
 * Conventions (shared with the library only through the documented ABI):
 *   - No Condon-Shortley phase: Pbar_m^m(x) > 0 on (-1,1).
 *   - int_{-1}^{1} Pbar_k^m(x)^2 dx = 1.
 *   - Orders are stored in the sequence m = 0, 1, -1, 2, -2, ..., 2N-1, -(2N-1).
 *     Coefficients: for each order, degrees k = |m|..2N-1 contiguous
 *     (4N^2 complex per field).  ALT values: for each order, the 2N nodes in
 *     ascending x ((4N-1)*2N complex per field).  Grid values: theta-major,
 *     2N rows of 4N-1 phi samples.  Complex numbers are interleaved (re, im).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Layout helpers: position of order m in the sequence 0, 1, -1, 2, -2, ...  */

static long order_slot(long m) { return m == 0 ? 0 : (m > 0 ? 2 * m - 1 : -2 * m); }

/* First coefficient of order m: orders before it hold 2N-|m'| degrees each. */
static long coef_offset(long N, long m) {
  long a = m < 0 ? -m : m;
  if (a == 0) return 0;
  long off_pos = 2 * N * (2 * a - 1) - a * (a - 1); /* 2N + 2*sum_{mu=1}^{a-1}(2N-mu) */
  return m > 0 ? off_pos : off_pos + (2 * N - a);
}

long oracle_coef_offset(long N, long m) { return coef_offset(N, m); }
long oracle_order_slot(long m) { return order_slot(m); }

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre rule (Sec. 1: 2N-point rule in x = cos(theta), ascending).  */
/* Newton's method on the Legendre polynomial P_n, evaluated by Bonnet's      */
/* recurrence; weights 2 / ((1 - x^2) P_n'(x)^2).                            */

static void legendre_p_and_dp(int n, double x, double* p, double* dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / (double)k;
    p0 = p1;
    p1 = p2;
  }
  *p = p1;
  *dp = (double)n * (x * p1 - p0) / (x * x - 1.0);
}

int oracle_gl_rule(int n, double* x, double* w) {
  if (n < 1) return 1;
  const double pi = 3.14159265358979323846;
#pragma omp parallel for schedule(dynamic, 16)
  for (int j = 0; j < n; ++j) {
    /* j-th largest root; stored at index n-1-j so that x is ascending. */
    double z = cos(pi * (j + 0.75) / (n + 0.5));
    double p, dp;
    for (int it = 0; it < 100; ++it) {
      legendre_p_and_dp(n, z, &p, &dp);
      double dz = p / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    legendre_p_and_dp(n, z, &p, &dp);
    x[n - 1 - j] = z;
    w[n - 1 - j] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Extended-exponent numbers: value = f * BIG^e with BIG = 2^960, |f| kept in */
/* [2^-480, 2^480).  This keeps Pbar_m^m(x), which can be far below 1e-308    */
/* for large m near the poles, representable until the recurrence in k       */
/* brings it back into range.                                                 */

typedef struct { double f; int e; } xnum;

static const double XBIG = 0x1p960;
static const double XBIGI = 0x1p-960;
static const double XHI = 0x1p480;
static const double XLO = 0x1p-480;

static xnum xnorm(xnum a) {
  double af = fabs(a.f);
  if (a.f == 0.0) { a.e = 0; return a; }
  if (af >= XHI) { a.f *= XBIGI; a.e += 1; }
  else if (af < XLO) { a.f *= XBIG; a.e -= 1; }
  return a;
}

static double xtod(xnum a) {
  if (a.e == 0) return a.f;
  if (a.e == -1) return a.f * XBIGI;
  if (a.e < -1) return 0.0;
  return a.f * XBIG; /* not reached for normalised Legendre values */
}

/* s * a + t * b for ordinary doubles s, t */
static xnum xlin(double s, xnum a, double t, xnum b) {
  xnum r;
  /* a zero carries no exponent: never align the other operand to it */
  if (b.f == 0.0 || t == 0.0) { r.f = s * a.f; r.e = a.e; return xnorm(r); }
  if (a.f == 0.0 || s == 0.0) { r.f = t * b.f; r.e = b.e; return xnorm(r); }
  int d = a.e - b.e;
  if (d == 0) { r.f = s * a.f + t * b.f; r.e = a.e; }
  else if (d == 1) { r.f = s * a.f + t * b.f * XBIGI; r.e = a.e; }
  else if (d == -1) { r.f = s * a.f * XBIGI + t * b.f; r.e = b.e; }
  else if (d > 1) { r.f = s * a.f; r.e = a.e; }
  else { r.f = t * b.f; r.e = b.e; }
  return xnorm(r);
}

/* Normalised associated Legendre functions Pbar_k^m(x), k = m..kmax, for one
 * order m >= 0 and one argument x in [-1, 1]; out[k-m].
 *   Pbar_0^0 = 1/sqrt(2)
 *   Pbar_m^m = sqrt((2m+1)/(2m)) sqrt(1-x^2) Pbar_{m-1}^{m-1}
 *   Pbar_{m+1}^m = sqrt(2m+3) x Pbar_m^m
 *   Pbar_k^m = a_k x Pbar_{k-1}^m - b_k Pbar_{k-2}^m,
 *     a_k = sqrt((4k^2-1)/(k^2-m^2)),
 *     b_k = sqrt((2k+1)(k-1-m)(k-1+m)/((2k-3)(k^2-m^2))).                     */
static void alf_column(int m, int kmax, double x, double* out) {
  double u = sqrt((1.0 - x) * (1.0 + x));
  xnum pmm = {1.0 / sqrt(2.0), 0};
  for (int j = 1; j <= m; ++j) {
    pmm.f *= sqrt((2.0 * j + 1.0) / (2.0 * j)) * u;
    pmm = xnorm(pmm);
  }
  if (kmax < m) return;
  out[0] = xtod(pmm);
  if (kmax == m) return;
  xnum zero = {0.0, 0};
  xnum p1 = xlin(sqrt(2.0 * m + 3.0) * x, pmm, 0.0, zero); /* k = m+1 */
  out[1] = xtod(p1);
  xnum p0 = pmm;
  for (int k = m + 2; k <= kmax; ++k) {
    double kk = (double)k, mm = (double)m;
    double den = kk * kk - mm * mm;
    double a = sqrt((4.0 * kk * kk - 1.0) / den);
    double b = sqrt((2.0 * kk + 1.0) * (kk - 1.0 - mm) * (kk - 1.0 + mm) / ((2.0 * kk - 3.0) * den));
    xnum p2 = xlin(a * x, p1, -b, p0);
    out[k - m] = xtod(p2);
    p0 = p1;
    p1 = p2;
  }
}

/* Table out[i*(kmax-m+1) + (k-m)] = Pbar_k^m(x_i). */
int oracle_alf_table(int m, int kmax, const double* x, int nx, double* out) {
  if (m < 0 || kmax < m) return 1;
  int nk = kmax - m + 1;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < nx; ++i) alf_column(m, kmax, x[i], out + (size_t)i * nk);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Forward ALT (Eq. sht_lt): for every order |m| <= 2N-1 and every node x_l,  */
/*   g(m, theta_l) = sum_{k=|m|}^{2N-1} beta_{k,m} Pbar_k^{|m|}(x_l),          */
/* for both signs of m (they share Pbar^{|m|}).  F fields, field stride 4N^2  */
/* complex for beta and (4N-1)*2N complex for g.                              */
int oracle_alt_forward(int N, const double* x, const double* beta, double* g, int F) {
  if (N < 1 || F < 0) return 1;
  const long K = 2L * N, ncoef = 4L * N * N, nval = (4L * N - 1) * K;
#pragma omp parallel
  {
    double* col = (double*)malloc(sizeof(double) * K);
#pragma omp for schedule(dynamic, 1)
    for (int am = 0; am < K; ++am) {
      for (int l = 0; l < K; ++l) {
        alf_column(am, (int)K - 1, x[l], col);
        for (int s = 0; s < (am == 0 ? 1 : 2); ++s) {
          long m = s == 0 ? am : -am;
          long co = coef_offset(N, m), go = order_slot(m) * K + l;
          for (int f = 0; f < F; ++f) {
            const double* b = beta + 2 * (f * ncoef + co);
            double re = 0.0, im = 0.0;
            for (int k = am; k < K; ++k) {
              re += b[2 * (k - am)] * col[k - am];
              im += b[2 * (k - am) + 1] * col[k - am];
            }
            g[2 * (f * nval + go)] = re;
            g[2 * (f * nval + go) + 1] = im;
          }
        }
      }
    }
    free(col);
  }
  return 0;
}

/* Inverse ALT (Sec. 3.1.1, B = A^T W): for every order and degree,           */
/*   beta_{k,m} = sum_{l=0}^{2N-1} w_l Pbar_k^{|m|}(x_l) g(m, theta_l).        */
int oracle_alt_inverse(int N, const double* x, const double* w, const double* g, double* beta, int F) {
  if (N < 1 || F < 0) return 1;
  const long K = 2L * N, ncoef = 4L * N * N, nval = (4L * N - 1) * K;
#pragma omp parallel
  {
    double* col = (double*)malloc(sizeof(double) * K);
#pragma omp for schedule(dynamic, 1)
    for (int am = 0; am < K; ++am) {
      for (int s = 0; s < (am == 0 ? 1 : 2); ++s) {
        long m = s == 0 ? am : -am;
        long co = coef_offset(N, m);
        for (int f = 0; f < F; ++f)
          memset(beta + 2 * (f * ncoef + co), 0, sizeof(double) * 2 * (K - am));
      }
      for (int l = 0; l < K; ++l) {
        alf_column(am, (int)K - 1, x[l], col);
        for (int s = 0; s < (am == 0 ? 1 : 2); ++s) {
          long m = s == 0 ? am : -am;
          long co = coef_offset(N, m), go = order_slot(m) * K + l;
          for (int f = 0; f < F; ++f) {
            double gr = w[l] * g[2 * (f * nval + go)];
            double gi = w[l] * g[2 * (f * nval + go) + 1];
            double* b = beta + 2 * (f * ncoef + co);
            for (int k = am; k < K; ++k) {
              b[2 * (k - am)] += col[k - am] * gr;
              b[2 * (k - am) + 1] += col[k - am] * gi;
            }
          }
        }
      }
    }
    free(col);
  }
  return 0;
}

/* Forward ALT restricted to one order m and an arbitrary list of nodes:      */
/* g[i] = sum_k beta_k Pbar_k^{|m|}(x_i), beta for that order only.  Used to  */
/* check sampled outputs at large N.                                          */
int oracle_alt_forward_m(int N, int m, const double* x, int nx, const double* beta_m, double* g_m) {
  int am = m < 0 ? -m : m;
  if (N < 1 || am > 2 * N - 1) return 1;
  const int K = 2 * N;
#pragma omp parallel
  {
    double* col = (double*)malloc(sizeof(double) * K);
#pragma omp for schedule(static)
    for (int i = 0; i < nx; ++i) {
      alf_column(am, K - 1, x[i], col);
      double re = 0.0, im = 0.0;
      for (int k = am; k < K; ++k) {
        re += beta_m[2 * (k - am)] * col[k - am];
        im += beta_m[2 * (k - am) + 1] * col[k - am];
      }
      g_m[2 * i] = re;
      g_m[2 * i + 1] = im;
    }
    free(col);
  }
  return 0;
}

/* Inverse ALT for one order: beta_m[k-|m|] = sum_l w_l Pbar_k^{|m|}(x_l) g_m[l]
 * over all 2N nodes. */
int oracle_alt_inverse_m(int N, int m, const double* x, const double* w, const double* g_m, double* beta_m) {
  int am = m < 0 ? -m : m;
  if (N < 1 || am > 2 * N - 1) return 1;
  const int K = 2 * N;
  double* col = (double*)malloc(sizeof(double) * K);
  memset(beta_m, 0, sizeof(double) * 2 * (K - am));
  for (int l = 0; l < K; ++l) {
    alf_column(am, K - 1, x[l], col);
    for (int k = am; k < K; ++k) {
      beta_m[2 * (k - am)] += col[k - am] * w[l] * g_m[2 * l];
      beta_m[2 * (k - am) + 1] += col[k - am] * w[l] * g_m[2 * l + 1];
    }
  }
  free(col);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* phi direction (Eq. sht_fft), direct sums.  M = 4N-1 samples              */
/* phi_j = 2 pi (j + 1/2) / M, so m phi_j = pi * (m (2j+1) mod 2M) / M; the   */
/* product is reduced exactly in integers before the cosine and sine.         */

static void phase(long m, long j, long M, double* c, double* s) {
  const double pi = 3.14159265358979323846;
  long r = (m * (2 * j + 1)) % (2 * M);
  if (r < 0) r += 2 * M;
  double ang = pi * (double)r / (double)M;
  *c = cos(ang);
  *s = sin(ang);
}

/* f[l][j] = sum_{m=-(2N-1)}^{2N-1} g(m, theta_l) e^{i m phi_j} */
int oracle_phi_synthesis(int N, const double* g, double* f, int F) {
  if (N < 1 || F < 0) return 1;
  const long K = 2L * N, M = 4L * N - 1, nval = M * K, ngrid = K * M;
#pragma omp parallel for collapse(2) schedule(static)
  for (long l = 0; l < K; ++l) {
    for (long j = 0; j < M; ++j) {
      for (int fi = 0; fi < F; ++fi) {
        double re = 0.0, im = 0.0;
        for (long m = -(K - 1); m <= K - 1; ++m) {
          double c, s;
          phase(m, j, M, &c, &s);
          const double* gv = g + 2 * (fi * nval + order_slot(m) * K + l);
          re += gv[0] * c - gv[1] * s;
          im += gv[0] * s + gv[1] * c;
        }
        f[2 * (fi * ngrid + l * M + j)] = re;
        f[2 * (fi * ngrid + l * M + j) + 1] = im;
      }
    }
  }
  return 0;
}

/* g(m, theta_l) = (1/M) sum_{j=0}^{M-1} f[l][j] e^{-i m phi_j} */
int oracle_phi_analysis(int N, const double* f, double* g, int F) {
  if (N < 1 || F < 0) return 1;
  const long K = 2L * N, M = 4L * N - 1, nval = M * K, ngrid = K * M;
#pragma omp parallel for collapse(2) schedule(static)
  for (long l = 0; l < K; ++l) {
    for (long m = -(K - 1); m <= K - 1; ++m) {
      for (int fi = 0; fi < F; ++fi) {
        double re = 0.0, im = 0.0;
        for (long j = 0; j < M; ++j) {
          double c, s;
          phase(m, j, M, &c, &s);
          const double* fv = f + 2 * (fi * ngrid + l * M + j);
          re += fv[0] * c + fv[1] * s;
          im += fv[1] * c - fv[0] * s;
        }
        double* gv = g + 2 * (fi * nval + order_slot(m) * K + l);
        gv[0] = re / (double)M;
        gv[1] = im / (double)M;
      }
    }
  }
  return 0;
}

/* The same two sums at a chosen set of nl nodes only (large N, where the   */
/* full grid is out of reach): g holds the nodes' values of every order,    */
/* (F x M x nl) in the order sequence above, f their grid rows (F x nl x M). */
int oracle_phi_synthesis_nodes(int N, int nl, const double* g, double* f, int F) {
  if (N < 1 || nl < 0 || F < 0) return 1;
  const long K = 2L * N, M = 4L * N - 1, L = nl;
#pragma omp parallel for collapse(2) schedule(static)
  for (long l = 0; l < L; ++l) {
    for (long j = 0; j < M; ++j) {
      for (int fi = 0; fi < F; ++fi) {
        double re = 0.0, im = 0.0;
        for (long m = -(K - 1); m <= K - 1; ++m) {
          double c, s;
          phase(m, j, M, &c, &s);
          const double* gv = g + 2 * ((fi * M + order_slot(m)) * L + l);
          re += gv[0] * c - gv[1] * s;
          im += gv[0] * s + gv[1] * c;
        }
        f[2 * ((fi * L + l) * M + j)] = re;
        f[2 * ((fi * L + l) * M + j) + 1] = im;
      }
    }
  }
  return 0;
}

int oracle_phi_analysis_nodes(int N, int nl, const double* f, double* g, int F) {
  if (N < 1 || nl < 0 || F < 0) return 1;
  const long K = 2L * N, M = 4L * N - 1, L = nl;
#pragma omp parallel for collapse(2) schedule(static)
  for (long l = 0; l < L; ++l) {
    for (long m = -(K - 1); m <= K - 1; ++m) {
      for (int fi = 0; fi < F; ++fi) {
        double re = 0.0, im = 0.0;
        for (long j = 0; j < M; ++j) {
          double c, s;
          phase(m, j, M, &c, &s);
          const double* fv = f + 2 * ((fi * L + l) * M + j);
          re += fv[0] * c + fv[1] * s;
          im += fv[1] * c - fv[0] * s;
        }
        double* gv = g + 2 * ((fi * M + order_slot(m)) * L + l);
        gv[0] = re / (double)M;
        gv[1] = im / (double)M;
      }
    }
  }
  return 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
