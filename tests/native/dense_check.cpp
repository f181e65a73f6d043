// Runs the plan builder's dense routines (csrc/dense.hpp) on a matrix read
// from a file, for comparison with numpy in tests/test_dense.py.
//
//   dense_check <mode> <in> <out> [tol]
//
// Files hold int32 rows, int32 cols, then the column-major float64 entries.
// Modes and what <out> receives (matrices in the same format, one after the
// other):
//   qr    pivoted_qr(A, tol): k (as a 1x1 matrix), perm (1 x n), R (k x n)
//   id    pivoted_qr + upper_solve: the interpolative decomposition
//         A ~ A(:, skel) V with V = [I T] P^T: skel (1 x k), V (k x n)
//   svd   jacobi_svd(A): U (m x n), s (1 x n), V (n x n)
//   thinq thin_q(A): Q
//   pinv  pinv(A)
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "dense.hpp"

using namespace sht;

static bool read_mat(const char* path, Mat& A) {
  std::FILE* f = std::fopen(path, "rb");
  if (!f) return false;
  int32_t rc[2];
  bool ok = std::fread(rc, sizeof rc, 1, f) == 1 && rc[0] >= 0 && rc[1] >= 0;
  if (ok) {
    A = Mat(rc[0], rc[1]);
    ok = A.a.empty() || std::fread(A.a.data(), sizeof(double), A.a.size(), f) == A.a.size();
  }
  std::fclose(f);
  return ok;
}

static void write_mat(std::FILE* f, const Mat& A) {
  const int32_t rc[2] = {A.r, A.c};
  std::fwrite(rc, sizeof rc, 1, f);
  if (!A.a.empty()) std::fwrite(A.a.data(), sizeof(double), A.a.size(), f);
}

static Mat row_of(const std::vector<double>& v) {
  Mat M(1, (int)v.size());
  for (size_t j = 0; j < v.size(); ++j) M(0, (int)j) = v[j];
  return M;
}

int main(int argc, char** argv) {
  if (argc < 4) return 2;
  const std::string mode = argv[1];
  const double tol = argc > 4 ? std::atof(argv[4]) : 0.0;
  Mat A;
  if (!read_mat(argv[2], A)) return 3;
  std::FILE* out = std::fopen(argv[3], "wb");
  if (!out) return 4;
  if (mode == "qr" || mode == "id") {
    Mat M = A;
    std::vector<int> perm;
    const int k = pivoted_qr(M, tol, std::min(M.r, M.c), perm);
    if (mode == "qr") {
      write_mat(out, row_of({(double)k}));
      write_mat(out, row_of(std::vector<double>(perm.begin(), perm.end())));
      Mat R(k, M.c);
      for (int j = 0; j < M.c; ++j)
        for (int i = 0; i < k && i <= j; ++i) R(i, j) = M(i, j);
      write_mat(out, R);
    } else {
      Mat T(k, M.c - k);
      for (int j = 0; j < M.c - k; ++j)
        for (int i = 0; i < k; ++i) T(i, j) = M(i, k + j);
      upper_solve(M, k, T);
      Mat V(k, M.c);
      for (int j = 0; j < k; ++j) V(j, perm[j]) = 1.0;
      for (int j = 0; j < M.c - k; ++j)
        for (int i = 0; i < k; ++i) V(i, perm[k + j]) = T(i, j);
      write_mat(out, row_of(std::vector<double>(perm.begin(), perm.begin() + k)));
      write_mat(out, V);
    }
  } else if (mode == "svd") {
    Mat U, V;
    std::vector<double> s;
    jacobi_svd(A, U, s, V);
    write_mat(out, U);
    write_mat(out, row_of(s));
    write_mat(out, V);
  } else if (mode == "thinq") {
    write_mat(out, thin_q(A));
  } else if (mode == "pinv") {
    write_mat(out, pinv(A));
  } else {
    std::fclose(out);
    return 5;
  }
  std::fclose(out);
  return 0;
}
