// Checks the tensor-core operand store the SHT_MIXED plan uploads
// (tc_build_images) against the per-op images of sht_plan_op_image, on the
// host.  The store is filled into a vector poisoned with 0xAAAA beforehand:
// its resize keeps existing elements, so an element the packing skipped would
// keep the poison and differ from the op's image.  Also checks that the op
// records' image offsets tile the store without gaps or overlaps.
//
//   tc_images_check N eps n0 n_leaf flags   -> prints "ok <elements>", exit 0
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "apply_tc.cuh"
#include "sht.h"

using namespace sht;

template <class T>
static bool fetch(sht_plan_t p, int what, std::vector<T>& v) {
  size_t bytes = 0;
  if (sht_plan_export(p, what, nullptr, &bytes) != SHT_OK || bytes % sizeof(T)) return false;
  v.resize(bytes / sizeof(T));
  return sht_plan_export(p, what, v.data(), &bytes) == SHT_OK;
}

int main(int argc, char** argv) {
  if (argc != 6) return 2;
  const int N = std::atoi(argv[1]);
  const double eps = std::atof(argv[2]);
  sht_opts o;
  sht_opts_default(N, eps, &o);
  o.n0 = std::atoi(argv[3]);
  o.n_leaf = std::atoi(argv[4]);
  o.flags = SHT_FLAG_HOST_ONLY | std::atoi(argv[5]);
  o.precision = SHT_MIXED;
  sht_plan_t p = nullptr;
  if (sht_plan_create(N, eps, &o, &p) != SHT_OK) return 3;
  std::vector<Unit> units;
  std::vector<Op> ops;
  std::vector<double> factors;
  if (!fetch(p, SHT_EXPORT_UNITS, units) || !fetch(p, SHT_EXPORT_OPS, ops) || !fetch(p, SHT_EXPORT_FACTORS, factors))
    return 4;
  TcImages img;
  std::vector<TcOp> tops;
  std::vector<int32_t> tiles;
  int max_rows = 0;
  tc_build_images(N, units, ops, factors.data(), img, tops, tiles, max_rows);
  const size_t total = img.size();
  std::fill(img.begin(), img.end(), (uint16_t)0xAAAA);
  tc_build_images(N, units, ops, factors.data(), img, tops, tiles, max_rows);
  if (img.size() != total || tops.size() != ops.size()) return 5;
  size_t at = 0;
  std::vector<uint16_t> want;
  for (size_t k = 0; k < ops.size(); ++k)
    for (int t = 0; t < 2; ++t) {
      size_t n = 0;
      if (sht_plan_op_image(p, (int64_t)k, t, nullptr, &n) != SHT_OK) return 6;
      want.assign(n, 0);
      if (n && sht_plan_op_image(p, (int64_t)k, t, want.data(), &n) != SHT_OK) return 6;
      if ((size_t)tops[k].img[t] != at) {
        std::printf("op %zu direction %d: image at %lld, expected %zu\n", k, t, (long long)tops[k].img[t], at);
        return 7;
      }
      for (size_t i = 0; i < n; ++i)
        if (img[at + i] != want[i]) {
          std::printf("op %zu direction %d element %zu: %04x, expected %04x\n", k, t, i, img[at + i], want[i]);
          return 8;
        }
      at += n;
    }
  // the store is exactly the images (at least 8 elements, the tail zero)
  if (at > total || (total > 8 && at != total)) return 9;
  for (size_t i = at; i < total; ++i)
    if (img[i] != 0) return 10;
  std::printf("ok %zu\n", at);
  sht_plan_destroy(p);
  return 0;
}
