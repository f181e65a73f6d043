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
  // packed in windows (the path of large stores): windows in order, end to
  // end, covering the images, and together equal to the whole store; small
  // windows, so that some ops are larger than one
  for (size_t window : {(size_t)2048, (size_t)65536}) {
    std::vector<TcOp> tops2;
    std::vector<int32_t> tiles2;
    int max_rows2 = 0;
    const size_t tot2 = tc_image_layout(N, units, ops, tops2, tiles2, max_rows2);
    if (tot2 != at || tiles2 != tiles || max_rows2 != max_rows) return 29;
    size_t next = 0, nwin = 0;
    bool same = true;
    tc_pack_windows(ops, tops2, factors.data(), tot2, window, [&](size_t first, const uint16_t* data, size_t n) {
      if (first != next) same = false;
      for (size_t i = 0; i < n && same; ++i) same = data[i] == img[first + i];
      next = first + n;
      ++nwin;
      return same;
    });
    if (!same || next != tot2 || (tot2 > window && nwin < 2)) return 30;
  }
  // first-writer marks and zero ranges: per order and direction, replay the
  // ops in processing order; a storing op may touch no row written before,
  // and every row the output step reads is first written by a storing op or
  // lies in one zero range -- exactly one of the two
  // processing orders: per unit and direction a permutation of its ops, the
  // phases ascending (forward) or descending (transposed), and within a phase
  // the first row of the side read non-decreasing
  std::vector<int32_t> ford, tord;
  tc_proc_order(units, tops, ford, tord);
  if (ford.size() != tops.size() || tord.size() != tops.size()) return 20;
  for (const Unit& un : units)
    for (int d = 0; d < 2; ++d) {
      const std::vector<int32_t>& o = d == 0 ? ford : tord;
      std::vector<char> seen((size_t)(un.op_end - un.op_begin), 0);
      for (int i = un.op_begin; i < un.op_end; ++i) {
        const int32_t k = o[(size_t)i];
        if (k < un.op_begin || k >= un.op_end || seen[(size_t)(k - un.op_begin)]) return 21;
        seen[(size_t)(k - un.op_begin)] = 1;
        if (i > un.op_begin) {
          const TcOp &a = tops[(size_t)o[(size_t)i - 1]], &b = tops[(size_t)k];
          if (d == 0 ? a.phase > b.phase : a.phase < b.phase) return 22;
          const int32_t* ao = d == 0 ? a.in_off : a.out_off;
          const int32_t* al = d == 0 ? a.in_len : a.out_len;
          const int32_t* bo = d == 0 ? b.in_off : b.out_off;
          const int32_t* bl = d == 0 ? b.in_len : b.out_len;
          if (a.phase == b.phase && (al[0] > 0 ? ao[0] : ao[1]) > (bl[0] > 0 ? bo[0] : bo[1])) return 23;
        }
      }
    }
  // live node rows: whole groups, within the Y regions, covering every Y row
  // written forward and every Y group read transposed, and tight (a write in
  // the last live group)
  std::vector<int32_t> live;
  tc_live_rows(N, units, tops, live);
  if (live.size() != units.size()) return 24;
  int dead_units = 0;  // orders with node rows no block reaches
  for (size_t u = 0; u < units.size(); ++u) {
    const Unit& un = units[u];
    const TcRows tr = tc_rows(un.nce, un.nco, N);
    const int lv = live[u];
    if (lv < 0 || lv % 8 != 0 || lv > tc_r8(N)) return 25;
    int top = 0;
    for (int q = un.op_begin; q < un.op_end; ++q) {
      const TcOp& t = tops[(size_t)q];
      for (int sg = 0; sg < 2; ++sg)
        for (int r = t.out_off[sg]; r < t.out_off[sg] + t.out_len[sg]; ++r) {
          const int i = r >= tr.yo ? r - tr.yo : r - tr.ye;  // node row in Y_e or Y_o
          if (r < tr.ye || r >= tr.yo + N) continue;
          if (i >= lv) return 26;
          top = std::max(top, i + 1);
        }
      const TcDir dt = tc_dir(t, false);
      for (int j = 0; j < dt.kg.ngt; ++j) {
        const int r0 = kTcGrpRows * tc_group(dt.kg, j);
        if (r0 < tr.ye || r0 >= tr.yo + N) continue;
        if ((r0 >= tr.yo ? r0 - tr.yo : r0 - tr.ye) >= lv) return 27;
      }
    }
    if (tc_r8(top) != lv) return 28;
    if (lv < N) ++dead_units;
  }
  std::vector<int32_t> zr, zri;
  tc_first_writers(N, units, tops, ford, tord, live, zr, zri);
  if (zri.size() != 2 * units.size() + 1 || zri[0] != 0) return 11;
  for (size_t u = 0; u < units.size(); ++u) {
    const Unit& un = units[u];
    const TcRows tr = tc_rows(un.nce, un.nco, N);
    for (int d = 0; d < 2; ++d) {
      const bool fwd = d == 0;
      const int acc0 = fwd ? tr.ye : 0;
      std::vector<int> state(tc_acc_rows(N), 0);  // 0 untouched, 1 stored first, 2 added first
      for (int q = 0; q < un.op_end - un.op_begin; ++q) {
        const TcOp& t = tops[(size_t)(fwd ? ford : tord)[(size_t)(un.op_begin + q)]];
        if (!(t.flags & (fwd ? OP_FWD_ACCUM : OP_BWD_ACCUM))) {
          if (t.flags & (fwd ? kTcFwdStore : kTcBwdStore)) return 12;
          continue;
        }
        const bool st = (t.flags & (fwd ? kTcFwdStore : kTcBwdStore)) != 0;
        const int32_t* oo = fwd ? t.out_off : t.in_off;
        const int32_t* ol = fwd ? t.out_len : t.in_len;
        for (int sg = 0; sg < 2; ++sg)
          for (int r = 0; r < ol[sg]; ++r) {
            const int a = oo[sg] + r - acc0;
            if (a < 0 || a >= tc_acc_rows(N)) return 13;
            if (st && state[a] != 0) return 14;
            if (state[a] == 0) state[a] = st ? 1 : 2;
          }
      }
      std::vector<int> zeroed(tc_acc_rows(N), 0);
      for (int z = zri[2 * u + d]; z < zri[2 * u + d + 1]; ++z)
        for (int r = zr[2 * z]; r < zr[2 * z] + zr[2 * z + 1]; ++r) {
          if (r < 0 || r >= tc_acc_rows(N)) return 15;
          ++zeroed[r];
        }
      // rows the output step reads (forward, the live node rows: the others
      // are neither written nor zeroed) are stored first or zeroed, once
      const int nl = std::min(N, (int)live[u]);
      const int rg[2][2] = {{0, fwd ? N : un.nce}, {fwd ? tr.yo - tr.ye : tr.xo, fwd ? N : un.nco}};
      for (const auto& g : rg)
        for (int r = g[0]; r < g[0] + g[1]; ++r) {
          const bool read = !fwd || r - g[0] < nl;
          if (read ? (state[r] == 1) + zeroed[r] != 1 : state[r] != 0 || zeroed[r] != 0) {
            std::printf("order %zu dir %d row %d: state %d zeroed %d\n", u, d, r, state[r], zeroed[r]);
            return 16;
          }
        }
    }
  }
  std::printf("ok %zu %d\n", at, dead_units);
  sht_plan_destroy(p);
  return 0;
}
