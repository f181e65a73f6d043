// Host-side plan: the packed apply program plus its device copies.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/sht.h"
#include "program.hpp"

namespace sht {

struct HostProgram {
  int N = 0;
  sht_opts opts{};
  std::vector<double> x, w;        // 2N Gauss-Legendre nodes (ascending) and weights
  std::vector<Unit> units;         // one per |m| = 0..2N-1, indexed by |m|
  std::vector<Op> ops;             // all units' ops, grouped by unit, sorted by phase
  std::vector<int32_t> phase_tab;  // per unit: nphase+1 op indices (absolute)
  FactorStore factors;             // packed blocks (column-major, ld % 4 == 0, 32-byte aligned)
  std::vector<int32_t> order;      // units by decreasing cost (schedule)
  std::vector<int32_t> unit_blocks;  // per unit: IDBF, low-rank, dense, dropped block counts (not in plan files)
  int32_t max_rows = 0;            // largest unit vector space (rows)
  sht_plan_info info{};
};

struct Mat;

// A source of the Legendre parity matrices of one order (Sec. 3.1.2) other
// than the builder's own host recurrence (e.g. the device).  Called from
// several host threads at once.  E(i, j) = Pbar_{am+2j}^{am}(xp_i) and
// O(i, j) = Pbar_{am+1+2j}^{am}(xp_i) at the N positive nodes xp (ascending),
// sized N x ceil((2N-am)/2) and N x floor((2N-am)/2); false on failure.
struct LegendreSource {
  virtual ~LegendreSource() = default;
  virtual bool parity_matrices(int N, int am, const double* xp, Mat& E, Mat& O) = 0;
};

// Build the apply program (Sec. 3.2-3.3), the Legendre matrices from `src`
// when given.  Returns SHT_OK or an error code (SHT_ERR_CUDA when the source
// fails).
sht_status build_program(int N, const sht_opts& opts, HostProgram& out, std::string& err,
                         LegendreSource* src = nullptr);

// One order built on its own, as in the per-order experiments of Sec. 5: the
// unit's ops (op_begin = 0) with its block statistics, and the time spent on
// its Legendre matrices (t_mat_s) and on partitioning, factoring and packing
// them (t_fac_s).  The factors themselves are not kept: this is for sizing
// and timing, never for a kernel.  The unit is bit for bit the one the full
// plan with the same N and options holds at that order.
struct OrderBuild {
  Unit unit{};
  std::vector<Op> ops;
  int64_t n_factors = 0;  // doubles in the unit's factor store
  int64_t n_idbf = 0, n_low = 0, n_dense = 0, n_drop = 0;
  int64_t e_idbf = 0, e_low = 0, e_dense = 0;
  int64_t max_rank = 0;
  double t_mat_s = 0.0, t_fac_s = 0.0;
};

// Build the orders |m| = am[0..count) (each in [0, 2N)) of an N plan, one
// host thread per order, the orders in parallel.
sht_status build_orders(int N, const sht_opts& opts, int count, const int* am, std::vector<OrderBuild>& out);

// Check that a program is internally consistent: unit layouts, op and phase
// ranges, factor offsets and the schedule.  Every program the kernels see
// (built or loaded from a file) passes this first, so no op can address rows
// or factors outside its buffers.
bool validate_program(const HostProgram& P, std::string& err);

// Gauss-Legendre rule on n points, ascending (used by the plan only).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);

}  // namespace sht
