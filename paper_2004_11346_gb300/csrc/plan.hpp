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
  std::vector<double> factors;     // packed blocks (column-major, ld % 4 == 0, 32-byte aligned)
  std::vector<int32_t> order;      // units by decreasing cost (schedule)
  std::vector<int32_t> unit_blocks;  // per unit: IDBF, low-rank, dense, dropped block counts (not in plan files)
  int32_t max_rows = 0;            // largest unit vector space (rows)
  sht_plan_info info{};
};

// Build the apply program (Sec. 3.2-3.3).  Returns SHT_OK or an error code.
sht_status build_program(int N, const sht_opts& opts, HostProgram& out, std::string& err);

// Check that a program is internally consistent: unit layouts, op and phase
// ranges, factor offsets and the schedule.  Every program the kernels see
// (built or loaded from a file) passes this first, so no op can address rows
// or factors outside its buffers.
bool validate_program(const HostProgram& P, std::string& err);

// Gauss-Legendre rule on n points, ascending (used by the plan only).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);

}  // namespace sht
