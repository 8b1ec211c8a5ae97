// Fine steps on the grid sides n = 32 R that are not powers of two (n = 96, 160, 192;
// Table 1's N_F = 160), on the warp-owned mixed-radix FFT kernels of kd_fine_mr.cuh
// (FineMrSet, kd_fine_sets.cuh), in both precisions and for the three IMEX schemes.  One
// launch plan (column variant 0, row variant 0); the step loop is the one of the other
// grids.
#include "kd_fine_sets.cuh"

namespace kd {

bool fine_mr_side(int n) { return n == 96 || n == 160 || n == 192; }

int fine_mr_run(int prec, const FineArgs& a, const StepCfg& cfg) {
  const bool f = prec == 0;
  switch (a.n) {
    case 96: return f ? run_steps<FineMrSet<float, 3>>(a, cfg) : run_steps<FineMrSet<double, 3>>(a, cfg);
    case 160: return f ? run_steps<FineMrSet<float, 5>>(a, cfg) : run_steps<FineMrSet<double, 5>>(a, cfg);
    case 192: return f ? run_steps<FineMrSet<float, 6>>(a, cfg) : run_steps<FineMrSet<double, 6>>(a, cfg);
  }
  return -1;
}

}  // namespace kd
