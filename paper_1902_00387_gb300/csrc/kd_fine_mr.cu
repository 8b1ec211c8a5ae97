// Fine steps on the grid sides n = 32 R that are not powers of two (n = 96, 160, 192;
// Table 1's N_F = 160), on the warp-owned mixed-radix FFT kernels of kd_fine_mr.cuh, in
// both precisions and for the three IMEX schemes.  One launch plan (column variant 0,
// row variant 0); the step loop is the one of the other grids (kd_fine_sets.cuh).
#include "kd_fine_sets.cuh"
#include "kd_fine_mr.cuh"

namespace kd {

template <typename T, int R>
struct FineMrSet {
  static constexpr int N = 32 * R;
  static constexpr bool FUSED = false;
  static constexpr int kFusedCol = -1;
  static constexpr unsigned BLOCK = 32 * kMrWarps;
  static int ncol() { return 1; }
  static int nrow() { return 1; }
  static unsigned blocks(long warps) { return (unsigned)((warps + kMrWarps - 1) / kMrWarps); }
  static void col(int, const FineArgs& a, int s, int j, cudaStream_t st, bool pdl) {
    launch_k(colmr_kernel<T, R>, blocks((long)a.batch * N), BLOCK, 0, st, pdl, a, s, j);
  }
  template <int SCH, int MODE>
  static void row_k(const FineArgs& a, int store, cudaStream_t st, bool pdl) {
    launch_k(rowmr_kernel<T, R, SCH, MODE>, blocks((long)a.batch * a.P), BLOCK, 0, st, pdl, a, store);
  }
  static void row(int, const FineArgs& a, int mode, int store, cudaStream_t st, bool pdl) {
    if (mode == 4) return row_k<SCHEME_RK443, 4>(a, store, st, pdl);   // prologue (scheme-free)
    if (a.scheme == SCHEME_RK111) return row_k<SCHEME_RK111, 0>(a, store, st, pdl);
    if (a.scheme == SCHEME_RK222)
      return mode == 0 ? row_k<SCHEME_RK222, 0>(a, store, st, pdl) : row_k<SCHEME_RK222, 1>(a, store, st, pdl);
    switch (mode) {
      case 0: return row_k<SCHEME_RK443, 0>(a, store, st, pdl);
      case 1: return row_k<SCHEME_RK443, 1>(a, store, st, pdl);
      case 2: return row_k<SCHEME_RK443, 2>(a, store, st, pdl);
      default: return row_k<SCHEME_RK443, 3>(a, store, st, pdl);
    }
  }
};

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
