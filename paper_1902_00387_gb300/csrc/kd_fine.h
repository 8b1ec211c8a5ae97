// Internal interfaces between the library's translation units.
#pragma once
#include "kd_common.cuh"

namespace kd {

// Optional per-launch hook (event timing of the fine kernels); kid 0 = column
// kernel, 1 = row kernel.  Called on the host around each launch.
struct LaunchProbe {
  void (*before)(void* user, int kid);
  void (*after)(void* user, int kid);
  void* user;
};

// Launch plan of the fine kernels: index of the column-kernel and row-kernel variant
// (tile shape, stage-update style) among those instantiated for the grid and precision;
// {0, 0} is the default ({6, 7} on the complex64 grid n = 1024, {5, 9} at n = 512 and
// {0, 9} at n = 256, {1, 9} at n = 128, fine_default_plan).
// Chosen per (n, precision, batch) by the autotuner.
struct FinePlan {
  int col = 0;
  int row = 0;
};

// One enqueue of fine steps.
struct StepCfg {
  int nsteps = 0;
  bool prologue = true;     // start with the inverse x transform of X (needed unless M holds it)
  bool store_last = false;  // leave M filled for the state after the last step
  // host [nsteps]: fields advanced at step s, a prefix of the batch (fields ordered by
  // decreasing step count); NULL: every field takes every step
  const int* active = nullptr;
  const LaunchProbe* probe = nullptr;
  FinePlan plan;
  bool pdl = false;         // launch the step kernels as programmatic dependent launches
  cudaStream_t st = nullptr;
};

// ---- kd_fine.cu
cudaError_t fine_prepare(int prec);
// bytes of the flow-phase table FineArgs::phases for `batch` fields and `nsteps` steps
size_t phase_table_bytes(int prec, long batch, int nsteps);
// fill FineArgs::phases (Galloway-Proctor, or any batch with per-slice parameters);
// returns kernels launched
int launch_phases(int prec, const FineArgs& a, int nsteps, cudaStream_t st);
// number of column / row variants instantiated for (fine_fft_grid(n), prec); false if none
bool fine_variants(int n, int prec, int* ncol, int* nrow);
// launch plan of a context before any autotuning or kd_set_plan
FinePlan fine_default_plan(int n, int prec);
// Row variant of the warp-transform row kernel of the complex64 n = 1024 grid
constexpr int kRow4Variant = 7;
// whether the plan's kernels read the first step's state from FineArgs::x_in_full and
// write the last step's to x_out_full (the caller's layout, no pack / unpack pass):
// RK443 steps of the row kernel kRow4Variant
bool fine_full_io(int n, int prec, const FinePlan& plan, int scheme);
// Enqueue cfg.nsteps RK443 steps on the compact state a.X after filling the phase table
// a.phases (which must hold phase_table_bytes(prec, a.batch, nsteps)).  Returns the
// number of kernels launched (negative on an unsupported grid size).
int fine_run(int prec, const FineArgs& a, const StepCfg& cfg);
// the same with the default plan and every field taking every step
int fine_launch_steps(int prec, const FineArgs& a, int nsteps, bool prologue, bool store_last,
                      cudaStream_t st, const LaunchProbe* probe = nullptr);

// ---- kd_fine_mr.cu: grid sides 32 R that are not powers of two (96, 160, 192)
bool fine_mr_side(int n);
int fine_mr_run(int prec, const FineArgs& a, const StepCfg& cfg);   // -1 for other sides
// FFT sides of the fine kernels: powers of two in [16, 1024] and fine_mr_side
inline bool fine_fft_side(int n) {
  return n == 16 || n == 32 || n == 64 || n == 128 || n == 256 || n == 512 || n == 1024 || fine_mr_side(n);
}
// FFT side the fine kernels use for the grid side n of a problem (kept set |k| <= K = n/3):
// n itself where it is an FFT side, else the smallest mixed-radix side m >= 2K + 2 (0 if
// none, i.e. n >= 288).  Both flows have only the wavenumbers +-1 in x and y, so u x b of
// a field with |k| <= K has |k| <= K + 1; on m >= 2K + 2 points no mode of it aliases onto
// the kept set, and the kept modes of the step are those of the n-point pseudo-spectral
// step (exactly, up to rounding).  Only the mixed-radix kernels take a kept set narrower
// or wider than m / 3 (the power-of-two kernels fix K = N / 3 at compile time).  This runs
// e.g. n = 240, the 3/2-padded grid of 160 kept modes a side, on the 192-point transform.
inline int fine_fft_grid(int n) {
  if (fine_fft_side(n)) return n;
  for (int m : {96, 160, 192})
    if (m >= 2 * (n / 3) + 2) return m;
  return 0;
}

// ---- kd_fine2_*.cu (register-FFT kernels, n <= 256) and kd_fine3_*.cu (n = 512, 1024):
// explicit instantiations per (T, N)
template <typename T, int N>
int fine2_run(const FineArgs& a, const StepCfg& cfg);
template <typename T, int N>
cudaError_t fine2_prep();
template <typename T, int N>
void fine2_variants(int* ncol, int* nrow);
template <typename T, int N>
FinePlan fine2_default_plan();
template <typename T, int N>
int fine3_run(const FineArgs& a, const StepCfg& cfg);
template <typename T, int N>
cudaError_t fine3_prep();
template <typename T, int N>
void fine3_variants(int* ncol, int* nrow);
template <typename T, int N>
FinePlan fine3_default_plan();

// ---- kd_ops.cu (layout conversions, Parareal update, norms)
// full [batch][3][n][n] (precision pin) -> compact [batch][3][P][P] (precision pout)
int full_to_compact(int pin, const void* full, int pout, void* comp, long batch, int n, cudaStream_t st);
// compact -> full, zeros outside the kept square
int compact_to_full(int pin, const void* comp, int pout, void* full, long batch, int n, cudaStream_t st);
// zeros at the entries of the full layout outside the kept square (the rest untouched)
int zero_outside_kept(int prec, void* full, long batch, int n, cudaStream_t st);
// compact (n_src grid, precision pin) -> compact (n_dst grid, precision pout):
// truncation when n_dst < n_src, zero padding when n_dst > n_src
int compact_resample(int pin, const void* src, int n_src, int pout, void* dst, int n_dst, long batch,
                     cudaStream_t st);
// Parareal update of one slice, FP64 (g given in precision pg on the coarse compact grid):
//   init = 0: U_next = F + prolong(g - Gold), Gold = g
//   init = 1: initial coarse sweep, U_next = prolong(g), Gold = g (F unused)
//   init = 2: increment form, U_next = F + prolong(g) (g = G of the increment; Gold unused)
// If partials != NULL: also per-block sums of |U_next - U_next_old|^2 and |U_next|^2
// into partials[2 * blockIdx + {0,1}] (deterministic order), returns the block count.
// (coarse set k in [-Kc, Pc - Kc)^2)
int parareal_update(const double* F, const void* g, int pg, double* Gold, double* U_next, int n, int Kc, int Pc,
                    int init, double* partials, cudaStream_t st);
// sigma = sqrt(sum diff / sum norm) of `nblocks` partial pairs -> out[0]; also the two sums
int finish_sigma(const double* partials, int nblocks, double* out, cudaStream_t st);
// partials of |a - ref| / |ref| over len complex FP64 values for finish_sigma; returns the
// block count (or -1)
int rel_error_partials(const double* a, const double* ref, long len, double* partials, cudaStream_t st);
// E[i] = sum |z|^2 over `len` complex128 entries of field i (stride len), i < count
int energy_kernel(const double* fields, long len, int count, double* E, cudaStream_t st);
// least-squares slope of 0.5 ln E_i against t_i = i * dt over t_i >= fit_from -> out[0];
// out[1] = 1 if every used E_i was finite and > 0
int growth_fit(const double* E, int count, double dt, double fit_from, double* out, cudaStream_t st);
// increment form: X = U - Uprev (U if first), Uprev = U (X in precision pout);
// Fv = X (first) or Fv + X.  `total` counts complex entries.
int delta_in(int pout, const double* U, double* Uprev, void* X, long total, int first, cudaStream_t st);
int accum_out(int pin, const void* X, double* Fv, long total, int first, cudaStream_t st);
// d = U - Uprev over `total` complex entries (FP64)
int diff_kernel(const double* U, const double* Uprev, double* d, long total, cudaStream_t st);
// dst[i] = t0 + i * dT
int fill_times(double* dst, int count, double t0, double dT, cudaStream_t st);
// dst[i] = (first + i) * dT: start times of slices first, first + 1, ...
int fill_slice_times(double* dst, int count, int first, double dT, cudaStream_t st);

}  // namespace kd
