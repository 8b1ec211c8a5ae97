// Fused pseudo-spectral IMEX RK443 fine step (the data-parallel fine propagator of
// Parareal, Sec. 3 Eq. 8 and Sec. 4), all slices of a batch advanced by every launch.
//
// This file holds the flow-phase table and the dispatch to the kernel families
// (kd_fine2.cuh for n <= 256, kd_fine3.cuh / kd_fine4.cuh for n = 512, 1024, instantiated
// per precision and grid in kd_fine2_*.cu / kd_fine3_*.cu; the mixed-radix kernels of
// kd_fine_mr.cuh for n = 96, 160, 192 in kd_fine_mr.cu).  One right-hand-side
// evaluation nabla_k x (u x b) followed by one IMEX stage is two kernels:
//   column kernel : mixed M (ky rows, x columns) -> inverse FFT in y -> u x b on the
//                   grid (u analytic, Sec. 2.1 / 2.2) -> forward FFT in y -> keep
//                   |ky| <= K -> W
//   row kernel    : W -> forward FFT in x -> keep |kx| <= K -> spectral curl
//                   i k3 x w_hat -> stage combine and diagonal implicit diffusion solve
//                   (Ascher-Ruuth-Spiteri (4,4,3)) -> inverse FFT in x of the next
//                   stage value -> M
// so a step is 4 x (column, row) and the state never leaves the compact 2/3 set.
//
// Accumulator form of the IMEX stages (A_ii = 1/2, d = 1 + dt lambda / 2):
//   stage 0: X1 = (X0 + dt/2 F0)/d ;  R_i = X0 + dt H_i0 F0 - dt A_i1 lambda X1  (i=2,3,4)
//   stage 1: X2 = (R2 + dt H21 F1)/d ; R_i += dt H_i1 F1 - dt A_i2 lambda X2    (i=3,4)
//   stage 2: X3 = (R3 + dt H32 F2)/d ; R4 += dt H42 F2 - dt A43 lambda X3
//   stage 3: X4 = (R4 + dt H43 F3)/d = new state
#include <math.h>

#include "kd_fine.h"
#include "kd_stage.cuh"

namespace kd {

// Stage times c_j of the explicit evaluations F_j of RK443, RK222 and RK111.
__constant__ double c_stage[3][4] = {{0.0, 0.5, 2.0 / 3.0, 0.5},
                                     {0.0, 0.29289321881345247560, 0.0, 0.0},
                                     {0.0, 0.0, 0.0, 0.0}};

// Flow phases of every (field, step, stage), in double, rounded to T:
// t = t0[b] + s dt + c_j dt, then (cos(cos t), sin(cos t), cos(sin t), sin(sin t)).
// With per-slice parameters dt is the field's own, and fields under a steady flow get
// the constant phases (1, 0, 1, 0).
template <typename T>
__global__ void phase_kernel(const double* t0, int batch, int nsteps, double dt, const SliceParams* sp, int sch,
                             T* out) {
  const long total = (long)batch * nsteps * 4;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int j = (int)(i & 3);
    const long bs = i >> 2;
    const int s = (int)(bs % nsteps);
    const long b = bs / nsteps;
    double dtb = dt;
    if (sp) {
      if (sp[b].flow != FLOW_GP) {
        out[i * 4 + 0] = T(1);
        out[i * 4 + 1] = T(0);
        out[i * 4 + 2] = T(1);
        out[i * 4 + 3] = T(0);
        continue;
      }
      dtb = sp[b].dt;
    }
    const double t = t0[b] + s * dtb + c_stage[sch][j] * dtb;
    const double px = cos(t), py = sin(t);
    out[i * 4 + 0] = (T)cos(px);
    out[i * 4 + 1] = (T)sin(px);
    out[i * 4 + 2] = (T)cos(py);
    out[i * 4 + 3] = (T)sin(py);
  }
}

size_t phase_table_bytes(int prec, long batch, int nsteps) {
  return (size_t)batch * nsteps * 16 * (prec == 0 ? 4 : 8);
}

int launch_phases(int prec, const FineArgs& a, int nsteps, cudaStream_t st) {
  if ((a.flow != FLOW_GP && !a.sp) || nsteps <= 0 || a.batch <= 0) return 0;
  const long total = (long)a.batch * nsteps * 4;
  long g = (total + 255) / 256;
  if (g > 65535L * 16) g = 65535L * 16;
  if (prec == 0)
    phase_kernel<float><<<(unsigned)g, 256, 0, st>>>(a.t0, a.batch, nsteps, a.dt, a.sp, a.scheme, (float*)a.phases);
  else
    phase_kernel<double><<<(unsigned)g, 256, 0, st>>>(a.t0, a.batch, nsteps, a.dt, a.sp, a.scheme, (double*)a.phases);
  return 1;
}

template <typename T>
static cudaError_t prepare_all() {
  cudaError_t e;
  if ((e = fine2_prep<T, 16>()) != cudaSuccess) return e;
  if ((e = fine2_prep<T, 32>()) != cudaSuccess) return e;
  if ((e = fine2_prep<T, 64>()) != cudaSuccess) return e;
  if ((e = fine2_prep<T, 128>()) != cudaSuccess) return e;
  if ((e = fine2_prep<T, 256>()) != cudaSuccess) return e;
  if ((e = fine3_prep<T, 512>()) != cudaSuccess) return e;
  return fine3_prep<T, 1024>();
}

cudaError_t fine_prepare(int prec) { return prec == 0 ? prepare_all<float>() : prepare_all<double>(); }

template <typename T>
static bool variants_T(int n, int* ncol, int* nrow) {
  switch (n) {
    case 16: fine2_variants<T, 16>(ncol, nrow); return true;
    case 32: fine2_variants<T, 32>(ncol, nrow); return true;
    case 64: fine2_variants<T, 64>(ncol, nrow); return true;
    case 128: fine2_variants<T, 128>(ncol, nrow); return true;
    case 256: fine2_variants<T, 256>(ncol, nrow); return true;
    case 512: fine3_variants<T, 512>(ncol, nrow); return true;
    case 1024: fine3_variants<T, 1024>(ncol, nrow); return true;
  }
  if (fine_mr_side(n)) {
    *ncol = *nrow = 1;
    return true;
  }
  return false;
}

FinePlan fine_default_plan(int n, int prec) {
  if (fine_fft_grid(n) == 1024 && prec == 0) return fine3_default_plan<float, 1024>();
  if (fine_fft_grid(n) == 512 && prec == 0) return fine3_default_plan<float, 512>();
  if (fine_fft_grid(n) == 256 && prec == 0) return fine2_default_plan<float, 256>();
  if (fine_fft_grid(n) == 128 && prec == 0) return fine2_default_plan<float, 128>();
  return FinePlan();
}

bool fine_full_io(int n, int prec, const FinePlan& plan, int scheme) {
  return n == 1024 && prec == 0 && plan.row == kRow4Variant && scheme == SCHEME_RK443;
}

bool fine_variants(int n, int prec, int* ncol, int* nrow) {
  const int m = fine_fft_grid(n);
  return prec == 0 ? variants_T<float>(m, ncol, nrow) : variants_T<double>(m, ncol, nrow);
}

template <typename T>
static int run_T(const FineArgs& a, const StepCfg& cfg) {
  switch (a.n) {
    case 16: return fine2_run<T, 16>(a, cfg);
    case 32: return fine2_run<T, 32>(a, cfg);
    case 64: return fine2_run<T, 64>(a, cfg);
    case 128: return fine2_run<T, 128>(a, cfg);
    case 256: return fine2_run<T, 256>(a, cfg);
    case 512: return fine3_run<T, 512>(a, cfg);
    case 1024: return fine3_run<T, 1024>(a, cfg);
  }
  return fine_mr_run(sizeof(T) == 4 ? 0 : 1, a, cfg);
}

int fine_run(int prec, const FineArgs& a, const StepCfg& cfg) {
  const int nph = launch_phases(prec, a, cfg.nsteps, cfg.st);
  const int r = prec == 0 ? run_T<float>(a, cfg) : run_T<double>(a, cfg);
  return r < 0 ? r : r + nph;
}

int fine_launch_steps(int prec, const FineArgs& a, int nsteps, bool prologue, bool store_last, cudaStream_t st,
                      const LaunchProbe* pr) {
  StepCfg cfg;
  cfg.nsteps = nsteps;
  cfg.prologue = prologue;
  cfg.store_last = store_last;
  cfg.probe = pr;
  cfg.st = st;
  return fine_run(prec, a, cfg);
}

}  // namespace kd
