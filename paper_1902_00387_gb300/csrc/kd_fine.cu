// Fused pseudo-spectral IMEX RK443 fine step (the data-parallel fine propagator of
// Parareal, Sec. 3 Eq. 8 and Sec. 4), all slices of a batch advanced by every launch.
//
// This file holds the flow-phase table and the dispatch to the kernel families
// (kd_fine2.cu for n <= 256, kd_fine3.cu for n = 512, 1024).  One right-hand-side
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

// Stage times c_j of the explicit evaluations F_j (RK443).
__constant__ double c_stage[4] = {0.0, 0.5, 2.0 / 3.0, 0.5};

// Flow phases of every (field, step, stage), in double, rounded to T:
// t = t0[b] + s dt + c_j dt, then (cos(cos t), sin(cos t), cos(sin t), sin(sin t)).
template <typename T>
__global__ void phase_kernel(const double* t0, int batch, int nsteps, double dt, T* out) {
  const long total = (long)batch * nsteps * 4;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int j = (int)(i & 3);
    const long bs = i >> 2;
    const int s = (int)(bs % nsteps);
    const long b = bs / nsteps;
    const double t = t0[b] + s * dt + c_stage[j] * dt;
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
  if (a.flow != FLOW_GP || nsteps <= 0 || a.batch <= 0) return 0;
  const long total = (long)a.batch * nsteps * 4;
  long g = (total + 255) / 256;
  if (g > 65535L * 16) g = 65535L * 16;
  if (prec == 0)
    phase_kernel<float><<<(unsigned)g, 256, 0, st>>>(a.t0, a.batch, nsteps, a.dt, (float*)a.phases);
  else
    phase_kernel<double><<<(unsigned)g, 256, 0, st>>>(a.t0, a.batch, nsteps, a.dt, (double*)a.phases);
  return 1;
}

cudaError_t fine_prepare(int prec) {
  cudaError_t e = fine2_prepare(prec);
  return e != cudaSuccess ? e : fine3_prepare(prec);
}

int fine_launch_steps(int prec, const FineArgs& a, int nsteps, bool prologue, bool store_last, cudaStream_t st,
                      const LaunchProbe* pr) {
  const int nph = launch_phases(prec, a, nsteps, st);
  const int r = a.n <= 256 ? fine2_launch_steps(prec, a, nsteps, prologue, store_last, st, pr)
                           : fine3_launch_steps(prec, a, nsteps, prologue, store_last, st, pr);
  return r < 0 ? r : r + nph;
}

}  // namespace kd
