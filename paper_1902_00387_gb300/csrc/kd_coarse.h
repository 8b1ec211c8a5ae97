// Persistent classical coarse propagator (kd_coarse.cu).
#pragma once
#include "kd_common.cuh"

namespace kd {

// COARSE_OUT: write G(U) to g64.  COARSE_INIT: U_{n+1} = G(U_n), Gold = G(U_n).
// COARSE_UPDATE: U_{n+1} = F + (G(U_n) - Gold), Gold = G(U_n).
// COARSE_INCR: U_{n+1} = F + G(U_n - Uprev_n)  (increment form; Gold unused).
enum { COARSE_OUT = 0, COARSE_INIT = 1, COARSE_UPDATE = 2, COARSE_INCR = 3 };

struct CoarseArgs {
  int Kc;             // coarse cutoff n_c / 3
  int Kf;             // fine cutoff n / 3 (input / update layout)
  int flow;
  double amp, kz, Rm, dt;
  int nsteps;
  const void* phases;   // [batch][nsteps][4][4] flow phases (precision T) or NULL (steady flow)
  const double* Un;     // fine compact FP64 inputs [batch][3][Pf][Pf] (complex interleaved)
  const double* Uprev;  // COARSE_INCR: previous iterate of the same slice (input is Un - Uprev)
  int mode;             // COARSE_OUT: write g64; COARSE_INIT / COARSE_UPDATE: Parareal update (batch 1)
  double* g64;          // COARSE_OUT: coarse compact FP64 outputs [batch][3][Pc][Pc]
  const double* Fv;     // COARSE_UPDATE: fine values F(U_n), fine compact FP64
  double* Gold;         // coarse values of the previous sweep (read, then replaced)
  double* Unext;        // U_{n+1}, fine compact FP64 (written)
  double* sigma_out;    // if not NULL: sigma, |U - U_old|^2, |U|^2 of Unext (3 doubles)
  int phase_smem;       // (internal) phase values the cluster kernel may stage in shared memory
};

bool coarse_conv_supported(int n_c);
size_t coarse_conv_smem(int prec, int n_c);
cudaError_t coarse_prepare(int prec);
// One block per field; returns 1 (kernels launched) or -1 if n_c is not supported.
int coarse_conv_launch(int prec, const CoarseArgs& a, int batch, int n_c, cudaStream_t st);

}  // namespace kd
