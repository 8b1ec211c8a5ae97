// Persistent classical coarse propagator (kd_coarse.cu).
#pragma once
#include "kd_common.cuh"

namespace kd {

// COARSE_OUT: write G(U) to g64.  COARSE_INIT: U_{n+1} = G(U_n), Gold = G(U_n).
// COARSE_UPDATE: U_{n+1} = F + (G(U_n) - Gold), Gold = G(U_n).
// COARSE_INCR: U_{n+1} = F + G(U_n - Uprev_n)  (increment form; Gold unused).
enum { COARSE_OUT = 0, COARSE_INIT = 1, COARSE_UPDATE = 2, COARSE_INCR = 3 };

// Mode sets are squares k in [-K, P - K)^2 per axis (the dealiased sets are K = n/3,
// P = 2K + 1; the learned operator's set is K = m/2, P = m).
struct CoarseArgs {
  int Kc, Pc;         // coarse set
  int Kf, Pf;         // input / update set (fine compact layout)
  int flow;
  double amp, kz, Rm, dt;
  int nsteps;
  const void* phases;   // [batch][nsteps][4][4] flow phases (precision T) or NULL (steady flow)
  const double* Un;     // fine compact FP64 inputs [batch][3][Pf][Pf] (complex interleaved)
  const double* Uprev;  // COARSE_INCR: previous iterate of the same slice (input is Un - Uprev)
  int mode;             // COARSE_OUT: write g64; otherwise the Parareal update (batch 1)
  double* g64;          // COARSE_OUT: coarse-set FP64 outputs [batch][3][Pc][Pc]
  const double* Fv;     // COARSE_UPDATE: fine values F(U_n), fine compact FP64
  double* Gold;         // coarse values of the previous sweep (read, then replaced)
  double* Unext;        // U_{n+1}, fine compact FP64 (written)
  double* sigma_out;    // if not NULL: sigma, |U - U_old|^2, |U|^2 of Unext (3 doubles per field)
  int phase_smem;       // (internal) phase values the cluster kernel may stage in shared memory
  // Batched instances (all optional): per-field parameters (kz, Rm, dt, amplitude; the
  // phase table then covers every field), per-field step counts (<= nsteps; the phase
  // table stride stays nsteps) and per-field slots: field b reads Un / Uprev / Fv at slot
  // map[b] (stride 3 Pf^2 complex) and writes slot map[b] + 1 of Unext.
  const SliceParams* sp;
  const int* steps;
  const int* map;
  int cluster;          // thread blocks per cluster (0: the default for Pc)
  int halo;             // halo exchange per stage: 0 halo stores + cluster barrier; 1 point-to-
                        // point (st.async counted on the receiver's mbarrier); 2 pull (the
                        // neighbours' rows read in place after a split cluster barrier)
};

bool coarse_conv_supported(int P);   // coarse set side P <= 88 (P <= 127 with 16-block clusters)
// whether a cluster of `cs` blocks can hold a P-row square (cs = 0: the default)
bool coarse_cluster_fits(int P, int cs);
cudaError_t coarse_prepare(int prec);
// the kernels of the alternative halo exchanges (CoarseArgs::halo 1, 2; kd_coarse_alt.cu)
cudaError_t coarse_alt_allow_nonportable(int prec);
cudaError_t coarse_alt_set_smem(int prec, int bytes);
cudaError_t coarse_alt_launch(int prec, const cudaLaunchConfig_t& cfg, int mpt, const CoarseArgs& a, int CS, int H);
// One thread-block cluster per field; returns 1 (kernels launched) or -1 if unsupported.
int coarse_conv_launch(int prec, const CoarseArgs& a, int batch, cudaStream_t st);

}  // namespace kd
