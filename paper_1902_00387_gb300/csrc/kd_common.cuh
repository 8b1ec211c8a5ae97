// Shared device/host definitions of the kd library (CUDA path only).
//
// Data layouts used inside the library (the public ABI layout is the full n x n grid,
// see include/kd.h):
//   K = n / 3 (2/3 dealiasing: |kx|, |ky| <= K are kept), P = 2K + 1.
//   compact spectral  S[b][c][iy][ix]  iy = ky + K, ix = kx + K       (P x P per component)
//   mixed             M[b][c][iy][x]   ky rows, physical x columns    (P x n per component)
// b = slice / batch index, c = field component (x, y, z).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace kd {

template <typename T>
struct alignas(2 * sizeof(T)) cx {
  T x, y;
};

template <typename T>
__host__ __device__ __forceinline__ cx<T> mk(T a, T b) {
  cx<T> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator*(cx<T> a, T s) { return mk(a.x * s, a.y * s); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// i * a
template <typename T>
__host__ __device__ __forceinline__ cx<T> mul_i(cx<T> a) { return mk(-a.y, a.x); }

// Programmatic dependent launch (kernels launched with the attribute
// cudaLaunchAttributeProgrammaticStreamSerialization may start while their predecessor in
// the stream drains): griddep_wait() returns once the predecessor has completed and its
// memory is visible (immediately for an ordinary launch); griddep_launch_dependents() lets
// the successor be scheduled.  A kernel reads its predecessor's outputs only after
// griddep_wait() and calls griddep_launch_dependents() only after its own wait, so data
// written two launches back is complete before the wait as well.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// Flow identifiers (match include/kd.h).
enum { FLOW_ROBERTS = 0, FLOW_GP = 1, FLOW_NONE = 2 };

// Per-grid device tables, one set per (n, precision): twiddles w_n^e = exp(-2 pi i e / n)
// and cos / sin of the collocation points 2 pi j / n.  Computed in double on the host.
struct GridTables {
  int n;
  void* tw;    // cx<T>[n]
  void* cosg;  // T[n]
  void* sing;  // T[n]
};

// Per-slice parameters of a batch whose fields belong to different problems (batched
// instances): flow amplitude, kz, Rm and the step dt of field b; flow is FLOW_*.
struct SliceParams {
  double amp, kz, Rm, dt;
  int flow, pad;
};

// Everything a fine-step kernel needs about one batched propagation.
struct FineArgs {
  int n, K, P;
  int batch;
  int flow;
  double amp;      // flow amplitude: 1 (Roberts), sqrt(3/2) (Galloway-Proctor), 0 (none)
  double kz, Rm, dt;
  const double* t0;  // [batch] absolute start time of each slice (device)
  void* X;           // compact state              [batch][3][P][P]
  void* R2;          // stage accumulators          [batch][3][P][P]
  void* R3;
  void* R4;          // holds R4 - X0 (the increment of the last stage over the state)
  void* Xlo;         // complex64 only (else NULL): low part of the state, X + Xlo (see kd_stage.cuh)
  int lo_valid;      // Xlo holds the low part of X (false before the first step of a call)
  void* M;           // mixed (inverse-x) field     [batch][3][P][n]
  void* W;           // mixed (forward-y) product   [batch][3][P][n]
  const void* tw;
  const void* cosg;
  const void* sing;
  const void* phases;  // Galloway-Proctor flow phases [batch][phase_steps][4 stages][4] (precision T)
  int phase_steps;     // steps covered by the phase table
  const SliceParams* sp;  // optional [batch] per-slice parameters (NULL: the scalars above);
                          // with sp the phase table is read for every field (flow = FLOW_GP)
  int scheme;             // IMEX scheme of the fine step: SCHEME_RK443 / RK222 / RK111
  // The state in the caller's full layout [batch][3][n][n] (FFT order), for kernels that
  // read or write it there directly (fine_full_io): x_in_full, if set, replaces X as the
  // state read before the first step's update; x_out_full, if set, receives the state
  // after the last step (its kept entries; X and Xlo are not written then).
  const void* x_in_full = nullptr;
  void* x_out_full = nullptr;
};

// IMEX Runge-Kutta schemes of the fine step (match include/kd.h KD_RK*) and their stage
// counts.
enum { SCHEME_RK443 = 0, SCHEME_RK222 = 1, SCHEME_RK111 = 2 };
__host__ __device__ constexpr int scheme_stages(int sch) { return sch == SCHEME_RK443 ? 4 : (sch == SCHEME_RK222 ? 2 : 1); }

}  // namespace kd
