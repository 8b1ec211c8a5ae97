// Fused pseudo-spectral IMEX RK443 fine step (the data-parallel fine propagator of
// Parareal, Sec. 3 Eq. 8 and Sec. 4), all slices of a batch advanced by every launch.
//
// One right-hand-side evaluation nabla_k x (u x b) followed by one IMEX stage is two
// kernels:
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

#include "kd_fft.cuh"
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

template <typename T>
struct Geo {
  // elements (transform length x transforms) held by one block, per component
  static constexpr int ELEMS = sizeof(T) == 4 ? 2048 : 1024;
};

template <typename T, int N>
struct ColGeo {
  static constexpr int TPT = N / 8;
  static constexpr int NTR = (Geo<T>::ELEMS / N) < 4 ? 4 : (Geo<T>::ELEMS / N);
  static constexpr int BLOCK = NTR * TPT;
};

template <typename T, int N>
struct RowGeo {
  static constexpr int TPT = N / 8;
  static constexpr int NTR = (Geo<T>::ELEMS / N) < 2 ? 2 : (Geo<T>::ELEMS / N);
  static constexpr int BLOCK = NTR * TPT;
};

template <typename T, int N, int NTR>
__device__ __forceinline__ void load_tables(cx<T>* s_tw, T* s_cos, T* s_sin, const FineArgs& a, bool grid) {
  const cx<T>* tw = (const cx<T>*)a.tw;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    s_tw[i] = tw[i];
    if (grid) {
      s_cos[i] = ((const T*)a.cosg)[i];
      s_sin[i] = ((const T*)a.sing)[i];
    }
  }
}

// ----------------------------------------------------------------- column kernel
template <typename T, int N>
__global__ void __launch_bounds__(ColGeo<T, N>::BLOCK) col_kernel(FineArgs a, int step, int stage) {
  using G = ColGeo<T, N>;
  constexpr int NTR = G::NTR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* buf = (cx<T>*)smem_raw;                  // [3][NTR][N]
  cx<T>* s_tw = buf + 3 * NTR * N;                // [N]
  T* s_cos = (T*)(s_tw + N);                      // [N]
  T* s_sin = s_cos + N;                           // [N]
  Phase<T>* s_ph = (Phase<T>*)(s_sin + N);       // [NTR]
  const int K = a.K, P = a.P;
  const long total = (long)a.batch * N;
  const long g0 = (long)blockIdx.x * NTR;
  const int cstride = NTR * N;

  load_tables<T, N, NTR>(s_tw, s_cos, s_sin, a, true);
  if (threadIdx.x < NTR) {
    const long g = g0 + threadIdx.x;
    s_ph[threadIdx.x] = load_phase<T>(a, g < total ? g / N : 0, step, stage);
  }
  // gather the kept ky entries of NTR columns; zero the rest
  const cx<T>* M = (const cx<T>*)a.M;
  for (int idx = threadIdx.x; idx < 3 * NTR * N; idx += blockDim.x) {
    const int c = idx / (NTR * N);
    const int r = idx - c * NTR * N;
    const int yy = r / NTR;  // FFT position (row index in y)
    const int t = r - yy * NTR;
    const long g = g0 + t;
    const int ky = yy < N / 2 ? yy : yy - N;
    cx<T> v = mk(T(0), T(0));
    if (ky >= -K && ky <= K && g < total) {
      const long b = g / N;
      const int x = (int)(g - b * N);
      v = M[((b * 3 + c) * P + (ky + K)) * (long)N + x];
    }
    buf[c * cstride + t * N + yy] = v;
  }
  __syncthreads();

  const int tr = threadIdx.x / G::TPT;
  const int lane = threadIdx.x - tr * G::TPT;
  fft3<T, N, +1>(buf + tr * N, cstride, lane, s_tw);   // ky -> y

  // w = u x b at (x, y) for every column of the block
  const T A = (T)a.amp;
  for (int idx = threadIdx.x; idx < NTR * N; idx += blockDim.x) {
    const int t = idx / N;
    const int y = idx - t * N;
    const long g = g0 + t;
    const int x = (int)(g % N);
    cross_u<T>(A, s_ph[t], s_cos[x], s_sin[x], s_cos[y], s_sin[y], buf[0 * cstride + idx], buf[1 * cstride + idx],
               buf[2 * cstride + idx]);
  }
  __syncthreads();

  fft3<T, N, -1>(buf + tr * N, cstride, lane, s_tw);   // y -> ky

  cx<T>* W = (cx<T>*)a.W;
  for (int idx = threadIdx.x; idx < 3 * P * NTR; idx += blockDim.x) {
    const int c = idx / (P * NTR);
    const int r = idx - c * P * NTR;
    const int iy = r / NTR;
    const int t = r - iy * NTR;
    const long g = g0 + t;
    if (g < total) {
      const long b = g / N;
      const int x = (int)(g - b * N);
      const int yy = (iy - K) & (N - 1);
      W[((b * 3 + c) * P + iy) * (long)N + x] = buf[c * cstride + t * N + yy];
    }
  }
}

// -------------------------------------------------------------------- row kernel
// mode: 0..3 = IMEX stage of the step whose explicit term W holds; 4 = prologue
// (inverse x transform of the state X only).  store_m: write the inverse x transform
// of the new stage value to M (false after the last stage of the last step).
template <typename T, int N>
__global__ void __launch_bounds__(RowGeo<T, N>::BLOCK) row_kernel(FineArgs a, int mode, int store_m) {
  using G = RowGeo<T, N>;
  constexpr int NTR = G::NTR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* buf = (cx<T>*)smem_raw;                  // [3][NTR][N]
  cx<T>* s_tw = buf + 3 * NTR * N;                // [N]
  const int K = a.K, P = a.P;
  const long total = (long)a.batch * P;
  const long r0 = (long)blockIdx.x * NTR;
  const int cstride = NTR * N;
  const int tr = threadIdx.x / G::TPT;
  const int lane = threadIdx.x - tr * G::TPT;
  load_tables<T, N, NTR>(s_tw, nullptr, nullptr, a, false);

  cx<T>* X = (cx<T>*)a.X;
  if (mode == 4) {
    for (int idx = threadIdx.x; idx < 3 * NTR * N; idx += blockDim.x) {
      const int c = idx / (NTR * N);
      const int r = idx - c * NTR * N;
      const int t = r / N;
      const int xx = r - t * N;
      const long row = r0 + t;
      const int kx = xx < N / 2 ? xx : xx - N;
      cx<T> v = mk(T(0), T(0));
      if (kx >= -K && kx <= K && row < total) {
        const long b = row / P;
        const int iy = (int)(row - b * P);
        v = X[((b * 3 + c) * P + iy) * (long)P + (kx + K)];
      }
      buf[c * cstride + t * N + xx] = v;
    }
    __syncthreads();
  } else {
    const cx<T>* W = (const cx<T>*)a.W;
    for (int idx = threadIdx.x; idx < 3 * NTR * N; idx += blockDim.x) {
      const int c = idx / (NTR * N);
      const int r = idx - c * NTR * N;
      const int t = r / N;
      const int xx = r - t * N;
      const long row = r0 + t;
      cx<T> v = mk(T(0), T(0));
      if (row < total) {
        const long b = row / P;
        const int iy = (int)(row - b * P);
        v = W[((b * 3 + c) * P + iy) * (long)N + xx];
      }
      buf[c * cstride + t * N + xx] = v;
    }
    __syncthreads();
    fft3<T, N, -1>(buf + tr * N, cstride, lane, s_tw);   // x -> kx

    const T inv_n2 = T(1) / (T(N) * T(N));
    for (int idx = threadIdx.x; idx < NTR * N; idx += blockDim.x) {
      const int t = idx / N;
      const int xx = idx - t * N;
      const long row = r0 + t;
      const int kx = xx < N / 2 ? xx : xx - N;
      cx<T>* e0 = &buf[0 * cstride + t * N + xx];
      cx<T>* e1 = &buf[1 * cstride + t * N + xx];
      cx<T>* e2 = &buf[2 * cstride + t * N + xx];
      if (kx < -K || kx > K || row >= total) {
        *e0 = mk(T(0), T(0));
        *e1 = mk(T(0), T(0));
        *e2 = mk(T(0), T(0));
        continue;
      }
      const long b = row / P;
      const int iy = (int)(row - b * P);
      cx<T> w0 = *e0 * inv_n2, w1 = *e1 * inv_n2, w2 = *e2 * inv_n2;
      stage_update<T>(a, stage_arrays<T>(a), mode, ((b * 3) * P + iy) * (long)P + (kx + K), (long)P * P, (T)kx,
                      (T)(iy - K), w0, w1, w2);
      *e0 = w0;
      *e1 = w1;
      *e2 = w2;
    }
    __syncthreads();
  }
  if (!store_m) return;   // uniform over the grid

  fft3<T, N, +1>(buf + tr * N, cstride, lane, s_tw);   // kx -> x
  cx<T>* Mo = (cx<T>*)a.M;
  for (int idx = threadIdx.x; idx < 3 * NTR * N; idx += blockDim.x) {
    const int c = idx / (NTR * N);
    const int r = idx - c * NTR * N;
    const int t = r / N;
    const int xx = r - t * N;
    const long row = r0 + t;
    if (row < total) {
      const long b = row / P;
      const int iy = (int)(row - b * P);
      Mo[((b * 3 + c) * P + iy) * (long)N + xx] = buf[c * cstride + t * N + xx];
    }
  }
}

// ------------------------------------------------------------------- launchers
template <typename T, int N>
static size_t col_smem() {
  using G = ColGeo<T, N>;
  return (size_t)3 * G::NTR * N * sizeof(cx<T>) + N * sizeof(cx<T>) + 2 * N * sizeof(T) + G::NTR * sizeof(Phase<T>);
}
template <typename T, int N>
static size_t row_smem() {
  using G = RowGeo<T, N>;
  return (size_t)3 * G::NTR * N * sizeof(cx<T>) + N * sizeof(cx<T>);
}

template <typename T, int N>
static cudaError_t prepare() {
  cudaError_t e = cudaFuncSetAttribute(col_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)col_smem<T, N>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(row_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem<T, N>());
}

template <typename T, int N>
static int launch_steps(const FineArgs& a, int nsteps, bool prologue, bool store_last, cudaStream_t st,
                        const LaunchProbe* pr) {
  using CG = ColGeo<T, N>;
  using RG = RowGeo<T, N>;
  const long cols = (long)a.batch * N;
  const long rows = (long)a.batch * a.P;
  const unsigned gc = (unsigned)((cols + CG::NTR - 1) / CG::NTR);
  const unsigned gr = (unsigned)((rows + RG::NTR - 1) / RG::NTR);
  const size_t sc = col_smem<T, N>(), sr = row_smem<T, N>();
  int launches = 0;
  if (prologue) {
    row_kernel<T, N><<<gr, RG::BLOCK, sr, st>>>(a, 4, 1);
    ++launches;
  }
  for (int s = 0; s < nsteps; ++s) {
    for (int j = 0; j < 4; ++j) {
      if (pr) pr->before(pr->user, 0);
      col_kernel<T, N><<<gc, CG::BLOCK, sc, st>>>(a, s, j);
      if (pr) pr->after(pr->user, 0);
      const int store = (s == nsteps - 1 && j == 3) ? (store_last ? 1 : 0) : 1;
      if (pr) pr->before(pr->user, 1);
      row_kernel<T, N><<<gr, RG::BLOCK, sr, st>>>(a, j, store);
      if (pr) pr->after(pr->user, 1);
      launches += 2;
    }
  }
  return launches;
}

template <typename T>
static cudaError_t prepare_all() {
  cudaError_t e;
  if ((e = prepare<T, 16>()) != cudaSuccess) return e;
  if ((e = prepare<T, 32>()) != cudaSuccess) return e;
  if ((e = prepare<T, 64>()) != cudaSuccess) return e;
  if ((e = prepare<T, 128>()) != cudaSuccess) return e;
  if ((e = prepare<T, 256>()) != cudaSuccess) return e;
  if ((e = prepare<T, 512>()) != cudaSuccess) return e;
  return prepare<T, 1024>();
}

cudaError_t fine_prepare(int prec) {
  cudaError_t e = prec == 0 ? prepare_all<float>() : prepare_all<double>();
  return e != cudaSuccess ? e : fine2_prepare(prec);
}

template <typename T>
static int launch_steps_T(const FineArgs& a, int nsteps, bool prologue, bool store_last, cudaStream_t st,
                          const LaunchProbe* pr) {
  switch (a.n) {
    case 16: return launch_steps<T, 16>(a, nsteps, prologue, store_last, st, pr);
    case 32: return launch_steps<T, 32>(a, nsteps, prologue, store_last, st, pr);
    case 64: return launch_steps<T, 64>(a, nsteps, prologue, store_last, st, pr);
    case 128: return launch_steps<T, 128>(a, nsteps, prologue, store_last, st, pr);
    case 256: return launch_steps<T, 256>(a, nsteps, prologue, store_last, st, pr);
    case 512: return launch_steps<T, 512>(a, nsteps, prologue, store_last, st, pr);
    case 1024: return launch_steps<T, 1024>(a, nsteps, prologue, store_last, st, pr);
  }
  return -1;
}

int fine_launch_steps(int prec, const FineArgs& a, int nsteps, bool prologue, bool store_last, cudaStream_t st,
                      const LaunchProbe* pr) {
  const int nph = launch_phases(prec, a, nsteps, st);
  int r;
  if (a.n <= 256)
    r = fine2_launch_steps(prec, a, nsteps, prologue, store_last, st, pr);
  else
    r = prec == 0 ? launch_steps_T<float>(a, nsteps, prologue, store_last, st, pr)
                  : launch_steps_T<double>(a, nsteps, prologue, store_last, st, pr);
  return r < 0 ? r : r + nph;
}

}  // namespace kd
