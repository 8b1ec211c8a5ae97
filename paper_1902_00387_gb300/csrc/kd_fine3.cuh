// Fine-step kernels for grids n = 512 and 1024 on the three-pass register FFT
// (kd_fft3.cuh).  Same two-kernels-per-stage structure and arithmetic as the n <= 256
// kernels of kd_fine2.cuh; a thread keeps its 16 elements per component in registers
// from the global load through both transforms and the pointwise step.  As there, the
// kernels are templates over the tile shape and the row kernel's stage-update style,
// and the instantiated shapes are the autotuner's candidates.
#pragma once
#include "kd_fft3.cuh"
#include "kd_fine2.cuh"

namespace kd {

// Candidate tile shapes of the n = 512, 1024 kernels (index 0 is the default plan).
template <typename T, int N>
struct Shapes3 {
  static constexpr int XT0 = (sizeof(T) == 4 ? 4096 : 2048) / N;
  static constexpr int RT0 = (sizeof(T) == 4 ? 4096 : 2048) / N;
  static constexpr int xt(int v) { return v == 0 ? XT0 : XT0 / 2; }
  static constexpr int rt(int v) { return (v & 1) == 0 ? RT0 : RT0 / 2; }
};

template <typename T, int N, int XT_>
struct Col3 {
  static constexpr int TPT = F3<N>::T;
  static constexpr int XT = XT_;                   // columns per block
  static constexpr int BLOCK = XT * TPT;
  static constexpr int NPAD = F3<N>::NPAD;
  static constexpr size_t smem =
      (size_t)3 * NPAD * XT * sizeof(cx<T>) + F3<N>::TWS * sizeof(cx<T>) + 2 * N * sizeof(T);
  static constexpr int MIN_BLOCKS = sizeof(T) == 4 ? fit_blocks(BLOCK, smem, 128) : 1;
};

template <typename T, int N, int RT_, int REGS = 128>
struct Row3 {
  static constexpr int TPT = F3<N>::T;
  static constexpr int RT = RT_;                   // rows per block
  static constexpr int BLOCK = RT * TPT;
  static constexpr int LROW0 = F3<N>::NPAD;
  static constexpr int LROW = LROW0 + ((8 - LROW0 % 16) + 16) % 16;
  static constexpr size_t smem = (size_t)3 * RT * LROW * sizeof(cx<T>) + F3<N>::TWS * sizeof(cx<T>);
  static constexpr int MIN_BLOCKS = sizeof(T) == 4 ? fit_blocks(BLOCK, smem, REGS) : 1;
};

template <typename T, int N, int XT>
__global__ void __launch_bounds__(Col3<T, N, XT>::BLOCK, Col3<T, N, XT>::MIN_BLOCKS)
    col3_kernel(FineArgs a, int step, int stage) {
  using G = Col3<T, N, XT>;
  constexpr int TT = G::TPT, NPAD = G::NPAD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* S = (cx<T>*)smem_raw;                    // [3][NPAD][XT]
  cx<T>* s_tw = S + 3 * NPAD * XT;
  T* s_cos = (T*)(s_tw + F3<N>::TWS);
  T* s_sin = s_cos + N;
  fft3_tables<T, N>(s_tw, (const cx<T>*)a.tw);
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    s_cos[i] = ((const T*)a.cosg)[i];
    s_sin[i] = ((const T*)a.sing)[i];
  }
  const int col = threadIdx.x % XT;
  const int lane = threadIdx.x / XT;
  const long total = (long)a.batch * N;
  const long g = (long)blockIdx.x * XT + col;
  const bool valid = g < total;
  const long b = valid ? g / N : 0;
  const int x = (int)(g - (g / N) * N);
  const int K = a.K, P = a.P;
  auto slot = [&](int c, int pi) { return S + ((long)c * NPAD + pi) * XT + col; };

  cx<T> v[3][16];
  const cx<T>* M = (const cx<T>*)a.M;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int yy = lane + TT * k;
    const int ky = yy < N / 2 ? yy : yy - N;
    const bool keep = valid && ky >= -K && ky <= K;
#pragma unroll
    for (int c = 0; c < 3; ++c)
      v[c][k] = keep ? M[((b * 3 + c) * P + (ky + K)) * (long)N + x] : mk(T(0), T(0));
  }
  __syncthreads();   // tables
  fft3_3<T, N, +1>(v, lane, s_tw, slot);           // ky -> y

  const Phase<T> ph = load_phase<T>(a, b, step, stage);
  const T A = flow_amp<T>(a, b);
  const T cxg = s_cos[x], sxg = s_sin[x];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int y = lane + TT * q;
    cross_u<T>(A, ph, cxg, sxg, s_cos[y], s_sin[y], v[0][q], v[1][q], v[2][q]);
  }
  __syncthreads();   // exchange buffer is reused
  fft3_3<T, N, -1>(v, lane, s_tw, slot);           // y -> ky

  if (!valid) return;
  cx<T>* W = (cx<T>*)a.W;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int yy = lane + TT * q;
    const int ky = yy < N / 2 ? yy : yy - N;
    if (ky >= -K && ky <= K) {
#pragma unroll
      for (int c = 0; c < 3; ++c) W[((b * 3 + c) * P + (ky + K)) * (long)N + x] = v[c][q];
    }
  }
}

// mode 0..3: stage update from W; mode 4: prologue (inverse x transform of X).
// STAGED as in row2_kernel; otherwise lane j updates its kept modes j + q T in registers.
template <typename T, int N, int RT, bool STAGED>
__global__ void __launch_bounds__(Row3<T, N, RT, STAGED ? 128 : 168>::BLOCK, Row3<T, N, RT, STAGED ? 128 : 168>::MIN_BLOCKS)
    row3_kernel(FineArgs a, int mode, int store_m) {
  using G = Row3<T, N, RT, STAGED ? 128 : 168>;
  constexpr int TT = G::TPT, LROW = G::LROW, BLOCK = G::BLOCK;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* S = (cx<T>*)smem_raw;                    // [3][RT][LROW]
  cx<T>* s_tw = S + 3 * RT * LROW;
  fft3_tables<T, N>(s_tw, (const cx<T>*)a.tw);
  const int lane = threadIdx.x % TT;
  const int rr = threadIdx.x / TT;
  const int K = a.K, P = a.P;
  const long total = (long)a.batch * P;
  const long row0 = (long)blockIdx.x * RT;
  const long row = row0 + rr;
  const bool valid = row < total;
  const long b = valid ? row / P : 0;
  const int iy = valid ? (int)(row - b * P) : 0;
  auto slot = [&](int c, int pi) { return S + (c * RT + rr) * LROW + pi; };
  auto hslot = [&](int c, int r, int ix) { return S + (c * RT + r) * LROW + ix; };

  cx<T> v[3][16];
  if (mode == 4) {
    const cx<T>* X = (const cx<T>*)a.X;
    const long sbase = ((b * 3) * P + iy) * (long)P + K;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int xx = lane + TT * k;
      const int kx = xx < N / 2 ? xx : xx - N;
      const bool keep = valid && kx >= -K && kx <= K;
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c][k] = keep ? X[sbase + c * (long)P * P + kx] : mk(T(0), T(0));
    }
    __syncthreads();
  } else {
    const cx<T>* W = (const cx<T>*)a.W;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int xx = lane + TT * k;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        v[c][k] = valid ? W[((b * 3 + c) * P + iy) * (long)N + xx] : mk(T(0), T(0));
    }
    __syncthreads();
    fft3_3<T, N, -1>(v, lane, s_tw, slot);         // x -> kx
    const T inv_n2 = T(1) / (T(N) * T(N));
    const StageArrays<T> sa = stage_arrays<T>(a);
    if (STAGED) {
      __syncthreads();   // every exchange read is done before the staging writes
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int xx = lane + TT * q;
        const int kx = xx < N / 2 ? xx : xx - N;
        if (kx >= -K && kx <= K) {
#pragma unroll
          for (int c = 0; c < 3; ++c) *hslot(c, rr, kx + K) = v[c][q] * inv_n2;
        }
      }
      __syncthreads();
      const long rows_here = total - row0 < RT ? total - row0 : RT;
      with_stage(mode, [&](auto m) {
        constexpr int MODE = decltype(m)::value;
#pragma unroll 4
        for (int idx = threadIdx.x; idx < rows_here * P; idx += BLOCK) {
          const int r = idx / P, ix = idx - r * P;
          const long grow = row0 + r;
          const long gb = grow / P;
          const int giy = (int)(grow - gb * P);
          cx<T> w0 = *hslot(0, r, ix), w1 = *hslot(1, r, ix), w2 = *hslot(2, r, ix);
          stage_update<MODE, T>(stage_coef<T>(a, gb), sa, ((gb * 3) * P + giy) * (long)P + ix, (long)P * P,
                                (T)(ix - K), (T)(giy - K), w0, w1, w2);
          *hslot(0, r, ix) = w0;
          *hslot(1, r, ix) = w1;
          *hslot(2, r, ix) = w2;
        }
      });
      if (!store_m) return;   // uniform over the grid
      __syncthreads();
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int xx = lane + TT * k;
        const int kx = xx < N / 2 ? xx : xx - N;
        const bool keep = kx >= -K && kx <= K;
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c][k] = keep ? *hslot(c, rr, kx + K) : mk(T(0), T(0));
      }
      __syncthreads();   // staging reads are done before the exchange writes
    } else {
      const StageCoef<T> sc = stage_coef<T>(a, b);
      const long s0 = ((b * 3) * P + iy) * (long)P + K;
      const T fky = (T)(iy - K);
      with_stage(mode, [&](auto m) {
        constexpr int MODE = decltype(m)::value;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int xx = lane + TT * q;
          const int kx = xx < N / 2 ? xx : xx - N;
          if (valid && kx >= -K && kx <= K) {
            cx<T> w0 = v[0][q] * inv_n2, w1 = v[1][q] * inv_n2, w2 = v[2][q] * inv_n2;
            stage_update<MODE, T>(sc, sa, s0 + kx, (long)P * P, (T)kx, fky, w0, w1, w2);
            v[0][q] = w0;
            v[1][q] = w1;
            v[2][q] = w2;
          } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) v[c][q] = mk(T(0), T(0));
          }
          if (q % kUpdateGroup == kUpdateGroup - 1) asm volatile("" ::: "memory");
        }
      });
      if (!store_m) return;   // uniform over the grid
      __syncthreads();   // exchange reads of the forward transform are done
    }
  }
  fft3_3<T, N, +1>(v, lane, s_tw, slot);           // kx -> x
  if (!valid) return;
  cx<T>* Mo = (cx<T>*)a.M;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int xx = lane + TT * q;
#pragma unroll
    for (int c = 0; c < 3; ++c) Mo[((b * 3 + c) * P + iy) * (long)N + xx] = v[c][q];
  }
}


template <typename T, int N, int XT>
static cudaError_t prepare_col3() {
  return cudaFuncSetAttribute(col3_kernel<T, N, XT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Col3<T, N, XT>::smem);
}

template <typename T, int N, int RT, bool STAGED>
static cudaError_t prepare_row3() {
  return cudaFuncSetAttribute(row3_kernel<T, N, RT, STAGED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Row3<T, N, RT, STAGED ? 128 : 168>::smem);
}

template <typename T, int N, int XT>
static void launch_col3(const FineArgs& a, int s, int j, cudaStream_t st) {
  using C = Col3<T, N, XT>;
  const unsigned gc = (unsigned)(((long)a.batch * N + XT - 1) / XT);
  col3_kernel<T, N, XT><<<gc, C::BLOCK, C::smem, st>>>(a, s, j);
}

template <typename T, int N, int RT, bool STAGED>
static void launch_row3(const FineArgs& a, int mode, int store, cudaStream_t st) {
  using R = Row3<T, N, RT, STAGED ? 128 : 168>;
  const unsigned gr = (unsigned)(((long)a.batch * a.P + RT - 1) / RT);
  row3_kernel<T, N, RT, STAGED><<<gr, R::BLOCK, R::smem, st>>>(a, mode, store);
}

template <typename T, int N>
struct Fine3Set {
  using Sh = Shapes3<T, N>;
  static constexpr bool WIDE = sizeof(T) == 4;
  static int ncol() { return WIDE ? 2 : 1; }
  static int nrow() { return WIDE ? 4 : 1; }
  static cudaError_t prepare() {
    cudaError_t e;
    if ((e = prepare_col3<T, N, Sh::xt(0)>()) != cudaSuccess) return e;
    if ((e = prepare_row3<T, N, Sh::rt(0), true>()) != cudaSuccess) return e;
    if (WIDE) {
      if ((e = prepare_col3<T, N, Sh::xt(1)>()) != cudaSuccess) return e;
      if ((e = prepare_row3<T, N, Sh::rt(1), true>()) != cudaSuccess) return e;
      if ((e = prepare_row3<T, N, Sh::rt(0), false>()) != cudaSuccess) return e;
      if ((e = prepare_row3<T, N, Sh::rt(1), false>()) != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  static void col(int v, const FineArgs& a, int s, int j, cudaStream_t st) {
    if (WIDE && v == 1)
      launch_col3<T, N, Sh::xt(1)>(a, s, j, st);
    else
      launch_col3<T, N, Sh::xt(0)>(a, s, j, st);
  }
  static void row(int v, const FineArgs& a, int mode, int store, cudaStream_t st) {
    if (!WIDE) v = 0;
    switch (v) {
      case 1: launch_row3<T, N, Sh::rt(1), true>(a, mode, store, st); break;
      case 2: launch_row3<T, N, Sh::rt(0), false>(a, mode, store, st); break;
      case 3: launch_row3<T, N, Sh::rt(1), false>(a, mode, store, st); break;
      default: launch_row3<T, N, Sh::rt(0), true>(a, mode, store, st); break;
    }
  }
};

template <typename T, int N>
int fine3_run(const FineArgs& a, const StepCfg& cfg) {
  return run_steps<Fine3Set<T, N>>(a, cfg);
}

template <typename T, int N>
cudaError_t fine3_prep() {
  return Fine3Set<T, N>::prepare();
}

template <typename T, int N>
void fine3_variants(int* ncol, int* nrow) {
  *ncol = Fine3Set<T, N>::ncol();
  *nrow = Fine3Set<T, N>::nrow();
}

}  // namespace kd

#define KD_FINE3_INSTANTIATE(T, N)                                        \
  template int kd::fine3_run<T, N>(const kd::FineArgs&, const kd::StepCfg&); \
  template cudaError_t kd::fine3_prep<T, N>();                             \
  template void kd::fine3_variants<T, N>(int*, int*);
