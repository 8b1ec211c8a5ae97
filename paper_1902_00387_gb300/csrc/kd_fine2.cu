// Fine-step kernels for grids n <= 256 built on the register-resident four-step FFT
// (kd_fft2.cuh): same two-kernels-per-stage structure and the same arithmetic as the
// shared-memory Stockham kernels of kd_fine.cu, with one shared-memory transpose per
// transform and loads / stores straight between global memory and registers.
//
// column kernel: thread (a, col), col fastest (XT columns per block), so that each
//   global access of a warp touches consecutive x of one ky row.
// row kernel:    thread (r, a), a fastest (RT rows per block), so that each global
//   access touches consecutive x (or kx) of one row.
#include "kd_fft2.cuh"
#include "kd_fine.h"
#include "kd_stage.cuh"

namespace kd {

template <typename T, int N>
struct Col2 {
  static constexpr int R1 = Split<N>::R1, R2 = Split<N>::R2;
  static constexpr int XT0 = N <= 64 ? 64 : (N == 128 ? 32 : 16);
  static constexpr int XT = sizeof(T) == 4 ? XT0 : (XT0 / 2 < 8 ? 8 : XT0 / 2);
  static constexpr int BLOCK = XT * R2;
  static constexpr size_t smem = (size_t)3 * N * XT * sizeof(cx<T>) + N * sizeof(cx<T>) + 2 * N * sizeof(T);
};

template <typename T, int N>
struct Row2 {
  static constexpr int R1 = Split<N>::R1, R2 = Split<N>::R2;
  static constexpr int BLOCK = sizeof(T) == 4 ? 256 : 128;
  static constexpr int RT = BLOCK / R2;
  // per-row exchange stride: R1 x (R2 + 1), padded to 8 (mod 16) complex slots
  static constexpr int LROW0 = R1 * (R2 + 1);
  static constexpr int LROW = LROW0 + ((8 - LROW0 % 16) + 16) % 16;
  static constexpr size_t smem = (size_t)3 * RT * LROW * sizeof(cx<T>) + N * sizeof(cx<T>);
};

template <typename T, int N>
__global__ void __launch_bounds__(Col2<T, N>::BLOCK) col2_kernel(FineArgs a, int step, int stage) {
  using G = Col2<T, N>;
  constexpr int R1 = G::R1, R2 = G::R2, XT = G::XT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* S = (cx<T>*)smem_raw;                    // [3][R1][R2][XT]
  cx<T>* s_tw = S + 3 * N * XT;                   // [N]
  T* s_cos = (T*)(s_tw + N);
  T* s_sin = s_cos + N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    s_tw[i] = ((const cx<T>*)a.tw)[i];
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
  auto slot = [&](int c, int q, int a2) { return S + ((c * R1 + q) * R2 + a2) * XT + col; };

  cx<T> v[3][R1];
  const cx<T>* M = (const cx<T>*)a.M;
#pragma unroll
  for (int k = 0; k < R1; ++k) {
    const int yy = lane + R2 * k;
    const int ky = yy < N / 2 ? yy : yy - N;
    const bool keep = valid && ky >= -K && ky <= K;
#pragma unroll
    for (int c = 0; c < 3; ++c)
      v[c][k] = keep ? M[((b * 3 + c) * P + (ky + K)) * (long)N + x] : mk(T(0), T(0));
  }
  __syncthreads();   // tables
  fft2_3<T, N, +1>(v, lane, s_tw, slot);           // ky -> y

  const Phase<T> ph = load_phase<T>(a, b, step, stage);
  const T A = (T)a.amp;
  const T cxg = s_cos[x], sxg = s_sin[x];
#pragma unroll
  for (int r = 0; r < R1; ++r) {
    const int y = lane + FFT2<N>::out_pos_base(r);
    cross_u<T>(A, ph, cxg, sxg, s_cos[y], s_sin[y], v[0][r], v[1][r], v[2][r]);
  }
  out_to_in<T, N>(v);
  __syncthreads();   // exchange buffers are reused
  fft2_3<T, N, -1>(v, lane, s_tw, slot);           // y -> ky

  if (!valid) return;
  cx<T>* W = (cx<T>*)a.W;
#pragma unroll
  for (int r = 0; r < R1; ++r) {
    const int yy = lane + FFT2<N>::out_pos_base(r);
    const int ky = yy < N / 2 ? yy : yy - N;
    if (ky >= -K && ky <= K) {
#pragma unroll
      for (int c = 0; c < 3; ++c) W[((b * 3 + c) * P + (ky + K)) * (long)N + x] = v[c][r];
    }
  }
}

// mode 0..3: stage update from W; mode 4: prologue (inverse x transform of X).
template <typename T, int N>
__global__ void __launch_bounds__(Row2<T, N>::BLOCK) row2_kernel(FineArgs a, int mode, int store_m) {
  using G = Row2<T, N>;
  constexpr int R1 = G::R1, R2 = G::R2, RT = G::RT, LROW = G::LROW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* S = (cx<T>*)smem_raw;                    // [3][RT][LROW]
  cx<T>* s_tw = S + 3 * RT * LROW;
  for (int i = threadIdx.x; i < N; i += blockDim.x) s_tw[i] = ((const cx<T>*)a.tw)[i];
  const int lane = threadIdx.x % R2;
  const int rr = threadIdx.x / R2;
  const int K = a.K, P = a.P;
  const long total = (long)a.batch * P;
  const long row = (long)blockIdx.x * RT + rr;
  const bool valid = row < total;
  const long b = valid ? row / P : 0;
  const int iy = valid ? (int)(row - b * P) : 0;
  auto slot = [&](int c, int q, int a2) { return S + (c * RT + rr) * LROW + q * (R2 + 1) + a2; };
  const long sbase = ((b * 3) * P + iy) * (long)P + K;   // compact index of (c = 0, iy, kx = 0)
  const long cst = (long)P * P;

  cx<T> v[3][R1];
  if (mode == 4) {
    const cx<T>* X = (const cx<T>*)a.X;
#pragma unroll
    for (int k = 0; k < R1; ++k) {
      const int xx = lane + R2 * k;
      const int kx = xx < N / 2 ? xx : xx - N;
      const bool keep = valid && kx >= -K && kx <= K;
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c][k] = keep ? X[sbase + c * cst + kx] : mk(T(0), T(0));
    }
    __syncthreads();
  } else {
    const cx<T>* W = (const cx<T>*)a.W;
#pragma unroll
    for (int k = 0; k < R1; ++k) {
      const int xx = lane + R2 * k;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        v[c][k] = valid ? W[((b * 3 + c) * P + iy) * (long)N + xx] : mk(T(0), T(0));
    }
    __syncthreads();
    fft2_3<T, N, -1>(v, lane, s_tw, slot);         // x -> kx
    const T inv_n2 = T(1) / (T(N) * T(N));
#pragma unroll
    for (int r = 0; r < R1; ++r) {
      const int xx = lane + FFT2<N>::out_pos_base(r);
      const int kx = xx < N / 2 ? xx : xx - N;
      if (valid && kx >= -K && kx <= K) {
        cx<T> w0 = v[0][r] * inv_n2, w1 = v[1][r] * inv_n2, w2 = v[2][r] * inv_n2;
        stage_update<T>(a, mode, sbase + kx, cst, (T)kx, (T)(iy - K), w0, w1, w2);
        v[0][r] = w0;
        v[1][r] = w1;
        v[2][r] = w2;
      } else {
        v[0][r] = v[1][r] = v[2][r] = mk(T(0), T(0));
      }
    }
    if (!store_m) return;   // uniform over the grid
    out_to_in<T, N>(v);
    __syncthreads();   // exchange buffers are reused
  }
  fft2_3<T, N, +1>(v, lane, s_tw, slot);           // kx -> x
  if (!valid) return;
  cx<T>* Mo = (cx<T>*)a.M;
#pragma unroll
  for (int r = 0; r < R1; ++r) {
    const int xx = lane + FFT2<N>::out_pos_base(r);
#pragma unroll
    for (int c = 0; c < 3; ++c) Mo[((b * 3 + c) * P + iy) * (long)N + xx] = v[c][r];
  }
}

template <typename T, int N>
static cudaError_t prepare2() {
  cudaError_t e = cudaFuncSetAttribute(col2_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Col2<T, N>::smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(row2_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Row2<T, N>::smem);
}

template <typename T>
static cudaError_t prepare2_all() {
  cudaError_t e;
  if ((e = prepare2<T, 16>()) != cudaSuccess) return e;
  if ((e = prepare2<T, 32>()) != cudaSuccess) return e;
  if ((e = prepare2<T, 64>()) != cudaSuccess) return e;
  if ((e = prepare2<T, 128>()) != cudaSuccess) return e;
  return prepare2<T, 256>();
}

cudaError_t fine2_prepare(int prec) { return prec == 0 ? prepare2_all<float>() : prepare2_all<double>(); }

template <typename T, int N>
static int steps2(const FineArgs& a, int nsteps, bool prologue, bool store_last, cudaStream_t st,
                  const LaunchProbe* pr) {
  using C = Col2<T, N>;
  using R = Row2<T, N>;
  const unsigned gc = (unsigned)(((long)a.batch * N + C::XT - 1) / C::XT);
  const unsigned gr = (unsigned)(((long)a.batch * a.P + R::RT - 1) / R::RT);
  int launches = 0;
  if (prologue) {
    row2_kernel<T, N><<<gr, R::BLOCK, R::smem, st>>>(a, 4, 1);
    ++launches;
  }
  for (int s = 0; s < nsteps; ++s) {
    for (int j = 0; j < 4; ++j) {
      if (pr) pr->before(pr->user, 0);
      col2_kernel<T, N><<<gc, C::BLOCK, C::smem, st>>>(a, s, j);
      if (pr) pr->after(pr->user, 0);
      const int store = (s == nsteps - 1 && j == 3) ? (store_last ? 1 : 0) : 1;
      if (pr) pr->before(pr->user, 1);
      row2_kernel<T, N><<<gr, R::BLOCK, R::smem, st>>>(a, j, store);
      if (pr) pr->after(pr->user, 1);
      launches += 2;
    }
  }
  return launches;
}

template <typename T>
static int steps2_T(const FineArgs& a, int nsteps, bool prologue, bool store_last, cudaStream_t st,
                    const LaunchProbe* pr) {
  switch (a.n) {
    case 16: return steps2<T, 16>(a, nsteps, prologue, store_last, st, pr);
    case 32: return steps2<T, 32>(a, nsteps, prologue, store_last, st, pr);
    case 64: return steps2<T, 64>(a, nsteps, prologue, store_last, st, pr);
    case 128: return steps2<T, 128>(a, nsteps, prologue, store_last, st, pr);
    case 256: return steps2<T, 256>(a, nsteps, prologue, store_last, st, pr);
  }
  return -1;
}

int fine2_launch_steps(int prec, const FineArgs& a, int nsteps, bool prologue, bool store_last, cudaStream_t st,
                       const LaunchProbe* pr) {
  return prec == 0 ? steps2_T<float>(a, nsteps, prologue, store_last, st, pr)
                   : steps2_T<double>(a, nsteps, prologue, store_last, st, pr);
}

}  // namespace kd
