// Fine-step kernels for grids n = 512 and 1024 on the three-pass register FFT
// (kd_fft3.cuh).  Same two-kernels-per-stage structure and arithmetic as the n <= 256
// kernels of kd_fine2.cu; a thread keeps its 16 elements per component in registers
// from the global load through both transforms and the pointwise step.
#include "kd_fft3.cuh"
#include "kd_fine.h"
#include "kd_stage.cuh"

namespace kd {

template <typename T, int N>
struct Col3 {
  static constexpr int TPT = F3<N>::T;
  static constexpr int XT = (sizeof(T) == 4 ? 4096 : 2048) / N;   // columns per block
  static constexpr int BLOCK = XT * TPT;
  static constexpr int NPAD = F3<N>::NPAD;
  static constexpr size_t smem = (size_t)3 * NPAD * XT * sizeof(cx<T>) + N * sizeof(cx<T>) + 2 * N * sizeof(T);
};

template <typename T, int N>
struct Row3 {
  static constexpr int TPT = F3<N>::T;
  static constexpr int RT = (sizeof(T) == 4 ? 4096 : 2048) / N;    // rows per block
  static constexpr int BLOCK = RT * TPT;
  static constexpr int LROW0 = F3<N>::NPAD;
  static constexpr int LROW = LROW0 + ((8 - LROW0 % 16) + 16) % 16;
  static constexpr size_t smem = (size_t)3 * RT * LROW * sizeof(cx<T>) + N * sizeof(cx<T>);
};

template <typename T, int N>
__global__ void __launch_bounds__(Col3<T, N>::BLOCK) col3_kernel(FineArgs a, int step, int stage) {
  using G = Col3<T, N>;
  constexpr int XT = G::XT, TT = G::TPT, NPAD = G::NPAD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* S = (cx<T>*)smem_raw;                    // [3][NPAD][XT]
  cx<T>* s_tw = S + 3 * NPAD * XT;
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
  const T A = (T)a.amp;
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

// mode 0..3: stage update from W; mode 4: prologue (inverse x transform of X)
template <typename T, int N>
__global__ void __launch_bounds__(Row3<T, N>::BLOCK) row3_kernel(FineArgs a, int mode, int store_m) {
  using G = Row3<T, N>;
  constexpr int RT = G::RT, TT = G::TPT, LROW = G::LROW, BLOCK = G::BLOCK;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* S = (cx<T>*)smem_raw;                    // [3][RT][LROW]
  cx<T>* s_tw = S + 3 * RT * LROW;
  for (int i = threadIdx.x; i < N; i += BLOCK) s_tw[i] = ((const cx<T>*)a.tw)[i];
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
    __syncthreads();   // every exchange read is done before the staging writes
    const T inv_n2 = T(1) / (T(N) * T(N));
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
    const StageArrays<T> sa = stage_arrays<T>(a);
    const long rows_here = total - row0 < RT ? total - row0 : RT;
#pragma unroll 2
    for (int idx = threadIdx.x; idx < rows_here * P; idx += BLOCK) {
      const int r = idx / P, ix = idx - r * P;
      const long grow = row0 + r;
      const long gb = grow / P;
      const int giy = (int)(grow - gb * P);
      cx<T> w0 = *hslot(0, r, ix), w1 = *hslot(1, r, ix), w2 = *hslot(2, r, ix);
      stage_update<T>(a, sa, mode, ((gb * 3) * P + giy) * (long)P + ix, (long)P * P, (T)(ix - K), (T)(giy - K), w0,
                      w1, w2);
      *hslot(0, r, ix) = w0;
      *hslot(1, r, ix) = w1;
      *hslot(2, r, ix) = w2;
    }
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

template <typename T, int N>
static cudaError_t prepare3() {
  cudaError_t e = cudaFuncSetAttribute(col3_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Col3<T, N>::smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(row3_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Row3<T, N>::smem);
}

cudaError_t fine3_prepare(int prec) {
  cudaError_t e = prec == 0 ? prepare3<float, 512>() : prepare3<double, 512>();
  if (e != cudaSuccess) return e;
  return prec == 0 ? prepare3<float, 1024>() : prepare3<double, 1024>();
}

template <typename T, int N>
static int steps3(const FineArgs& a, int nsteps, bool prologue, bool store_last, cudaStream_t st,
                  const LaunchProbe* pr) {
  using C = Col3<T, N>;
  using R = Row3<T, N>;
  const unsigned gc = (unsigned)(((long)a.batch * N + C::XT - 1) / C::XT);
  const unsigned gr = (unsigned)(((long)a.batch * a.P + R::RT - 1) / R::RT);
  int launches = 0;
  if (prologue) {
    row3_kernel<T, N><<<gr, R::BLOCK, R::smem, st>>>(a, 4, 1);
    ++launches;
  }
  for (int s = 0; s < nsteps; ++s) {
    for (int j = 0; j < 4; ++j) {
      if (pr) pr->before(pr->user, 0);
      col3_kernel<T, N><<<gc, C::BLOCK, C::smem, st>>>(a, s, j);
      if (pr) pr->after(pr->user, 0);
      const int store = (s == nsteps - 1 && j == 3) ? (store_last ? 1 : 0) : 1;
      if (pr) pr->before(pr->user, 1);
      row3_kernel<T, N><<<gr, R::BLOCK, R::smem, st>>>(a, j, store);
      if (pr) pr->after(pr->user, 1);
      launches += 2;
    }
  }
  return launches;
}

int fine3_launch_steps(int prec, const FineArgs& a, int nsteps, bool prologue, bool store_last, cudaStream_t st,
                       const LaunchProbe* pr) {
  if (a.n == 512)
    return prec == 0 ? steps3<float, 512>(a, nsteps, prologue, store_last, st, pr)
                     : steps3<double, 512>(a, nsteps, prologue, store_last, st, pr);
  if (a.n == 1024)
    return prec == 0 ? steps3<float, 1024>(a, nsteps, prologue, store_last, st, pr)
                     : steps3<double, 1024>(a, nsteps, prologue, store_last, st, pr);
  return -1;
}

}  // namespace kd
