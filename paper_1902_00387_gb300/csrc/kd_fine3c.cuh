// Component-split fine-step kernels for grids n = 512, 1024 (three-pass register FFT with
// 16 values per thread, kd_fft3.cuh): every thread transforms one field component, the
// components meeting in shared memory for u x b (column kernel) and for the curl and
// stage update (row kernel, staged).  Three times the threads of col3_kernel /
// row3_kernel at a third of the registers each; same arithmetic.
#pragma once
#include "kd_fine3.cuh"

namespace kd {

template <typename T, int N, int XT_>
struct Col3C {
  static constexpr int TPT = F3<N>::T, XT = XT_, BLOCK = XT * 3 * TPT;
  static constexpr int NPAD = F3<N>::NPAD;
  static constexpr size_t smem =
      (size_t)3 * NPAD * XT * sizeof(cx<T>) + F3<N>::TWS * sizeof(cx<T>) + 2 * N * sizeof(T);
  static constexpr int MIN_BLOCKS = fit_blocks(BLOCK, smem, 80);
};

template <typename T, int N, int RT_>
struct Row3C {
  static constexpr int TPT = F3<N>::T, RT = RT_, BLOCK = RT * 3 * TPT;
  static constexpr int LROW0 = F3<N>::NPAD;
  static constexpr int LROW = LROW0 + ((8 - LROW0 % 16) + 16) % 16;
  static constexpr size_t smem = (size_t)3 * RT * LROW * sizeof(cx<T>) + F3<N>::TWS * sizeof(cx<T>);
  static constexpr int MIN_BLOCKS = fit_blocks(BLOCK, smem, 80);
};

// thread (col, c, lane), col fastest
template <typename T, int N, int XT>
__global__ void __launch_bounds__(Col3C<T, N, XT>::BLOCK, Col3C<T, N, XT>::MIN_BLOCKS)
    col3c_kernel(FineArgs a, int step, int stage) {
  using G = Col3C<T, N, XT>;
  constexpr int TT = G::TPT, NPAD = G::NPAD;
  constexpr int K = N / 3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* S = (cx<T>*)smem_raw;                    // [3][NPAD][XT] exchange, then [3][N][XT] grid staging
  cx<T>* s_tw = S + 3 * NPAD * XT;
  T* s_cos = (T*)(s_tw + F3<N>::TWS);
  T* s_sin = s_cos + N;
  fft3_tables<T, N>(s_tw, (const cx<T>*)a.tw);
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    s_cos[i] = ((const T*)a.cosg)[i];
    s_sin[i] = ((const T*)a.sing)[i];
  }
  const int col = threadIdx.x % XT;
  const int rest = threadIdx.x / XT;
  const int c = rest % 3;
  const int lane = rest / 3;
  const long total = (long)a.batch * N;
  const long g = (long)blockIdx.x * XT + col;
  const bool valid = g < total;
  const long b = valid ? g / N : 0;
  const int x = (int)(g - (g / N) * N);
  const int P = a.P;
  auto slot = [&](int pi) { return S + ((long)c * NPAD + pi) * XT + col; };
  auto grid = [&](int cc, int y) { return S + ((long)cc * N + y) * XT + col; };

  cx<T> v[16];
  const cx<T>* M = (const cx<T>*)a.M;
  griddep_wait();    // M is the predecessor's output
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int yy = lane + TT * k;
    const int ky = yy < N / 2 ? yy : yy - N;
    const bool keep = valid && ky >= -K && ky <= K;
    v[k] = keep ? M[((b * 3 + c) * P + (ky + K)) * (long)N + x] : mk(T(0), T(0));
  }
  __syncthreads();   // tables
  fft3r_1<T, N, 16, +1>(v, lane, s_tw, slot);      // ky -> y
  __syncthreads();   // exchange reads are done: the buffer now stages b on the grid
#pragma unroll
  for (int q = 0; q < 16; ++q) *grid(c, lane + TT * q) = v[q];
  __syncthreads();
  const Phase<T> ph = load_phase<T>(a, b, step, stage);
  const T A = flow_amp<T>(a, b);
  const T cxg = s_cos[x], sxg = s_sin[x];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int y = lane + TT * q;
    cx<T> bx = *grid(0, y), by = *grid(1, y), bz = *grid(2, y);
    cross_u<T>(A, ph, cxg, sxg, s_cos[y], s_sin[y], bx, by, bz);
    v[q] = c == 0 ? bx : (c == 1 ? by : bz);
    if (q % 4 == 3) asm volatile("" ::: "memory");   // bounds the loads in flight (registers)
  }
  griddep_launch_dependents();
  __syncthreads();   // staging reads are done before the exchange writes
  fft3r_1<T, N, 16, -1>(v, lane, s_tw, slot);      // y -> ky
  if (!valid) return;
  cx<T>* W = (cx<T>*)a.W;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int yy = lane + TT * q;
    const int ky = yy < N / 2 ? yy : yy - N;
    if (ky >= -K && ky <= K) W[((b * 3 + c) * P + (ky + K)) * (long)N + x] = v[q];
  }
}

// thread (lane, c, r), lane fastest; mode 0..3: stage update from W; mode 4: prologue
template <typename T, int N, int RT>
__global__ void __launch_bounds__(Row3C<T, N, RT>::BLOCK, Row3C<T, N, RT>::MIN_BLOCKS)
    row3c_kernel(FineArgs a, int mode, int store_m) {
  using G = Row3C<T, N, RT>;
  constexpr int TT = G::TPT, LROW = G::LROW, BLOCK = G::BLOCK;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* S = (cx<T>*)smem_raw;                    // [3][RT][LROW]
  cx<T>* s_tw = S + 3 * RT * LROW;
  fft3_tables<T, N>(s_tw, (const cx<T>*)a.tw);
  const int lane = threadIdx.x % TT;
  const int rest = threadIdx.x / TT;
  const int c = rest % 3;
  const int rr = rest / 3;
  const int K = a.K, P = a.P;
  const long total = (long)a.batch * P;
  const long row0 = (long)blockIdx.x * RT;
  const long row = row0 + rr;
  const bool valid = row < total;
  const long b = valid ? row / P : 0;
  const int iy = valid ? (int)(row - b * P) : 0;
  auto slot = [&](int pi) { return S + (c * RT + rr) * LROW + pi; };
  auto hslot = [&](int cc, int r, int ix) { return S + (cc * RT + r) * LROW + ix; };

  cx<T> v[16];
  griddep_wait();    // W (and, for the prologue, X) come from the predecessors
  if (mode == 4) {
    const cx<T>* X = (const cx<T>*)a.X;
    const long sbase = ((b * 3 + c) * P + iy) * (long)P + K;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int xx = lane + TT * k;
      const int kx = xx < N / 2 ? xx : xx - N;
      const bool keep = valid && kx >= -K && kx <= K;
      v[k] = keep ? X[sbase + kx] : mk(T(0), T(0));
    }
    __syncthreads();
  } else {
    const cx<T>* W = (const cx<T>*)a.W;
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = valid ? W[((b * 3 + c) * P + iy) * (long)N + lane + TT * k] : mk(T(0), T(0));
    __syncthreads();
    fft3r_1<T, N, 16, -1>(v, lane, s_tw, slot);    // x -> kx
    const T inv_n2 = T(1) / (T(N) * T(N));
    __syncthreads();   // every exchange read is done before the staging writes
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int xx = lane + TT * q;
      const int kx = xx < N / 2 ? xx : xx - N;
      if (kx >= -K && kx <= K) *hslot(c, rr, kx + K) = v[q] * inv_n2;
    }
    __syncthreads();
    const StageArrays<T> sa = stage_arrays<T>(a);
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
      v[k] = (kx >= -K && kx <= K) ? *hslot(c, rr, kx + K) : mk(T(0), T(0));
    }
    __syncthreads();   // staging reads are done before the exchange writes
  }
  griddep_launch_dependents();
  fft3r_1<T, N, 16, +1>(v, lane, s_tw, slot);      // kx -> x
  if (!valid) return;
  cx<T>* Mo = (cx<T>*)a.M;
#pragma unroll
  for (int q = 0; q < 16; ++q) Mo[((b * 3 + c) * P + iy) * (long)N + lane + TT * q] = v[q];
}

}  // namespace kd
