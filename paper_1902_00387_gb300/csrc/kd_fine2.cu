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
  static constexpr int MIN_BLOCKS = BLOCK <= 256 ? 2 : 1;   // register cap: two blocks per SM
  static constexpr size_t smem = (size_t)3 * N * XT * sizeof(cx<T>) + N * sizeof(cx<T>) + 2 * N * sizeof(T);
};

// RT rows per block; BLOCK = RT * R2 threads.
template <typename T, int N, int RT_>
struct Row2 {
  static constexpr int R1 = Split<N>::R1, R2 = Split<N>::R2;
  static constexpr int RT = RT_;
  static constexpr int BLOCK = RT * R2;
  static constexpr int K = N / 3, P = 2 * K + 1;
  // per-row exchange stride: R1 x (R2 + 1), padded to 8 (mod 16) complex slots
  static constexpr int LROW0 = R1 * (R2 + 1);
  static constexpr int LROW = LROW0 + ((8 - LROW0 % 16) + 16) % 16;
  static_assert(LROW >= P, "staging of the kept modes reuses the exchange buffer");
  static constexpr size_t smem = (size_t)3 * RT * LROW * sizeof(cx<T>) + N * sizeof(cx<T>);
};

// default rows per block: keep 128-thread blocks (several blocks per SM)
template <typename T, int N>
struct RowDefault {
  static constexpr int R2 = Split<N>::R2;
  static constexpr int RT = (sizeof(T) == 4 ? 128 : 64) / R2;
};

template <typename T, int N>
__global__ void __launch_bounds__(Col2<T, N>::BLOCK, Col2<T, N>::MIN_BLOCKS) col2_kernel(FineArgs a, int step, int stage) {
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
// The stage update runs from shared memory: after the forward transform the kept
// modes are staged row-major in the (then free) exchange buffer, every thread updates
// consecutive kx of a row (coalesced stage arrays, independent loads), and the new
// stage values are read back in the layout of the inverse transform.
template <typename T, int N, int RT>
__global__ void __launch_bounds__(Row2<T, N, RT>::BLOCK) row2_kernel(FineArgs a, int mode, int store_m) {
  using G = Row2<T, N, RT>;
  constexpr int R1 = G::R1, R2 = G::R2, LROW = G::LROW, BLOCK = G::BLOCK;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* S = (cx<T>*)smem_raw;                    // [3][RT][LROW]
  cx<T>* s_tw = S + 3 * RT * LROW;
  for (int i = threadIdx.x; i < N; i += BLOCK) s_tw[i] = ((const cx<T>*)a.tw)[i];
  const int lane = threadIdx.x % R2;
  const int rr = threadIdx.x / R2;
  const int K = a.K, P = a.P;
  const long total = (long)a.batch * P;
  const long row0 = (long)blockIdx.x * RT;
  const long row = row0 + rr;
  const bool valid = row < total;
  const long b = valid ? row / P : 0;
  const int iy = valid ? (int)(row - b * P) : 0;
  auto slot = [&](int c, int q, int a2) { return S + (c * RT + rr) * LROW + q * (R2 + 1) + a2; };
  // staged kept modes: H(c, r, ix) for row r of the block, ix = kx + K
  auto hslot = [&](int c, int r, int ix) { return S + (c * RT + r) * LROW + ix; };

  cx<T> v[3][R1];
  if (mode == 4) {
    const cx<T>* X = (const cx<T>*)a.X;
    const long sbase = ((b * 3) * P + iy) * (long)P + K;
#pragma unroll
    for (int k = 0; k < R1; ++k) {
      const int xx = lane + R2 * k;
      const int kx = xx < N / 2 ? xx : xx - N;
      const bool keep = valid && kx >= -K && kx <= K;
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c][k] = keep ? X[sbase + c * (long)P * P + kx] : mk(T(0), T(0));
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
    __syncthreads();   // every exchange read is done before the staging writes
    const T inv_n2 = T(1) / (T(N) * T(N));
#pragma unroll
    for (int r = 0; r < R1; ++r) {
      const int xx = lane + FFT2<N>::out_pos_base(r);
      const int kx = xx < N / 2 ? xx : xx - N;
      if (kx >= -K && kx <= K) {
#pragma unroll
        for (int c = 0; c < 3; ++c) *hslot(c, rr, kx + K) = v[c][r] * inv_n2;
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
    for (int k = 0; k < R1; ++k) {
      const int xx = lane + R2 * k;
      const int kx = xx < N / 2 ? xx : xx - N;
      const bool keep = kx >= -K && kx <= K;
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c][k] = keep ? *hslot(c, rr, kx + K) : mk(T(0), T(0));
    }
    __syncthreads();   // staging reads are done before the exchange writes
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
  constexpr int RT = RowDefault<T, N>::RT;
  cudaError_t e = cudaFuncSetAttribute(col2_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Col2<T, N>::smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(row2_kernel<T, N, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Row2<T, N, RT>::smem);
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
  constexpr int RT = RowDefault<T, N>::RT;
  using R = Row2<T, N, RT>;
  const unsigned gc = (unsigned)(((long)a.batch * N + C::XT - 1) / C::XT);
  const unsigned gr = (unsigned)(((long)a.batch * a.P + R::RT - 1) / R::RT);
  int launches = 0;
  if (prologue) {
    row2_kernel<T, N, RT><<<gr, R::BLOCK, R::smem, st>>>(a, 4, 1);
    ++launches;
  }
  for (int s = 0; s < nsteps; ++s) {
    for (int j = 0; j < 4; ++j) {
      if (pr) pr->before(pr->user, 0);
      col2_kernel<T, N><<<gc, C::BLOCK, C::smem, st>>>(a, s, j);
      if (pr) pr->after(pr->user, 0);
      const int store = (s == nsteps - 1 && j == 3) ? (store_last ? 1 : 0) : 1;
      if (pr) pr->before(pr->user, 1);
      row2_kernel<T, N, RT><<<gr, R::BLOCK, R::smem, st>>>(a, j, store);
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
