// Fine-step kernels for grids n <= 256 built on the register-resident four-step FFT
// (kd_fft2.cuh): two kernels per RK443 stage, loads / stores straight between global
// memory and registers, one shared-memory transpose per transform.
//
// column kernel: thread (a, col), col fastest (XT columns per block), so that each
//   global access of a warp touches consecutive x of one ky row.
// row kernel:    thread (r, a), a fastest (RT rows per block), so that each global
//   access touches consecutive x (or kx) of one row.
//
// Every kernel is a template over its tile shape (XT columns or RT rows per block) and,
// for the row kernel, over where the stage update runs (STAGED: the kept modes go
// through shared memory so that consecutive threads update consecutive kx of a row;
// otherwise each thread updates the modes its transform left in its registers).  The
// instantiated shapes are the candidates of the launch-plan autotuner; this header is
// included by the translation units that instantiate them.
#pragma once
#include "kd_fft2.cuh"
#include "kd_fine.h"
#include "kd_stage.cuh"

namespace kd {

// Blocks per SM asked of the compiler: as many as shared memory allows (228 KB per SM,
// 1 KB reserved per block) while keeping at least `min_regs` registers per thread.
constexpr int fit_blocks(int block, size_t smem, int min_regs) {
  const int by_smem = (int)(233472 / (smem + 1024));
  const int by_regs = 65536 / (block * min_regs);
  const int m = by_smem < by_regs ? by_smem : by_regs;
  return m < 1 ? 1 : m;
}

// Candidate tile shapes of the n <= 256 kernels (index 0 is the default plan).
template <typename T, int N>
struct Shapes2 {
  static constexpr int R2 = Split<N>::R2;
  static constexpr int XT0 = sizeof(T) == 4 ? (N <= 64 ? 64 : (N == 128 ? 32 : 16))
                                            : (N <= 64 ? 32 : (N == 128 ? 16 : 8));
  static constexpr int RT0 = (sizeof(T) == 4 ? 128 : 64) / R2;
  static constexpr int xt(int v) { return v == 0 ? XT0 : XT0 / 2; }
  static constexpr int rt(int v) { return (v & 1) == 0 ? RT0 : (RT0 / 2 < 1 ? 1 : RT0 / 2); }
};

template <typename T, int N, int XT_>
struct Col2 {
  static constexpr int R1 = Split<N>::R1, R2 = Split<N>::R2;
  static constexpr int XT = XT_;
  static constexpr int BLOCK = XT * R2;
  static constexpr size_t smem = (size_t)3 * N * XT * sizeof(cx<T>) + N * sizeof(cx<T>) + 2 * N * sizeof(T);
  static constexpr int MIN_BLOCKS = sizeof(T) == 4 ? fit_blocks(BLOCK, smem, 128) : (BLOCK <= 256 ? 2 : 1);
};

// RT rows per block; BLOCK = RT * R2 threads.  The in-register stage update keeps the
// whole row transform live while its loads are in flight, so its variants are given
// more registers per thread (REGS).
template <typename T, int N, int RT_, int REGS = 128>
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
  static constexpr int MIN_BLOCKS = sizeof(T) == 4 ? fit_blocks(BLOCK, smem, REGS) : 1;
};

// Points of the in-register stage update whose loads may be in flight together: a
// compiler fence after every group keeps the loads of later points from being hoisted
// (which would need more registers than the thread has).
constexpr int kUpdateGroup = 4;

template <typename T, int N, int XT>
__global__ void __launch_bounds__(Col2<T, N, XT>::BLOCK, Col2<T, N, XT>::MIN_BLOCKS)
    col2_kernel(FineArgs a, int step, int stage) {
  using G = Col2<T, N, XT>;
  constexpr int R1 = G::R1, R2 = G::R2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* S = (cx<T>*)smem_raw;                    // [3][R1][R2][XT]
  cx<T>* s_tw = S + 3 * N * XT;                   // [N]
  T* s_cos = (T*)(s_tw + N);
  T* s_sin = s_cos + N;
  fft2_tables<T, N>(s_tw, (const cx<T>*)a.tw);
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
  auto slot = [&](int c, int q, int a2) { return S + ((c * R1 + q) * R2 + a2) * XT + col; };

  cx<T> v[3][R1];
  const cx<T>* M = (const cx<T>*)a.M;
  griddep_wait();    // M is the predecessor's output
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
  const T A = flow_amp<T>(a, b);
  const T cxg = s_cos[x], sxg = s_sin[x];
#pragma unroll
  for (int r = 0; r < R1; ++r) {
    const int y = lane + FFT2<N>::out_pos_base(r);
    cross_u<T>(A, ph, cxg, sxg, s_cos[y], s_sin[y], v[0][r], v[1][r], v[2][r]);
  }
  out_to_in<T, N>(v);
  griddep_launch_dependents();
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
// STAGED: after the forward transform the kept modes are staged row-major in the
// (then free) exchange buffer, every thread updates consecutive kx of a row (coalesced
// stage arrays, independent loads), and the new stage values are read back in the
// layout of the inverse transform.  Otherwise the update runs on the registers the
// forward transform left (lanes hold consecutive kx, so the accesses still coalesce).
template <typename T, int N, int RT, bool STAGED, int SCH = SCHEME_RK443>
__global__ void __launch_bounds__(Row2<T, N, RT, STAGED ? 128 : 168>::BLOCK, Row2<T, N, RT, STAGED ? 128 : 168>::MIN_BLOCKS)
    row2_kernel(FineArgs a, int mode, int store_m) {
  using G = Row2<T, N, RT, STAGED ? 128 : 168>;
  constexpr int R1 = G::R1, R2 = G::R2, LROW = G::LROW, BLOCK = G::BLOCK;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* S = (cx<T>*)smem_raw;                    // [3][RT][LROW]
  cx<T>* s_tw = S + 3 * RT * LROW;
  fft2_tables<T, N>(s_tw, (const cx<T>*)a.tw);
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
  griddep_wait();    // W (and, for the prologue, X) come from the predecessors
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
    const T inv_n2 = T(1) / (T(N) * T(N));
    const StageArrays<T> sa = stage_arrays<T>(a);
    if (STAGED) {
      __syncthreads();   // every exchange read is done before the staging writes
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
          stage_update_s<SCH, MODE, T>(stage_coef<T>(a, gb), sa, ((gb * 3) * P + giy) * (long)P + ix, (long)P * P,
                                (T)(ix - K), (T)(giy - K), w0, w1, w2);
          *hslot(0, r, ix) = w0;
          *hslot(1, r, ix) = w1;
          *hslot(2, r, ix) = w2;
        }
      });
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
    } else {
      const StageCoef<T> q = stage_coef<T>(a, b);
      const long s0 = ((b * 3) * P + iy) * (long)P + K;
      const T fky = (T)(iy - K);
      with_stage(mode, [&](auto m) {
        constexpr int MODE = decltype(m)::value;
#pragma unroll
        for (int r = 0; r < R1; ++r) {
          const int xx = lane + FFT2<N>::out_pos_base(r);
          const int kx = xx < N / 2 ? xx : xx - N;
          if (valid && kx >= -K && kx <= K) {
            cx<T> w0 = v[0][r] * inv_n2, w1 = v[1][r] * inv_n2, w2 = v[2][r] * inv_n2;
            stage_update_s<SCH, MODE, T>(q, sa, s0 + kx, (long)P * P, (T)kx, fky, w0, w1, w2);
            v[0][r] = w0;
            v[1][r] = w1;
            v[2][r] = w2;
          } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) v[c][r] = mk(T(0), T(0));
          }
          if (r % kUpdateGroup == kUpdateGroup - 1) asm volatile("" ::: "memory");
        }
      });
      if (!store_m) return;   // uniform over the grid
      out_to_in<T, N>(v);
      __syncthreads();   // exchange reads of the forward transform are done
    }
  }
  griddep_launch_dependents();
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

}  // namespace kd
