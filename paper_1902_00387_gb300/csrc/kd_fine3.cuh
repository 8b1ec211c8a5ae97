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

template <typename T, int N, int XT_, int R = 16>
struct Col3 {
  static constexpr int TPT = F3<N, R>::T;
  static constexpr int XT = XT_;                   // columns per block
  static constexpr int BLOCK = XT * TPT;
  static constexpr int NPAD = F3<N, R>::NPAD;
  static constexpr size_t smem =
      (size_t)3 * NPAD * XT * sizeof(cx<T>) + F3<N, R>::TWS * sizeof(cx<T>) + 2 * N * sizeof(T);
  static constexpr int MIN_BLOCKS = sizeof(T) == 4 ? fit_blocks(BLOCK, smem, 128) : 1;
};

template <typename T, int N, int RT_, int REGS = 128, int R = 16>
struct Row3 {
  static constexpr int TPT = F3<N, R>::T;
  static constexpr int RT = RT_;                   // rows per block
  static constexpr int BLOCK = RT * TPT;
  static constexpr int LROW0 = F3<N, R>::NPAD;
  static constexpr int LROW = LROW0 + ((8 - LROW0 % 16) + 16) % 16;
  static constexpr size_t smem = (size_t)3 * RT * LROW * sizeof(cx<T>) + F3<N, R>::TWS * sizeof(cx<T>);
  static constexpr int MIN_BLOCKS = sizeof(T) == 4 ? fit_blocks(BLOCK, smem, REGS) : 1;
};

template <typename T, int N, int XT, int R>
__global__ void __launch_bounds__(Col3<T, N, XT, R>::BLOCK, Col3<T, N, XT, R>::MIN_BLOCKS)
    col3_kernel(FineArgs a, int step, int stage) {
  using G = Col3<T, N, XT, R>;
  constexpr int TT = G::TPT, NPAD = G::NPAD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* S = (cx<T>*)smem_raw;                    // [3][NPAD][XT]
  cx<T>* s_tw = S + 3 * NPAD * XT;
  T* s_cos = (T*)(s_tw + F3<N, R>::TWS);
  T* s_sin = s_cos + N;
  fft3_tables<T, N, R>(s_tw, (const cx<T>*)a.tw);
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

  cx<T> v[3][R];
  const cx<T>* M = (const cx<T>*)a.M;
  griddep_wait();    // M is the predecessor's output
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int yy = lane + TT * k;
    const int ky = yy < N / 2 ? yy : yy - N;
    const bool keep = valid && ky >= -K && ky <= K;
#pragma unroll
    for (int c = 0; c < 3; ++c)
      v[c][k] = keep ? M[((b * 3 + c) * P + (ky + K)) * (long)N + x] : mk(T(0), T(0));
  }
  __syncthreads();   // tables
  fft3r<T, N, R, +1>(v, lane, s_tw, slot);           // ky -> y

  const Phase<T> ph = load_phase<T>(a, b, step, stage);
  const T A = flow_amp<T>(a, b);
  const T cxg = s_cos[x], sxg = s_sin[x];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int y = lane + TT * q;
    cross_u<T>(A, ph, cxg, sxg, s_cos[y], s_sin[y], v[0][q], v[1][q], v[2][q]);
  }
  griddep_launch_dependents();
  __syncthreads();   // exchange buffer is reused
  fft3r<T, N, R, -1>(v, lane, s_tw, slot);           // y -> ky

  if (!valid) return;
  cx<T>* W = (cx<T>*)a.W;
#pragma unroll
  for (int q = 0; q < R; ++q) {
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
template <typename T, int N, int RT, bool STAGED, int R, int SCH = SCHEME_RK443>
__global__ void __launch_bounds__(Row3<T, N, RT, STAGED ? 128 : 168, R>::BLOCK,
                                  Row3<T, N, RT, STAGED ? 128 : 168, R>::MIN_BLOCKS)
    row3_kernel(FineArgs a, int mode, int store_m) {
  using G = Row3<T, N, RT, STAGED ? 128 : 168, R>;
  constexpr int TT = G::TPT, LROW = G::LROW, BLOCK = G::BLOCK;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* S = (cx<T>*)smem_raw;                    // [3][RT][LROW]
  cx<T>* s_tw = S + 3 * RT * LROW;
  fft3_tables<T, N, R>(s_tw, (const cx<T>*)a.tw);
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

  cx<T> v[3][R];
  griddep_wait();    // W (and, for the prologue, X) come from the predecessors
  if (mode == 4) {
    const cx<T>* X = (const cx<T>*)a.X;
    const long sbase = ((b * 3) * P + iy) * (long)P + K;
#pragma unroll
    for (int k = 0; k < R; ++k) {
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
    for (int k = 0; k < R; ++k) {
      const int xx = lane + TT * k;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        v[c][k] = valid ? W[((b * 3 + c) * P + iy) * (long)N + xx] : mk(T(0), T(0));
    }
    __syncthreads();
    fft3r<T, N, R, -1>(v, lane, s_tw, slot);         // x -> kx
    const T inv_n2 = T(1) / (T(N) * T(N));
    const StageArrays<T> sa = stage_arrays<T>(a);
    if (STAGED) {
      __syncthreads();   // every exchange read is done before the staging writes
#pragma unroll
      for (int q = 0; q < R; ++q) {
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
      for (int k = 0; k < R; ++k) {
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
        for (int q = 0; q < R; ++q) {
          const int xx = lane + TT * q;
          const int kx = xx < N / 2 ? xx : xx - N;
          if (valid && kx >= -K && kx <= K) {
            cx<T> w0 = v[0][q] * inv_n2, w1 = v[1][q] * inv_n2, w2 = v[2][q] * inv_n2;
            stage_update_s<SCH, MODE, T>(sc, sa, s0 + kx, (long)P * P, (T)kx, fky, w0, w1, w2);
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
  griddep_launch_dependents();
  fft3r<T, N, R, +1>(v, lane, s_tw, slot);           // kx -> x
  if (!valid) return;
  cx<T>* Mo = (cx<T>*)a.M;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int xx = lane + TT * q;
#pragma unroll
    for (int c = 0; c < 3; ++c) Mo[((b * 3 + c) * P + iy) * (long)N + xx] = v[c][q];
  }
}


// ---------------------------------------------------------------------------------
// Persistent variants: one block per SM loops over tiles and copies the next tile's
// input into shared memory with cp.async while it transforms the current one, so the
// global-memory latency of the loads overlaps the FFT work (the register-resident
// transforms leave room for only 8-16 warps per SM, too few to hide it otherwise).

// 16-byte asynchronous global -> shared copy; `valid` false fills the 16 bytes with zeros.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int sz = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename T, int N, int XT_>
struct Col3P {
  static constexpr int TPT = F3<N>::T, XT = XT_, BLOCK = XT * TPT;
  static constexpr int NPAD = F3<N>::NPAD;
  static constexpr int P = 2 * (N / 3) + 1;
  static constexpr int CPC = 16 / sizeof(cx<T>);   // complex values per 16-byte copy
  static constexpr size_t smem = (size_t)3 * NPAD * XT * sizeof(cx<T>) + F3<N>::TWS * sizeof(cx<T>) +
                                 2 * N * sizeof(T) + (size_t)3 * P * XT * sizeof(cx<T>);
};

template <typename T, int N, int XT>
__global__ void __launch_bounds__(Col3P<T, N, XT>::BLOCK, 1) col3p_kernel(FineArgs a, int step, int stage) {
  using G = Col3P<T, N, XT>;
  constexpr int TT = G::TPT, NPAD = G::NPAD, P = G::P, CPC = G::CPC, BLOCK = G::BLOCK;
  constexpr int K = N / 3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* S = (cx<T>*)smem_raw;                    // [3][NPAD][XT] exchange
  cx<T>* s_tw = S + 3 * NPAD * XT;
  T* s_cos = (T*)(s_tw + F3<N>::TWS);
  T* s_sin = s_cos + N;
  cx<T>* Bf = (cx<T>*)(s_sin + N);                // [3][P][XT] prefetched kept rows of the tile
  fft3_tables<T, N>(s_tw, (const cx<T>*)a.tw);
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    s_cos[i] = ((const T*)a.cosg)[i];
    s_sin[i] = ((const T*)a.sing)[i];
  }
  const int col = threadIdx.x % XT;
  const int lane = threadIdx.x / XT;
  const long ntiles = (long)a.batch * N / XT;     // XT divides N: a tile never spans two fields
  const cx<T>* M = (const cx<T>*)a.M;
  cx<T>* W = (cx<T>*)a.W;
  auto slot = [&](int c, int pi) { return S + ((long)c * NPAD + pi) * XT + col; };
  auto prefetch = [&](long tile) {
    const long g0 = tile * XT;
    const long b = g0 / N;
    const int x0 = (int)(g0 - b * N);
    for (int i = threadIdx.x; i < 3 * P * (XT / CPC); i += BLOCK) {
      const int ch = i % (XT / CPC), r = i / (XT / CPC);
      const int c = r / P, iy = r - c * P;
      cp_async16(Bf + ((long)c * P + iy) * XT + ch * CPC, M + ((b * 3 + c) * P + iy) * (long)N + x0 + ch * CPC, true);
    }
    cp_async_commit();
  };
  griddep_wait();    // M is the predecessor's output
  if ((long)blockIdx.x < ntiles) prefetch(blockIdx.x);
  for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    cp_async_wait_all();
    __syncthreads();   // the tile's rows (and, first time, the tables) are visible
    const long g = tile * XT + col;
    const long b = g / N;
    const int x = (int)(g - b * N);
    cx<T> v[3][16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int yy = lane + TT * k;
      const int ky = yy < N / 2 ? yy : yy - N;
      const bool keep = ky >= -K && ky <= K;
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c][k] = keep ? Bf[((long)c * P + (ky + K)) * XT + col] : mk(T(0), T(0));
    }
    __syncthreads();   // Bf is free for the next tile
    if (tile + gridDim.x < ntiles) prefetch(tile + gridDim.x);
    fft3_3<T, N, +1>(v, lane, s_tw, slot);         // ky -> y
    const Phase<T> ph = load_phase<T>(a, b, step, stage);
    const T A = flow_amp<T>(a, b);
    const T cxg = s_cos[x], sxg = s_sin[x];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int y = lane + TT * q;
      cross_u<T>(A, ph, cxg, sxg, s_cos[y], s_sin[y], v[0][q], v[1][q], v[2][q]);
    }
    __syncthreads();   // exchange buffer is reused
    fft3_3<T, N, -1>(v, lane, s_tw, slot);         // y -> ky
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
  cp_async_wait_all();
}

template <typename T, int N, int RT_>
struct Row3P {
  static constexpr int TPT = F3<N>::T, RT = RT_, BLOCK = RT * TPT;
  static constexpr int LROW0 = F3<N>::NPAD;
  static constexpr int LROW = LROW0 + ((8 - LROW0 % 16) + 16) % 16;
  static constexpr int CPC = 16 / sizeof(cx<T>);
  static constexpr size_t smem = (size_t)3 * RT * LROW * sizeof(cx<T>) + F3<N>::TWS * sizeof(cx<T>) +
                                 (size_t)RT * 3 * N * sizeof(cx<T>);
};

// Stage update (mode 0..3) only; the prologue (mode 4) uses row3_kernel.
template <typename T, int N, int RT>
__global__ void __launch_bounds__(Row3P<T, N, RT>::BLOCK, 1) row3p_kernel(FineArgs a, int mode, int store_m) {
  using G = Row3P<T, N, RT>;
  constexpr int TT = G::TPT, LROW = G::LROW, CPC = G::CPC, BLOCK = G::BLOCK;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* S = (cx<T>*)smem_raw;                    // [3][RT][LROW] exchange
  cx<T>* s_tw = S + 3 * RT * LROW;
  cx<T>* Bf = s_tw + F3<N>::TWS;                  // [RT][3][N] prefetched W rows of the tile
  fft3_tables<T, N>(s_tw, (const cx<T>*)a.tw);
  const int lane = threadIdx.x % TT;
  const int rr = threadIdx.x / TT;
  const int K = a.K, P = a.P;
  const long total = (long)a.batch * P;
  const long ntiles = (total + RT - 1) / RT;
  const cx<T>* W = (const cx<T>*)a.W;
  cx<T>* Mo = (cx<T>*)a.M;
  auto slot = [&](int c, int pi) { return S + (c * RT + rr) * LROW + pi; };
  auto prefetch = [&](long tile) {
    for (int i = threadIdx.x; i < RT * 3 * (N / CPC); i += BLOCK) {
      const int ch = i % (N / CPC), rc = i / (N / CPC);
      const int r = rc / 3, c = rc - r * 3;
      const long row = tile * RT + r;
      const bool ok = row < total;
      const long b = ok ? row / P : 0;
      const int iy = ok ? (int)(row - b * P) : 0;
      cp_async16(Bf + ((long)r * 3 + c) * N + ch * CPC, W + ((b * 3 + c) * P + iy) * (long)N + ch * CPC, ok);
    }
    cp_async_commit();
  };
  const StageArrays<T> sa = stage_arrays<T>(a);
  const T inv_n2 = T(1) / (T(N) * T(N));
  griddep_wait();    // W is the predecessor's output
  if ((long)blockIdx.x < ntiles) prefetch(blockIdx.x);
  for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    cp_async_wait_all();
    __syncthreads();
    const long row = tile * RT + rr;
    const bool valid = row < total;
    const long b = valid ? row / P : 0;
    const int iy = valid ? (int)(row - b * P) : 0;
    cx<T> v[3][16];
#pragma unroll
    for (int k = 0; k < 16; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c][k] = Bf[((long)rr * 3 + c) * N + lane + TT * k];
    __syncthreads();   // Bf is free for the next tile
    if (tile + gridDim.x < ntiles) prefetch(tile + gridDim.x);
    fft3_3<T, N, -1>(v, lane, s_tw, slot);         // x -> kx
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
    if (!store_m) continue;   // uniform over the grid
    __syncthreads();          // exchange reads of the forward transform are done
    fft3_3<T, N, +1>(v, lane, s_tw, slot);         // kx -> x
    if (valid) {
#pragma unroll
      for (int q = 0; q < 16; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) Mo[((b * 3 + c) * P + iy) * (long)N + lane + TT * q] = v[c][q];
    }
  }
  cp_async_wait_all();
}

// blocks of a persistent launch: one per SM
inline unsigned persistent_grid(long tiles) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 132;
  }
  return (unsigned)(tiles < sms ? (tiles < 1 ? 1 : tiles) : sms);
}

}  // namespace kd
