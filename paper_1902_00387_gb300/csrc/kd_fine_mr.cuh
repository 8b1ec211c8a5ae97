// Fine-step kernels for grid sides n = 32 R, on a mixed-radix FFT owned by one warp: the
// only kernels of the sides that are not powers of two (R = 3, 5, 6: n = 96, 160, 192;
// Table 1's N_F = 160 and the refinement 96 / 128 / 160 of Sec. 5.2), and a launch-plan
// variant of the sides 32, 64, 128, 256 (R = 1, 2, 4, 8).
//
// Transform of N = 32 R points, R values a lane (Cooley-Tukey with factors R and 32):
//   layout A: lane a holds x[a + 32 k], register k < R
//   layout B: lane l holds x[q + R rev(l)], register q < R (rev = 5-bit bit reversal)
// a_to_b: an R-point DFT inside the lane (over k), the twiddle w_N^(a q), then for each q a
//   32-point radix-2 decimation-in-frequency DFT across the lanes (shuffles), which leaves
//   its outputs in bit-reversed lane order;
// b_to_a: the transposed sequence: a 32-point decimation-in-time DFT across the lanes
//   (bit-reversed input, natural output), the twiddle, the R-point DFT inside the lane.
// Both compute X[m] = sum_n x[n] exp(DIR 2 pi i n m / N) (no normalisation).  The inverse
// transforms of the step go A -> B (spectral to physical) and the forward ones B -> A,
// so a pass never re-orders data: the column pass keeps ky in layout A and y in layout B,
// the row pass x in layout B and kx in layout A.  The three field components of a column
// or row live in one warp's registers (3 R complex values a lane), so u x b and the curl
// need no exchange; a warp barrier is never needed (shuffles only).
#pragma once
#include "kd_fft2.cuh"
#include "kd_fine.h"
#include "kd_stage.cuh"

namespace kd {

// (cos, sin)(2 pi m / R) for the in-lane DFTs, m < R.
template <int R>
__device__ __forceinline__ double mr_cos(int m);
template <int R>
__device__ __forceinline__ double mr_sin(int m);
template <>
__device__ __forceinline__ double mr_cos<3>(int m) { return m == 0 ? 1.0 : -0.5; }
template <>
__device__ __forceinline__ double mr_sin<3>(int m) {
  return m == 0 ? 0.0 : (m == 1 ? 0.86602540378443864676 : -0.86602540378443864676);
}
template <>
__device__ __forceinline__ double mr_cos<5>(int m) {
  switch (m) {
    case 0: return 1.0;
    case 1: case 4: return 0.30901699437494742410;
    default: return -0.80901699437494742410;
  }
}
template <>
__device__ __forceinline__ double mr_sin<5>(int m) {
  switch (m) {
    case 0: return 0.0;
    case 1: return 0.95105651629515357212;
    case 2: return 0.58778525229247312917;
    case 3: return -0.58778525229247312917;
    default: return -0.95105651629515357212;
  }
}
template <>
__device__ __forceinline__ double mr_cos<6>(int m) {
  switch (m) {
    case 0: return 1.0;
    case 1: case 5: return 0.5;
    case 2: case 4: return -0.5;
    default: return -1.0;
  }
}
template <>
__device__ __forceinline__ double mr_sin<6>(int m) {
  switch (m) {
    case 0: case 3: return 0.0;
    case 1: case 2: return 0.86602540378443864676;
    default: return -0.86602540378443864676;
  }
}

// In-lane R-point DFT, X[k] = sum_j x[j] exp(DIR 2 pi i j k / R): radix 2 for R = 1, 2,
// 4, 8 (the sides 32, 64, 128, 256), direct for R = 3, 5, 6.
template <typename T, int R, int DIR>
__device__ __forceinline__ void mr_dft(cx<T> (&v)[R]) {
  if constexpr (R == 1) {
    return;
  } else if constexpr ((R & (R - 1)) == 0) {
    dft_dif<T, R, DIR>(v);                         // X[k] at v[bitrev(k)]
    cx<T> t[R];
#pragma unroll
    for (int k = 0; k < R; ++k) t[k] = v[bitrev<R>(k)];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = t[k];
    return;
  }
  cx<T> out[R];
#pragma unroll
  for (int k = 0; k < R; ++k) {
    cx<T> acc = v[0];
#pragma unroll
    for (int j = 1; j < R; ++j) {
      const int m = (j * k) % R;
      const T c = (T)mr_cos<R>(m), s = (T)(DIR * mr_sin<R>(m));
      acc = acc + mk(v[j].x * c - v[j].y * s, v[j].x * s + v[j].y * c);
    }
    out[k] = acc;
  }
#pragma unroll
  for (int k = 0; k < R; ++k) v[k] = out[k];
}

template <typename T>
__device__ __forceinline__ cx<T> shfl_xor(cx<T> v, int m) {
  return mk(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// Per-lane twiddles of a warp transform: wl[i] = w_32^(lane mod h) for the across-lane stage
// of half size h = 16 >> i (w_32 = exp(-2 pi i / 32) composed as exp(-2 pi i (lane mod h) / 2h)),
// wq[q] = w_N^(lane q) (q < R); both for the forward sign, conjugated for the inverse.
template <typename T, int R>
struct MrTw {
  cx<T> wl[5];
  cx<T> wq[R];
};

template <typename T, int R>
__device__ __forceinline__ MrTw<T, R> mr_twiddles(int lane, const cx<T>* tw) {
  constexpr int N = 32 * R;
  MrTw<T, R> t;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int h = 16 >> i;
    const int e = (lane % h) * (N / (2 * h));   // exp(-2 pi i (lane mod h) / 2h) = w_N^e
    t.wl[i] = tw[e];
  }
#pragma unroll
  for (int q = 0; q < R; ++q) t.wq[q] = tw[(lane * q) % N];
  return t;
}

template <typename T, int DIR>
__device__ __forceinline__ cx<T> mr_apply(cx<T> v, cx<T> w) {
  return cmul(v, DIR < 0 ? w : mk(w.x, -w.y));
}

// layout A -> layout B (see above)
template <typename T, int R, int DIR>
__device__ __forceinline__ void mr_a_to_b(cx<T> (&v)[R], int lane, const MrTw<T, R>& t) {
  mr_dft<T, R, DIR>(v);
#pragma unroll
  for (int q = 1; q < R; ++q) v[q] = mr_apply<T, DIR>(v[q], t.wq[q]);
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int h = 16 >> i;
    const bool up = (lane & h) != 0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const cx<T> p = shfl_xor(v[q], h);
      v[q] = up ? mr_apply<T, DIR>(p - v[q], t.wl[i]) : v[q] + p;
    }
  }
}

// layout B -> layout A
template <typename T, int R, int DIR>
__device__ __forceinline__ void mr_b_to_a(cx<T> (&v)[R], int lane, const MrTw<T, R>& t) {
#pragma unroll
  for (int i = 4; i >= 0; --i) {
    const int h = 16 >> i;
    const bool up = (lane & h) != 0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const cx<T> own = up ? mr_apply<T, DIR>(v[q], t.wl[i]) : v[q];
      const cx<T> p = shfl_xor(own, h);
      v[q] = up ? p - own : own + p;
    }
  }
#pragma unroll
  for (int q = 1; q < R; ++q) v[q] = mr_apply<T, DIR>(v[q], t.wq[q]);
  mr_dft<T, R, DIR>(v);
}

__device__ __forceinline__ int mr_rev5(int l) { return __brev((unsigned)l) >> 27; }

constexpr int kMrWarps = 4;   // warps (columns or rows) per block

// Column pass of one RK stage: M (kept ky rows) -> inverse FFT in y -> u x b -> forward
// FFT in y -> kept ky rows -> W.  One warp per grid column.
template <typename T, int R>
__global__ void __launch_bounds__(32 * kMrWarps) colmr_kernel(FineArgs a, int step, int stage) {
  constexpr int N = 32 * R;
  const int lane = threadIdx.x & 31;
  const long col = (long)blockIdx.x * kMrWarps + (threadIdx.x >> 5);
  const MrTw<T, R> tw = mr_twiddles<T, R>(lane, (const cx<T>*)a.tw);
  const T* cosg = (const T*)a.cosg;
  const T* sing = (const T*)a.sing;
  griddep_wait();    // M is the predecessor's output
  if (col >= (long)a.batch * N) return;
  const long b = col / N;
  const int x = (int)(col - b * N);
  const int K = a.K, P = a.P;
  const cx<T>* M = (const cx<T>*)a.M;
  cx<T> v[3][R];
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int yy = lane + 32 * k;
    const int ky = yy < N / 2 ? yy : yy - N;
    const bool keep = ky >= -K && ky <= K;
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c][k] = keep ? M[((b * 3 + c) * P + ky + K) * (long)N + x] : mk(T(0), T(0));
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) mr_a_to_b<T, R, +1>(v[c], lane, tw);   // ky -> y (layout B)
  const Phase<T> ph = load_phase<T>(a, b, step, stage);
  const T A = flow_amp<T>(a, b);
  const int rl = mr_rev5(lane);
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int y = q + R * rl;
    cross_u<T>(A, ph, cosg[x], sing[x], cosg[y], sing[y], v[0][q], v[1][q], v[2][q]);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) mr_b_to_a<T, R, -1>(v[c], lane, tw);   // y -> ky (layout A)
  cx<T>* W = (cx<T>*)a.W;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int yy = lane + 32 * k;
    const int ky = yy < N / 2 ? yy : yy - N;
    if (ky >= -K && ky <= K) {
#pragma unroll
      for (int c = 0; c < 3; ++c) W[((b * 3 + c) * P + ky + K) * (long)N + x] = v[c][k];
    }
  }
}

// Row pass (MODE 0..3 stage update, 4 = prologue: inverse x transform of X): W row (x in
// layout B) -> forward FFT in x -> kept kx (layout A) -> curl, stage update -> inverse FFT
// in x -> M.  One warp per ky row.
template <typename T, int R, int SCH, int MODE>
__global__ void __launch_bounds__(32 * kMrWarps) rowmr_kernel(FineArgs a, int store_m) {
  constexpr int N = 32 * R;
  const int lane = threadIdx.x & 31;
  const long row = (long)blockIdx.x * kMrWarps + (threadIdx.x >> 5);
  const MrTw<T, R> tw = mr_twiddles<T, R>(lane, (const cx<T>*)a.tw);
  griddep_wait();    // W (and the stage arrays) come from the predecessors
  const int K = a.K, P = a.P;
  if (row >= (long)a.batch * P) return;
  const long b = row / P;
  const int iy = (int)(row - b * P);
  const int rl = mr_rev5(lane);
  StageArrays<T> sa = stage_arrays<T>(a);
  const long s0 = ((b * 3) * P + iy) * (long)P + K;   // compact index of (iy, kx = 0), component 0
  cx<T> v[3][R];
  if constexpr (MODE == 4) {
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int xx = lane + 32 * k;
      const int kx = xx < N / 2 ? xx : xx - N;
      const bool keep = kx >= -K && kx <= K;
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c][k] = keep ? sa.X[s0 + c * (long)P * P + kx] : mk(T(0), T(0));
    }
  } else {
    const cx<T>* W = (const cx<T>*)a.W;
#pragma unroll
    for (int q = 0; q < R; ++q)
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c][q] = W[((b * 3 + c) * P + iy) * (long)N + q + R * rl];
#pragma unroll
    for (int c = 0; c < 3; ++c) mr_b_to_a<T, R, -1>(v[c], lane, tw);   // x -> kx (layout A)
    const StageCoef<T> sc = stage_coef<T>(a, b);
    const T inv_n2 = T(1) / (T(N) * T(N));
    const T fky = (T)(iy - K);
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int xx = lane + 32 * k;
      const int kx = xx < N / 2 ? xx : xx - N;
      if (kx >= -K && kx <= K) {
        cx<T> w0 = v[0][k] * inv_n2, w1 = v[1][k] * inv_n2, w2 = v[2][k] * inv_n2;
        stage_update_s<SCH, MODE, T>(sc, sa, s0 + kx, (long)P * P, (T)kx, fky, w0, w1, w2);
        v[0][k] = w0;
        v[1][k] = w1;
        v[2][k] = w2;
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c][k] = mk(T(0), T(0));
      }
    }
    if (!store_m) return;   // uniform over the grid
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) mr_a_to_b<T, R, +1>(v[c], lane, tw);   // kx -> x (layout B)
  cx<T>* Mo = (cx<T>*)a.M;
#pragma unroll
  for (int q = 0; q < R; ++q)
#pragma unroll
    for (int c = 0; c < 3; ++c) Mo[((b * 3 + c) * P + iy) * (long)N + q + R * rl] = v[c][q];
}

}  // namespace kd
