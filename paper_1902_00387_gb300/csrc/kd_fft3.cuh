// Register-resident Stockham FFT in three passes of radices (R, N/R^2, R), R = 16
// (N = 512, 1024) or R = 8 (N = 128, 256, 512), all three field components at once.
// A transform is owned by T = N/R threads ("lane" j); every lane keeps R values per
// component in registers:
//   input  v[k] = x[j + k T]     output  v[q] = X[j + q T]     (k, q < R)
// so the output of one transform is in place as the input of the next (no exchange
// between the inverse transform, the pointwise step and the forward transform).
// Pass p with radix Rp and stride Ns: butterfly b reads x[b + k N/Rp], twiddles by
// w_N^(k (b mod Ns) N/(Ns Rp)), does an Rp-point DFT and writes to
// (b / Ns) Ns Rp + (b mod Ns) + q Ns; the last pass (Ns = N/R) writes to j + q T, which
// stays in registers.  Shared-memory indices are padded by one slot per R so that the
// stride-R stores of the first pass spread over the banks.  The packed butterflies of
// dft_dif are used below N = 512 only: the 1024 kernels measured slower with them.
#pragma once
#include "kd_fft2.cuh"

namespace kd {

// Three-pass transform with R = 8 or 16 values per thread (N = R * RM * R, RM = N / R^2):
// T = N / R lanes per transform; shared-memory index i is padded to i + i / R so that the
// stride-R stores of the first pass spread over the banks.
template <int N, int R = 16>
struct F3 {
  static_assert(R == 8 || R == 16, "8 or 16 values per thread");
  static constexpr int T = N / R, RM = N / (R * R), NB2 = R / RM;
  static_assert(RM >= 2 && RM <= R && N == R * RM * R, "N = R x RM x R with 2 <= RM <= R");
  static constexpr int NPAD = N + N / R;
  // twiddles re-laid for conflict-free reads: pass 3 [k][j] (R x T), pass 2 [k][b mod R]
  static constexpr int TWS = N + R * RM;
  __device__ __forceinline__ static int pad(int i) { return i + i / R; }
};

// Fill the shared twiddle tables of fft3_3 / fft3r from tw[e] = exp(-2 pi i e / N).
template <typename T, int N, int R = 16>
__device__ __forceinline__ void fft3_tables(cx<T>* s_tw, const cx<T>* tw) {
  constexpr int TT = F3<N, R>::T, RM = F3<N, R>::RM;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int k = i / TT, j = i - k * TT;
    s_tw[i] = tw[k * j];                               // pass 3: w^(k j)
  }
  for (int i = threadIdx.x; i < R * RM; i += blockDim.x) {
    const int k = i / R, bm = i - k * R;
    s_tw[N + i] = tw[k * bm * (N / (R * RM))];         // pass 2: w^(k (b mod R) N / (R RM))
  }
}

// S(c, i): shared slot of element i (already padded, F3::pad) of component c;
// tw: the tables written by fft3_tables.  Lane j holds v[c][k] = x[j + k T] on input and
// v[c][q] = X[j + q T] on output.  Ends after the last exchange read; the caller
// synchronises before the exchange is written again.
template <typename T, int N, int R, int DIR, class Slot>
__device__ __forceinline__ void fft3r(cx<T> (&v)[3][R], int j, const cx<T>* tw, Slot S) {
  using F = F3<N, R>;
  constexpr int TT = F::T, RM = F::RM, NB2 = F::NB2;
  // pass 1: radix R, Ns = 1 (no twiddles)
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    dft_dif<T, R, DIR, (N < 512)>(v[c]);
#pragma unroll
    for (int q = 0; q < R; ++q) *S(c, F::pad(j * R + q)) = v[c][bitrev<R>(q)];
  }
  __syncthreads();
  // pass 2: radix RM, Ns = R; NB2 butterflies per lane
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int i = 0; i < NB2; ++i) {
      const int b = j + i * TT;
#pragma unroll
      for (int k = 0; k < RM; ++k) v[c][i * RM + k] = *S(c, F::pad(b + k * (N / RM)));
    }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NB2; ++i) {
    const int b = j + i * TT;
    const int bm = b % R;
    cx<T> w[RM];
#pragma unroll
    for (int k = 1; k < RM; ++k) {
      const cx<T> t = tw[N + k * R + bm];
      w[k] = DIR < 0 ? t : mk(t.x, -t.y);
    }
    const int idxD = (b / R) * R * RM + bm;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      cx<T>* vv = &v[c][i * RM];
#pragma unroll
      for (int k = 1; k < RM; ++k) vv[k] = cmul(vv[k], w[k]);
      dft_dif<T, RM, DIR, (N < 512)>(vv);
#pragma unroll
      for (int q = 0; q < RM; ++q) *S(c, F::pad(idxD + q * R)) = vv[bitrev<RM>(q)];
    }
  }
  __syncthreads();
  // pass 3: radix R, Ns = N / R; outputs stay in registers at j + q T
  cx<T> w[R];
#pragma unroll
  for (int k = 1; k < R; ++k) {
    const cx<T> t = tw[k * TT + j];
    w[k] = DIR < 0 ? t : mk(t.x, -t.y);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cx<T> u[R];
#pragma unroll
    for (int k = 0; k < R; ++k) u[k] = *S(c, F::pad(j + k * TT));
#pragma unroll
    for (int k = 1; k < R; ++k) u[k] = cmul(u[k], w[k]);
    dft_dif<T, R, DIR, (N < 512)>(u);
#pragma unroll
    for (int q = 0; q < R; ++q) v[c][q] = u[bitrev<R>(q)];
  }
}

// One-component three-pass transform (the component-split kernels): S(i) is the slot of
// padded index i of this thread's component.
template <typename T, int N, int R, int DIR, class Slot>
__device__ __forceinline__ void fft3r_1(cx<T> (&v)[R], int j, const cx<T>* tw, Slot S) {
  using F = F3<N, R>;
  constexpr int TT = F::T, RM = F::RM, NB2 = F::NB2;
  dft_dif<T, R, DIR, (N < 512)>(v);
#pragma unroll
  for (int q = 0; q < R; ++q) *S(F::pad(j * R + q)) = v[bitrev<R>(q)];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NB2; ++i) {
    const int b = j + i * TT;
#pragma unroll
    for (int k = 0; k < RM; ++k) v[i * RM + k] = *S(F::pad(b + k * (N / RM)));
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NB2; ++i) {
    const int b = j + i * TT;
    const int bm = b % R;
    cx<T>* vv = &v[i * RM];
#pragma unroll
    for (int k = 1; k < RM; ++k) {
      const cx<T> t = tw[N + k * R + bm];
      vv[k] = cmul(vv[k], DIR < 0 ? t : mk(t.x, -t.y));
    }
    dft_dif<T, RM, DIR, (N < 512)>(vv);
    const int idxD = (b / R) * R * RM + bm;
#pragma unroll
    for (int q = 0; q < RM; ++q) *S(F::pad(idxD + q * R)) = vv[bitrev<RM>(q)];
  }
  __syncthreads();
  cx<T> u[R];
#pragma unroll
  for (int k = 0; k < R; ++k) u[k] = *S(F::pad(j + k * TT));
#pragma unroll
  for (int k = 1; k < R; ++k) {
    const cx<T> t = tw[k * TT + j];
    u[k] = cmul(u[k], DIR < 0 ? t : mk(t.x, -t.y));
  }
  dft_dif<T, R, DIR, (N < 512)>(u);
#pragma unroll
  for (int q = 0; q < R; ++q) v[q] = u[bitrev<R>(q)];
}

// The 16-values-per-thread transform of the n = 512, 1024 kernels.
template <typename T, int N, int DIR, class Slot>
__device__ __forceinline__ void fft3_3(cx<T> (&v)[3][16], int j, const cx<T>* tw, Slot S) {
  fft3r<T, N, 16, DIR>(v, j, tw, S);
}

}  // namespace kd
