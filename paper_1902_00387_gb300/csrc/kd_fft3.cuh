// Register-resident Stockham FFT for N = 512 and 1024 (three passes, radices 16,
// N/256, 16), all three field components at once.  A transform is owned by
// T = N/16 threads ("lane" j); every lane keeps 16 values per component in registers:
//   input  v[k] = x[j + k T]     output  v[q] = X[j + q T]     (k, q < 16)
// so the output of one transform is in place as the input of the next (no exchange
// between the inverse transform, the pointwise step and the forward transform).
// Pass p with radix R and stride Ns: butterfly b reads x[b + k N/R], twiddles by
// w_N^(k (b mod Ns) N/(Ns R)), does an R-point DFT and writes to
// (b / Ns) Ns R + (b mod Ns) + q Ns; the last pass (Ns = N/16) writes to j + q T, which
// stays in registers.  Shared-memory indices are padded by one slot per 16 (pad16) so
// that the stride-16 stores of the first pass spread over the banks.
#pragma once
#include "kd_fft2.cuh"

namespace kd {

__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

template <int N>
struct F3 {
  static constexpr int T = N / 16, RM = N / 256, NB2 = 16 / RM;
  static constexpr int NPAD = N + N / 16;
  // twiddles re-laid for conflict-free reads: pass 3 [k][j] (16 x T), pass 2 [k][b mod 16]
  static constexpr int TWS = N + 16 * RM;
};

// Fill the shared twiddle tables of fft3_3 from tw[e] = exp(-2 pi i e / N).
template <typename T, int N>
__device__ __forceinline__ void fft3_tables(cx<T>* s_tw, const cx<T>* tw) {
  constexpr int TT = F3<N>::T, RM = F3<N>::RM;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int k = i / TT, j = i - k * TT;
    s_tw[i] = tw[k * j];                               // pass 3: w^(k j)
  }
  for (int i = threadIdx.x; i < 16 * RM; i += blockDim.x) {
    const int k = i / 16, bm = i - k * 16;
    s_tw[N + i] = tw[k * bm * (N / (16 * RM))];        // pass 2: w^(k (b mod 16) N / (16 RM))
  }
}

// S(c, i): shared slot of element i (already padded by the caller's layout) of component c;
// tw: the tables written by fft3_tables
template <typename T, int N, int DIR, class Slot>
__device__ __forceinline__ void fft3_3(cx<T> (&v)[3][16], int j, const cx<T>* tw, Slot S) {
  constexpr int TT = F3<N>::T, RM = F3<N>::RM, NB2 = F3<N>::NB2;
  // pass 1: radix 16, Ns = 1 (no twiddles)
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    dft_dif<T, 16, DIR>(v[c]);
#pragma unroll
    for (int q = 0; q < 16; ++q) *S(c, pad16(j * 16 + q)) = v[c][bitrev<16>(q)];
  }
  __syncthreads();
  // pass 2: radix RM, Ns = 16; NB2 butterflies per lane
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int i = 0; i < NB2; ++i) {
      const int b = j + i * TT;
#pragma unroll
      for (int k = 0; k < RM; ++k) v[c][i * RM + k] = *S(c, pad16(b + k * (N / RM)));
    }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NB2; ++i) {
    const int b = j + i * TT;
    const int bm = b & 15;
    cx<T> w[RM];
#pragma unroll
    for (int k = 1; k < RM; ++k) {
      const cx<T> t = tw[N + k * 16 + bm];
      w[k] = DIR < 0 ? t : mk(t.x, -t.y);
    }
    const int idxD = (b >> 4) * 16 * RM + bm;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      cx<T>* vv = &v[c][i * RM];
#pragma unroll
      for (int k = 1; k < RM; ++k) vv[k] = cmul(vv[k], w[k]);
      dft_dif<T, RM, DIR>(vv);
#pragma unroll
      for (int q = 0; q < RM; ++q) *S(c, pad16(idxD + q * 16)) = vv[bitrev<RM>(q)];
    }
  }
  __syncthreads();
  // pass 3: radix 16, Ns = N / 16; outputs stay in registers at j + q T
  cx<T> w[16];
#pragma unroll
  for (int k = 1; k < 16; ++k) {
    const cx<T> t = tw[k * TT + j];
    w[k] = DIR < 0 ? t : mk(t.x, -t.y);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cx<T> u[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) u[k] = *S(c, pad16(j + k * TT));
#pragma unroll
    for (int k = 1; k < 16; ++k) u[k] = cmul(u[k], w[k]);
    dft_dif<T, 16, DIR>(u);
#pragma unroll
    for (int q = 0; q < 16; ++q) v[c][q] = u[bitrev<16>(q)];
  }
}

}  // namespace kd
