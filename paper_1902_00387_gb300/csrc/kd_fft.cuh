// Batched complex FFT of power-of-two length N in shared memory, all three field
// components at once.  Stockham auto-sort formulation (no bit reversal): pass p with
// radix R and stride Ns reads x[j + k N/R], twiddles by w_N^(k (j mod Ns) N/(Ns R)),
// does an R-point DFT in registers and writes to (j / Ns) Ns R + (j mod Ns) + q Ns.
// Radix-8 passes first, then one radix-2 or radix-4 pass for the remaining bits.
//
// Each transform is owned by TPT = N / 8 consecutive threads ("lanes"); every lane
// holds 8 values per component per pass.  All threads of the block must call the
// pass functions (they contain __syncthreads).
#pragma once
#include "kd_common.cuh"

namespace kd {

// R-point DFT in registers; DIR = -1 forward (exp(-i ...)), +1 inverse.
template <typename T, int DIR>
__device__ __forceinline__ void dft2(cx<T>& a, cx<T>& b) {
  cx<T> t = a - b;
  a = a + b;
  b = t;
}

// multiply by (-i)^{DIR<0} / (+i)^{DIR>0}: w_4 = exp(DIR * 2 pi i / 4)
template <typename T, int DIR>
__device__ __forceinline__ cx<T> rot4(cx<T> a) {
  return DIR < 0 ? mk(a.y, -a.x) : mk(-a.y, a.x);
}

template <typename T, int DIR>
__device__ __forceinline__ void dft4(cx<T>& a0, cx<T>& a1, cx<T>& a2, cx<T>& a3) {
  cx<T> t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3, t3 = rot4<T, DIR>(a1 - a3);
  a0 = t0 + t2;
  a2 = t0 - t2;
  a1 = t1 + t3;
  a3 = t1 - t3;
}

template <typename T, int DIR>
__device__ __forceinline__ void dft8(cx<T>* v) {
  // even / odd split: E = DFT4(v0, v2, v4, v6), O = DFT4(v1, v3, v5, v7)
  cx<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  cx<T> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<T, DIR>(e0, e1, e2, e3);
  dft4<T, DIR>(o0, o1, o2, o3);
  const T h = T(0.70710678118654752440);
  // w_8^q = exp(DIR * 2 pi i q / 8)
  cx<T> w1o = DIR < 0 ? mk(h * (o1.x + o1.y), h * (o1.y - o1.x)) : mk(h * (o1.x - o1.y), h * (o1.y + o1.x));
  cx<T> w2o = rot4<T, DIR>(o2);
  cx<T> w3o = DIR < 0 ? mk(h * (-o3.x + o3.y), h * (-o3.y - o3.x)) : mk(h * (-o3.x - o3.y), h * (-o3.y + o3.x));
  v[0] = e0 + o0;
  v[4] = e0 - o0;
  v[1] = e1 + w1o;
  v[5] = e1 - w1o;
  v[2] = e2 + w2o;
  v[6] = e2 - w2o;
  v[3] = e3 + w3o;
  v[7] = e3 - w3o;
}

template <typename T, int R, int DIR>
__device__ __forceinline__ void dftR(cx<T>* v) {
  if constexpr (R == 2) {
    dft2<T, DIR>(v[0], v[1]);
  } else if constexpr (R == 4) {
    dft4<T, DIR>(v[0], v[1], v[2], v[3]);
  } else {
    dft8<T, DIR>(v);
  }
}

// One Stockham pass over all transforms of the block.
//   buf     : shared memory, component c of transform t at buf + c * cstride + t * tstride
//   tw      : shared twiddles tw[e] = exp(-2 pi i e / N), e in [0, N)
template <typename T, int N, int DIR, int NS, int R>
__device__ __forceinline__ void fft_pass(cx<T>* buf, int cstride, int lane, const cx<T>* tw) {
  constexpr int TPT = N / 8;
  constexpr int NB = 8 / R;  // butterflies per lane in this pass
  cx<T> v[3][8];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int j = lane + i * TPT;
#pragma unroll
      for (int k = 0; k < R; ++k) v[c][i * R + k] = buf[c * cstride + j + k * (N / R)];
    }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int j = lane + i * TPT;
    const int jm = j % NS;
    cx<T> w[8];
    if constexpr (NS > 1) {
#pragma unroll
      for (int k = 1; k < R; ++k) {
        cx<T> t = tw[k * jm * (N / (NS * R))];
        w[k] = DIR < 0 ? t : mk(t.x, -t.y);
      }
    }
    const int idxD = (j / NS) * NS * R + jm;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      cx<T>* vv = &v[c][i * R];
      if constexpr (NS > 1) {
#pragma unroll
        for (int k = 1; k < R; ++k) vv[k] = cmul(vv[k], w[k]);
      }
      dftR<T, R, DIR>(vv);
#pragma unroll
      for (int k = 0; k < R; ++k) buf[c * cstride + idxD + k * NS] = vv[k];
    }
  }
  __syncthreads();
}

template <typename T, int N, int DIR, int NS>
__device__ __forceinline__ void fft_passes(cx<T>* buf, int cstride, int lane, const cx<T>* tw) {
  if constexpr (NS < N) {
    constexpr int R = (N / NS >= 8) ? 8 : (N / NS);
    fft_pass<T, N, DIR, NS, R>(buf, cstride, lane, tw);
    fft_passes<T, N, DIR, NS * R>(buf, cstride, lane, tw);
  }
}

// Unnormalised length-N transforms of the 3 components of every transform in the
// block: out[q] = sum_k in[k] exp(DIR * 2 pi i k q / N).  `buf` points at this
// thread's transform (component 0); the result replaces the input.
template <typename T, int N, int DIR>
__device__ __forceinline__ void fft3(cx<T>* buf, int cstride, int lane, const cx<T>* tw) {
  fft_passes<T, N, DIR, 1>(buf, cstride, lane, tw);
}

}  // namespace kd
