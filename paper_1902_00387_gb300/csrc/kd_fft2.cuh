// Register-resident complex FFT of length N = R1 * R2 (N <= 256) with one shared-memory
// transpose (the "four-step" factorisation):
//   n = a + R2 k (a < R2, k < R1),  m = q + R1 p (q < R1, p < R2)
//   X[q + R1 p] = sum_a w_R2^{a p} [ w_N^{a q} sum_k x[a + R2 k] w_R1^{k q} ]
// A transform is owned by R2 threads ("lane" a).  Pass 1: lane a does the R1-point DFT
// over k of its own R1 values and the twiddle w_N^{a q}; the R1 x R2 matrix goes
// through shared memory; pass 2: lane a does the R2-point DFTs for q = a + R2 j.
//
// Register contract (v[r], r < R1):
//   input  v[k]           = x[a + R2 k]
//   output v[j * R2 + p]  = X[(a + R2 j) + R1 p]      (j < R1 / R2, p < R2)
// Since (a + R2 j) + R1 p = a + R2 (j + (R1 / R2) p), the output of one transform holds
// exactly the inputs another transform needs in the same lane, after the compile-time
// register permutation in_from_out().  The three field components are transformed
// together so that a pass needs one barrier.
#pragma once
#include "kd_common.cuh"

namespace kd {

template <int N>
struct Split;
template <>
struct Split<16> { static constexpr int R1 = 4, R2 = 4; };
template <>
struct Split<32> { static constexpr int R1 = 8, R2 = 4; };
template <>
struct Split<64> { static constexpr int R1 = 8, R2 = 8; };
template <>
struct Split<128> { static constexpr int R1 = 16, R2 = 8; };
template <>
struct Split<256> { static constexpr int R1 = 16, R2 = 16; };

// cos / sin (e pi / 16), e = 0..8
__device__ __forceinline__ double cpi16(int e) {
  switch (e) {
    case 0: return 1.0;
    case 1: return 0.98078528040323044913;
    case 2: return 0.92387953251128675613;
    case 3: return 0.83146961230254523708;
    case 4: return 0.70710678118654752440;
    case 5: return 0.55557023301960222474;
    case 6: return 0.38268343236508977173;
    case 7: return 0.19509032201612826785;
    default: return 0.0;
  }
}

// a * w_32^e with w_32 = exp(DIR 2 pi i / 32), 0 <= e < 16 (e is a compile-time
// constant after unrolling, so the branches fold away).
template <typename T, int DIR>
__device__ __forceinline__ cx<T> mul_w32(cx<T> a, int e) {
  if (e == 0) return a;
  if (e == 8) return DIR < 0 ? mk(a.y, -a.x) : mk(-a.y, a.x);
  const T c = (T)(e <= 8 ? cpi16(e) : -cpi16(16 - e));
  const T s = (T)(DIR * (e <= 8 ? cpi16(8 - e) : cpi16(e - 8)));
  return mk(a.x * c - a.y * s, a.x * s + a.y * c);
}

// cos(e pi / 16) for any integer e (folded into the range of cpi16)
__device__ __forceinline__ double c16(int e) {
  e &= 31;
  if (e > 16) e = 32 - e;
  return e <= 8 ? cpi16(e) : -cpi16(16 - e);
}

// a * w_32^e for any integer e (compile-time after unrolling): multiples of 8 are the
// quarter turns (no multiply), the rest one complex product with constant factors.
template <typename T, int DIR>
__device__ __forceinline__ cx<T> mul_w32_any(cx<T> a, int e) {
  e &= 31;
  if (e == 0) return a;
  if (e == 8) return DIR < 0 ? mk(a.y, -a.x) : mk(-a.y, a.x);     // times DIR i
  if (e == 16) return mk(-a.x, -a.y);
  if (e == 24) return DIR < 0 ? mk(-a.y, a.x) : mk(a.y, -a.x);    // times -DIR i
  const T c = (T)c16(e), s = (T)(DIR * c16(8 - e));
  return mk(a.x * c - a.y * s, a.x * s + a.y * c);
}

template <int R>
__host__ __device__ constexpr int bitrev(int q) {
  int r = 0;
  for (int b = 1; b < R; b <<= 1) {
    r = (r << 1) | (q & 1);
    q >>= 1;
  }
  return r;
}

// Butterfly: (a, b) <- (a + b, a - b).  For float both components go through one packed
// FP32x2 instruction each (sm_100 and later): the sum as a packed add, the difference as
// a packed a + (-1) b, whose product is exact, so both round once, as two scalar adds do.
template <typename T>
__device__ __forceinline__ void bfly(cx<T>& a, cx<T>& b) {
  const cx<T> x0 = a, x1 = b;
  a = x0 + x1;
  b = x0 - x1;
}
template <>
__device__ __forceinline__ void bfly<float>(cx<float>& a, cx<float>& b) {
  const float2 x0 = make_float2(a.x, a.y), x1 = make_float2(b.x, b.y);
  const float2 s = __fadd2_rn(x0, x1);
  const float2 d = __ffma2_rn(x1, make_float2(-1.f, -1.f), x0);
  a = mk(s.x, s.y);
  b = mk(d.x, d.y);
}

// Radix-2^2 decimation in frequency on the block v[O .. O + L) (L a power of two <= 32):
// the data flow and output order of radix-2, with the non-trivial twiddles of two
// stages applied once after the second.  With d = the block's upper-half differences,
// the second stage's lower half combines d[i] and d[i + L/4] times w_4 (a quarter turn),
// and the four quarter blocks then carry the twiddles w_L^(r' i), r' = 0, 2, 1, 3 (the
// output residue mod 4 that each quarter block computes, in bit-reversed order).  32
// points: 28 twiddle products instead of radix-2's 34; 16 points: 8 instead of 10.
template <typename T, int DIR, int L, int O>
__device__ __forceinline__ void dft_r22(cx<T>* v) {
  if constexpr (L == 2) {
    bfly(v[O], v[O + 1]);
  } else if constexpr (L >= 4) {
    constexpr int H = L / 2, Q = L / 4, U = 32 / L;   // w_L = w_32^U
#pragma unroll
    for (int i = 0; i < H; ++i) bfly(v[O + i], v[O + i + H]);
#pragma unroll
    for (int i = 0; i < Q; ++i) v[O + H + Q + i] = mul_w32_any<T, DIR>(v[O + H + Q + i], 8);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      bfly(v[O + i], v[O + i + Q]);
      bfly(v[O + H + i], v[O + H + i + Q]);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      v[O + Q + i] = mul_w32_any<T, DIR>(v[O + Q + i], 2 * i * U);
      v[O + H + i] = mul_w32_any<T, DIR>(v[O + H + i], i * U);
      v[O + H + Q + i] = mul_w32_any<T, DIR>(v[O + H + Q + i], 3 * i * U);
    }
    dft_r22<T, DIR, Q, O>(v);
    dft_r22<T, DIR, Q, O + Q>(v);
    dft_r22<T, DIR, Q, O + H>(v);
    dft_r22<T, DIR, Q, O + H + Q>(v);
  }
}

// In-register R-point DFT (R = 2, 4, 8, 16, 32), decimation in frequency: radix-2 up to 8
// points, radix-2^2 (dft_r22, same output order) at 16 and 32.
// In: v[n] natural order.  Out: X[q] at v[bitrev<R>(q)].  PACKED selects the packed
// butterflies of bfly in the radix-2 loop (same results).
template <typename T, int R, int DIR, bool PACKED = true>
__device__ __forceinline__ void dft_dif(cx<T>* v) {
  if constexpr (R >= 16) {
    dft_r22<T, DIR, R, 0>(v);
    return;
  }
#pragma unroll
  for (int span = R / 2; span >= 1; span >>= 1) {
#pragma unroll
    for (int start = 0; start < R; start += 2 * span) {
#pragma unroll
      for (int i = 0; i < span; ++i) {
        cx<T> x0 = v[start + i], x1 = v[start + i + span];
        if (PACKED) {
          bfly(x0, x1);
        } else {
          const cx<T> a = x0;
          x0 = a + x1;
          x1 = a - x1;
        }
        v[start + i] = x0;
        v[start + i + span] = mul_w32<T, DIR>(x1, i * (32 / (2 * span)));
      }
    }
  }
}

template <int N>
struct FFT2 {
  static constexpr int R1 = Split<N>::R1, R2 = Split<N>::R2, J = R1 / R2;
  // register holding input element k (= x[a + R2 k]) when taken from an output set
  __host__ __device__ static constexpr int in_from_out(int k) { return (k % J) * R2 + k / J; }
  // element index (along the transform) of output register r in lane a
  __host__ __device__ static constexpr int out_pos_base(int r) { return R2 * (r / R2) + R1 * (r % R2); }
};

// Shared twiddles of fft2_3, laid out [q][a] = w_N^(a q) (q < R1, a < R2) so that the
// lanes of a transform read consecutive words.  tw[e] = exp(-2 pi i e / N).
template <typename T, int N>
__device__ __forceinline__ void fft2_tables(cx<T>* s_tw, const cx<T>* tw) {
  constexpr int R2 = Split<N>::R2;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int q = i / R2, a = i - q * R2;
    s_tw[i] = tw[(a * q) & (N - 1)];
  }
}

// Three-component transform.  S(c, q, a2) returns the shared-memory slot of matrix
// element (q, a2) of component c for this thread's transform; tw: fft2_tables.
// Ends with the results in registers; the caller must __syncthreads() before the
// shared exchange buffers are written again.
template <typename T, int N, int DIR, class Slot>
__device__ __forceinline__ void fft2_3(cx<T> (&v)[3][Split<N>::R1], int a, const cx<T>* tw, Slot S) {
  constexpr int R1 = Split<N>::R1, R2 = Split<N>::R2, J = R1 / R2;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    dft_dif<T, R1, DIR>(v[c]);
#pragma unroll
    for (int q = 0; q < R1; ++q) {
      cx<T> y = v[c][bitrev<R1>(q)];
      if (q != 0) {
        const cx<T> w = tw[q * R2 + a];
        y = cmul(y, DIR < 0 ? w : mk(w.x, -w.y));
      }
      *S(c, q, a) = y;
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int q = a + R2 * j;
      cx<T> u[R2];
#pragma unroll
      for (int a2 = 0; a2 < R2; ++a2) u[a2] = *S(c, q, a2);
      dft_dif<T, R2, DIR>(u);
#pragma unroll
      for (int p = 0; p < R2; ++p) v[c][j * R2 + p] = u[bitrev<R2>(p)];
    }
  }
}

// One-component transform (the component-split kernels): the same passes as fft2_3 with
// S(q, a2) the slot of matrix element (q, a2) of this thread's transform.
// WARP: the R2 lanes of every transform are consecutive threads of one warp and the
// slots are the transform's own, so a warp barrier orders the exchange (no block barrier).
template <typename T, int N, int DIR, class Slot, bool WARP = false>
__device__ __forceinline__ void fft2_1(cx<T> (&v)[Split<N>::R1], int a, const cx<T>* tw, Slot S) {
  constexpr int R1 = Split<N>::R1, R2 = Split<N>::R2, J = R1 / R2;
  dft_dif<T, R1, DIR>(v);
#pragma unroll
  for (int q = 0; q < R1; ++q) {
    cx<T> y = v[bitrev<R1>(q)];
    if (q != 0) {
      const cx<T> w = tw[q * R2 + a];
      y = cmul(y, DIR < 0 ? w : mk(w.x, -w.y));
    }
    *S(q, a) = y;
  }
  if (WARP)
    __syncwarp();
  else
    __syncthreads();
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int q = a + R2 * j;
    cx<T> u[R2];
#pragma unroll
    for (int a2 = 0; a2 < R2; ++a2) u[a2] = *S(q, a2);
    dft_dif<T, R2, DIR>(u);
#pragma unroll
    for (int p = 0; p < R2; ++p) v[j * R2 + p] = u[bitrev<R2>(p)];
  }
}

template <typename T, int N>
__device__ __forceinline__ void out_to_in_1(cx<T> (&v)[Split<N>::R1]) {
  constexpr int R1 = Split<N>::R1;
  cx<T> t[R1];
#pragma unroll
  for (int k = 0; k < R1; ++k) t[k] = v[FFT2<N>::in_from_out(k)];
#pragma unroll
  for (int k = 0; k < R1; ++k) v[k] = t[k];
}

// Re-order registers from the output layout of one transform to the input layout of
// the next (same lane): in[k] = out[in_from_out(k)].
template <typename T, int N>
__device__ __forceinline__ void out_to_in(cx<T> (&v)[3][Split<N>::R1]) {
  constexpr int R1 = Split<N>::R1;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cx<T> t[R1];
#pragma unroll
    for (int k = 0; k < R1; ++k) t[k] = v[c][FFT2<N>::in_from_out(k)];
#pragma unroll
    for (int k = 0; k < R1; ++k) v[c][k] = t[k];
  }
}

}  // namespace kd
