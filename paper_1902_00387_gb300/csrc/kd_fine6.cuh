// Column kernel for n = 1024 on a 1024-point FFT owned by a PAIR of warps (64 lanes x 16
// values), complex64: twice the warps per SM of the one-warp-per-column kernel (col5 in
// kd_fine4.cuh) at 16 values of each field component a lane.
//
// Lane L = 32 w + lane (w: the pair's warp) of a column holds, per component, either
//   layout A: x[L + 64 k], k < 16 (the spectral side, ky)
//   layout B: x[m1 + 16 p + 256 brev2(j)], p < 16, L = 4 m1 + j (the physical side, y)
// wp_a_to_b: a 16-point DFT over k inside the lane, the twiddle w_1024^(L m1), a transpose
// through the column's shared buffer (both warps, a named barrier of the pair) after which
// L = 4 m1 + e holds the a = 4 a' + e of row m1, a 16-point DFT over a', the twiddle
// w_64^(e p), and a 4-point DFT over e between the lanes 4 m1 .. 4 m1 + 3 of one warp
// (radix-2 decimation in frequency by shuffles, output in bit-reversed lane order).
// wp_b_to_a runs the same steps backwards.  Both compute X[m] = sum_n x[n] exp(DIR 2 pi i
// n m / 1024) without normalisation.  The rest follows col5: inputs staged two components
// ahead with 16-byte cp.async, u x b in registers, outputs through a padded staging area.
#pragma once
#include "kd_fine4.cuh"

namespace kd {

constexpr int kWPPitch = 20;               // complex per row of a pair's transpose buffer:
constexpr int kWPBuf = 64 * kWPPitch;      // conflict-free column accesses of a half warp

__device__ __forceinline__ int wp_brev2(int j) { return ((j & 1) << 1) | (j >> 1); }

template <int DIR>
__device__ __forceinline__ cx<float> wp_apply(cx<float> v, cx<float> w) {
  return cmul(v, DIR < 0 ? w : conjf2(w));
}

__device__ __forceinline__ cx<float> wp_shfl(cx<float> v, int m) {
  return mk(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// v * (DIR i)^(b): the 4-point twiddle exp(DIR 2 pi i b / 4) for b = 0, 1
template <int DIR>
__device__ __forceinline__ cx<float> wp_rot(cx<float> v, int b) {
  return b ? (DIR > 0 ? mk(-v.y, v.x) : mk(v.y, -v.x)) : v;
}

// Twiddles in shared memory: s_tw[m1 * 64 + L] = w_1024^(L m1) (m1 < 16, L < 64), so that
// w_64^(e p) = w_1024^(16 e p) = s_tw[p * 64 + 16 e].
__device__ __forceinline__ void wp_table(cx<float>* s_tw, const cx<float>* tw) {
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) s_tw[i] = tw[((i & 63) * (i >> 6)) & 1023];
}

// layout A -> layout B.  S: the pair's buffer (kWPBuf complex); bar: the pair's barrier.
template <int DIR, class BAR>
__device__ __forceinline__ void wp_a_to_b(cx<float> (&v)[16], int L, cx<float>* S, const cx<float>* tw, BAR bar) {
  dft_dif<float, 16, DIR>(v);                      // Y[m1] at v[bitrev(m1)]
#pragma unroll
  for (int m1 = 0; m1 < 16; m1 += 2) {
    cx<float> y0 = v[bitrev<16>(m1)], y1 = v[bitrev<16>(m1 + 1)];
    if (m1 != 0) y0 = wp_apply<DIR>(y0, tw[m1 * 64 + L]);
    y1 = wp_apply<DIR>(y1, tw[(m1 + 1) * 64 + L]);
    *(float4*)&S[L * kWPPitch + m1] = make_float4(y0.x, y0.y, y1.x, y1.y);
  }
  bar();
  const int m1 = L >> 2, e = L & 3;
#pragma unroll
  for (int ap = 0; ap < 16; ++ap) v[ap] = S[(4 * ap + e) * kWPPitch + m1];
  bar();                                           // the buffer is read before it is rewritten
  dft_dif<float, 16, DIR>(v);                      // E_e[p] at v[bitrev(p)]
  cx<float> u[16];
#pragma unroll
  for (int p = 0; p < 16; ++p) {
    const cx<float> x = v[bitrev<16>(p)];
    u[p] = (e == 0 || p == 0) ? x : wp_apply<DIR>(x, tw[p * 64 + 16 * e]);
  }
  // 4-point DFT over e between lanes 4 m1 + e (lane bits 1, 0), decimation in frequency
#pragma unroll
  for (int p = 0; p < 16; ++p) {
    const cx<float> q = wp_shfl(u[p], 2);
    u[p] = (L & 2) ? wp_rot<DIR>(q - u[p], L & 1) : u[p] + q;
  }
#pragma unroll
  for (int p = 0; p < 16; ++p) {
    const cx<float> q = wp_shfl(u[p], 1);
    v[p] = (L & 1) ? q - u[p] : u[p] + q;          // X[m1 + 16 p + 256 brev2(L & 3)]
  }
}

// layout B -> layout A
template <int DIR, class BAR>
__device__ __forceinline__ void wp_b_to_a(cx<float> (&v)[16], int L, cx<float>* S, const cx<float>* tw, BAR bar) {
  const int m1 = L >> 2, e = L & 3;
  // 4-point DFT over the lanes' h (bit-reversed input), decimation in time
#pragma unroll
  for (int p = 0; p < 16; ++p) {
    const cx<float> q = wp_shfl(v[p], 1);
    v[p] = (L & 1) ? q - v[p] : v[p] + q;
  }
#pragma unroll
  for (int p = 0; p < 16; ++p) {
    const cx<float> own = (L & 2) ? wp_rot<DIR>(v[p], L & 1) : v[p];
    const cx<float> q = wp_shfl(own, 2);
    v[p] = (L & 2) ? q - own : own + q;            // T_e[p]
  }
#pragma unroll
  for (int p = 1; p < 16; ++p)
    if (e != 0) v[p] = wp_apply<DIR>(v[p], tw[p * 64 + 16 * e]);
  dft_dif<float, 16, DIR>(v);                      // V[a'] at v[bitrev(a')], a = 4 a' + e
#pragma unroll
  for (int ap = 0; ap < 16; ++ap) S[(4 * ap + e) * kWPPitch + m1] = v[bitrev<16>(ap)];
  bar();
#pragma unroll
  for (int q = 0; q < 16; q += 2) {
    const float4 r = *(const float4*)&S[L * kWPPitch + q];
    cx<float> y0 = mk(r.x, r.y), y1 = mk(r.z, r.w);
    if (q != 0) y0 = wp_apply<DIR>(y0, tw[q * 64 + L]);
    y1 = wp_apply<DIR>(y1, tw[(q + 1) * 64 + L]);
    v[q] = y0;
    v[q + 1] = y1;
  }
  bar();
  dft_dif<float, 16, DIR>(v);                      // Z[L + 64 k] at v[bitrev(k)]
  cx<float> t[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) t[k] = v[bitrev<16>(k)];
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = t[k];
}

// physical index of register p of pair lane L in layout B
__device__ __forceinline__ int wp_phys(int L, int p) { return (L >> 2) + 16 * p + 256 * wp_brev2(L & 3); }

// Register k of pair lane L never holds a kept wavenumber (|k| <= N/3) when L + 64 k lies
// in (N/3, N - N/3) for every L.
template <int N>
__host__ __device__ constexpr bool wp_never_kept(int k) {
  return 64 * k > N / 3 && 64 * k + 63 < N - N / 3;
}

template <int N>
struct Col7 {
  static_assert(N == 1024, "1024-point transforms on a warp pair");
  static constexpr int XG = 8, BLOCK = 64 * XG, MINB = 1;   // 8 columns, 16 warps
  static constexpr int K = N / 3, P = 2 * K + 1;
  static constexpr int OP = XG + 1;
  static constexpr int OUTSZ = (P * OP + 1) & ~1;
  static constexpr size_t smem = ((size_t)XG * kWPBuf + 2 * (size_t)P * XG + OUTSZ + N) * sizeof(cx<float>);
  static_assert(smem + 1024 <= 233472, "the block fits the shared memory of an SM");
  __device__ __forceinline__ static int in_at(int iy, int xi) {
    return iy * XG + ((((xi >> 1) ^ (iy >> 1)) & 3) << 1) + (xi & 1);
  }
};

template <int N>
__global__ void __launch_bounds__(Col7<N>::BLOCK, Col7<N>::MINB) col7_kernel(FineArgs a, int step, int stage) {
  using G = Col7<N>;
  constexpr int K = G::K, P = G::P, OP = G::OP, XG = G::XG, GPF = N / XG, H = XG / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* Tb = (cx<float>*)smem_raw;             // [XG][kWPBuf] the pairs' transpose buffers
  cx<float>* In = Tb + XG * kWPBuf;                 // [2][P][XG]
  cx<float>* Out = In + 2 * P * XG;                 // [P][OP]
  cx<float>* s_tw = Out + G::OUTSZ;                 // [16][64]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int col = warp >> 1, L = 32 * (warp & 1) + lane;   // column of the pair, pair lane
  cx<float>* S = Tb + col * kWPBuf;
  auto bar = [&]() { named_bar(1 + col, 64); };
  const float* g_cos = (const float*)a.cosg;
  const float* g_sin = (const float*)a.sing;
  wp_table(s_tw, (const cx<float>*)a.tw);
  const long groups = (long)a.batch * GPF;
  const long mine = groups > (long)blockIdx.x ? (groups - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const cx<float>* M = (const cx<float>*)a.M;
  cx<float>* W = (cx<float>*)a.W;
  auto load = [&](long k) {
    if (k < 3 * mine) {
      const long g = blockIdx.x + (k / 3) * (long)gridDim.x;
      const int c = (int)(k % 3);
      const long b = g / GPF;
      const int x0 = (int)(g - b * GPF) * XG;
      const cx<float>* src = M + ((b * 3 + c) * (long)P) * N + x0;
      cx<float>* dst = In + (k & 1) * P * XG;
      for (int i = threadIdx.x; i < P * H; i += G::BLOCK) {
        const int h = i & (H - 1), iy = i / H;
        cp_async16(dst + G::in_at(iy, 2 * h), src + (long)iy * N + 2 * h, true);
      }
    }
    cp_async_commit();
  };
  griddep_wait();    // M is the predecessor's output
  load(0);
  load(1);
  for (long j = 0; j < mine; ++j) {
    const long g = blockIdx.x + j * (long)gridDim.x;
    const long b = g / GPF;
    const int x0 = (int)(g - b * GPF) * XG;
    const int x = x0 + col;
    const Phase<float> ph = load_phase<float>(a, b, step, stage);
    const float A = flow_amp<float>(a, b);
    cx<float> v0[16], v1[16], v2[16];
    auto fetch = [&](cx<float>(&v)[16], int c) {
      const long k = 3 * j + c;
      cp_async_wait_group1();
      __syncthreads();   // load k visible to the block (and, first time, the table)
      const cx<float>* buf = In + (k & 1) * P * XG;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int yy = L + 64 * q;
        const int ky = yy < N / 2 ? yy : yy - N;
        if (wp_never_kept<N>(q))
          v[q] = mk(0.f, 0.f);
        else
          v[q] = (ky >= -K && ky <= K) ? buf[G::in_at(ky + K, col)] : mk(0.f, 0.f);
      }
      __syncthreads();   // the buffer is read: it takes load k + 2
      load(k + 2);
      wp_a_to_b<+1>(v, L, S, s_tw, bar);          // ky -> y (layout B)
    };
    fetch(v0, 0);
    fetch(v1, 1);
    fetch(v2, 2);
    {
      const float cxg = __ldg(&g_cos[x]), sxg = __ldg(&g_sin[x]);
      const float uy = A * (sxg * ph.cpx + cxg * ph.spx);
      const float uzx = cxg * ph.cpx - sxg * ph.spx;
#pragma unroll
      for (int p = 0; p < 16; ++p) {
        const int y = wp_phys(L, p);
        const float cyg = __ldg(&g_cos[y]), syg = __ldg(&g_sin[y]);
        const float ux = A * (cyg * ph.cpy - syg * ph.spy);
        const float uz = A * (uzx + (syg * ph.cpy + cyg * ph.spy));
        const cx<float> bx = v0[p], by = v1[p], bz = v2[p];
        v0[p] = bz * uy - by * uz;
        v1[p] = bx * uz - bz * ux;
        v2[p] = by * ux - bx * uy;
      }
    }
    auto emit = [&](cx<float>(&v)[16], int c) {
      wp_b_to_a<-1>(v, L, S, s_tw, bar);          // y -> ky (layout A)
      __syncthreads();   // the staging area is free
#pragma unroll
      for (int p = 0; p < 16; ++p) {
        if (wp_never_kept<N>(p)) continue;
        const int yy = L + 64 * p;
        const int ky = yy < N / 2 ? yy : yy - N;
        if (ky >= -K && ky <= K) Out[(ky + K) * OP + col] = v[p];
      }
      __syncthreads();
      cx<float>* dst = W + ((b * 3 + c) * (long)P) * N + x0;
      for (int i = threadIdx.x; i < P * H; i += G::BLOCK) {
        const int h = i & (H - 1), row = i / H;
        const cx<float> e0 = Out[row * OP + 2 * h], e1 = Out[row * OP + 2 * h + 1];
        *(float4*)(dst + (long)row * N + 2 * h) = make_float4(e0.x, e0.y, e1.x, e1.y);
      }
    };
    emit(v0, 0);
    emit(v1, 1);
    emit(v2, 2);
  }
  cp_async_wait_all();
}

}  // namespace kd
