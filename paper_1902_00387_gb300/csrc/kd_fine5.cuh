// Fine-step kernels for n = 512, 256 and 128 on a warp-owned FFT of n = 32 R points
// (R = 16, 8, 4 values a lane), complex64.
//
// A transform of one field component of one grid column (column kernel) or one ky row
// (row kernel) belongs to one warp, R values a lane, in one of two layouts:
//   layout A: lane a holds x[a + 32 k], k < R (the spectral side: ky or kx)
//   layout B: lane l = m1 + R e holds x[m1 + R p + R^2 brev_G(e)], p < R, G = 32 / R
//             (the physical side: y or x; brev_G reverses the bits of e < G)
// wr_a_to_b (n = a + 32 k, m = m1 + R m2): an R-point DFT over k inside the lane, the
// twiddle w_n^(a m1), a transpose through a shared buffer private to the warp after
// which lane m1 + R e holds a = G a' + e of row m1, an R-point DFT over a', the twiddle
// w_32^(e p), and a G-point DFT over e between the lanes m1 + R e (decimation in frequency
// by shuffles: one stage for n = 512, two for n = 256, three for n = 128).  wr_b_to_a is the same sequence
// backwards.  Both compute X[m] = sum_n x[n] exp(DIR 2 pi i n m / n) without
// normalisation.  The column pass takes ky in layout A to y in layout B and back; the row
// pass x in layout B to kx in layout A and back, so nothing is re-ordered between the
// transforms and the pointwise steps.  The kernels follow the 1024-point ones
// (kd_fine4.cuh): a column kernel with one warp per column and all three components in
// registers (u x b formed in registers), a row kernel with one warp per component of a
// row (the curl exchanged in shared memory).
#pragma once
#include "kd_fine4.cuh"

namespace kd {

template <int N>
struct WR {
  static_assert(N == 512 || N == 256 || N == 128, "warp transforms of 512, 256 or 128 points");
  static constexpr int R = N / 32;                // values a lane
  static constexpr int LR = R == 16 ? 4 : (R == 8 ? 3 : 2);   // log2 R
  static constexpr int G = 32 / R;                // lanes sharing a row of the second pass
  // complex per row of a warp's transpose buffer: 16-byte row starts, quarter-warp row
  // stores and half-warp column reads at most 2-way in conflict
  static constexpr int PITCH = R == 16 ? 18 : (R == 8 ? 10 : 4);
  static constexpr int BUF = 32 * PITCH;
};

// Twiddle table of the warp transforms in shared memory: s_tw[m1 * 32 + a] = w_N^(a m1)
// (m1 < R), so that w_32^(e p) = w_N^(R e p) = s_tw[p * 32 + R e].
template <int N>
__device__ __forceinline__ void wr_table(cx<float>* s_tw, const cx<float>* tw) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) s_tw[i] = tw[((i & 31) * (i >> 5)) & (N - 1)];
}

template <int DIR>
__device__ __forceinline__ cx<float> wr_apply(cx<float> v, cx<float> w) {
  return cmul(v, DIR < 0 ? w : conjf2(w));
}

__device__ __forceinline__ cx<float> wr_shfl(cx<float> v, int m) {
  return mk(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// v * exp(DIR 2 pi i b / 4) for b = 0, 1 (the 4-point twiddle)
template <int DIR>
__device__ __forceinline__ cx<float> wr_rot(cx<float> v, int b) {
  return b ? (DIR > 0 ? mk(-v.y, v.x) : mk(v.y, -v.x)) : v;
}

// bit reversal of e < G (G = 2, 4, 8)
__host__ __device__ constexpr int wr_brev(int e, int G) {
  return G == 2 ? e : (G == 4 ? (((e & 1) << 1) | (e >> 1)) : (((e & 1) << 2) | (e & 2) | (e >> 2)));
}

// The cross-lane stage of half size s (s = G/2 .. 1, lanes l and l ^ s R) of the G-point
// DFT over e, decimation in frequency: the upper lane takes (partner - own) w_2s^(e mod s).
// w_8^t (s = 4) comes from the table: w_8^t = w_N^(N t / 8) = s_tw[t * 32 + 4 R] (t < 4).
template <int N, int DIR, int S_>
__device__ __forceinline__ cx<float> wr_dif_stage(cx<float> x, int e, const cx<float>* tw) {
  constexpr int R = WR<N>::R;
  const cx<float> q = wr_shfl(x, S_ * R);
  if (!(e & S_)) return x + q;
  const cx<float> d = q - x;
  if constexpr (S_ == 1) return d;
  else if constexpr (S_ == 2) return wr_rot<DIR>(d, e & 1);
  else return (e & 3) ? wr_apply<DIR>(d, tw[(e & 3) * 32 + 4 * R]) : d;
}

// The same stage for decimation in time (input bit-reversed): the upper lane's value is
// multiplied first, then (partner - own) / (own + partner).
template <int N, int DIR, int S_>
__device__ __forceinline__ cx<float> wr_dit_stage(cx<float> x, int e, const cx<float>* tw) {
  constexpr int R = WR<N>::R;
  cx<float> own = x;
  if (e & S_) {
    if constexpr (S_ == 2) own = wr_rot<DIR>(x, e & 1);
    else if constexpr (S_ == 4) own = (e & 3) ? wr_apply<DIR>(x, tw[(e & 3) * 32 + 4 * R]) : x;
  }
  const cx<float> q = wr_shfl(own, S_ * R);
  return (e & S_) ? q - own : own + q;
}

// layout A -> layout B; tw: s_tw of wr_table
template <int N, int DIR>
__device__ __forceinline__ void wr_a_to_b(cx<float> (&v)[N / 32], int lane, cx<float>* S, const cx<float>* tw) {
  using W = WR<N>;
  constexpr int R = W::R, G = W::G, PI = W::PITCH;
  dft_dif<float, R, DIR>(v);                       // Y[m1] at v[bitrev(m1)]
#pragma unroll
  for (int m1 = 0; m1 < R; m1 += 2) {
    cx<float> y0 = v[bitrev<R>(m1)], y1 = v[bitrev<R>(m1 + 1)];
    if (m1 != 0) y0 = wr_apply<DIR>(y0, tw[m1 * 32 + lane]);
    y1 = wr_apply<DIR>(y1, tw[(m1 + 1) * 32 + lane]);
    *(float4*)&S[lane * PI + m1] = make_float4(y0.x, y0.y, y1.x, y1.y);
  }
  __syncwarp();
  const int m1 = lane & (R - 1), e = lane >> W::LR;
#pragma unroll
  for (int ap = 0; ap < R; ++ap) v[ap] = S[(G * ap + e) * PI + m1];
  __syncwarp();
  dft_dif<float, R, DIR>(v);                       // E_e[p] at v[bitrev(p)]
  // w_32^(e p), then the G-point DFT over e between the lanes m1 + R e (decimation in
  // frequency), all in place at the bit-reversed registers
#pragma unroll
  for (int p = 1; p < R; ++p)
    if (e != 0) v[bitrev<R>(p)] = wr_apply<DIR>(v[bitrev<R>(p)], tw[p * 32 + R * e]);
  if constexpr (G == 8) {
#pragma unroll
    for (int p = 0; p < R; ++p) v[bitrev<R>(p)] = wr_dif_stage<N, DIR, 4>(v[bitrev<R>(p)], e, tw);
  }
  if constexpr (G >= 4) {
#pragma unroll
    for (int p = 0; p < R; ++p) v[bitrev<R>(p)] = wr_dif_stage<N, DIR, 2>(v[bitrev<R>(p)], e, tw);
  }
#pragma unroll
  for (int p = 0; p < R; ++p) v[bitrev<R>(p)] = wr_dif_stage<N, DIR, 1>(v[bitrev<R>(p)], e, tw);
  cx<float> t[R];                                  // X[m1 + R p + R^2 brev(e)] into v[p]
#pragma unroll
  for (int p = 0; p < R; ++p) t[p] = v[bitrev<R>(p)];
#pragma unroll
  for (int p = 0; p < R; ++p) v[p] = t[p];
}

// layout B -> layout A
template <int N, int DIR>
__device__ __forceinline__ void wr_b_to_a(cx<float> (&v)[N / 32], int lane, cx<float>* S, const cx<float>* tw) {
  using W = WR<N>;
  constexpr int R = W::R, G = W::G, PI = W::PITCH;
  const int m1 = lane & (R - 1), e = lane >> W::LR;
  // G-point DFT over the lanes' (bit-reversed) h, decimation in time
#pragma unroll
  for (int p = 0; p < R; ++p) v[p] = wr_dit_stage<N, DIR, 1>(v[p], e, tw);
  if constexpr (G >= 4) {
#pragma unroll
    for (int p = 0; p < R; ++p) v[p] = wr_dit_stage<N, DIR, 2>(v[p], e, tw);
  }
  if constexpr (G == 8) {
#pragma unroll
    for (int p = 0; p < R; ++p) v[p] = wr_dit_stage<N, DIR, 4>(v[p], e, tw);
  }
#pragma unroll
  for (int p = 1; p < R; ++p)                      // T_e[p] w_32^(e p)
    if (e != 0) v[p] = wr_apply<DIR>(v[p], tw[p * 32 + R * e]);
  dft_dif<float, R, DIR>(v);                       // V[a'] at v[bitrev(a')], a = G a' + e
#pragma unroll
  for (int ap = 0; ap < R; ++ap) S[(G * ap + e) * PI + m1] = v[bitrev<R>(ap)];
  __syncwarp();
#pragma unroll
  for (int q = 0; q < R; q += 2) {
    const float4 r = *(const float4*)&S[lane * PI + q];
    cx<float> y0 = mk(r.x, r.y), y1 = mk(r.z, r.w);
    if (q != 0) y0 = wr_apply<DIR>(y0, tw[q * 32 + lane]);
    y1 = wr_apply<DIR>(y1, tw[(q + 1) * 32 + lane]);
    v[q] = y0;
    v[q + 1] = y1;
  }
  __syncwarp();
  dft_dif<float, R, DIR>(v);                       // Z[a + 32 k] at v[bitrev(k)]
  cx<float> t[R];
#pragma unroll
  for (int k = 0; k < R; ++k) t[k] = v[bitrev<R>(k)];
#pragma unroll
  for (int k = 0; k < R; ++k) v[k] = t[k];
}

// physical index (y or x) of register p of `lane` in layout B
template <int N>
__device__ __forceinline__ int wr_phys(int lane, int p) {
  using W = WR<N>;
  return (lane & (W::R - 1)) + W::R * p + W::R * W::R * wr_brev(lane >> W::LR, W::G);
}

// ------------------------------------------------------------------ column kernel
// One warp per grid column with all three components; XG = 8 adjacent columns per block
// (64-byte runs of a row), input rows staged two components ahead with 16-byte cp.async,
// output through a padded staging area; MINB blocks per SM.
template <int N>
struct ColW {
  using W = WR<N>;
  static constexpr int XG = 8, BLOCK = 32 * XG, MINB = N == 512 ? 2 : (N == 256 ? 3 : 4);
  static constexpr int K = N / 3, P = 2 * K + 1;
  static constexpr int OP = XG + 1;
  static constexpr int OUTSZ = (P * OP + 1) & ~1;
  static constexpr size_t smem =
      ((size_t)XG * W::BUF + 2 * (size_t)P * XG + OUTSZ + N) * sizeof(cx<float>) + (size_t)N * sizeof(float2);
  static_assert(MINB * (smem + 1024) <= 233472, "blocks fit the shared memory of an SM");
  __device__ __forceinline__ static int in_at(int iy, int xi) {
    return iy * XG + ((((xi >> 1) ^ (iy >> 1)) & 3) << 1) + (xi & 1);
  }
};

template <int N>
__global__ void __launch_bounds__(ColW<N>::BLOCK, ColW<N>::MINB) colw_kernel(FineArgs a, int step, int stage) {
  using G = ColW<N>;
  constexpr int K = G::K, P = G::P, OP = G::OP, XG = G::XG, GPF = N / XG, H = XG / 2, R = G::W::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* Tb = (cx<float>*)smem_raw;             // [XG][BUF]
  cx<float>* In = Tb + XG * G::W::BUF;              // [2][P][XG]
  cx<float>* Out = In + 2 * P * XG;                 // [P][OP]
  cx<float>* s_tw = Out + G::OUTSZ;                 // [R][32]
  float2* s_cs = (float2*)(s_tw + N);               // (cos, sin)(2 pi j / N)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  cx<float>* S = Tb + warp * G::W::BUF;
  wr_table<N>(s_tw, (const cx<float>*)a.tw);
  {
    const float* g_cos = (const float*)a.cosg;
    const float* g_sin = (const float*)a.sing;
    for (int i = threadIdx.x; i < N; i += blockDim.x) s_cs[i] = make_float2(g_cos[i], g_sin[i]);
  }
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
    const int x = x0 + warp;
    const Phase<float> ph = load_phase<float>(a, b, step, stage);
    const float A = flow_amp<float>(a, b);
    cx<float> v0[R], v1[R], v2[R];
    auto fetch = [&](cx<float>(&v)[R], int c) {
      const long k = 3 * j + c;
      cp_async_wait_group1();
      __syncthreads();   // load k visible to the block (and, first time, the tables)
      const cx<float>* buf = In + (k & 1) * P * XG;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int yy = lane + 32 * q;
        const int ky = yy < N / 2 ? yy : yy - N;
        if (wfft_never_kept<N>(q))
          v[q] = mk(0.f, 0.f);
        else
          v[q] = (ky >= -K && ky <= K) ? buf[G::in_at(ky + K, warp)] : mk(0.f, 0.f);
      }
      __syncthreads();   // the buffer is read: it takes load k + 2
      load(k + 2);
      wr_a_to_b<N, +1>(v, lane, S, s_tw);         // ky -> y (layout B)
    };
    fetch(v0, 0);
    fetch(v1, 1);
    fetch(v2, 2);
    {
      const float2 csx = s_cs[x];
      const float uy = A * (csx.y * ph.cpx + csx.x * ph.spx);
      const float uzx = csx.x * ph.cpx - csx.y * ph.spx;
#pragma unroll
      for (int p = 0; p < R; ++p) {
        const float2 csy = s_cs[wr_phys<N>(lane, p)];
        const float ux = A * (csy.x * ph.cpy - csy.y * ph.spy);
        const float uz = A * (uzx + (csy.y * ph.cpy + csy.x * ph.spy));
        const cx<float> bx = v0[p], by = v1[p], bz = v2[p];
        v0[p] = bz * uy - by * uz;
        v1[p] = bx * uz - bz * ux;
        v2[p] = by * ux - bx * uy;
      }
    }
    auto emit = [&](cx<float>(&v)[R], int c) {
      wr_b_to_a<N, -1>(v, lane, S, s_tw);         // y -> ky (layout A)
      __syncthreads();   // the staging area is free
#pragma unroll
      for (int p = 0; p < R; ++p) {
        if (wfft_never_kept<N>(p)) continue;
        const int yy = lane + 32 * p;
        const int ky = yy < N / 2 ? yy : yy - N;
        if (ky >= -K && ky <= K) Out[(ky + K) * OP + warp] = v[p];
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

// --------------------------------------------------------------------- row kernel
// Slots of a lane's registers that can hold a kept kx (the others never do): slot(p) =
// the number of such registers below p.
template <int N>
__host__ __device__ constexpr int wr_slot(int p) {
  int s = 0;
  for (int q = 0; q < p; ++q) s += wfft_never_kept<N>(q) ? 0 : 1;
  return s;
}

template <int N, int MODE>
struct RowW {
  using W = WR<N>;
  static constexpr int WARPS = 3, BLOCK = 96;
  static constexpr int K = N / 3, P = 2 * K + 1;
  static constexpr int NPRE = row4_reads(MODE);
  static constexpr int SLOTS = wr_slot<N>(N / 32);
  static constexpr int WSMEM = W::BUF + NPRE * SLOTS * 32;
  static constexpr size_t smem = ((size_t)WARPS * WSMEM + N) * sizeof(cx<float>);
  static constexpr int MINB = (int)(233472 / (smem + 1024)) > 8 ? 8 : (int)(233472 / (smem + 1024));
};

template <int N, int MODE>
__global__ void __launch_bounds__(RowW<N, MODE>::BLOCK, RowW<N, MODE>::MINB) roww_kernel(FineArgs a, int store_m) {
  using G = RowW<N, MODE>;
  constexpr int K = G::K, P = G::P, NPRE = G::NPRE, R = G::W::R, PI = G::W::PITCH, SL = G::SLOTS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = warp, c1 = c == 2 ? 0 : c + 1, c2 = c == 0 ? 2 : c - 1;
  cx<float>* Tb = (cx<float>*)smem_raw;             // [3][WSMEM]
  cx<float>* s_tw = Tb + G::WARPS * G::WSMEM;       // [R][32]
  cx<float>* S = Tb + warp * G::WSMEM;
  cx<float>* Q = S + G::W::BUF;                     // [NPRE][slot][lane]
  wr_table<N>(s_tw, (const cx<float>*)a.tw);
  __syncthreads();
  const StageArrays<float> sa = stage_arrays<float>(a);
  const cx<float>* src[3] = {MODE == 0 ? sa.X : (MODE == 1 ? sa.R2 : (MODE == 2 ? sa.R3 : sa.R4)),
                             MODE == 1 ? sa.R3 : (MODE == 2 ? sa.R4 : sa.X), MODE == 1 ? sa.R4 : sa.Xlo};
  const int npre = MODE == 3 && !sa.lo_valid ? 2 : NPRE;
  const long rows = (long)a.batch * P;
  griddep_wait();    // W (and the stage arrays) come from the predecessors
  for (long row = blockIdx.x; row < rows; row += gridDim.x) {
    const long b = row / P;
    const int iy = (int)(row - b * P);
    const long sbase = ((b * 3 + c) * P + iy) * (long)P + K;   // compact index of kx = 0
    cx<float> v[R];
    if (MODE == 4) {
#pragma unroll
      for (int k = 0; k < R; ++k) {
        const int xx = lane + 32 * k;
        const int kx = xx < N / 2 ? xx : xx - N;
        v[k] = !wfft_never_kept<N>(k) && kx >= -K && kx <= K ? sa.X[sbase + kx] : mk(0.f, 0.f);
      }
    } else {
#pragma unroll
      for (int j = 0; j < NPRE; ++j)
#pragma unroll
        for (int p = 0; p < R; ++p) {
          if (wfft_never_kept<N>(p) || j >= npre) continue;
          const int xx = lane + 32 * p;
          const int kx = xx < N / 2 ? xx : xx - N;
          if (kx >= -K && kx <= K) cp_async8(Q + (j * SL + wr_slot<N>(p)) * 32 + lane, src[j] + sbase + kx);
        }
      cp_async_commit();
      const cx<float>* Wr = (const cx<float>*)a.W + ((b * 3 + c) * P + iy) * (long)N;
#pragma unroll
      for (int p = 0; p < R; ++p) v[p] = Wr[wr_phys<N>(lane, p)];
      wr_b_to_a<N, -1>(v, lane, S, s_tw);         // x -> kx: v[k] = n^2 w_hat_c(kx index lane + 32 k)
#pragma unroll
      for (int p = 0; p < R; p += 2)
        *(float4*)&S[lane * PI + p] = make_float4(v[p].x, v[p].y, v[p + 1].x, v[p + 1].y);
      __syncthreads();                             // the row's three components are in place
      cp_async_wait_all();
      const StageCoef<float> sc = stage_coef<float>(a, b);
      const float inv_n2 = 1.f / ((float)N * (float)N);
      const float fky = (float)(iy - K);
      const float lam_y = (fky * fky + sc.kz * sc.kz);
      const cx<float>* S1 = Tb + c1 * G::WSMEM;
      const cx<float>* S2 = Tb + c2 * G::WSMEM;
#pragma unroll
      for (int p = 0; p < R; p += 2) {
        const float4 e1 = *(const float4*)&S1[lane * PI + p], e2 = *(const float4*)&S2[lane * PI + p];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int pp = p + h;
          const int xx = lane + 32 * pp;
          const int kx = xx < N / 2 ? xx : xx - N;
          if (wfft_never_kept<N>(pp) || kx < -K || kx > K) {
            v[pp] = mk(0.f, 0.f);
          } else {
            const float fkx = (float)kx;
            const float k1 = (c == 0 ? fky : (c == 1 ? sc.kz : fkx)) * inv_n2;
            const float k2 = (c == 0 ? sc.kz : (c == 1 ? fkx : fky)) * inv_n2;
            const cx<float> w1 = h ? mk(e1.z, e1.w) : mk(e1.x, e1.y), w2 = h ? mk(e2.z, e2.w) : mk(e2.x, e2.y);
            const cx<float> f = mul_i(w2 * k1 - w1 * k2);
            const float lam = (fkx * fkx + lam_y) * sc.inv_rm;
            const float g = implicit_gain(sc.dt * 0.5f * lam);
            cx<float> r[3];
#pragma unroll
            for (int j = 0; j < NPRE; ++j)
              r[j] = j < npre ? Q[(j * SL + wr_slot<N>(pp)) * 32 + lane] : mk(0.f, 0.f);
            v[pp] = stage_update_1<MODE>(sc, sa, sbase + kx, g, sc.dt * lam, r, f, nullptr);
          }
        }
      }
      __syncthreads();                             // the exchange is read before S is rewritten
      if (!store_m) continue;                      // uniform over the grid
    }
    wr_a_to_b<N, +1>(v, lane, S, s_tw);           // kx -> x (layout B)
    cx<float>* Mr = (cx<float>*)a.M + ((b * 3 + c) * P + iy) * (long)N;
#pragma unroll
    for (int p = 0; p < R; ++p) Mr[wr_phys<N>(lane, p)] = v[p];
  }
}

}  // namespace kd
