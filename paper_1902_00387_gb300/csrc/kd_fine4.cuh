// Fine-step kernels for n = 1024 on a warp-owned four-step FFT (1024 = 32 x 32).
//
// Every field component of one grid column (column kernel) or one ky row (row kernel) is
// transformed by one warp: lane a keeps the 32 values x[a + 32 k] in registers, does a
// 32-point DFT over k, twiddles, exchanges through a shared-memory transpose private to
// the warp (ordered by __syncwarp, no block barrier), and does a second 32-point DFT;
// the result X[a + 32 p] lands in the same registers in the same layout, so an inverse
// transform, the pointwise step and a forward transform follow each other without any
// re-ordering.  The radix-2 butterflies are packed FP32x2 instructions (bfly).
//
// The three components meet only where the method couples them: in physical space for
// u x b (column kernel, Sec. 2 Eq. 1) and in spectral space for the curl (row kernel).
// There the warps of one column / row exchange their values through shared memory
// behind a named barrier over just those warps.
//
// Memory traffic (complex64, layouts of kd_common.cuh: M and W are [b][c][P][n] with x
// contiguous):
//   column kernel: reads M and writes W along columns.  A block owns 4 adjacent columns
//     (12 warps), so both directions move 32-byte runs of a row: the input rows of the
//     next group are prefetched with 8-byte cp.async into a padded staging buffer while
//     the current group is transformed, and the output goes through the transpose
//     buffers of the component's 4 warps and leaves as 16-byte stores.
//   row kernel: reads W, writes M and touches the compact stage arrays along rows;
//     every access is a whole warp over consecutive elements.
#pragma once
#include "kd_fft2.cuh"
#include "kd_fine3.cuh"
#include "kd_stage.cuh"

namespace kd {

// Barrier over `count` threads (whole warps) that share the hardware barrier `id` (1..15).
__device__ __forceinline__ void named_bar(int id, int count) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(count) : "memory");
}

// 8-byte asynchronous global -> shared copy, cached in L1 so that the 4 columns of a
// row share one sector fetch.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ cx<float> conjf2(cx<float> w) { return mk(w.x, -w.y); }

// Wait until at most one committed cp.async group of this thread is still in flight.
__device__ __forceinline__ void cp_async_wait_group1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// A warp's transpose buffer: 32 rows of 34 complex (the pad keeps 16-byte row starts and
// spreads the 16-byte stores of a quarter warp over all banks).
constexpr int kWPitch = 34;
constexpr int kWBuf = 32 * kWPitch;

// 1024-point transform owned by one warp.
//   in : v[k] = x[lane + 32 k]        out: v[p] = X[lane + 32 p]
//   X[m] = sum_n x[n] exp(DIR 2 pi i n m / 1024)   (no normalisation)
// tw(q) returns w_1024^(lane q) = exp(-2 pi i lane q / 1024) for q = 1..31; S is the warp's
// buffer (kWBuf complex).  Leaves S free for the caller (ends with __syncwarp).
template <int DIR, class TW>
__device__ __forceinline__ void wfft1024(cx<float> (&v)[32], int lane, cx<float>* S, TW tw) {
  // pass 1: DFT over k of this lane's column of the 32 x 32 matrix, then w_1024^(lane q)
  dft_dif<float, 32, DIR>(v);
#pragma unroll
  for (int q = 0; q < 32; q += 2) {
    cx<float> y0 = v[bitrev<32>(q)], y1 = v[bitrev<32>(q + 1)];
    if (q != 0) {
      const cx<float> w = tw(q);
      y0 = cmul(y0, DIR < 0 ? w : conjf2(w));
    }
    const cx<float> w1 = tw(q + 1);
    y1 = cmul(y1, DIR < 0 ? w1 : conjf2(w1));
    *(float4*)&S[lane * kWPitch + q] = make_float4(y0.x, y0.y, y1.x, y1.y);
  }
  __syncwarp();
  // pass 2: lane takes row q = lane of the transposed matrix, DFT over a
#pragma unroll
  for (int a = 0; a < 32; ++a) v[a] = S[a * kWPitch + lane];
  __syncwarp();
  dft_dif<float, 32, DIR>(v);
  cx<float> t[32];
#pragma unroll
  for (int p = 0; p < 32; ++p) t[p] = v[bitrev<32>(p)];
#pragma unroll
  for (int p = 0; p < 32; ++p) v[p] = t[p];
}

// Twiddle table of the warp transforms in shared memory: s_tw[q * 32 + a] = w_1024^(a q),
// read by lane a as consecutive words.
__device__ __forceinline__ void wfft_table(cx<float>* s_tw, const cx<float>* tw) {
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) s_tw[i] = tw[((i & 31) * (i >> 5)) & 1023];
}

// Registers of one lane's 32 values that hold no kept wavenumber (|k| <= K) for any lane:
// index lane + 32 k lies in (K, N - K) for every lane.
template <int N>
__host__ __device__ constexpr bool wfft_never_kept(int k) {
  return 32 * k > N / 3 && 32 * k + 31 < N - N / 3;
}

// ------------------------------------------------------------------ column kernel
// CB: bytes per asynchronous copy of the input staging: 8 (one complex, L1-allocating,
// pitch 5: conflict-free column reads) or 16 (two complex, L2 only, pitch 6: half the
// copies, two-way bank conflicts on the column reads).
template <int N, int CB>
struct Col4 {
  static_assert(N == 1024, "warp-owned transforms of 1024 points");
  static_assert(CB == 8 || CB == 16, "8- or 16-byte copies");
  static constexpr int XG = 4;                  // adjacent columns per group (32-byte runs)
  static constexpr int WARPS = 3 * XG;          // warp (c, xi): component c of column xi
  static constexpr int BLOCK = 32 * WARPS;
  static constexpr int K = N / 3, P = 2 * K + 1;
  static constexpr int IP = CB == 8 ? 5 : 6;    // input staging pitch in complex
  static constexpr int OP = 5;                  // output staging pitch (conflict-free writes)
  static_assert(XG * kWBuf >= P * OP, "the output staging of a component fits its warps' buffers");
  static constexpr size_t smem = ((size_t)WARPS * kWBuf + (size_t)3 * P * IP + N) * sizeof(cx<float>) +
                                 (size_t)N * sizeof(float2);
};

// One RK stage's column pass: M (kept ky rows, physical x) -> inverse FFT in y -> u x b ->
// forward FFT in y -> kept ky rows -> W.  Persistent: one block per SM walks the groups of
// 4 columns; the staging buffer holds the next group's rows while this one is computed.
template <int N, int CB>
__global__ void __launch_bounds__(Col4<N, CB>::BLOCK, 1) col4_kernel(FineArgs a, int step, int stage) {
  using G = Col4<N, CB>;
  constexpr int K = G::K, P = G::P, IP = G::IP, OP = G::OP, XG = G::XG, GPF = N / XG;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* Tb = (cx<float>*)smem_raw;             // [WARPS][kWBuf] transpose buffers
  cx<float>* St = Tb + G::WARPS * kWBuf;            // [3 P][IP] staged input rows of a group
  cx<float>* s_tw = St + 3 * P * IP;                // [32][32] twiddles
  float2* s_cs = (float2*)(s_tw + N);               // (cos, sin)(2 pi j / N)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = warp / XG, xi = warp - (warp / XG) * XG;
  const int c1 = c == 2 ? 0 : c + 1, c2 = c == 0 ? 2 : c - 1;
  cx<float>* S = Tb + warp * kWBuf;
  wfft_table(s_tw, (const cx<float>*)a.tw);
  for (int i = threadIdx.x; i < N; i += blockDim.x)
    s_cs[i] = make_float2(((const float*)a.cosg)[i], ((const float*)a.sing)[i]);
  const long groups = (long)a.batch * GPF;
  const cx<float>* M = (const cx<float>*)a.M;
  cx<float>* W = (cx<float>*)a.W;
  auto prefetch = [&](long g) {
    const long b = g / GPF;
    const int x0 = (int)(g - b * GPF) * XG;
    const cx<float>* src = M + (b * 3) * (long)P * N + x0;
    if constexpr (CB == 8) {
      for (int i = threadIdx.x; i < 3 * P * XG; i += G::BLOCK) {
        const int xx = i & (XG - 1), r = i / XG;   // r = c P + iy
        cp_async8(St + r * IP + xx, src + (long)r * N + xx);
      }
    } else {
      for (int i = threadIdx.x; i < 3 * P * (XG / 2); i += G::BLOCK) {
        const int xx = (i & (XG / 2 - 1)) * 2, r = i / (XG / 2);
        cp_async16(St + r * IP + xx, src + (long)r * N + xx, true);
      }
    }
    cp_async_commit();
  };
  auto twf = [&](int q) { return s_tw[q * 32 + lane]; };
  griddep_wait();    // M is the predecessor's output
  if ((long)blockIdx.x < groups) prefetch(blockIdx.x);
  for (long g = blockIdx.x; g < groups; g += gridDim.x) {
    cp_async_wait_all();
    __syncthreads();   // the group's rows (and, first time, the tables) are visible
    const long b = g / GPF;
    const int x0 = (int)(g - b * GPF) * XG;
    const int x = x0 + xi;
    cx<float> v[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const int yy = lane + 32 * k;
      const int ky = yy < N / 2 ? yy : yy - N;
      if (wfft_never_kept<N>(k))
        v[k] = mk(0.f, 0.f);
      else
        v[k] = (ky >= -K && ky <= K) ? St[(c * P + ky + K) * IP + xi] : mk(0.f, 0.f);
    }
    __syncthreads();   // every warp has its rows: the staging buffer takes the next group
    if (g + gridDim.x < groups) prefetch(g + gridDim.x);
    const Phase<float> ph = load_phase<float>(a, b, step, stage);
    const float A = flow_amp<float>(a, b);

    wfft1024<+1>(v, lane, S, twf);                 // ky -> y: v[p] = b_c(x, y = lane + 32 p)

    // u x b at (x, y): component c of w = u_c1 b_c2 - u_c2 b_c1 (cyclic c, c1, c2)
#pragma unroll
    for (int p = 0; p < 32; p += 2)
      *(float4*)&S[lane * kWPitch + p] = make_float4(v[p].x, v[p].y, v[p + 1].x, v[p + 1].y);
    named_bar(1 + xi, 96);                         // the column's three components are in place
    {
      const float2 csx = s_cs[x];
      const float uy = A * (csx.y * ph.cpx + csx.x * ph.spx);
      const float uzx = csx.x * ph.cpx - csx.y * ph.spx;
      const cx<float>* S1 = Tb + (c1 * XG + xi) * kWBuf;
      const cx<float>* S2 = Tb + (c2 * XG + xi) * kWBuf;
#pragma unroll
      for (int p = 0; p < 32; p += 2) {
        const float4 q1 = *(const float4*)&S1[lane * kWPitch + p], q2 = *(const float4*)&S2[lane * kWPitch + p];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float2 csy = s_cs[lane + 32 * (p + h)];
          const float ux = A * (csy.x * ph.cpy - csy.y * ph.spy);
          const float uz = A * (uzx + (csy.y * ph.cpy + csy.x * ph.spy));
          const float u1 = c == 0 ? uy : (c == 1 ? uz : ux);
          const float u2 = c == 0 ? uz : (c == 1 ? ux : uy);
          const cx<float> b1 = h ? mk(q1.z, q1.w) : mk(q1.x, q1.y), b2 = h ? mk(q2.z, q2.w) : mk(q2.x, q2.y);
          v[p + h] = b2 * u1 - b1 * u2;
        }
      }
    }
    named_bar(1 + xi, 96);                         // the exchange is read before S is rewritten
    wfft1024<-1>(v, lane, S, twf);                 // y -> ky: v[p] = w_c(x, yy = lane + 32 p)

    // kept ky rows -> W through the staging area formed by the component's 4 buffers
    named_bar(5 + c, 32 * XG);                     // the component's warps are done with their buffers
    cx<float>* R = Tb + c * XG * kWBuf;            // [P][OP]
#pragma unroll
    for (int p = 0; p < 32; ++p) {
      if (wfft_never_kept<N>(p)) continue;
      const int yy = lane + 32 * p;
      const int ky = yy < N / 2 ? yy : yy - N;
      if (ky >= -K && ky <= K) R[(ky + K) * OP + xi] = v[p];
    }
    named_bar(5 + c, 32 * XG);
    {
      cx<float>* dst = W + ((b * 3 + c) * (long)P) * N + x0;
      for (int i = xi * 32 + lane; i < 2 * P; i += 32 * XG) {
        const int row = i >> 1, h = (i & 1) * 2;
        const cx<float> e0 = R[row * OP + h], e1 = R[row * OP + h + 1];
        *(float4*)(dst + (long)row * N + h) = make_float4(e0.x, e0.y, e1.x, e1.y);
      }
    }
  }
  cp_async_wait_all();
}

// ------------------------------------------ column kernel, one warp per column
// Col5: a warp owns one grid column and all three of its components (96 complex values a
// lane), so u x b is formed in registers: no exchange between warps and the flow is
// evaluated once per point.  A group of XG warps owns XG adjacent columns; a block holds GR
// groups.  XG = 8, GR = 1: 64-byte runs of a row, one block per SM, block barriers.  XG = 4,
// GR = 2: two groups of four warps in one block, each with its own staging buffers and
// named barriers, so that one group copies while the other transforms; the tables stay in
// shared memory.  XG = 4, GR = 1: two blocks per SM with the tables read from global memory
// (L1), measured slower at 1024^2 x 256 (3.88 against 3.32 ms per launch, 292 bytes of
// spills).  The input rows arrive one component at a time through two staging buffers,
// loaded two components ahead with 16-byte cp.async; a row of a buffer is XG / 2 chunks of
// 16 bytes (columns 2h, 2h + 1), chunk h stored at h ^ (row bits), which keeps the column
// reads of a half warp to two rows per bank.  The output of each component goes through a
// padded staging area (odd pitch: conflict-free column writes) and leaves as 16-byte
// stores.
template <int N, int XG_, int GR_ = 1>
struct Col5 {
  static_assert(N == 1024, "warp-owned transforms of 1024 points");
  static_assert((XG_ == 4 || XG_ == 8) && (GR_ == 1 || (GR_ == 2 && XG_ == 4)), "8 x 1 or 4 x 1 / 4 x 2 columns");
  static constexpr int XG = XG_;                // columns per group = warps per group
  static constexpr int GR = GR_;                // independent groups per block (own buffers, own barriers)
  static constexpr int BLOCK = 32 * XG * GR;
  static constexpr int K = N / 3, P = 2 * K + 1;
  static constexpr int OP = XG + 1;             // output staging pitch (complex)
  static constexpr bool STAB = XG * GR == 8;    // tables in shared memory (one 8-warp block per SM)
  static constexpr int MINB = 8 / (XG * GR);
  // complex per group, rounded up to 16 bytes: every group's staging buffers start on the
  // 16-byte boundary the cp.async copies into them need
  static constexpr size_t group_smem = (2 * (size_t)P * XG + (size_t)P * OP + 1) & ~(size_t)1;
  static_assert((XG * GR * kWBuf) % 2 == 0 && (2 * P * XG) % 2 == 0, "16-byte aligned staging buffers");
  static constexpr size_t smem = ((size_t)XG * GR * kWBuf + GR * group_smem + (STAB ? N : 0)) * sizeof(cx<float>) +
                                 (STAB ? (size_t)N * sizeof(float2) : 0);
  static_assert(MINB * (smem + 1024) <= 233472, "blocks fit the shared memory of an SM");
  // complex index of column xi of staged row iy in an input buffer
  __device__ __forceinline__ static int in_at(int iy, int xi) {
    constexpr int H = XG / 2;                   // 16-byte chunks per row
    const int swz = XG == 8 ? (iy >> 1) : (iy >> 2);
    return iy * XG + ((((xi >> 1) ^ swz) & (H - 1)) << 1) + (xi & 1);
  }
};

// The barrier of a group: the whole block when it is one group, else a named barrier of
// the group's warps (ids 1 and 2), so that the groups run out of step with each other.
template <int GR>
__device__ __forceinline__ void group_bar(int grp, int threads) {
  if constexpr (GR == 1)
    __syncthreads();
  else
    named_bar(1 + grp, threads);
}

template <int N, int XG, int GR>
__global__ void __launch_bounds__(Col5<N, XG, GR>::BLOCK, Col5<N, XG, GR>::MINB)
    col5_kernel(FineArgs a, int step, int stage) {
  using G = Col5<N, XG, GR>;
  constexpr int K = G::K, P = G::P, OP = G::OP, GPF = N / XG, H = XG / 2, GT = 32 * XG;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = warp / XG, wl = warp - grp * XG, gtid = threadIdx.x - grp * GT;
  cx<float>* Tb = (cx<float>*)smem_raw;                        // [XG GR][kWBuf] transpose buffers
  cx<float>* In = Tb + XG * GR * kWBuf + grp * G::group_smem;  // [2][P][XG] staged input rows (swizzled chunks)
  cx<float>* Out = In + 2 * P * XG;                            // [P][OP] output staging
  cx<float>* s_tw = Tb + XG * GR * kWBuf + GR * G::group_smem; // [32][32] twiddles (STAB)
  float2* s_cs = (float2*)(s_tw + N);                          // (cos, sin)(2 pi j / N) (STAB)
  cx<float>* S = Tb + warp * kWBuf;
  const cx<float>* g_tw = (const cx<float>*)a.tw;
  const float* g_cos = (const float*)a.cosg;
  const float* g_sin = (const float*)a.sing;
  if constexpr (G::STAB) {
    wfft_table(s_tw, g_tw);
    for (int i = threadIdx.x; i < N; i += blockDim.x) s_cs[i] = make_float2(g_cos[i], g_sin[i]);
  }
  if constexpr (GR > 1) __syncthreads();   // the tables, before the groups part ways
  auto twf = [&](int q) {
    if constexpr (G::STAB) {
      return s_tw[q * 32 + lane];
    } else {
      const float2 w = __ldg((const float2*)&g_tw[(lane * q) & (N - 1)]);
      return mk(w.x, w.y);
    }
  };
  auto csf = [&](int j) { return G::STAB ? s_cs[j] : make_float2(__ldg(&g_cos[j]), __ldg(&g_sin[j])); };
  const long groups = (long)a.batch * GPF;
  const long first = (long)blockIdx.x * GR + grp, stride = (long)gridDim.x * GR;
  const long mine = groups > first ? (groups - 1 - first) / stride + 1 : 0;
  const cx<float>* M = (const cx<float>*)a.M;
  cx<float>* W = (cx<float>*)a.W;
  // load k of this group: component k % 3 of its column group k / 3 into buffer k % 2
  auto load = [&](long k) {
    if (k < 3 * mine) {
      const long g = first + (k / 3) * stride;
      const int c = (int)(k % 3);
      const long b = g / GPF;
      const int x0 = (int)(g - b * GPF) * XG;
      const cx<float>* src = M + ((b * 3 + c) * (long)P) * N + x0;
      cx<float>* dst = In + (k & 1) * P * XG;
      for (int i = gtid; i < P * H; i += GT) {
        const int h = i & (H - 1), iy = i / H;
        cp_async16(dst + G::in_at(iy, 2 * h), src + (long)iy * N + 2 * h, true);
      }
    }
    cp_async_commit();   // possibly empty: keeps one group per load for the waits
  };
  griddep_wait();    // M is the predecessor's output
  load(0);
  load(1);
  for (long j = 0; j < mine; ++j) {
    const long g = first + j * stride;
    const long b = g / GPF;
    const int x0 = (int)(g - b * GPF) * XG;
    const int x = x0 + wl;
    const Phase<float> ph = load_phase<float>(a, b, step, stage);
    const float A = flow_amp<float>(a, b);
    cx<float> v0[32], v1[32], v2[32];
    // component c: staged ky rows -> registers -> inverse FFT in y
    auto fetch = [&](cx<float>(&v)[32], int c) {
      const long k = 3 * j + c;
      cp_async_wait_group1();
      group_bar<GR>(grp, GT);   // load k visible to the group (and, first time, the tables)
      const cx<float>* buf = In + (k & 1) * P * XG;
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int yy = lane + 32 * q;
        const int ky = yy < N / 2 ? yy : yy - N;
        if (wfft_never_kept<N>(q))
          v[q] = mk(0.f, 0.f);
        else
          v[q] = (ky >= -K && ky <= K) ? buf[G::in_at(ky + K, wl)] : mk(0.f, 0.f);
      }
      group_bar<GR>(grp, GT);   // the buffer is read: it takes load k + 2
      load(k + 2);
      wfft1024<+1>(v, lane, S, twf);               // ky -> y: v[p] = b_c(x, y = lane + 32 p)
    };
    fetch(v0, 0);
    fetch(v1, 1);
    fetch(v2, 2);
    // w = u x b at (x, y = lane + 32 p)
    {
      const float2 csx = csf(x);
      const float uy = A * (csx.y * ph.cpx + csx.x * ph.spx);
      const float uzx = csx.x * ph.cpx - csx.y * ph.spx;
#pragma unroll
      for (int p = 0; p < 32; ++p) {
        const float2 csy = csf(lane + 32 * p);
        const float ux = A * (csy.x * ph.cpy - csy.y * ph.spy);
        const float uz = A * (uzx + (csy.y * ph.cpy + csy.x * ph.spy));
        const cx<float> bx = v0[p], by = v1[p], bz = v2[p];
        v0[p] = bz * uy - by * uz;
        v1[p] = bx * uz - bz * ux;
        v2[p] = by * ux - bx * uy;
      }
    }
    // component c: forward FFT in y -> kept ky rows -> staging -> W
    auto emit = [&](cx<float>(&v)[32], int c) {
      wfft1024<-1>(v, lane, S, twf);               // y -> ky: v[p] = w_c(x, yy = lane + 32 p)
      group_bar<GR>(grp, GT);   // the staging area is free (previous component stored)
#pragma unroll
      for (int p = 0; p < 32; ++p) {
        if (wfft_never_kept<N>(p)) continue;
        const int yy = lane + 32 * p;
        const int ky = yy < N / 2 ? yy : yy - N;
        if (ky >= -K && ky <= K) Out[(ky + K) * OP + wl] = v[p];
      }
      group_bar<GR>(grp, GT);
      cx<float>* dst = W + ((b * 3 + c) * (long)P) * N + x0;
      for (int i = gtid; i < P * H; i += GT) {
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
// Compact arrays a row pass of stage MODE reads (X; R2, R3, R4; R3, R4; R4, X, Xlo), in the
// order stage_update_1 takes them; the prologue (MODE 4) reads X before anything else and
// stages nothing.
__host__ __device__ constexpr int row4_reads(int mode) { return mode == 1 || mode == 3 ? 3 : (mode == 2 ? 2 : (mode == 4 ? 0 : 1)); }

// Slots of a lane's kept kx registers: p <= 10 and p >= 21 (the others never hold a kept
// wavenumber at n = 1024).
constexpr int kRow4Slots = 22;
__host__ __device__ constexpr int row4_slot(int p) { return p <= 10 ? p : p - 10; }

// ROWS rows per block (3 warps each).  Shared memory per warp: its transpose buffer and
// the stage arrays of its row component, [array][slot][lane], filled by cp.async when the
// row starts and read after the forward transform.
template <int N, int ROWS, int MODE>
struct Row4 {
  static_assert(N == 1024, "warp-owned transforms of 1024 points");
  static constexpr int WARPS = 3 * ROWS;        // warp (rr, c): component c of row rr
  static constexpr int BLOCK = 32 * WARPS;
  static constexpr int K = N / 3, P = 2 * K + 1;
  static constexpr int NPRE = row4_reads(MODE);
  static constexpr int WSMEM = kWBuf + NPRE * kRow4Slots * 32;   // complex per warp
  static constexpr size_t smem = ((size_t)WARPS * WSMEM + N) * sizeof(cx<float>);
  static constexpr int MINB = (int)(233472 / (smem + 1024)) > 5 ? 5 : (int)(233472 / (smem + 1024));
  static_assert(!(N == 1024) || (wfft_never_kept<N>(11) && wfft_never_kept<N>(20) && !wfft_never_kept<N>(10) &&
                                 !wfft_never_kept<N>(21)), "kept registers are p <= 10 and p >= 21");
};

// One component of one IMEX RK443 stage at compact index s (the expressions of
// stage_update): f = F_c(X_j) (already scaled); r[0..] = the arrays the stage reads, in
// the order X (stage 0), R2 R3 R4 (stage 1), R3 R4 (stage 2), R4 X Xlo (stage 3; Xlo
// zero before the first step).  R4 holds R4 - X0 and the state is the pair (X, Xlo) as
// in state_add.  Returns X_{j+1}.  Stage 3 stores the state in X and Xlo, or, with xout
// set (the last step of a call), its rounded value at *xout only.
template <int MODE>
__device__ __forceinline__ cx<float> stage_update_1(const StageCoef<float>& q, const StageArrays<float>& sa, long s,
                                                    float g, float dl, const cx<float>* r, cx<float> f,
                                                    cx<float>* xout) {
  const float dt = q.dt;
  if (MODE == 0) {
    const cx<float> x0 = r[0];
    const cx<float> x1 = implicit_solve(x0 + f * (dt * 0.5f), g);
    sa.R2[s] = x0 + f * (dt * float(11.0 / 18.0)) - x1 * (dl * float(1.0 / 6.0));
    sa.R3[s] = x0 + f * (dt * float(5.0 / 6.0)) + x1 * (dl * 0.5f);
    sa.R4[s] = f * (dt * 0.25f) - x1 * (dl * 1.5f);
    return x1;
  } else if (MODE == 1) {
    const cx<float> x2 = implicit_solve(r[0] + f * (dt * float(1.0 / 18.0)), g);
    sa.R3[s] = r[1] - f * (dt * float(5.0 / 6.0)) - x2 * (dl * 0.5f);
    sa.R4[s] = r[2] + f * (dt * 1.75f) + x2 * (dl * 1.5f);
    return x2;
  } else if (MODE == 2) {
    const cx<float> x3 = implicit_solve(r[0] + f * (dt * 0.5f), g);
    sa.R4[s] = r[1] + f * (dt * 0.75f) - x3 * (dl * 0.5f);
    return x3;
  } else {
    const cx<float> x0 = r[1], lo = r[2];
    const cx<float> e = final_increment(x0, r[0] - f * (dt * 1.75f), g);
    float s0, e0, s1, e1, h0, l0, h1, l1;
    two_sum(x0.x, e.x, s0, e0);
    two_sum(x0.y, e.y, s1, e1);
    two_sum(s0, lo.x + e0, h0, l0);
    two_sum(s1, lo.y + e1, h1, l1);
    if (xout) {
      *xout = mk(h0, h1);
    } else {
      sa.X[s] = mk(h0, h1);
      sa.Xlo[s] = mk(l0, l1);
    }
    return mk(h0, h1);
  }
}

// One RK stage's row pass (MODE 0..3): W -> forward FFT in x -> kept kx -> curl i k3 x w_hat
// -> stage update -> inverse FFT in x of the next stage value -> M.  MODE 4 is the
// prologue, the inverse x transform of X.  Persistent blocks of ROWS rows; the stage
// arrays of a row are copied to shared memory while its W row is transformed.
template <int N, int ROWS, int MODE>
__global__ void __launch_bounds__(Row4<N, ROWS, MODE>::BLOCK, Row4<N, ROWS, MODE>::MINB)
    row4_kernel(FineArgs a, int store_m) {
  using G = Row4<N, ROWS, MODE>;
  constexpr int K = G::K, P = G::P, NPRE = G::NPRE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rr = warp / 3, c = warp - (warp / 3) * 3;
  const int c1 = c == 2 ? 0 : c + 1, c2 = c == 0 ? 2 : c - 1;
  cx<float>* Tb = (cx<float>*)smem_raw;             // [WARPS][WSMEM]
  cx<float>* s_tw = Tb + G::WARPS * G::WSMEM;       // [32][32] twiddles
  cx<float>* S = Tb + warp * G::WSMEM;              // transpose buffer
  cx<float>* Q = S + kWBuf;                         // [NPRE][slot][lane] staged stage arrays
  wfft_table(s_tw, (const cx<float>*)a.tw);
  __syncthreads();
  auto twf = [&](int q) { return s_tw[q * 32 + lane]; };
  const StageArrays<float> sa = stage_arrays<float>(a);
  const cx<float>* src[3] = {MODE == 0 ? sa.X : (MODE == 1 ? sa.R2 : (MODE == 2 ? sa.R3 : sa.R4)),
                             MODE == 1 ? sa.R3 : (MODE == 2 ? sa.R4 : sa.X), MODE == 1 ? sa.R4 : sa.Xlo};
  // the array holding the state X among src (stages 0 and 3), read from the caller's
  // layout [batch][3][N][N] in the first step when x_in_full is set
  constexpr int XSRC = MODE == 0 ? 0 : (MODE == 3 ? 1 : -1);
  const cx<float>* xin = (const cx<float>*)a.x_in_full;
  cx<float>* xout = MODE == 3 ? (cx<float>*)a.x_out_full : nullptr;
  // stage 3 before the first step of a call: the low part of the state is zero
  const int npre = MODE == 3 && !sa.lo_valid ? 2 : NPRE;
  const long rows = (long)a.batch * P;
  griddep_wait();    // W (and the stage arrays) come from the predecessors
  for (long r0 = (long)blockIdx.x * ROWS; r0 < rows; r0 += (long)gridDim.x * ROWS) {
    const long row = r0 + rr;
    if (row >= rows) break;                        // uniform over the row's three warps
    const long b = row / P;
    const int iy = (int)(row - b * P);
    const long sbase = ((b * 3 + c) * P + iy) * (long)P + K;   // compact index of kx = 0
    // the row (b, c, ky = iy - K) in the caller's layout: element kx at (kx mod N)
    const long fbase = ((b * 3 + c) * N + (iy - K < 0 ? iy - K + N : iy - K)) * (long)N;
    cx<float> v[32];
    if (MODE == 4) {
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        const int xx = lane + 32 * k;
        const int kx = xx < N / 2 ? xx : xx - N;
        if (wfft_never_kept<N>(k))
          v[k] = mk(0.f, 0.f);
        else
          v[k] = (kx >= -K && kx <= K) ? (xin ? xin[fbase + xx] : sa.X[sbase + kx]) : mk(0.f, 0.f);
      }
    } else {
      // the stage arrays of this lane's kept kx -> Q (each lane later reads only its own copies)
#pragma unroll
      for (int j = 0; j < NPRE; ++j)
#pragma unroll
        for (int p = 0; p < 32; ++p) {
          if (wfft_never_kept<N>(p) || j >= npre) continue;
          const int xx = lane + 32 * p;
          const int kx = xx < N / 2 ? xx : xx - N;
          if (kx >= -K && kx <= K)
            cp_async8(Q + (j * kRow4Slots + row4_slot(p)) * 32 + lane,
                      j == XSRC && xin ? xin + fbase + xx : src[j] + sbase + kx);
        }
      cp_async_commit();
      const cx<float>* Wr = (const cx<float>*)a.W + ((b * 3 + c) * P + iy) * (long)N;
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] = Wr[lane + 32 * k];
      wfft1024<-1>(v, lane, S, twf);               // x -> kx: v[p] = n^2 w_hat_c(kx index lane + 32 p)
      // curl: F_c = i (k_c1 w_c2 - k_c2 w_c1), k = (kx, ky, kz), w = v / n^2
#pragma unroll
      for (int p = 0; p < 32; p += 2)
        *(float4*)&S[lane * kWPitch + p] = make_float4(v[p].x, v[p].y, v[p + 1].x, v[p + 1].y);
      named_bar(1 + rr, 96);
      cp_async_wait_all();                         // this lane's staged values
      const StageCoef<float> sc = stage_coef<float>(a, b);
      const float inv_n2 = 1.f / ((float)N * (float)N);
      const float fky = (float)(iy - K);
      const float lam_y = (fky * fky + sc.kz * sc.kz);
      const cx<float>* S1 = Tb + (rr * 3 + c1) * G::WSMEM;
      const cx<float>* S2 = Tb + (rr * 3 + c2) * G::WSMEM;
#pragma unroll
      for (int p = 0; p < 32; p += 2) {
        const float4 e1 = *(const float4*)&S1[lane * kWPitch + p], e2 = *(const float4*)&S2[lane * kWPitch + p];
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
              r[j] = j < npre ? Q[(j * kRow4Slots + row4_slot(pp)) * 32 + lane] : mk(0.f, 0.f);
            v[pp] = stage_update_1<MODE>(sc, sa, sbase + kx, g, sc.dt * lam, r, f,
                                         xout ? xout + fbase + xx : nullptr);
          }
        }
      }
      named_bar(1 + rr, 96);                       // the exchange is read before S is rewritten
      if (!store_m) continue;                      // uniform over the grid
    }
    wfft1024<+1>(v, lane, S, twf);                 // kx -> x
    cx<float>* Mr = (cx<float>*)a.M + ((b * 3 + c) * P + iy) * (long)N;
#pragma unroll
    for (int p = 0; p < 32; ++p) Mr[lane + 32 * p] = v[p];
  }
}

}  // namespace kd
