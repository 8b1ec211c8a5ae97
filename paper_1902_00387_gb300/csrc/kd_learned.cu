// Learned coarse propagator kernels (see kd_learned.h): layout maps between the
// learned mode set and the fine compact set, the BF16 GEMV used in the serial
// Parareal sweep, the BF16 tensor-core GEMM used for training, and the training
// helpers (residual and loss, gradient operand, Adam).
#include <cuda_bf16.h>
#include <math.h>

#include "kd_learned.h"

namespace kd {

namespace {

constexpr int TB = 256;

unsigned grid1(long total) {
  long g = (total + TB - 1) / TB;
  if (g < 1) g = 1;
  if (g > 65535L * 16) g = 65535L * 16;
  return (unsigned)g;
}

// fixed-order block reduction of two doubles; thread 0 writes out[0..1] (out[2*blockIdx])
__device__ __forceinline__ void block_sum2(double a, double b, double* out) {
  __shared__ double sa[TB / 32], sb[TB / 32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sa[threadIdx.x >> 5] = a;
    sb[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int w = 0; w < TB / 32; ++w) {
      x += sa[w];
      y += sb[w];
    }
    out[2 * blockIdx.x] = x;
    out[2 * blockIdx.x + 1] = y;
  }
}

}  // namespace

// ------------------------------------------------------------------ layouts
__global__ void k_lgather(const double* U, const double* Uprev, int Kf, int Pf, float* x, int K, int P, long total) {
  const long nc = 3L * P * P;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long b = i / nc;
    const int j = (int)(i - b * nc);
    const int c = j / (P * P), r = j - c * P * P;
    const int ky = r / P - K, kx = r % P - K;
    const long f = (b * 3 + c) * (long)Pf * Pf + (long)(ky + Kf) * Pf + (kx + Kf);
    double re = U[2 * f], im = U[2 * f + 1];
    if (Uprev) {
      re -= Uprev[2 * f];
      im -= Uprev[2 * f + 1];
    }
    x[2 * i] = (float)re;
    x[2 * i + 1] = (float)im;
  }
}

int learned_gather(const double* U, const double* Uprev, int Kf, int Pf, float* x, int K, int P, int batch,
                   cudaStream_t st) {
  const long total = (long)batch * 3 * P * P;
  k_lgather<<<grid1(total), TB, 0, st>>>(U, Uprev, Kf, Pf, x, K, P, total);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

__global__ void __launch_bounds__(TB) k_lupdate(const double* Fv, const float* y, int K, int P, double* U, int Kf,
                                                int Pf, int init, double* partials, long total) {
  double acc_d = 0.0, acc_n = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i / ((long)Pf * Pf));
    const int r = (int)(i - (long)c * Pf * Pf);
    const int ky = r / Pf - Kf, kx = r % Pf - Kf;
    double gx = 0.0, gy = 0.0;
    if (ky >= -K && ky < P - K && kx >= -K && kx < P - K) {
      const long j = ((long)c * P + ky + K) * P + kx + K;
      gx = (double)y[2 * j];
      gy = (double)y[2 * j + 1];
    }
    const double ux = init ? gx : Fv[2 * i] + gx;
    const double uy = init ? gy : Fv[2 * i + 1] + gy;
    if (partials) {
      const double dx = ux - U[2 * i], dy = uy - U[2 * i + 1];
      acc_d += dx * dx + dy * dy;
      acc_n += ux * ux + uy * uy;
    }
    U[2 * i] = ux;
    U[2 * i + 1] = uy;
  }
  if (partials) block_sum2(acc_d, acc_n, partials);
}

int learned_update(const double* Fv, const float* y, int K, int P, double* Unext, int Kf, int Pf, int init,
                   double* partials, cudaStream_t st) {
  const long total = 3L * Pf * Pf;
  unsigned g = grid1(total);
  if (g > 1024) g = 1024;
  k_lupdate<<<g, TB, 0, st>>>(Fv, y, K, P, Unext, Kf, Pf, init, partials, total);
  cudaError_t e = cudaGetLastError();
  return e != cudaSuccess ? -(int)e : (int)g;
}

template <typename T>
__global__ void k_l2f(const float* x, int K, int P, cx<T>* X, int Kf, int Pf, long total) {
  const long fs = 3L * Pf * Pf, nc = 3L * P * P;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long b = i / fs;
    const int f = (int)(i - b * fs);
    const int c = f / (Pf * Pf), r = f - c * Pf * Pf;
    const int ky = r / Pf - Kf, kx = r % Pf - Kf;
    cx<T> v = mk(T(0), T(0));
    if (ky >= -K && ky < P - K && kx >= -K && kx < P - K) {
      const long j = b * nc + ((long)c * P + ky + K) * P + kx + K;
      v = mk((T)x[2 * j], (T)x[2 * j + 1]);
    }
    X[i] = v;
  }
}

template <typename T>
__global__ void k_f2l(const cx<T>* X, int Kf, int Pf, float* y, int K, int P, long total) {
  const long fs = 3L * Pf * Pf, nc = 3L * P * P;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long b = i / nc;
    const int j = (int)(i - b * nc);
    const int c = j / (P * P), r = j - c * P * P;
    const int ky = r / P - K, kx = r % P - K;
    const cx<T> v = X[b * fs + ((long)c * Pf + ky + Kf) * Pf + kx + Kf];
    y[2 * i] = (float)v.x;
    y[2 * i + 1] = (float)v.y;
  }
}

int learned_to_fine(const float* x, int K, int P, void* X, int prec, int Kf, int Pf, long batch, cudaStream_t st) {
  const long total = batch * 3 * (long)Pf * Pf;
  if (prec == 0)
    k_l2f<float><<<grid1(total), TB, 0, st>>>(x, K, P, (cx<float>*)X, Kf, Pf, total);
  else
    k_l2f<double><<<grid1(total), TB, 0, st>>>(x, K, P, (cx<double>*)X, Kf, Pf, total);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int fine_to_learned(const void* X, int prec, int Kf, int Pf, float* y, int K, int P, long batch, cudaStream_t st) {
  const long total = batch * 3 * (long)P * P;
  if (prec == 0)
    k_f2l<float><<<grid1(total), TB, 0, st>>>((const cx<float>*)X, Kf, Pf, y, K, P, total);
  else
    k_f2l<double><<<grid1(total), TB, 0, st>>>((const cx<double>*)X, Kf, Pf, y, K, P, total);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

__global__ void k_f32_f64(const float* x, double* d, long n2) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n2; i += (long)gridDim.x * blockDim.x)
    d[i] = (double)x[i];
}

int learned_f32_to_f64(const float* x, double* d, long n_complex, cudaStream_t st) {
  k_f32_f64<<<grid1(2 * n_complex), TB, 0, st>>>(x, d, 2 * n_complex);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

__global__ void k_f64_f32(const double* d, float* x, long n2) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n2; i += (long)gridDim.x * blockDim.x)
    x[i] = (float)d[i];
}

int learned_f64_to_f32(const double* d, float* x, long n_complex, cudaStream_t st) {
  k_f64_f32<<<grid1(2 * n_complex), TB, 0, st>>>(d, x, 2 * n_complex);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

__global__ void k_units(double* d, int nc, int j0, long total) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long t = i / nc;
    const int j = (int)(i - t * nc);
    d[2 * i] = (j == j0 + t) ? 1.0 : 0.0;
    d[2 * i + 1] = 0.0;
  }
}

int learned_unit_vectors(double* d, int nc, int j0, int count, cudaStream_t st) {
  const long total = (long)count * nc;
  k_units<<<grid1(total), TB, 0, st>>>(d, nc, j0, total);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

__global__ void k_columns(const double* g64, int nc, int ld, int j0, int count, float* W, long total) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    // i = row * count + t  (t fastest keeps the W stores of a warp on one row)
    const long row = i / count;
    const int t = (int)(i - row * count);
    const double re = g64[2 * ((long)t * nc + row)], im = g64[2 * ((long)t * nc + row) + 1];
    W[row * ld + j0 + t] = (float)re;
    W[(row + nc) * ld + j0 + t] = (float)im;
  }
}

int learned_columns(const double* g64, int nc, int ld, int j0, int count, float* W, cudaStream_t st) {
  const long total = (long)nc * count;
  k_columns<<<grid1(total), TB, 0, st>>>(g64, nc, ld, j0, count, W, total);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

// -------------------------------------------------------------------- GEMV
// One warp per output j: rows j (Re W) and nc + j (Im W), 8 BF16 per 16-byte load.
constexpr int GV_WARPS = 8;

__global__ void __launch_bounds__(GV_WARPS * 32)
k_gemv(const __nv_bfloat16* __restrict__ W, const float* __restrict__ x, float* __restrict__ y, int nc, int ld) {
  extern __shared__ __align__(16) float sx[];   // [2][ld]: re, im (zero beyond nc)
  const int f = blockIdx.y;
  const float* xf = x + 2L * f * nc;
  for (int i = threadIdx.x; i < ld; i += blockDim.x) {
    sx[i] = i < nc ? xf[2 * i] : 0.f;
    sx[ld + i] = i < nc ? xf[2 * i + 1] : 0.f;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * GV_WARPS + warp;
  if (j >= nc) return;
  const uint4* ra = (const uint4*)(W + (long)j * ld);
  const uint4* rb = (const uint4*)(W + (long)(nc + j) * ld);
  const int chunks = ld / 8;
  float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
#pragma unroll 4
  for (int q = lane; q < chunks; q += 32) {
    const uint4 va = __ldg(ra + q), vb = __ldg(rb + q);
    const __nv_bfloat162* pa = (const __nv_bfloat162*)&va;
    const __nv_bfloat162* pb = (const __nv_bfloat162*)&vb;
    const float* xr = sx + 8 * q;
    const float* xi = sx + ld + 8 * q;
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const float2 a2 = __bfloat1622float2(pa[h]), b2 = __bfloat1622float2(pb[h]);
      ar = fmaf(a2.x, xr[2 * h], fmaf(a2.y, xr[2 * h + 1], ar));
      ai = fmaf(a2.x, xi[2 * h], fmaf(a2.y, xi[2 * h + 1], ai));
      br = fmaf(b2.x, xr[2 * h], fmaf(b2.y, xr[2 * h + 1], br));
      bi = fmaf(b2.x, xi[2 * h], fmaf(b2.y, xi[2 * h + 1], bi));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    ar += __shfl_down_sync(0xffffffffu, ar, o);
    ai += __shfl_down_sync(0xffffffffu, ai, o);
    br += __shfl_down_sync(0xffffffffu, br, o);
    bi += __shfl_down_sync(0xffffffffu, bi, o);
  }
  if (lane == 0) {
    y[2L * f * nc + 2 * j] = ar - bi;
    y[2L * f * nc + 2 * j + 1] = br + ai;
  }
}

cudaError_t learned_gemv_prepare(int ld_max) {
  return cudaFuncSetAttribute(k_gemv, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * ld_max * (int)sizeof(float));
}

int learned_gemv(const __nv_bfloat16* W, const float* x, float* y, int nc, int ld, int batch, cudaStream_t st) {
  if (ld % 8 != 0 || ld < nc || batch <= 0) return -1;
  dim3 grid((unsigned)((nc + GV_WARPS - 1) / GV_WARPS), (unsigned)batch);
  k_gemv<<<grid, GV_WARPS * 32, 2 * ld * sizeof(float), st>>>(W, x, y, nc, ld);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

// -------------------------------------------------------------------- GEMM
// 128 x 128 block tile, BK = 32, 8 warps (2 x 4), warp tile 64 x 32; operands staged
// with cp.async (zero fill outside the matrix), fragments by ldmatrix, mma.sync
// m16n8k16 BF16 with FP32 accumulation.
constexpr int BM = 128, BN = 128, BK = 32, SKEW = 8, LDS = BK + SKEW;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool pred) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int sz = pred ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(sz));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ __forceinline__ void ldsm_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* p) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(s));
}

__device__ __forceinline__ void mma_bf16(float* d, const unsigned* a, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(256) k_gemm_tn(const __nv_bfloat16* __restrict__ A,
                                                 const __nv_bfloat16* __restrict__ Bt, float* __restrict__ C, int M,
                                                 int N, int K, int ldc) {
  __shared__ __align__(16) __nv_bfloat16 As[2][BM][LDS];
  __shared__ __align__(16) __nv_bfloat16 Bs[2][BN][LDS];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 2, wn = warp & 3;   // 2 x 4 warps
  const long m0 = (long)blockIdx.y * BM, n0 = (long)blockIdx.x * BN;
  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

  auto load_tile = [&](int buf, int k0) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int chunk = tid + t * 256;   // 512 chunks of 16 bytes per operand tile
      const int r = chunk >> 2, kc = (chunk & 3) * 8;
      const long gm = m0 + r, gn = n0 + r;
      const bool pa = gm < M && k0 + kc < K;
      const bool pb = gn < N && k0 + kc < K;
      cp_async16(&As[buf][r][kc], A + (pa ? gm * K + k0 + kc : 0), pa);
      cp_async16(&Bs[buf][r][kc], Bt + (pb ? gn * K + k0 + kc : 0), pb);
    }
    cp_async_commit();
  };

  const int ktiles = (K + BK - 1) / BK;
  load_tile(0, 0);
  for (int kt = 0; kt < ktiles; ++kt) {
    const int cur = kt & 1;
    cp_async_wait0();
    __syncthreads();
    if (kt + 1 < ktiles) load_tile(cur ^ 1, (kt + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      unsigned af[4][4], bf[4][2];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int row = wm * 64 + i * 16 + (lane & 15);
        const int col = kk + (lane >> 4) * 8;
        ldsm_x4(af[i][0], af[i][1], af[i][2], af[i][3], &As[cur][row][col]);
      }
#pragma unroll
      for (int j = 0; j < 4; j += 2) {
        // two n8 tiles: matrices (n0-7,k0-7), (n0-7,k8-15), (n8-15,k0-7), (n8-15,k8-15)
        const int nrow = wn * 32 + j * 8 + (lane & 7) + ((lane >> 4) << 3);
        const int col = kk + ((lane >> 3) & 1) * 8;
        ldsm_x4(bf[j][0], bf[j][1], bf[j + 1][0], bf[j + 1][1], &Bs[cur][nrow][col]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j][0], bf[j][1]);
    }
    __syncthreads();
  }
  // epilogue: c0,c1 at (row = lane/4, col = 2 (lane%4) + {0,1}), c2,c3 at row + 8
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const long row = m0 + wm * 64 + i * 16 + (lane >> 2) + h * 8;
        const long col = n0 + wn * 32 + j * 8 + (lane & 3) * 2;
        if (row < M) {
          if (col < N) C[row * ldc + col] = acc[i][j][2 * h];
          if (col + 1 < N) C[row * ldc + col + 1] = acc[i][j][2 * h + 1];
        }
      }
}

int gemm_bf16_tn(const __nv_bfloat16* A, const __nv_bfloat16* Bt, float* C, int M, int N, int K, int ldc,
                 cudaStream_t st) {
  if (K % 8 != 0 || M <= 0 || N <= 0 || (((uintptr_t)A) & 15) || (((uintptr_t)Bt) & 15)) return -1;
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM));
  k_gemm_tn<<<grid, 256, 0, st>>>(A, Bt, C, M, N, K, ldc);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

// ---------------------------------------------------------------- training
__global__ void k_pack_x(const float* x, int m, int nc, int ld, __nv_bfloat16* Xs, __nv_bfloat16* XtT, long total) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long n = i / ld;
    const int j = (int)(i - n * ld);
    const bool in = j < nc;
    const __nv_bfloat16 re = __float2bfloat16(in ? x[2 * (n * nc + j)] : 0.f);
    const __nv_bfloat16 im = __float2bfloat16(in ? x[2 * (n * nc + j) + 1] : 0.f);
    Xs[n * ld + j] = re;
    Xs[(m + n) * ld + j] = im;
    if (in) {
      XtT[(long)j * 2 * m + n] = re;
      XtT[(long)j * 2 * m + m + n] = im;
    }
  }
}

int learned_pack_x(const float* x, int m, int nc, int ld, __nv_bfloat16* Xs, __nv_bfloat16* XtT, cudaStream_t st) {
  const long total = (long)m * ld;
  k_pack_x<<<grid1(total), TB, 0, st>>>(x, m, nc, ld, Xs, XtT, total);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

__global__ void k_transpose_y(const float* y, int m, int nc, float* yT, long total) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long n = i / nc;
    const int j = (int)(i - n * nc);
    yT[2 * ((long)j * m + n)] = y[2 * i];
    yT[2 * ((long)j * m + n) + 1] = y[2 * i + 1];
  }
}

int learned_transpose_y(const float* y, int m, int nc, float* yT, cudaStream_t st) {
  const long total = (long)m * nc;
  k_transpose_y<<<grid1(total), TB, 0, st>>>(y, m, nc, yT, total);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

__global__ void __launch_bounds__(TB) k_residual(const float* C1, const float* yT, int m, int nc,
                                                 __nv_bfloat16* A2, double* partials, long total) {
  double acc = 0.0;
  const long m2 = 2L * m;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long j = i / m;
    const int n = (int)(i - j * m);
    const float pr = C1[j * m2 + n] - C1[(nc + j) * m2 + m + n];
    const float pi = C1[(nc + j) * m2 + n] + C1[j * m2 + m + n];
    const float rr = pr - yT[2 * i], ri = pi - yT[2 * i + 1];
    acc += (double)rr * rr + (double)ri * ri;
    A2[j * m2 + n] = __float2bfloat16(rr);
    A2[j * m2 + m + n] = __float2bfloat16(ri);
    A2[(nc + j) * m2 + n] = __float2bfloat16(ri);
    A2[(nc + j) * m2 + m + n] = __float2bfloat16(-rr);
  }
  if (partials) block_sum2(acc, 0.0, partials);
}

int learned_residual(const float* C1, const float* yT, int m, int nc, __nv_bfloat16* A2, double* partials,
                     cudaStream_t st) {
  const long total = (long)nc * m;
  unsigned g = grid1(total);
  if (g > 1024) g = 1024;
  k_residual<<<g, TB, 0, st>>>(C1, yT, m, nc, A2, partials, total);
  cudaError_t e = cudaGetLastError();
  return e != cudaSuccess ? -(int)e : (int)g;
}

__global__ void __launch_bounds__(TB) k_adam(float* W, const float* W0, const float* C2, float* m1, float* v,
                                             __nv_bfloat16* Wbf, long count, float scale, float wd, float lr, float b1,
                                             float b2, float eps, float c1, float c2, double* partials2) {
  double acc = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
    const float w = W[i];
    const float d0 = W0 ? w - W0[i] : w;
    const float g = scale * C2[i] + 2.f * wd * d0;
    const float mm = b1 * m1[i] + (1.f - b1) * g;
    const float vv = b2 * v[i] + (1.f - b2) * g * g;
    m1[i] = mm;
    v[i] = vv;
    const float wn = w - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    W[i] = wn;
    Wbf[i] = __float2bfloat16(wn);
    const float dn = W0 ? wn - W0[i] : wn;
    acc += (double)dn * dn;
  }
  if (partials2) block_sum2(acc, 0.0, partials2);
}

int learned_adam(float* W, const float* W0, const float* C2, float* m1, float* v, __nv_bfloat16* Wbf, long count,
                 float scale, float wd, float lr, float beta1, float beta2, float eps, int step, double* partials2,
                 cudaStream_t st) {
  unsigned g = grid1(count);
  if (g > 1024) g = 1024;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  k_adam<<<g, TB, 0, st>>>(W, W0, C2, m1, v, Wbf, count, scale, wd, lr, beta1, beta2, eps, c1, c2, partials2);
  cudaError_t e = cudaGetLastError();
  return e != cudaSuccess ? -(int)e : (int)g;
}

// heavy-ball gradient descent: v = mu v + g, W -= eta v (updates stay in the span of
// the gradients, i.e. of the training inputs, when started from W0 with wd = 0)
__global__ void k_momentum(float* W, const float* W0, const float* C2, float* v, __nv_bfloat16* Wbf, long count,
                           float scale, float wd, float eta, float mu) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
    const float w = W[i];
    const float g = scale * C2[i] + 2.f * wd * (W0 ? w - W0[i] : w);
    const float vv = mu * v[i] + g;
    v[i] = vv;
    const float wn = w - eta * vv;
    W[i] = wn;
    Wbf[i] = __float2bfloat16(wn);
  }
}

int learned_momentum(float* W, const float* W0, const float* C2, float* v, __nv_bfloat16* Wbf, long count,
                     float scale, float wd, float eta, float mu, cudaStream_t st) {
  k_momentum<<<grid1(count), TB, 0, st>>>(W, W0, C2, v, Wbf, count, scale, wd, eta, mu);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

__global__ void k_grad(const float* W, const float* W0, const float* C2, float* grad, long count, float scale,
                       float wd) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
    const float d0 = W0 ? W[i] - W0[i] : W[i];
    grad[i] = scale * C2[i] + 2.f * wd * d0;
  }
}

int learned_grad(const float* W, const float* W0, const float* C2, float* grad, long count, float scale, float wd,
                 cudaStream_t st) {
  k_grad<<<grid1(count), TB, 0, st>>>(W, W0, C2, grad, count, scale, wd);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

__global__ void k_f2bf(const float* x, __nv_bfloat16* y, long count) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

int f32_to_bf16(const float* x, __nv_bfloat16* y, long count, cudaStream_t st) {
  k_f2bf<<<grid1(count), TB, 0, st>>>(x, y, count);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

__global__ void __launch_bounds__(TB) k_sum(const double* p, int count, double* out) {
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < count; i += TB) {
    a += p[2 * i];
    b += p[2 * i + 1];
  }
  block_sum2(a, b, out);
}

int sum_partials(const double* p, int count, double* out, cudaStream_t st) {
  k_sum<<<1, TB, 0, st>>>(p, count, out);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

__global__ void __launch_bounds__(TB) k_diff_norms(const float* a, const float* b, long count, double* partials) {
  double d = 0.0, n = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
    const double x = (double)a[i] - (double)b[i];
    d += x * x;
    n += (double)b[i] * b[i];
  }
  block_sum2(d, n, partials);
}

int diff_norms(const float* a, const float* b, long count, double* partials, cudaStream_t st) {
  unsigned g = grid1(count);
  if (g > 1024) g = 1024;
  k_diff_norms<<<g, TB, 0, st>>>(a, b, count, partials);
  cudaError_t e = cudaGetLastError();
  return e != cudaSuccess ? -(int)e : (int)g;
}

// ------------------------------------------------------------ minimum-norm correction
// Gram matrix G[i][j] = x_i^H x_j of m learned vectors (complex FP32 [m][nc]), as complex
// FP64 [m][m].  A block computes a 16 x 16 tile; the products of a 32-wide chunk of the
// unknowns are summed in FP32 and the chunk sums in FP64.
constexpr int GT = 16, GK = 32;

__global__ void __launch_bounds__(GT * GT) k_gram(const float2* x, int m, int nc, double2* G) {
  __shared__ float2 xi[GT][GK + 1], xj[GT][GK + 1];
  const int ti = threadIdx.x / GT, tj = threadIdx.x % GT;
  const int i0 = blockIdx.y * GT, j0 = blockIdx.x * GT;
  double ar = 0.0, ai = 0.0;
  for (int k0 = 0; k0 < nc; k0 += GK) {
    for (int e = threadIdx.x; e < GT * GK; e += GT * GT) {
      const int r = e / GK, k = k0 + e % GK;
      const bool in = k < nc;
      xi[r][e % GK] = in && i0 + r < m ? x[(long)(i0 + r) * nc + k] : make_float2(0.f, 0.f);
      xj[r][e % GK] = in && j0 + r < m ? x[(long)(j0 + r) * nc + k] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float sr = 0.f, si = 0.f;
#pragma unroll 8
    for (int k = 0; k < GK; ++k) {
      const float2 a = xi[ti][k], b = xj[tj][k];   // conj(a) b
      sr = fmaf(a.x, b.x, fmaf(a.y, b.y, sr));
      si = fmaf(a.x, b.y, fmaf(-a.y, b.x, si));
    }
    ar += sr;
    ai += si;
    __syncthreads();
  }
  if (i0 + ti < m && j0 + tj < m) G[(long)(i0 + ti) * m + j0 + tj] = make_double2(ar, ai);
}

int learned_gram(const float* x, int m, int nc, double* G, cudaStream_t st) {
  const dim3 grid((m + GT - 1) / GT, (m + GT - 1) / GT);
  k_gram<<<grid, GT * GT, 0, st>>>((const float2*)x, m, nc, (double2*)G);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

// R[l] = y[l] - g[l], rounded to complex FP32 (g: FP64 classical outputs)
__global__ void k_resid64(const float* y, const double* g, float* R, long total) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x)
    R[i] = (float)((double)y[i] - g[i]);
}

int learned_resid64(const float* y, const double* g, float* R, long n_complex, cudaStream_t st) {
  k_resid64<<<grid1(2 * n_complex), TB, 0, st>>>(y, g, R, 2 * n_complex);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

// A_n = sum_{l < m} R_l Ginv[l][n] (complex FP32 sums) written as the gradient GEMM's left
// operand A2[2 nc][2 mp]: row j (Re A_n[j], Im A_n[j]), row nc + j (Im A_n[j], -Re A_n[j]);
// columns n in [m, mp) zero.  A block computes 16 n x 64 j; Ginv is FP32 complex [m][m].
constexpr int CJ = 64, CN = 16, CL = 16;

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16(v);
  lo = __float2bfloat16(v - __bfloat162float(hi));
}

__global__ void __launch_bounds__(256) k_minnorm_operand(const float2* R, const float2* Gi, int m, int mp, int nc,
                                                         __nv_bfloat16* A2, __nv_bfloat16* A2lo) {
  __shared__ float2 sR[CL][CJ], sG[CL][CN + 1];
  const int j0 = blockIdx.x * CJ, n0 = blockIdx.y * CN;
  const int tj = threadIdx.x % CJ, tn = threadIdx.x / CJ;   // 64 x 4 threads, 4 n each
  float2 acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q] = make_float2(0.f, 0.f);
  for (int l0 = 0; l0 < m; l0 += CL) {
    for (int e = threadIdx.x; e < CL * CJ; e += 256) {
      const int l = l0 + e / CJ, j = j0 + e % CJ;
      sR[e / CJ][e % CJ] = l < m && j < nc ? R[(long)l * nc + j] : make_float2(0.f, 0.f);
    }
    for (int e = threadIdx.x; e < CL * CN; e += 256) {
      const int l = l0 + e / CN, n = n0 + e % CN;
      sG[e / CN][e % CN] = l < m && n < m ? Gi[(long)l * m + n] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 4
    for (int l = 0; l < CL; ++l) {
      const float2 r = sR[l][tj];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 g = sG[l][tn * 4 + q];
        acc[q].x = fmaf(r.x, g.x, fmaf(-r.y, g.y, acc[q].x));
        acc[q].y = fmaf(r.x, g.y, fmaf(r.y, g.x, acc[q].y));
      }
    }
    __syncthreads();
  }
  const int j = j0 + tj;
  if (j >= nc) return;
  const long m2 = 2L * mp;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int n = n0 + tn * 4 + q;
    if (n >= mp) continue;
    const float2 a = n < m ? acc[q] : make_float2(0.f, 0.f);
    __nv_bfloat16 rh, rl, ih, il, mh, ml;
    split_bf16(a.x, rh, rl);
    split_bf16(a.y, ih, il);
    split_bf16(-a.x, mh, ml);
    A2[(long)j * m2 + n] = rh;
    A2[(long)j * m2 + mp + n] = ih;
    A2[(long)(nc + j) * m2 + n] = ih;
    A2[(long)(nc + j) * m2 + mp + n] = mh;
    A2lo[(long)j * m2 + n] = rl;
    A2lo[(long)j * m2 + mp + n] = il;
    A2lo[(long)(nc + j) * m2 + n] = il;
    A2lo[(long)(nc + j) * m2 + mp + n] = ml;
  }
}

int learned_minnorm_operand(const float* R, const float* Ginv, int m, int mp, int nc, __nv_bfloat16* A2,
                            __nv_bfloat16* A2lo, cudaStream_t st) {
  const dim3 grid((nc + CJ - 1) / CJ, (mp + CN - 1) / CN);
  k_minnorm_operand<<<grid, 256, 0, st>>>((const float2*)R, (const float2*)Ginv, m, mp, nc, A2, A2lo);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

// XtTlo: x - bf16(x) in BF16, laid out as learned_pack_x's XtT ([nc][2 m])
__global__ void k_pack_x_lo(const float* x, int m, int nc, __nv_bfloat16* XtTlo, long total) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long n = i / nc;
    const int j = (int)(i - n * nc);
    __nv_bfloat16 h, l;
    split_bf16(x[2 * i], h, l);
    XtTlo[(long)j * 2 * m + n] = l;
    split_bf16(x[2 * i + 1], h, l);
    XtTlo[(long)j * 2 * m + m + n] = l;
  }
}

int learned_pack_x_lo(const float* x, int m, int nc, __nv_bfloat16* XtTlo, cudaStream_t st) {
  const long total = (long)m * nc;
  k_pack_x_lo<<<grid1(total), TB, 0, st>>>(x, m, nc, XtTlo, total);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

// Wbf = bf16(W0 + D0 + D1 + D2) (stacked operators)
__global__ void k_add_bf16(const float* W0, const float* D0, const float* D1, const float* D2, __nv_bfloat16* Wbf,
                           long count) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x)
    Wbf[i] = __float2bfloat16(W0[i] + (D0[i] + (D1[i] + D2[i])));
}

int learned_add_bf16(const float* W0, const float* D0, const float* D1, const float* D2, __nv_bfloat16* Wbf,
                     long count, cudaStream_t st) {
  k_add_bf16<<<grid1(count), TB, 0, st>>>(W0, D0, D1, D2, Wbf, count);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace kd
