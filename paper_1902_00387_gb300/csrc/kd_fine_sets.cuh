// Launch plans of the fine step: the kernel variants of every (precision, grid) and the
// step loop (kd_fine.h: fine_run).  Included by the instantiation units kd_fine2_*.cu
// and kd_fine3_*.cu.
//
// complex64 variants (complex128 has variant 0 only):
//   n <= 256  column: 0, 1 = four-step kernels with XT0, XT0/2 columns per block;
//                     2 = component-split four-step kernel (one component per thread);
//                     3 = three-pass kernel with 8 values per thread (n = 128, 256)
//             row:    0..3 = four-step kernels, (RT0 | RT0/2 rows) x (staged | registers);
//                     4, 5 = component-split kernels with 8 | 4 rows per block;
//                     6, 7 = three-pass, 8 values per thread, staged | registers (n = 128, 256)
//             both:   the next variant = the warp-owned mixed-radix kernels of kd_fine_mr.cuh
//                     (one warp per column / row with its three components; n = 32 .. 256);
//                     at n = 256 the last = the 256-point warp-transform kernels of
//                     kd_fine5.cuh (the row kernel for RK443)
//   n >= 512  column: 0, 1 = three-pass, 16 values per thread, XT0, XT0/2 columns;
//                     2 = persistent prefetching kernel; 3 = component-split kernel;
//                     4 = 8 values per thread (n = 512); 5 = 512-point warp transforms,
//                     one warp per column (kd_fine5.cuh; n = 512)
//             row:    0..3 = three-pass, 16 values, (RT0 | RT0/2) x (staged | registers);
//                     4 = persistent prefetching kernel (in registers);
//                     5, 6 = component-split kernels with RT0 | RT0/2 rows per block;
//                     7, 8 = 8 values per thread, staged | registers (n = 512);
//                     9 = 512-point warp transforms, one warp per component of a row
//                     (kd_fine5.cuh; n = 512)
//   n = 1024  column: 4 = warp-owned transforms (kd_fine4.cuh), one warp per component,
//                     4 columns per block; 5 = warp-owned transforms, one warp per column,
//                     8 columns per block; 6 = the same with two independent groups of
//                     4 columns per block
//             row:    7 = warp-owned transforms, one row per block
#pragma once
#include "kd_fine2c.cuh"
#include "kd_fine3.cuh"
#include "kd_fine3c.cuh"
#include "kd_fine2f.cuh"
#include "kd_fine4.cuh"
#include "kd_fine5.cuh"
#include "kd_fine_mr.cuh"

namespace kd {

// Launch `k` on stream st; with pdl the launch may overlap its predecessor's tail
// (programmatic dependent launch; the kernels synchronise with griddep_wait()).
template <typename... KArgs, typename... Args>
static void launch_k(void (*k)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st, bool pdl,
                     Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(block, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k, args...);
}

// The warp-owned mixed-radix kernels (kd_fine_mr.cuh) of the side 32 R as a launch plan
// (no shared memory to set up).
template <typename T, int R>
struct FineMrSet {
  static constexpr int N = 32 * R;
  static constexpr bool FUSED = false;
  static constexpr int kFusedCol = -1;
  static constexpr unsigned BLOCK = 32 * kMrWarps;
  static int ncol() { return 1; }
  static int nrow() { return 1; }
  static unsigned blocks(long warps) { return (unsigned)((warps + kMrWarps - 1) / kMrWarps); }
  static void col(int, const FineArgs& a, int s, int j, cudaStream_t st, bool pdl) {
    launch_k(colmr_kernel<T, R>, blocks((long)a.batch * N), BLOCK, 0, st, pdl, a, s, j);
  }
  template <int SCH, int MODE>
  static void row_k(const FineArgs& a, int store, cudaStream_t st, bool pdl) {
    launch_k(rowmr_kernel<T, R, SCH, MODE>, blocks((long)a.batch * a.P), BLOCK, 0, st, pdl, a, store);
  }
  static void row(int, const FineArgs& a, int mode, int store, cudaStream_t st, bool pdl) {
    if (mode == 4) return row_k<SCHEME_RK443, 4>(a, store, st, pdl);   // prologue (scheme-free)
    if (a.scheme == SCHEME_RK111) return row_k<SCHEME_RK111, 0>(a, store, st, pdl);
    if (a.scheme == SCHEME_RK222)
      return mode == 0 ? row_k<SCHEME_RK222, 0>(a, store, st, pdl) : row_k<SCHEME_RK222, 1>(a, store, st, pdl);
    switch (mode) {
      case 0: return row_k<SCHEME_RK443, 0>(a, store, st, pdl);
      case 1: return row_k<SCHEME_RK443, 1>(a, store, st, pdl);
      case 2: return row_k<SCHEME_RK443, 2>(a, store, st, pdl);
      default: return row_k<SCHEME_RK443, 3>(a, store, st, pdl);
    }
  }
};

// Warp-transform kernels of the n = 512 and 256 complex64 grids (kd_fine5.cuh).
template <int N>
static void launch_colw(const FineArgs& a, int s, int j, cudaStream_t st, bool pdl) {
  using C = ColW<N>;
  const long groups = (long)a.batch * (N / C::XG);
  const long cap = (long)persistent_grid(1L << 30) * C::MINB;
  launch_k(colw_kernel<N>, (unsigned)(groups < cap ? groups : cap), C::BLOCK, C::smem, st, pdl, a, s, j);
}

template <int N, int MODE>
static void launch_roww_mode(const FineArgs& a, int store, cudaStream_t st, bool pdl) {
  using G = RowW<N, MODE>;
  const long rows = (long)a.batch * a.P;
  const long cap = (long)persistent_grid(1L << 30) * G::MINB;
  launch_k(roww_kernel<N, MODE>, (unsigned)(rows < cap ? rows : cap), G::BLOCK, G::smem, st, pdl, a, store);
}

template <int N>
static void launch_roww(const FineArgs& a, int mode, int store, cudaStream_t st, bool pdl) {
  switch (mode) {
    case 0: return launch_roww_mode<N, 0>(a, store, st, pdl);
    case 1: return launch_roww_mode<N, 1>(a, store, st, pdl);
    case 2: return launch_roww_mode<N, 2>(a, store, st, pdl);
    case 3: return launch_roww_mode<N, 3>(a, store, st, pdl);
    default: return launch_roww_mode<N, 4>(a, store, st, pdl);
  }
}

template <int N>
static cudaError_t prepare_w() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(colw_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ColW<N>::smem)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(roww_kernel<N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)RowW<N, 0>::smem)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(roww_kernel<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)RowW<N, 1>::smem)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(roww_kernel<N, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)RowW<N, 2>::smem)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(roww_kernel<N, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)RowW<N, 3>::smem)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(roww_kernel<N, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RowW<N, 4>::smem);
}

template <typename T, int N, int XT>
static cudaError_t prepare_col2() {
  return cudaFuncSetAttribute(col2_kernel<T, N, XT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Col2<T, N, XT>::smem);
}

template <typename T, int N, int RT, bool STAGED, int SCH = SCHEME_RK443>
static cudaError_t prepare_row2() {
  return cudaFuncSetAttribute(row2_kernel<T, N, RT, STAGED, SCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Row2<T, N, RT, STAGED ? 128 : 168>::smem);
}

template <typename T, int N, int XT>
static void launch_col2(const FineArgs& a, int s, int j, cudaStream_t st, bool pdl) {
  using C = Col2<T, N, XT>;
  const unsigned gc = (unsigned)(((long)a.batch * N + XT - 1) / XT);
  launch_k(col2_kernel<T, N, XT>, gc, C::BLOCK, C::smem, st, pdl, a, s, j);
}

template <typename T, int N, int RT, bool STAGED, int SCH = SCHEME_RK443>
static void launch_row2(const FineArgs& a, int mode, int store, cudaStream_t st, bool pdl) {
  using R = Row2<T, N, RT, STAGED ? 128 : 168>;
  const unsigned gr = (unsigned)(((long)a.batch * a.P + RT - 1) / RT);
  launch_k(row2_kernel<T, N, RT, STAGED, SCH>, gr, R::BLOCK, R::smem, st, pdl, a, mode, store);
}

template <typename T, int N, int XT, int R>
static cudaError_t prepare_col3() {
  return cudaFuncSetAttribute(col3_kernel<T, N, XT, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Col3<T, N, XT, R>::smem);
}

template <typename T, int N, int RT, bool STAGED, int R, int SCH = SCHEME_RK443>
static cudaError_t prepare_row3() {
  return cudaFuncSetAttribute(row3_kernel<T, N, RT, STAGED, R, SCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Row3<T, N, RT, STAGED ? 128 : 168, R>::smem);
}

template <typename T, int N, int XT, int R>
static void launch_col3(const FineArgs& a, int s, int j, cudaStream_t st, bool pdl) {
  using C = Col3<T, N, XT, R>;
  const unsigned gc = (unsigned)(((long)a.batch * N + XT - 1) / XT);
  launch_k(col3_kernel<T, N, XT, R>, gc, C::BLOCK, C::smem, st, pdl, a, s, j);
}

template <typename T, int N, int RT, bool STAGED, int R, int SCH = SCHEME_RK443>
static void launch_row3(const FineArgs& a, int mode, int store, cudaStream_t st, bool pdl) {
  using G = Row3<T, N, RT, STAGED ? 128 : 168, R>;
  const unsigned gr = (unsigned)(((long)a.batch * a.P + RT - 1) / RT);
  launch_k(row3_kernel<T, N, RT, STAGED, R, SCH>, gr, G::BLOCK, G::smem, st, pdl, a, mode, store);
}

// 8-values-per-thread shapes: 256-thread blocks
template <int N>
struct Shapes8 {
  static constexpr int TPT = N / 8;
  static constexpr int XT = 256 / TPT, RT = 256 / TPT;
};

template <typename T, int N, int XT>
static void launch_col2c(const FineArgs& a, int s, int j, cudaStream_t st, bool pdl) {
  using C = Col2C<T, N, XT>;
  const unsigned gc = (unsigned)(((long)a.batch * N + XT - 1) / XT);
  launch_k(col2c_kernel<T, N, XT>, gc, C::BLOCK, C::smem, st, pdl, a, s, j);
}

template <typename T, int N, int RT>
static void launch_row2c(const FineArgs& a, int mode, int store, cudaStream_t st, bool pdl) {
  using R = Row2C<T, N, RT>;
  const unsigned gr = (unsigned)(((long)a.batch * a.P + RT - 1) / RT);
  launch_k(row2c_kernel<T, N, RT>, gr, R::BLOCK, R::smem, st, pdl, a, mode, store);
}

// component-split shapes
template <int N>
struct ShapesC {
  static constexpr int XT = N <= 64 ? 32 : 16;
  static constexpr int RT0 = 8, RT1 = 4;
};

template <typename T, int N>
struct Fine2Set {
  using Sh = Shapes2<T, N>;
  using ShC = ShapesC<N>;
  static constexpr bool WIDE = sizeof(T) == 4;
  static constexpr bool R8 = WIDE && (N == 128 || N == 256);
  // FP32 n = 128: column variant 4 is the persistent 2-block fused step (the row
  // variant does not apply)
  static constexpr bool FUSED = WIDE && N == 128;
  static constexpr int kFusedCol = 4;
  // the warp-owned mixed-radix kernels (FineMrSet) as a further column / row variant of
  // the sides 32 R, complex64 (complex128 keeps one plan: the serial fine run, tuned for
  // one field, and the batched sweeps then take the same kernels, so a Parareal run of N
  // iterations reproduces the serial fine run bit for bit)
  static constexpr bool MR = WIDE && N % 32 == 0;
  // complex64 n = 256 and 128: the warp-transform kernels (kd_fine5.cuh) after that
  static constexpr bool WT = WIDE && (N == 256 || N == 128);
  static int ncol0() { return WIDE ? (R8 ? (FUSED ? 5 : 4) : 3) : 1; }
  static int nrow0() { return WIDE ? (R8 ? 8 : 6) : 1; }
  static int ncol() { return ncol0() + (MR ? 1 : 0) + (WT ? 1 : 0); }
  static int nrow() { return nrow0() + (MR ? 1 : 0) + (WT ? 1 : 0); }
  // plan of a context that is not autotuned: the warp-transform row kernel with the
  // four-step column kernel (n = 256) or its second tile shape (n = 128), measured fastest
  // of the fixed plans
  static FinePlan default_plan() {
    FinePlan p;
    if (WT) p.row = nrow0() + 1;
    if (WT && N == 128) p.col = 1;
    return p;
  }
  static cudaError_t prepare() {
    cudaError_t e;
    if ((e = prepare_col2<T, N, Sh::xt(0)>()) != cudaSuccess) return e;
    if ((e = prepare_row2<T, N, Sh::rt(0), true>()) != cudaSuccess) return e;
    if ((e = prepare_row2<T, N, Sh::rt(0), true, SCHEME_RK222>()) != cudaSuccess) return e;
    if ((e = prepare_row2<T, N, Sh::rt(0), true, SCHEME_RK111>()) != cudaSuccess) return e;
    if (WIDE) {
      if ((e = prepare_col2<T, N, Sh::xt(1)>()) != cudaSuccess) return e;
      if ((e = prepare_row2<T, N, Sh::rt(1), true>()) != cudaSuccess) return e;
      if ((e = prepare_row2<T, N, Sh::rt(0), false>()) != cudaSuccess) return e;
      if ((e = prepare_row2<T, N, Sh::rt(1), false>()) != cudaSuccess) return e;
    }
    if constexpr (WIDE) {
      if ((e = cudaFuncSetAttribute(col2c_kernel<T, N, ShC::XT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)Col2C<T, N, ShC::XT>::smem)) != cudaSuccess)
        return e;
      if ((e = cudaFuncSetAttribute(row2c_kernel<T, N, ShC::RT0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)Row2C<T, N, ShC::RT0>::smem)) != cudaSuccess)
        return e;
      if ((e = cudaFuncSetAttribute(row2c_kernel<T, N, ShC::RT1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)Row2C<T, N, ShC::RT1>::smem)) != cudaSuccess)
        return e;
    }
    if constexpr (FUSED) {
      if ((e = cudaFuncSetAttribute(fused128_kernel<>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)Fused128::smem)) != cudaSuccess)
        return e;
    }
    if constexpr (R8) {
      if ((e = prepare_col3<T, N, Shapes8<N>::XT, 8>()) != cudaSuccess) return e;
      if ((e = prepare_row3<T, N, Shapes8<N>::RT, true, 8>()) != cudaSuccess) return e;
      if ((e = prepare_row3<T, N, Shapes8<N>::RT, false, 8>()) != cudaSuccess) return e;
    }
    if constexpr (WT) {
      if ((e = prepare_w<N>()) != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  static void col(int v, const FineArgs& a, int s, int j, cudaStream_t st, bool pdl) {
    if constexpr (MR) {
      if (v == ncol0()) return FineMrSet<T, N / 32>::col(0, a, s, j, st, pdl);
    }
    if constexpr (WT) {
      if (v == ncol0() + 1) return launch_colw<N>(a, s, j, st, pdl);
    }
    if constexpr (WIDE) {
      if (v == 2) return launch_col2c<T, N, ShC::XT>(a, s, j, st, pdl);
    }
    if constexpr (R8) {
      if (v == 3) return launch_col3<T, N, Shapes8<N>::XT, 8>(a, s, j, st, pdl);
    }
    if (WIDE && v == 1)
      launch_col2<T, N, Sh::xt(1)>(a, s, j, st, pdl);
    else
      launch_col2<T, N, Sh::xt(0)>(a, s, j, st, pdl);
  }
  static void row(int v, const FineArgs& a, int mode, int store, cudaStream_t st, bool pdl) {
    if constexpr (MR) {
      if (v == nrow0()) return FineMrSet<T, N / 32>::row(0, a, mode, store, st, pdl);   // every scheme
    }
    if constexpr (WT) {   // RK443 only; the lower-order schemes take the default row kernel below
      if (v == nrow0() + 1 && a.scheme == SCHEME_RK443) return launch_roww<N>(a, mode, store, st, pdl);
    }
    if (!WIDE) v = 0;
    // the lower-order schemes run on the default row kernel (prologue included)
    if (a.scheme == SCHEME_RK222) return launch_row2<T, N, Sh::rt(0), true, SCHEME_RK222>(a, mode, store, st, pdl);
    if (a.scheme == SCHEME_RK111) return launch_row2<T, N, Sh::rt(0), true, SCHEME_RK111>(a, mode, store, st, pdl);
    if constexpr (WIDE) {
      if (v == 4) return launch_row2c<T, N, ShC::RT0>(a, mode, store, st, pdl);
      if (v == 5) return launch_row2c<T, N, ShC::RT1>(a, mode, store, st, pdl);
    }
    if constexpr (R8) {
      if (v == 6) return launch_row3<T, N, Shapes8<N>::RT, true, 8>(a, mode, store, st, pdl);
      if (v == 7) return launch_row3<T, N, Shapes8<N>::RT, false, 8>(a, mode, store, st, pdl);
    }
    switch (v) {
      case 1: launch_row2<T, N, Sh::rt(1), true>(a, mode, store, st, pdl); break;
      case 2: launch_row2<T, N, Sh::rt(0), false>(a, mode, store, st, pdl); break;
      case 3: launch_row2<T, N, Sh::rt(1), false>(a, mode, store, st, pdl); break;
      default: launch_row2<T, N, Sh::rt(0), true>(a, mode, store, st, pdl); break;
    }
  }
};

template <typename T, int N, int XT>
static void launch_col3c(const FineArgs& a, int s, int j, cudaStream_t st, bool pdl) {
  using C = Col3C<T, N, XT>;
  const unsigned gc = (unsigned)(((long)a.batch * N + XT - 1) / XT);
  launch_k(col3c_kernel<T, N, XT>, gc, C::BLOCK, C::smem, st, pdl, a, s, j);
}

template <typename T, int N, int RT>
static void launch_row3c(const FineArgs& a, int mode, int store, cudaStream_t st, bool pdl) {
  using R = Row3C<T, N, RT>;
  const unsigned gr = (unsigned)(((long)a.batch * a.P + RT - 1) / RT);
  launch_k(row3c_kernel<T, N, RT>, gr, R::BLOCK, R::smem, st, pdl, a, mode, store);
}

// Warp-transform kernels (kd_fine4.cuh) of the n = 1024 complex64 grid: the row kernel
// runs one row per block, 5 blocks per SM.
#ifndef KD_COL4_COPY
#define KD_COL4_COPY 16
#endif
constexpr int kRow4Rows = 1, kCol4Copy = KD_COL4_COPY;

template <int N, int MODE>
static void launch_row4(const FineArgs& a, int store, cudaStream_t st, bool pdl) {
  using G = Row4<N, kRow4Rows, MODE>;
  const long blocks = ((long)a.batch * a.P + kRow4Rows - 1) / kRow4Rows;
  const long cap = (long)persistent_grid(1L << 30) * G::MINB;
  launch_k(row4_kernel<N, kRow4Rows, MODE>, (unsigned)(blocks < cap ? blocks : cap), G::BLOCK, G::smem, st, pdl, a,
           store);
}

template <int N, int MODE>
static cudaError_t prepare_row4() {
  using G = Row4<N, kRow4Rows, MODE>;
  return cudaFuncSetAttribute(row4_kernel<N, kRow4Rows, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)G::smem);
}

template <typename T, int N>
struct Fine3Set {
  using Sh = Shapes3<T, N>;
  static constexpr bool WIDE = sizeof(T) == 4;
  static constexpr bool R8 = WIDE && N == 512;
  static constexpr bool W4 = WIDE && N == 1024;
  static constexpr int kW4Col = 4, kW5Col = 5, kW6Col = 6, kW4Row = kRow4Variant;
  // n = 512: column variant 5 and row variant 9 are the 512-point warp-transform kernels
  static constexpr int kC512Col = 5, kC512Row = 9;
  static constexpr int XTC = Sh::XT0, RTC0 = Sh::RT0, RTC1 = Sh::RT0 / 2;
  static constexpr bool FUSED = false;   // no persistent fused step at these sizes
  static constexpr int kFusedCol = -1;
  static int ncol() { return WIDE ? (R8 ? 6 : (W4 ? 7 : 4)) : 1; }
  // plan of a context that is not autotuned: the warp-transform kernels where they exist
  static FinePlan default_plan() {
    FinePlan p;
    if (W4) {
      p.col = kW6Col;
      p.row = kW4Row;
    } else if (R8) {
      p.col = kC512Col;
      p.row = kC512Row;
    }
    return p;
  }
  static int nrow() { return WIDE ? (R8 ? 10 : (W4 ? 8 : 7)) : 1; }
  static cudaError_t prepare() {
    cudaError_t e;
    if constexpr (R8) {
      if ((e = prepare_w<N>()) != cudaSuccess) return e;
    }
    if constexpr (W4) {
      if ((e = cudaFuncSetAttribute(col4_kernel<N, kCol4Copy>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)Col4<N, kCol4Copy>::smem)) != cudaSuccess)
        return e;
      if ((e = cudaFuncSetAttribute(col5_kernel<N, 8, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)Col5<N, 8, 1>::smem)) != cudaSuccess)
        return e;
      if ((e = cudaFuncSetAttribute(col5_kernel<N, 4, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)Col5<N, 4, 2>::smem)) != cudaSuccess)
        return e;
      if ((e = prepare_row4<N, 0>()) != cudaSuccess) return e;
      if ((e = prepare_row4<N, 1>()) != cudaSuccess) return e;
      if ((e = prepare_row4<N, 2>()) != cudaSuccess) return e;
      if ((e = prepare_row4<N, 3>()) != cudaSuccess) return e;
      if ((e = prepare_row4<N, 4>()) != cudaSuccess) return e;
    }
    if ((e = prepare_col3<T, N, Sh::xt(0), 16>()) != cudaSuccess) return e;
    if ((e = prepare_row3<T, N, Sh::rt(0), true, 16>()) != cudaSuccess) return e;
    if ((e = prepare_row3<T, N, Sh::rt(0), true, 16, SCHEME_RK222>()) != cudaSuccess) return e;
    if ((e = prepare_row3<T, N, Sh::rt(0), true, 16, SCHEME_RK111>()) != cudaSuccess) return e;
    if (WIDE) {
      if ((e = prepare_col3<T, N, Sh::xt(1), 16>()) != cudaSuccess) return e;
      if ((e = prepare_row3<T, N, Sh::rt(1), true, 16>()) != cudaSuccess) return e;
      if ((e = prepare_row3<T, N, Sh::rt(0), false, 16>()) != cudaSuccess) return e;
      if ((e = prepare_row3<T, N, Sh::rt(1), false, 16>()) != cudaSuccess) return e;
      if ((e = cudaFuncSetAttribute(col3p_kernel<T, N, Sh::XT0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)Col3P<T, N, Sh::XT0>::smem)) != cudaSuccess)
        return e;
      if ((e = cudaFuncSetAttribute(row3p_kernel<T, N, Sh::RT0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)Row3P<T, N, Sh::RT0>::smem)) != cudaSuccess)
        return e;
    }
    if constexpr (WIDE) {
      if ((e = cudaFuncSetAttribute(col3c_kernel<T, N, XTC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)Col3C<T, N, XTC>::smem)) != cudaSuccess)
        return e;
      if ((e = cudaFuncSetAttribute(row3c_kernel<T, N, RTC0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)Row3C<T, N, RTC0>::smem)) != cudaSuccess)
        return e;
      if ((e = cudaFuncSetAttribute(row3c_kernel<T, N, RTC1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)Row3C<T, N, RTC1>::smem)) != cudaSuccess)
        return e;
    }
    if constexpr (R8) {
      if ((e = prepare_col3<T, N, Shapes8<N>::XT, 8>()) != cudaSuccess) return e;
      if ((e = prepare_row3<T, N, Shapes8<N>::RT, true, 8>()) != cudaSuccess) return e;
      if ((e = prepare_row3<T, N, Shapes8<N>::RT, false, 8>()) != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  static void col(int v, const FineArgs& a, int s, int j, cudaStream_t st, bool pdl) {
    if constexpr (W4) {
      if (v == kW5Col) {
        using C5 = Col5<N, 8, 1>;
        launch_k(col5_kernel<N, 8, 1>, persistent_grid((long)a.batch * (N / C5::XG)), C5::BLOCK, C5::smem, st, pdl,
                 a, s, j);
        return;
      }
      if (v == kW6Col) {
        using C6 = Col5<N, 4, 2>;
        const long groups = (long)a.batch * (N / C6::XG);
        launch_k(col5_kernel<N, 4, 2>, persistent_grid((groups + 1) / 2), C6::BLOCK, C6::smem, st, pdl, a, s, j);
        return;
      }
      if (v == kW4Col) {
        using C4 = Col4<N, kCol4Copy>;
        launch_k(col4_kernel<N, kCol4Copy>, persistent_grid((long)a.batch * (N / C4::XG)), C4::BLOCK, C4::smem, st,
                 pdl, a, s, j);
        return;
      }
    }
    if constexpr (WIDE) {
      if (v == 3) return launch_col3c<T, N, XTC>(a, s, j, st, pdl);
    }
    if constexpr (R8) {
      if (v == 4) return launch_col3<T, N, Shapes8<N>::XT, 8>(a, s, j, st, pdl);
      if (v == kC512Col) return launch_colw<N>(a, s, j, st, pdl);
    }
    if (WIDE && v == 2) {
      using C = Col3P<T, N, Sh::XT0>;
      launch_k(col3p_kernel<T, N, Sh::XT0>, persistent_grid((long)a.batch * N / Sh::XT0), C::BLOCK, C::smem, st, pdl,
               a, s, j);
    } else if (WIDE && v == 1) {
      launch_col3<T, N, Sh::xt(1), 16>(a, s, j, st, pdl);
    } else {
      launch_col3<T, N, Sh::xt(0), 16>(a, s, j, st, pdl);
    }
  }
  static void row(int v, const FineArgs& a, int mode, int store, cudaStream_t st, bool pdl) {
    if (!WIDE) v = 0;
    if (a.scheme == SCHEME_RK222) return launch_row3<T, N, Sh::rt(0), true, 16, SCHEME_RK222>(a, mode, store, st, pdl);
    if (a.scheme == SCHEME_RK111) return launch_row3<T, N, Sh::rt(0), true, 16, SCHEME_RK111>(a, mode, store, st, pdl);
    if constexpr (W4) {
      if (v == kW4Row) {
        switch (mode) {
          case 0: return launch_row4<N, 0>(a, store, st, pdl);
          case 1: return launch_row4<N, 1>(a, store, st, pdl);
          case 2: return launch_row4<N, 2>(a, store, st, pdl);
          case 3: return launch_row4<N, 3>(a, store, st, pdl);
          default: return launch_row4<N, 4>(a, store, st, pdl);
        }
      }
    }
    if constexpr (WIDE) {
      if (v == 5) return launch_row3c<T, N, RTC0>(a, mode, store, st, pdl);
      if (v == 6) return launch_row3c<T, N, RTC1>(a, mode, store, st, pdl);
    }
    if constexpr (R8) {
      if (v == 7) return launch_row3<T, N, Shapes8<N>::RT, true, 8>(a, mode, store, st, pdl);
      if (v == 8) return launch_row3<T, N, Shapes8<N>::RT, false, 8>(a, mode, store, st, pdl);
      if (v == kC512Row) return launch_roww<N>(a, mode, store, st, pdl);
    }
    if (v == 4 && mode == 4) v = 0;   // the prologue runs on the tiled kernel
    if (v == 4) {
      using G = Row3P<T, N, Sh::RT0>;
      const long tiles = ((long)a.batch * a.P + Sh::RT0 - 1) / Sh::RT0;
      launch_k(row3p_kernel<T, N, Sh::RT0>, persistent_grid(tiles), G::BLOCK, G::smem, st, pdl, a, mode, store);
      return;
    }
    switch (v) {
      case 1: launch_row3<T, N, Sh::rt(1), true, 16>(a, mode, store, st, pdl); break;
      case 2: launch_row3<T, N, Sh::rt(0), false, 16>(a, mode, store, st, pdl); break;
      case 3: launch_row3<T, N, Sh::rt(1), false, 16>(a, mode, store, st, pdl); break;
      default: launch_row3<T, N, Sh::rt(0), true, 16>(a, mode, store, st, pdl); break;
    }
  }
};

// The step loop shared by both kernel families.
template <class Set>
static int run_steps(const FineArgs& a0, const StepCfg& cfg) {
  const FinePlan pl = cfg.plan;
  int cv = pl.col >= 0 && pl.col < Set::ncol() ? pl.col : 0;
  if constexpr (Set::FUSED) {
    if (cv == Set::kFusedCol) cv = 0;   // (only for the calls the fused step does not cover)
  }
  const int rv = pl.row >= 0 && pl.row < Set::nrow() ? pl.row : 0;
  int launches = 0;
  if constexpr (Set::FUSED) {
    // the persistent fused step: every step of every field in one launch (RK443, from X,
    // no mixed field kept at the end, all fields for all steps)
    if (pl.col == Set::kFusedCol && cfg.prologue && !cfg.store_last && !cfg.active &&
        a0.scheme == SCHEME_RK443 && cfg.nsteps > 0) {
      FineArgs af = a0;
      af.lo_valid = 0;
      launch_k(fused128_kernel<>, (unsigned)(2 * a0.batch), Fused128::THREADS, Fused128::smem, cfg.st, cfg.pdl, af,
               cfg.nsteps);
      return 1;
    }
  }
  if (cfg.prologue) {
    Set::row(rv, a0, 4, 1, cfg.st, cfg.pdl);
    ++launches;
  }
  FineArgs a = a0;
  const int stages = scheme_stages(a0.scheme);
  for (int s = 0; s < cfg.nsteps; ++s) {
    a.lo_valid = s > 0;   // the low part of the state (kd_stage.cuh) exists from the second step
    // the caller's layout holds the state before the first step and receives it after the last
    a.x_in_full = s == 0 ? a0.x_in_full : nullptr;
    a.x_out_full = s == cfg.nsteps - 1 ? a0.x_out_full : nullptr;
    if (cfg.active) {
      a.batch = cfg.active[s];
      if (a.batch <= 0) break;
    }
    for (int j = 0; j < stages; ++j) {
      if (cfg.probe) cfg.probe->before(cfg.probe->user, 0);
      Set::col(cv, a, s, j, cfg.st, cfg.pdl);
      if (cfg.probe) cfg.probe->after(cfg.probe->user, 0);
      const int store = (s == cfg.nsteps - 1 && j == stages - 1) ? (cfg.store_last ? 1 : 0) : 1;
      if (cfg.probe) cfg.probe->before(cfg.probe->user, 1);
      Set::row(rv, a, j, store, cfg.st, cfg.pdl);
      if (cfg.probe) cfg.probe->after(cfg.probe->user, 1);
      launches += 2;
    }
  }
  return launches;
}

template <typename T, int N>
int fine2_run(const FineArgs& a, const StepCfg& cfg) {
  return run_steps<Fine2Set<T, N>>(a, cfg);
}

template <typename T, int N>
cudaError_t fine2_prep() {
  return Fine2Set<T, N>::prepare();
}

template <typename T, int N>
void fine2_variants(int* ncol, int* nrow) {
  *ncol = Fine2Set<T, N>::ncol();
  *nrow = Fine2Set<T, N>::nrow();
}

template <typename T, int N>
FinePlan fine2_default_plan() {
  return Fine2Set<T, N>::default_plan();
}

template <typename T, int N>
int fine3_run(const FineArgs& a, const StepCfg& cfg) {
  return run_steps<Fine3Set<T, N>>(a, cfg);
}

template <typename T, int N>
cudaError_t fine3_prep() {
  return Fine3Set<T, N>::prepare();
}

template <typename T, int N>
void fine3_variants(int* ncol, int* nrow) {
  *ncol = Fine3Set<T, N>::ncol();
  *nrow = Fine3Set<T, N>::nrow();
}

template <typename T, int N>
FinePlan fine3_default_plan() {
  return Fine3Set<T, N>::default_plan();
}

}  // namespace kd

// Explicit instantiation of one (T, N) in the including translation unit.
#define KD_FINE2_INSTANTIATE(T, N)                                        \
  template int kd::fine2_run<T, N>(const kd::FineArgs&, const kd::StepCfg&); \
  template cudaError_t kd::fine2_prep<T, N>();                             \
  template void kd::fine2_variants<T, N>(int*, int*);                       \
  template kd::FinePlan kd::fine2_default_plan<T, N>();
#define KD_FINE3_INSTANTIATE(T, N)                                        \
  template int kd::fine3_run<T, N>(const kd::FineArgs&, const kd::StepCfg&); \
  template cudaError_t kd::fine3_prep<T, N>();                             \
  template void kd::fine3_variants<T, N>(int*, int*);              \
  template kd::FinePlan kd::fine3_default_plan<T, N>();
