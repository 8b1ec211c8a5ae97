// Persistent fine propagator for n = 128, complex64, RK443: every step of a field in
// one launch, the field in a cluster of 2 thread blocks (Sec. 4's pseudo-spectral IMEX
// step: inverse FFT, u x b on the grid, forward FFT, curl, implicit diffusion).
//
// Block r of a field's cluster owns the kept ky rows [43 r, 43 r + 43) (42 for r = 1)
// and the physical x columns [64 r, 64 r + 64).  Its shared buffer B holds the mixed
// field for ALL kept ky rows and ITS x columns: B[c][ky][x - 64 r], complex64, rows
// padded to 65 entries, 133 KB.
// A stage is
//   column pass (block-local): for each own column, the kept ky values of the 3
//     components -> inverse y transform -> u x b at (x, y) -> forward y transform ->
//     kept ky, in place in B;
//   cluster barrier;
//   row pass: for each own ky row, the 128 x values come from the own B (own half) and
//     from the peer's B (distributed shared memory); forward x transform -> curl, IMEX
//     update (stage accumulators X, R2..R4 in global memory, as in the row kernels) ->
//     inverse x transform -> written back to both halves;
//   cluster barrier.
// Before the first step the row pass transforms X (the prologue of the two-kernel path).
// Rows of different blocks are disjoint, and columns within a block are disjoint, so
// the passes need no barrier between their reads and writes of B.  The transforms are
// the one-component register FFT of kd_fft2.cuh, one component at a time.  Each transform
// has its own shared exchange slots (the row and column passes reuse them), and its 8
// lanes are one warp's consecutive threads, so its exchange needs only warp barriers: the
// only block-wide barriers of a stage are the two cluster barriers.
#pragma once
#include <cooperative_groups.h>

#include "kd_fft2.cuh"
#include "kd_stage.cuh"

namespace kd {

struct Fused128 {
  static constexpr int N = 128, K = 42, P = 85;
  static constexpr int R1 = Split<N>::R1, R2 = Split<N>::R2;   // 16 values x 8 lanes a transform
  static constexpr int XH = 64;                                  // x columns per block
  static constexpr int XP = XH + 1;                              // padded row of B (no bank conflicts
                                                                 // between the lanes of a column)
  static constexpr int ROWS = 43;                                // ky rows of block 0 (42 for block 1)
  static constexpr int THREADS = 384;                            // 48 transforms at once
  static constexpr int SLOTS = THREADS / R2;                     // 48
  static constexpr int LS = R1 * (R2 + 1) + 4;                   // exchange slots of one transform (the
                                                                 // 4 transforms of a warp on different banks)
  static constexpr size_t buf_bytes = (size_t)3 * P * XP * 8;    // 132,600
  static constexpr size_t smem = buf_bytes + (size_t)SLOTS * LS * 8 + (size_t)N * 8 + 2 * (size_t)N * 4;
};

template <int SCH = SCHEME_RK443>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(Fused128::THREADS, 1)
    fused128_kernel(FineArgs a, int nsteps) {
  using T = float;
  using F = Fused128;
  constexpr int N = F::N, R1 = F::R1, R2 = F::R2, XH = F::XH, XP = F::XP;
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* B = (cx<T>*)smem_raw;                                 // [3][P][XP]
  cx<T>* X_s = B + 3 * F::P * XP;                              // [SLOTS][LS] exchange slots
  cx<T>* s_tw = X_s + F::SLOTS * F::LS;                        // [N]
  T* s_cos = (T*)(s_tw + N);
  T* s_sin = s_cos + N;
  fft2_tables<T, N>(s_tw, (const cx<T>*)a.tw);
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    s_cos[i] = ((const T*)a.cosg)[i];
    s_sin[i] = ((const T*)a.sing)[i];
  }
  const int r = (int)cluster.block_rank();
  const long b = blockIdx.x / 2;                               // field of this cluster
  cx<T>* Bpeer = cluster.map_shared_rank(B, r ^ 1);
  const int slot = threadIdx.x / R2, lane = threadIdx.x % R2;
  cx<T>* my_slots = X_s + slot * F::LS;
  auto S = [&](int q, int a2) { return my_slots + q * (R2 + 1) + a2; };
  const int K = F::K, P = F::P;
  const long PP = (long)P * P;
  // the ky row of this thread's row transform (kept index), valid for slot < rows
  const int rows = r == 0 ? F::ROWS : P - F::ROWS;
  const bool row_valid = slot < rows;
  const int iy = r * F::ROWS + (row_valid ? slot : 0);
  const T inv_n2 = T(1) / (T(N) * T(N));
  StageArrays<T> sa = stage_arrays<T>(a);
  const StageCoef<T> q = stage_coef<T>(a, b);
  const T A = flow_amp<T>(a, b);
  const long s0 = ((b * 3) * P + iy) * (long)P + K;            // compact index of (iy, kx = 0), component 0
  const T fky = (T)(iy - K);
  // element (c, ky, x) of the mixed field, in the block that owns column x
  auto mixed = [&](int c, int ky, int x) -> cx<T>* {
    cx<T>* base = (x / XH) == r ? B : Bpeer;
    return base + ((long)c * P + ky) * XP + (x % XH);
  };
  cx<T> v[3][R1];

  // one-component transforms of v[0..2] through this transform's own exchange slots: its 8
  // lanes are consecutive threads of one warp, so warp barriers order the exchange
  auto transform3 = [&](auto dir) {
    constexpr int DIR = decltype(dir)::value;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      fft2_1<T, N, DIR, decltype(S), true>(v[c], lane, s_tw, S);
      __syncwarp();   // the slots are written again by the next component
    }
  };
  // inverse x transform of v (kept kx in input order) and its store into both halves
  auto row_inverse_store = [&]() {
    transform3(std::integral_constant<int, +1>());
    if (row_valid) {
#pragma unroll
      for (int k = 0; k < R1; ++k) {
        const int xx = lane + FFT2<N>::out_pos_base(k);
#pragma unroll
        for (int c = 0; c < 3; ++c) *mixed(c, iy, xx) = v[c][k];
      }
    }
  };

  griddep_wait();   // X comes from the predecessor
  // prologue: mixed field of stage 0 from X
  {
    const cx<T>* X = (const cx<T>*)a.X;
#pragma unroll
    for (int k = 0; k < R1; ++k) {
      const int xx = lane + R2 * k;
      const int kx = xx < N / 2 ? xx : xx - N;
      const bool keep = row_valid && kx >= -K && kx <= K;
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c][k] = keep ? X[s0 + c * PP + kx] : mk(T(0), T(0));
    }
    __syncthreads();   // tables
    row_inverse_store();
  }
  cluster.sync();

  const int stages = 4;
  for (int s = 0; s < nsteps; ++s) {
    sa.lo_valid = s > 0 || a.lo_valid;   // the low part of the state exists from the second step
#pragma unroll 1
    for (int j = 0; j < stages; ++j) {
      // ---- column pass: own columns, two rounds of 48
      const Phase<T> ph = load_phase<T>(a, b, s, j);
#pragma unroll 1
      for (int round = 0; round < 2; ++round) {
        const int xl = round * F::SLOTS + slot;
        const bool col_valid = xl < XH;
        const int x = r * XH + (col_valid ? xl : 0);
#pragma unroll
        for (int k = 0; k < R1; ++k) {
          const int yy = lane + R2 * k;
          const int ky = yy < N / 2 ? yy : yy - N;
          const bool keep = col_valid && ky >= -K && ky <= K;
#pragma unroll
          for (int c = 0; c < 3; ++c)
            v[c][k] = keep ? B[((long)c * P + (ky + K)) * XP + xl] : mk(T(0), T(0));
        }
        transform3(std::integral_constant<int, +1>());   // ky -> y
        const T cxg = s_cos[x], sxg = s_sin[x];
#pragma unroll
        for (int k = 0; k < R1; ++k) {
          const int y = lane + FFT2<N>::out_pos_base(k);
          cross_u<T>(A, ph, cxg, sxg, s_cos[y], s_sin[y], v[0][k], v[1][k], v[2][k]);
        }
        out_to_in<T, N>(v);
        transform3(std::integral_constant<int, -1>());   // y -> ky
        if (col_valid) {
#pragma unroll
          for (int k = 0; k < R1; ++k) {
            const int yy = lane + FFT2<N>::out_pos_base(k);
            const int ky = yy < N / 2 ? yy : yy - N;
            if (ky >= -K && ky <= K) {
#pragma unroll
              for (int c = 0; c < 3; ++c) B[((long)c * P + (ky + K)) * XP + xl] = v[c][k];
            }
          }
        }
      }
      cluster.sync();   // every column of both blocks is done before rows read them

      // ---- row pass: own rows, x from both halves
#pragma unroll
      for (int k = 0; k < R1; ++k) {
        const int xx = lane + R2 * k;
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c][k] = row_valid ? *mixed(c, iy, xx) : mk(T(0), T(0));
      }
      transform3(std::integral_constant<int, -1>());   // x -> kx
      with_stage(j, [&](auto m) {
        constexpr int MODE = decltype(m)::value;
#pragma unroll
        for (int k = 0; k < R1; ++k) {
          const int xx = lane + FFT2<N>::out_pos_base(k);
          const int kx = xx < N / 2 ? xx : xx - N;
          if (row_valid && kx >= -K && kx <= K) {
            cx<T> w0 = v[0][k] * inv_n2, w1 = v[1][k] * inv_n2, w2 = v[2][k] * inv_n2;
            stage_update_s<SCH, MODE, T>(q, sa, s0 + kx, PP, (T)kx, fky, w0, w1, w2);
            v[0][k] = w0;
            v[1][k] = w1;
            v[2][k] = w2;
          } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) v[c][k] = mk(T(0), T(0));
          }
          if (k % kUpdateGroup == kUpdateGroup - 1) asm volatile("" ::: "memory");
        }
      });
      if (s == nsteps - 1 && j == stages - 1) break;   // X holds the result
      out_to_in<T, N>(v);
      row_inverse_store();
      cluster.sync();   // both halves of every row are written before the next column pass
    }
  }
  griddep_launch_dependents();
  cluster.sync();   // no block leaves while its peer may still read its buffer
}

}  // namespace kd
