// BF16 GEMM on the 5th-generation tensor cores (tcgen05) for the training of the learned
// coarse propagator: C[M][N] = A[M][K] B[N][K]^T, both operands K-major (row-major with K
// innermost), FP32 accumulation in tensor memory (TMEM), FP32 output.
//
// One CTA of 128 threads computes a 128 x 128 tile of C.  Operand tiles of 128 rows x 64 K
// (128 bytes a row) sit in shared memory in the 128-byte swizzled K-major layout the tensor
// core reads (16-byte chunk c of row r at r * 128 + ((c ^ (r mod 8)) * 16), tiles 1024-byte
// aligned), zero outside the matrices, in a ring of stages.  One thread issues tcgen05.mma
// (M = 128, N = 128, K = 16; 4 per 64-wide K tile) into a 128-column TMEM accumulator and
// commits each K tile to that stage's "empty" mbarrier.  The epilogue reads the accumulator
// with tcgen05.ld (warp w owns TMEM lanes = tile rows 32 w .. 32 w + 31, one row per
// thread) and stores the rows of C in range.
//
// Main kernel (k_gemm_tn_tma): warp-specialised.  One thread of warp 0 loads the stages
// with TMA (cp.async.bulk.tensor, 128-byte swizzle; out-of-range boxes read as zeros),
// counted on the stage's "full" mbarrier; one thread of warp 1 waits on "full", issues
// the MMAs and commits to "empty", which the loader waits on before refilling the stage;
// no block barrier inside the K loop.  Where the driver offers no tensor-map encoder,
// k_gemm_tn_tc stages the same layout with cp.async from all threads.  Both move 16-byte
// pieces: A and B start on 16-byte boundaries and K is a multiple of 8.
//
// Every mbarrier wait has an iteration limit; a wait that runs out sets *err and the CTA
// stops issuing work, waits (again bounded) for its committed MMAs, frees its TMEM and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <stdio.h>

#include <mutex>

#include "../../include/kd.h"
#include "kd_learned.h"
#include "kd_wait.cuh"

namespace kd {

namespace {

constexpr int kBM = 128, kBN = 128, kBK = 64;   // CTA tile; K tile = one 128-byte swizzle row
constexpr int kStages = 4;
constexpr int kThreads = 128;
constexpr int kTileBytes = kBM * kBK * 2;        // 16 KB per operand tile
constexpr int kSmemBytes = kStages * 2 * kTileBytes + 1024;   // + alignment slack
constexpr long long kWaitCycles = 20000000;      // ~10 ms at 2 GHz

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp16(uint32_t dst, const void* src, bool pred) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(pred ? 16 : 0));
}

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  return mbar_wait_bounded<false>(bar, parity, kWaitCycles);
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF)        // start address
         | ((uint64_t)1 << 16)                   // leading byte offset (unused with swizzle)
         | ((uint64_t)(1024 >> 4) << 32)         // stride byte offset: next 8-row group
         | ((uint64_t)1 << 46)                   // descriptor version
         | ((uint64_t)2 << 61);                  // 128-byte swizzle
}

// instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major, N = 128, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate,
                                    uint32_t idesc = kIdesc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tn_tc(const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ Bt, float* __restrict__ C,
                 int M, int N, int K, int ldc, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[kStages + 1];   // per stage, + the final commit
  __shared__ uint32_t tmem_base;
  __shared__ int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // 1024-byte aligned tile ring: [stage][A | B]
  const uint32_t raw = saddr(smem_raw);
  const uint32_t ring = (raw + 1023u) & ~1023u;
  const long m0 = (long)blockIdx.y * kBM, n0 = (long)blockIdx.x * kBN;
  const int ktiles = (K + kBK - 1) / kBK;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                 "r"(kBN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    s_bad = 0;
    for (int s = 0; s <= kStages; ++s) mbar_init(saddr(&bars[s]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  // copy K tile kt into stage s: 2 x 128 rows x 8 chunks of 16 bytes, 16 chunks a thread
  auto load = [&](int kt, int s) {
    const uint32_t a_s = ring + (uint32_t)(s * 2 * kTileBytes), b_s = a_s + kTileBytes;
    const long k0 = (long)kt * kBK;
#pragma unroll
    for (int t = 0; t < (kBM * 8) / kThreads; ++t) {
      const int q = tid + t * kThreads;
      const int r = q >> 3, c = q & 7;
      const long k = k0 + c * 8;
      const uint32_t off = (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
      const bool pa = m0 + r < M && k < K, pb = n0 + r < N && k < K;
      cp16(a_s + off, A + (pa ? (m0 + r) * (long)K + k : 0), pa);
      cp16(b_s + off, Bt + (pb ? (n0 + r) * (long)K + k : 0), pb);
    }
  };

  // The copy runs kAhead tiles ahead of the MMAs.  A stage is refilled two K tiles after
  // its MMAs were issued (tile kt + kAhead goes into the stage of tile kt - 2), so the wait
  // for the tensor core to release it overlaps the MMAs of tile kt - 1.
  constexpr int kAhead = kStages - 2;
  for (int kt = 0; kt < kAhead; ++kt) {
    if (kt < ktiles) load(kt, kt);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  for (int kt = 0; kt < ktiles; ++kt) {
    const int nt = kt + kAhead;
    if (nt < ktiles) {
      const int s = nt % kStages;
      if (nt >= kStages && !*(volatile int*)&s_bad) {
        // tile nt - kStages (= kt - 2) was committed to bars[s]: its (nt / kStages - 1)-th completion
        if (!mbar_wait(saddr(&bars[s]), (uint32_t)((nt / kStages - 1) & 1))) *(volatile int*)&s_bad = 1;
      }
      if (!*(volatile int*)&s_bad) load(nt, s);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group %0;" ::"n"(kAhead) : "memory");      // tile kt has landed
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");           // visible to the tensor core
    __syncthreads();
    if (tid == 0 && !*(volatile int*)&s_bad) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_s = ring + (uint32_t)((kt % kStages) * 2 * kTileBytes), b_s = a_s + kTileBytes;
#pragma unroll
      for (int j = 0; j < kBK / 16; ++j)   // K = 16 per MMA: 32 bytes further along the swizzled row
        mma(tmem, sw128_desc(a_s + 32 * j), sw128_desc(b_s + 32 * j), (kt > 0 || j > 0) ? 1u : 0u);
      commit(saddr(&bars[kt % kStages]));
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  // all MMAs of this thread are done when the final commit arrives
  if (tid == 0) {
    commit(saddr(&bars[kStages]));
    if (!mbar_wait(saddr(&bars[kStages]), 0u)) *(volatile int*)&s_bad = 1;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool bad = *(volatile int*)&s_bad != 0;
  if (bad && tid == 0) atomicExch(err, 1);

  // epilogue: row 32 warp + lane of the tile, 32 columns per load
  const long row = m0 + warp * 32 + lane;
#pragma unroll 1
  for (int c0 = 0; c0 < kBN && !bad; c0 += 32) {
    uint32_t v[32];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (row < M) {
      float* crow = C + row * (long)ldc + n0 + c0;
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (n0 + c0 + i < N) crow[i] = __uint_as_float(v[i]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kBN) : "memory");
  }
}

// TMA kernel: A tiles 128 x 64, B tiles BN x 64 (BN = 128 or 256: one UMMA of N = BN)
template <int BN>
struct TmaCfg {
  static constexpr int kATile = kBM * kBK * 2, kBTile = BN * kBK * 2, kStage = kATile + kBTile;
  static constexpr int kStages = BN == 256 ? 4 : 6;
  static constexpr int kSmem = kStages * kStage + 1024;
  static constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                     ((uint32_t)(kBM >> 4) << 24);
};

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// box {64 K, 128 rows} at element (x = K index, y = row) of the tensor map into dst
__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tn_tma(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, float* __restrict__ C,
                  int M, int N, int K, int ldc, int* err) {
  using G = TmaCfg<BN>;
  constexpr int kTmaStages = G::kStages;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[kTmaStages], empty[kTmaStages], done;
  __shared__ uint32_t tmem_base;
  __shared__ int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t ring = (saddr(smem_raw) + 1023u) & ~1023u;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
  const int ktiles = (K + kBK - 1) / kBK;

  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    s_bad = 0;
    for (int s = 0; s < kTmaStages; ++s) {
      mbar_init(saddr(&full[s]));
      mbar_init(saddr(&empty[s]));
    }
    mbar_init(saddr(&done));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&ta) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tb) : "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {
    // loader
    int issued = 0;
    for (int kt = 0; kt < ktiles; ++kt) {
      const int s = kt % kTmaStages;
      if (kt >= kTmaStages && !mbar_wait(saddr(&empty[s]), (uint32_t)((kt / kTmaStages - 1) & 1))) {
        *(volatile int*)&s_bad = 1;
        break;
      }
      const uint32_t a_s = ring + (uint32_t)(s * G::kStage);
      mbar_expect_tx(saddr(&full[s]), G::kStage);
      tma_load(a_s, &ta, kt * kBK, m0, saddr(&full[s]));
      tma_load(a_s + G::kATile, &tb, kt * kBK, n0, saddr(&full[s]));
      issued = kt + 1;
    }
    if (issued < ktiles) {
      // gave up: the copies already issued still write this CTA's shared memory; wait
      // (bounded) until the last ring's worth of them has landed before the CTA may exit
      for (int kt = issued > kTmaStages ? issued - kTmaStages : 0; kt < issued; ++kt)
        mbar_wait(saddr(&full[kt % kTmaStages]), (uint32_t)((kt / kTmaStages) & 1));
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    for (int kt = 0; kt < ktiles; ++kt) {
      const int s = kt % kTmaStages;
      if (!mbar_wait(saddr(&full[s]), (uint32_t)((kt / kTmaStages) & 1))) {
        *(volatile int*)&s_bad = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_s = ring + (uint32_t)(s * G::kStage), b_s = a_s + G::kATile;
#pragma unroll
      for (int j = 0; j < kBK / 16; ++j)
        mma(tmem, sw128_desc(a_s + 32 * j), sw128_desc(b_s + 32 * j), (kt > 0 || j > 0) ? 1u : 0u, G::kIdesc);
      commit(saddr(&empty[s]));
    }
    commit(saddr(&done));   // arrives when every MMA issued above has completed
  }
  // the accumulator is complete once `done` arrives
  if (!mbar_wait(saddr(&done), 0u)) *(volatile int*)&s_bad = 1;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool bad = *(volatile int*)&s_bad != 0;
  if (bad && tid == 0) atomicExch(err, 1);

  const long row = (long)m0 + warp * 32 + lane;
#pragma unroll 1
  for (int c0 = 0; c0 < BN && !bad; c0 += 32) {
    uint32_t v[32];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (row < M && n0 + c0 < N) {
      float* crow = C + row * (long)ldc + n0 + c0;
      if (n0 + c0 + 32 <= N && (((uintptr_t)crow) & 15) == 0) {
#pragma unroll
        for (int i = 0; i < 32; i += 4)
          *(float4*)(crow + i) = make_float4(__uint_as_float(v[i]), __uint_as_float(v[i + 1]),
                                             __uint_as_float(v[i + 2]), __uint_as_float(v[i + 3]));
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i)
          if (n0 + c0 + i < N) crow[i] = __uint_as_float(v[i]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 2) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

// 2-D tensor map of a row-major BF16 matrix [rows][K]: boxes of box_rows rows x 64 K, 128-byte swizzle
bool make_map(CUtensorMap* map, const void* base, int rows, int K, int box_rows) {
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return false;
    }
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int gemm_bf16_tn_tc(const __nv_bfloat16* A, const __nv_bfloat16* Bt, float* C, int M, int N, int K, int ldc,
                    int* err, cudaStream_t st) {
  if (K % 8 != 0 || M <= 0 || N <= 0 || K <= 0 || !err || (((uintptr_t)A) & 15) || (((uintptr_t)Bt) & 15)) return -1;
  dim3 grid((unsigned)((N + kBN - 1) / kBN), (unsigned)((M + kBM - 1) / kBM));
  // B tiles of 256 rows (one N = 256 MMA per K step) when they make at least two tiles
  // per SM; fewer, larger tiles leave SMs idle, and there the 128-row tiles (and their
  // deeper 6-stage ring) win: measured 567 vs 302 TFLOP/s at 14406 x 512 x 7208, while
  // 256-row tiles win at 4096^3 (875 vs 636) and 8192^3
  // the current device's SM count and shared-memory opt-in, set on every call (host-side
  // attribute calls): nothing cached outlives a device switch or a cudaDeviceReset
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms <= 0)
    return -1;
  const long tiles256 = (long)((M + kBM - 1) / kBM) * ((N + 255) / 256);
  const bool wide = N > 128 && tiles256 >= 2L * sms;
  CUtensorMap ta, tb;
  if (make_map(&ta, A, M, K, kBM) && make_map(&tb, Bt, N, K, wide ? 256 : 128)) {
    const int smem = wide ? TmaCfg<256>::kSmem : TmaCfg<128>::kSmem;
    if (cudaFuncSetAttribute(wide ? k_gemm_tn_tma<256> : k_gemm_tn_tma<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem) != cudaSuccess)
      return -1;
    dim3 g2((unsigned)((N + (wide ? 255 : 127)) / (wide ? 256 : 128)), grid.y);
    if (wide)
      k_gemm_tn_tma<256><<<g2, kThreads, smem, st>>>(ta, tb, C, M, N, K, ldc, err);
    else
      k_gemm_tn_tma<128><<<g2, kThreads, smem, st>>>(ta, tb, C, M, N, K, ldc, err);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
  }
  if (cudaFuncSetAttribute(k_gemm_tn_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) != cudaSuccess)
    return -1;
  k_gemm_tn_tc<<<grid, kThreads, kSmemBytes, st>>>(A, Bt, C, M, N, K, ldc, err);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

// one CTA waits on an mbarrier that receives its only arrival (arrive = 1) or none
__global__ void k_wait_selftest(int arrive, long long max_cycles, int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(saddr(&bar));
  __syncthreads();
  if (arrive && threadIdx.x == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&bar)) : "memory");
  const bool ok = mbar_wait_bounded<false>(saddr(&bar), 0u, max_cycles);
  __syncthreads();
  if (threadIdx.x == 0) *status = ok ? 0 : 1;
}

}  // namespace kd

extern "C" kd_status kd_selftest_wait(int arrive, double max_ms, void* cuda_stream) {
  using namespace kd;
  if (!(max_ms > 0) || max_ms > 1000.0) return KD_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int* status = nullptr;
  if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) return KD_ENOMEM;
  int clock_khz = 0, dev = 0, h = -1;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev) != cudaSuccess || clock_khz <= 0)
    clock_khz = 2070000;
  const long long cycles = (long long)(max_ms * clock_khz);
  k_wait_selftest<<<1, 32, 0, st>>>(arrive ? 1 : 0, cycles, status);
  kd_status s = KD_OK;
  if (cudaGetLastError() != cudaSuccess || cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    s = KD_ECUDA;
  else
    s = h == 0 ? KD_OK : KD_ETIMEOUT;
  cudaFree(status);
  return s;
}

extern "C" kd_status kd_gemm_bf16_tn(const void* A, const void* Bt, float* C, int M, int N, int K, int ldc, int engine,
                                     void* cuda_stream) {
  using namespace kd;
  if (!A || !Bt || !C || M < 1 || N < 1 || K < 8 || K % 8 != 0 || ldc < N || (((uintptr_t)A) & 15) ||
      (((uintptr_t)Bt) & 15) ||
      (engine != KD_GEMM_TCGEN05 && engine != KD_GEMM_MMA_SYNC)) {
    fprintf(stderr, "kd_gemm_bf16_tn: bad arguments\n");
    return KD_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (engine == KD_GEMM_MMA_SYNC) {
    if (gemm_bf16_tn((const __nv_bfloat16*)A, (const __nv_bfloat16*)Bt, C, M, N, K, ldc, st) < 0) return KD_ECUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? KD_OK : KD_ECUDA;
  }
  // the status word of the kernel's bounded waits: one per device for the process lifetime
  static int* err_of[64] = {nullptr};
  static std::mutex err_mutex;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return KD_ECUDA;
  int* err = nullptr;
  {
    std::lock_guard<std::mutex> lock(err_mutex);
    if (!err_of[dev] && cudaMalloc(&err_of[dev], sizeof(int)) != cudaSuccess) {
      err_of[dev] = nullptr;
      return KD_ENOMEM;
    }
    err = err_of[dev];
  }
  int e = 0;
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess ||
      gemm_bf16_tn_tc((const __nv_bfloat16*)A, (const __nv_bfloat16*)Bt, C, M, N, K, ldc, err, st) < 0 ||
      cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return KD_ECUDA;
  return e ? KD_ECUDA : KD_OK;
}
