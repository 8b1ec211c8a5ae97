// Library-internal view of the context of include/kd.h and the helpers shared by the
// C-ABI translation units (kd_abi.cu, kd_tune.cu, kd_sweep.cu).
#pragma once
#include <nvtx3/nvToolsExt.h>
#include <cuda_bf16.h>

#include <string>
#include <functional>
#include <map>
#include <tuple>
#include <vector>

#include "../../include/kd.h"
#include "kd_fine.h"

namespace kdi {

struct Tables {
  int n = 0, prec = -1;
  void* tw = nullptr;
  void* cosg = nullptr;
  void* sing = nullptr;
};

struct FineWs {
  long cap = 0;
  int n = 0, prec = 0;
  void* X = nullptr;
  void* R2 = nullptr;
  void* R3 = nullptr;
  void* R4 = nullptr;
  void* Xlo = nullptr;     // complex64: low part of the state within a propagation call
  void* M = nullptr;
  void* W = nullptr;
  void* ph = nullptr;      // flow-phase table
  size_t ph_bytes = 0;
};

inline size_t csize(int prec) { return prec == KD_C128 ? 16 : 8; }

}  // namespace kdi

struct kd_ctx {
  kd_params p;
  kd::FinePlan plan[2];        // launch plans of the fine (0) and coarse (1) grid
  kd::FinePlan plan_serial;    // fine-grid plan for one field at a time (kd_fine_serial)
  int plan_serial_ok = 0;
  int pdl = 1;                 // fine-step kernels as programmatic dependent launches
  // pipelined Parareal: the fine sweep of iteration k + 1 runs in `overlap` slice chunks on
  // st2 while the serial sweep of iteration k runs on st (0: one batched sweep, no overlap)
  int overlap = 0;
  int coarse_cluster = 0;          // blocks per cluster of the coarse solver (0: default)
  // captured CUDA graphs of fine sweeps (kd_set_graphs; run_graph), keyed by a signature
  // of the sweep's shape and launch plan that includes the allocation generation (any
  // device allocation or free invalidates them)
  int graphs = 1;
  unsigned long long alloc_gen = 0;
  cudaStream_t st_g = nullptr;     // the graphs run here (a capturable stream), fenced by gev
  cudaEvent_t gev[2] = {nullptr, nullptr};
  struct GraphEntry {
    cudaGraphExec_t exec;
    long long launches;
  };
  std::map<std::string, GraphEntry> gcache;
  double* ref_T = nullptr;         // kd_set_reference: compact FP64 reference field at t = T
  int gemm_engine = 0;             // learned-operator training GEMM: KD_GEMM_TCGEN05 (0) or KD_GEMM_MMA_SYNC
  int coarse_sync = 0;             // coarse solver halo exchange: KD_SYNC_CLUSTER (0) or KD_SYNC_P2P
  cudaStream_t st2 = nullptr;      // fine chunks (lowest priority)
  cudaStream_t st_hi = nullptr;    // serial sweeps (highest priority)
  std::vector<cudaEvent_t> pev2;   // chunk release / fine-done / timing events
  void* conv_tmp = nullptr;        // FP64 staging of the convolution fine operator
  size_t conv_tmp_bytes = 0;
  // kd_fine_batched_host: device slots of the chunks in flight (in 0, in 1, out 0, out 1),
  // the start times, the copy streams and their events
  void* hio[4] = {nullptr, nullptr, nullptr, nullptr};
  size_t hio_bytes = 0;
  double* hio_t0 = nullptr;
  int hio_t0_cap = 0;
  cudaStream_t st_h2d = nullptr, st_d2h = nullptr;
  cudaEvent_t hev[12] = {};   // host-buffer calls: per device slot copied in / computed / copied out
  cudaStream_t st = nullptr;
  int device = 0;
  kdi::Tables tab_f, tab_c;
  kdi::FineWs ws_f, ws_c;
  // Parareal / serial buffers
  long cap_slices = 0;
  double* U = nullptr;
  double* Fv = nullptr;
  double* Gv = nullptr;
  double* Uprev = nullptr;    // previous iterate (increment form of the fine sweep)
  void* ph_c = nullptr;       // coarse flow-phase table of all slices
  size_t ph_c_bytes = 0;
  double* t0f = nullptr;
  double* t0c = nullptr;
  double* partials = nullptr;
  double* scal = nullptr;     // device scalars (sigma, fit)
  double* Ebuf = nullptr;
  void* full_tmp = nullptr;   // full-grid FP64 staging [max(N+1, batch)][3][n][n]
  size_t full_tmp_bytes = 0;
  double* host_scal = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // the context's device buffers (dalloc / dfree): allocs[i] of alloc_sizes[i] bytes, a
  // null entry once freed; alloc_held is their sum and alloc_limit its cap (0: none,
  // kd_set_alloc_limit)
  std::vector<void*> allocs;
  std::vector<size_t> alloc_sizes;
  size_t alloc_held = 0;
  size_t alloc_limit = 0;
  std::string err;
  long long launches = 0;     // kernels launched by this context
  int cK = 0, cP = 0;         // coarse mode set k in [-cK, cP - cK)^2
  // learned coarse propagator (kd_learned_*)
  int l_nphase = 0;
  double l_sliceT = 0.0;
  __nv_bfloat16* l_W = nullptr;   // [nphase][2 nc][nc] BF16 stacked operators
  float* l_W0 = nullptr;          // [nphase][2 nc][nc] FP32 classical-propagator matrices
  std::vector<int> l_valid;       // phase operator passed validation against the classical one
  float* l_x = nullptr;           // sweep vectors [2][nc] complex
  int fallback = 0;
  // slice block of a multi-rank run (kd_block_*): global index of local slice 0 and sizes
  int blk_lo = 0, blk_n = 0, blk_N = 0, blk_S = 0, blk_Sc = 0;
  double blk_dt = 0.0, blk_dtc = 0.0;
  // optional event timing of the fine column / row kernels
  int prof = 0;
  std::vector<cudaEvent_t> pev;
  std::vector<int> pkid;
  size_t pev_used = 0;
  double prof_ms[2] = {0.0, 0.0};
  long long prof_n[2] = {0, 0};
};


namespace kdi {

constexpr int kMaxChunks = 16;   // slice chunks of the pipelined fine sweep

kd_status fail(kd_ctx* c, kd_status s, const std::string& m);
kd_status cuda_fail(kd_ctx* c, cudaError_t e, const char* where);

#define KD_CUDA(call, where)                                 \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return kdi::cuda_fail(ctx, e_, where); \
  } while (0)

#define KD_LAUNCH(expr, where)                                                          \
  do {                                                                                  \
    int r_ = (expr);                                                                    \
    if (r_ < 0) return kdi::fail(ctx, KD_ECUDA, std::string(where) + ": launch failed"); \
    ctx->launches += r_ > 0 ? r_ : 1;                                                   \
    cudaError_t e_ = cudaGetLastError();                                                \
    if (e_ != cudaSuccess) return kdi::cuda_fail(ctx, e_, where);                       \
  } while (0)

bool valid_n(int n);
// NVTX range for the duration of a scope: the phases of a solve show up by name in a
// profiler timeline (no cost when no tool is attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

inline int kept(int n) { return 2 * (n / 3) + 1; }
inline long compact_len(int n) { return 3L * kept(n) * kept(n); }  // complex entries per field
int steps_for(double dT, double dt);
kd_status dalloc(kd_ctx* ctx, void** p, size_t bytes, const char* what);
void dfree(kd_ctx* ctx, void* p);
kd_status make_tables(kd_ctx* ctx, Tables& t, int n, int prec);
kd_status ensure_ws(kd_ctx* ctx, FineWs& w, int n, int prec, long batch);
kd::FineArgs fine_args(const kd_ctx* ctx, const FineWs& w, const Tables& t, int n, long batch, double dt,
                       const double* t0);
// point a.phases at a table of the workspace large enough for `nsteps` steps
kd_status with_phases(kd_ctx* ctx, FineWs& w, kd::FineArgs& a, int nsteps);
// Parareal building blocks (kd_abi.cu) on local slice indices of the context's slice
// arrays U / Fv / Uprev / Gv (slice i starts at t0f[i]):
kd_status ensure_slices(kd_ctx* ctx, long N);
kd_status coarse_phases(kd_ctx* ctx, int N, int Sc, double dtc);
kd_status coarse_step(kd_ctx* ctx, int i, int Sc, double dtc, bool init, bool last);
kd_status learned_step(kd_ctx* ctx, int i, bool init, bool last);
bool use_learned(const kd_ctx* ctx, int i);
kd_status fine_sweep(kd_ctx* ctx, int first, int N, int S, double dt, int iter);
// Enqueue `launches` (work on ctx->st) through a CUDA graph captured once per `key` and
// replayed on the context's graph stream, fenced against ctx->st; the values are those of
// the direct launches.  The caller makes every allocation the launches need beforehand
// and puts into `key` everything the launches depend on besides device data.
kd_status run_graph(kd_ctx* ctx, const std::string& key, const std::function<kd_status()>& launches);
kd_status copy_in_b0(kd_ctx* ctx, const double* b0);
kd_status ensure_full_tmp(kd_ctx* ctx, size_t bytes);
// the convolution-form fine operator (fine_operator KD_FINE_CONV) on FP64 compact fields
bool conv_op(const kd_ctx* ctx);
kd_status ensure_conv_tmp(kd_ctx* ctx, size_t bytes);
kd_status conv_fine(kd_ctx* ctx, const double* in, double* out, long batch, int nsteps, double dt, const double* t0);
// fine steps on grid g (0 fine, 1 coarse) with the context's plan for that grid
int run_fine(kd_ctx* ctx, int g, int prec, const kd::FineArgs& a, int nsteps, bool prologue, bool store_last,
             const kd::LaunchProbe* probe = nullptr, const int* active = nullptr);

}  // namespace kdi
