// Slice blocks of a multi-rank Parareal run (include/kd.h: kd_block_*).
//
// The time communicator of the paper's implementation (Sec. 4.1, Algorithms 1-3) gives
// each rank a contiguous block of slices [lo, lo + n_local): the parallel step is local to
// the rank, and the serial sweep passes one slice state from rank r to rank r + 1.  Here a
// context holds one block in the same device arrays as kd_parareal_run (local slice i is
// global slice lo + i, starting at t = (lo + i) dT), and the host moves the boundary states
// between ranks (kd_block_get_boundary / kd_block_set_boundary, FP64 compact form).  The
// arithmetic is that of kd_parareal_run: the increment form of the correction, slices
// n < k - 1 left untouched in iteration k (they are exact), and U_{k} = F(U_{k-1}) for the
// slice n = k - 1 whose input no longer changes.
#include <math.h>

#include <string>

#include "kd_ctx.h"

using namespace kd;
using namespace kdi;

namespace {

kd_status need_block(kd_ctx* ctx, const char* who) {
  if (ctx->blk_n <= 0) return fail(ctx, KD_EINVAL, std::string(who) + ": call kd_block_init first");
  return KD_OK;
}

}  // namespace

extern "C" {

kd_status kd_block_init(kd_ctx* ctx, int lo, int n_local, double T, int n_slices) {
  if (!ctx) return KD_EINVAL;
  if (n_slices < 1 || n_slices > KD_MAX_SLICES) return fail(ctx, KD_EINVAL, "kd_block_init: n_slices out of range");
  if (lo < 0 || n_local < 1 || lo + n_local > n_slices)
    return fail(ctx, KD_EINVAL, "kd_block_init: the block must lie in [0, n_slices)");
  if (!(T > 0) || !isfinite(T)) return fail(ctx, KD_EINVAL, "kd_block_init: T must be > 0");
  if (ctx->p.fine_form != KD_FINE_INCREMENT)
    return fail(ctx, KD_EINVAL, "kd_block_init: slice blocks use fine_form KD_FINE_INCREMENT");
  const double dT = T / n_slices;
  if (ctx->p.coarse_kind == KD_COARSE_LEARNED) {
    if (ctx->l_nphase == 0) return fail(ctx, KD_EINVAL, "kd_block_init: call kd_learned_init first");
    if (fabs(dT - ctx->l_sliceT) > 1e-9 * dT)
      return fail(ctx, KD_EINVAL, "kd_block_init: slice length differs from the learned operators' slice");
  }
  const int n = ctx->p.n, nc = ctx->p.n_coarse;
  const int S = steps_for(dT, ctx->p.dt_fine), Sc = steps_for(dT, ctx->p.dt_coarse);
  kd_status s;
  if ((s = ensure_slices(ctx, n_local)) != KD_OK) return s;
  if ((s = ensure_ws(ctx, ctx->ws_f, n, ctx->p.prec_fine, n_local)) != KD_OK) return s;
  if ((s = ensure_ws(ctx, ctx->ws_c, nc, ctx->p.prec_coarse, 1)) != KD_OK) return s;
  ctx->blk_lo = lo;
  ctx->blk_n = n_local;
  ctx->blk_N = n_slices;
  ctx->blk_S = S;
  ctx->blk_Sc = Sc;
  ctx->blk_dt = dT / S;
  ctx->blk_dtc = dT / Sc;
  ctx->fallback = 0;
  KD_LAUNCH(fill_slice_times(ctx->t0f, n_local + 1, lo, dT, ctx->st), "times");
  KD_LAUNCH(fill_slice_times(ctx->t0c, n_local + 1, lo, dT, ctx->st), "times");
  if ((s = coarse_phases(ctx, n_local, Sc, ctx->blk_dtc)) != KD_OK) return s;
  KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
  return KD_OK;
}

size_t kd_block_boundary_bytes(kd_ctx* ctx) { return ctx ? (size_t)compact_len(ctx->p.n) * 16 : 0; }

kd_status kd_block_set_initial(kd_ctx* ctx, const double* b0) {
  if (!ctx) return KD_EINVAL;
  kd_status s = need_block(ctx, "kd_block_set_initial");
  if (s != KD_OK) return s;
  if (!b0) return fail(ctx, KD_EINVAL, "kd_block_set_initial: b0 is NULL");
  if ((s = copy_in_b0(ctx, b0)) != KD_OK) return s;
  KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
  return KD_OK;
}

kd_status kd_block_set_boundary(kd_ctx* ctx, const double* u_lo) {
  if (!ctx) return KD_EINVAL;
  kd_status s = need_block(ctx, "kd_block_set_boundary");
  if (s != KD_OK) return s;
  if (!u_lo) return fail(ctx, KD_EINVAL, "kd_block_set_boundary: NULL buffer");
  KD_CUDA(cudaMemcpyAsync(ctx->U, u_lo, kd_block_boundary_bytes(ctx), cudaMemcpyDefault, ctx->st), "boundary in");
  KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
  return KD_OK;
}

kd_status kd_block_get_boundary(kd_ctx* ctx, double* u_hi) {
  if (!ctx) return KD_EINVAL;
  kd_status s = need_block(ctx, "kd_block_get_boundary");
  if (s != KD_OK) return s;
  if (!u_hi) return fail(ctx, KD_EINVAL, "kd_block_get_boundary: NULL buffer");
  const long len = compact_len(ctx->p.n);
  KD_CUDA(cudaMemcpyAsync(u_hi, ctx->U + 2 * (long)ctx->blk_n * len, kd_block_boundary_bytes(ctx), cudaMemcpyDefault,
                          ctx->st),
          "boundary out");
  KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
  return KD_OK;
}

kd_status kd_block_fine(kd_ctx* ctx, int k) {
  if (!ctx) return KD_EINVAL;
  kd_status s = need_block(ctx, "kd_block_fine");
  if (s != KD_OK) return s;
  if (k < 1 || k > KD_MAX_ITERS) return fail(ctx, KD_EINVAL, "kd_block_fine: k must be in [1, KD_MAX_ITERS]");
  // slices n >= k - 1 can still change; the global last slice is always swept so that
  // its defect is measured (as in kd_parareal_run)
  int first = k - 1 - ctx->blk_lo;
  const bool has_last = ctx->blk_lo + ctx->blk_n == ctx->blk_N;
  if (has_last && first > ctx->blk_n - 1) first = ctx->blk_n - 1;
  if (first < 0) first = 0;
  if (first >= ctx->blk_n) return KD_OK;
  if ((s = fine_sweep(ctx, first, ctx->blk_n, ctx->blk_S, ctx->blk_dt, k)) != KD_OK) return s;
  KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
  return KD_OK;
}

kd_status kd_block_sweep(kd_ctx* ctx, int k, double* sigma) {
  if (!ctx) return KD_EINVAL;
  kd_status s = need_block(ctx, "kd_block_sweep");
  if (s != KD_OK) return s;
  if (k < 0 || k > KD_MAX_ITERS) return fail(ctx, KD_EINVAL, "kd_block_sweep: k must be in [0, KD_MAX_ITERS]");
  const int nl = ctx->blk_n, lo = ctx->blk_lo;
  const bool want_sigma = sigma && k >= 1;
  if (sigma) *sigma = 0.0;
  if (k == 0) {
    for (int i = 0; i < nl; ++i)
      if ((s = use_learned(ctx, i) ? learned_step(ctx, i, true, false)
                                   : coarse_step(ctx, i, ctx->blk_Sc, ctx->blk_dtc, true, false)) != KD_OK)
        return s;
    KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
    return KD_OK;
  }
  const int n = ctx->p.n;
  const long len = compact_len(n), lenc = 3L * ctx->cP * ctx->cP;
  const bool has_last = lo + nl == ctx->blk_N;
  int first = k - 1 - lo;                       // local index of the slice whose input is exact
  if (has_last && first > nl - 1) first = nl - 1;
  bool measured = false;
  for (int i = first < 0 ? 0 : first; i < nl; ++i) {
    const bool last = want_sigma && i == nl - 1;
    if (i == first) {
      // U_{first+1} = F(U_first): the coarse terms cancel exactly
      int nb = parareal_update(ctx->Fv + 2 * i * len, ctx->Gv + 2 * i * lenc, KD_C128, ctx->Gv + 2 * i * lenc,
                               ctx->U + 2 * (i + 1) * len, n, ctx->cK, ctx->cP, 0, last ? ctx->partials : nullptr,
                               ctx->st);
      if (nb < 0) return fail(ctx, KD_ECUDA, "parareal update launch failed");
      ctx->launches += 1;
      if (last) KD_LAUNCH(finish_sigma(ctx->partials, nb, ctx->scal, ctx->st), "sigma");
    } else if ((s = use_learned(ctx, i) ? learned_step(ctx, i, false, last)
                                        : coarse_step(ctx, i, ctx->blk_Sc, ctx->blk_dtc, false, last)) != KD_OK) {
      return s;
    }
    measured = measured || last;
  }
  if (measured) KD_CUDA(cudaMemcpyAsync(ctx->host_scal, ctx->scal, 8, cudaMemcpyDeviceToHost, ctx->st), "sigma copy");
  KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
  if (measured) {
    *sigma = ctx->host_scal[0];
    if (!isfinite(*sigma)) return fail(ctx, KD_ENONFINITE, "kd_block_sweep: non-finite defect");
  }
  return KD_OK;
}

kd_status kd_block_get_state(kd_ctx* ctx, int i, double* u) {
  if (!ctx) return KD_EINVAL;
  kd_status s = need_block(ctx, "kd_block_get_state");
  if (s != KD_OK) return s;
  if (i < 0 || i > ctx->blk_n || !u) return fail(ctx, KD_EINVAL, "kd_block_get_state: bad index or NULL buffer");
  const int n = ctx->p.n;
  const size_t fb = 3UL * n * n * 16;
  if ((s = ensure_full_tmp(ctx, fb)) != KD_OK) return s;
  KD_LAUNCH(compact_to_full(KD_C128, ctx->U + 2 * (long)i * compact_len(n), KD_C128, ctx->full_tmp, 1, n, ctx->st),
            "state to full");
  KD_CUDA(cudaMemcpyAsync(u, ctx->full_tmp, fb, cudaMemcpyDefault, ctx->st), "state copy");
  KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
  return KD_OK;
}

}  // extern "C"
