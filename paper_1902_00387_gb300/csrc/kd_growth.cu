// Direct growth rate by power iteration of the fine propagator (include/kd.h:
// kd_growth_power).
//
// The growth rate of a kinematic dynamo (Sec. 1) is the real part of the leading
// eigenvalue of the linear operator for a steady flow, and ln|mu| / period for the
// leading Floquet multiplier mu of a time-periodic flow.  Both are the growth of the
// dominant mode of the propagator M over an interval tau, M = exp(L tau) (steady) or the
// one-period map (tau = period): iterate b <- M b / |M b|; |M b| / |b| -> |mu| and
// gamma = ln(|M b| / |b|) / tau.  M is applied by the fine propagator on the device; the
// norms are fixed-order FP64 reductions.
#include <math.h>

#include "kd_ctx.h"

using namespace kd;
using namespace kdi;

namespace {

constexpr int kNormBlocks = 256;

// partial sums of |x|^2 per block (fixed order), x complex of precision T
template <typename T>
__global__ void k_norm2_partials(const cx<T>* x, long len, double* partials) {
  double acc = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < len; i += (long)gridDim.x * blockDim.x) {
    const double a = (double)x[i].x, b = (double)x[i].y;
    acc += a * a + b * b;
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void k_norm2_finish(const double* partials, int nb, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += partials[b];
  *out = s;
}

// x *= 1 / sqrt(*norm2), the factor computed in FP64 and applied in precision T
template <typename T>
__global__ void k_normalise(cx<T>* x, long len, const double* norm2) {
  const double f = 1.0 / sqrt(*norm2);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < len; i += (long)gridDim.x * blockDim.x)
    x[i] = mk((T)((double)x[i].x * f), (T)((double)x[i].y * f));
}

int norm2(int prec, const void* x, long len, double* partials, double* out, cudaStream_t st) {
  if (prec == KD_C64)
    k_norm2_partials<float><<<kNormBlocks, 256, 0, st>>>((const cx<float>*)x, len, partials);
  else
    k_norm2_partials<double><<<kNormBlocks, 256, 0, st>>>((const cx<double>*)x, len, partials);
  k_norm2_finish<<<1, 32, 0, st>>>(partials, kNormBlocks, out);
  return cudaPeekAtLastError() == cudaSuccess ? 2 : -1;
}

int normalise(int prec, void* x, long len, const double* n2, cudaStream_t st) {
  long g = (len + 255) / 256;
  if (g > 65535L * 8) g = 65535L * 8;
  if (prec == KD_C64)
    k_normalise<float><<<(unsigned)g, 256, 0, st>>>((cx<float>*)x, len, n2);
  else
    k_normalise<double><<<(unsigned)g, 256, 0, st>>>((cx<double>*)x, len, n2);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace

extern "C" kd_status kd_growth_power(kd_ctx* ctx, const double* b0, double t0, double tau, int max_iter, double tol,
                                     double* rate, int* iters, double* b_out) {
  if (!ctx) return KD_EINVAL;
  if (!b0 || !rate) return fail(ctx, KD_EINVAL, "kd_growth_power: NULL buffer");
  if (!(tau > 0) || !isfinite(tau) || !isfinite(t0)) return fail(ctx, KD_EINVAL, "kd_growth_power: tau must be > 0");
  if (max_iter < 1 || !(tol >= 0)) return fail(ctx, KD_EINVAL, "kd_growth_power: max_iter >= 1, tol >= 0");
  const int n = ctx->p.n;
  const bool conv = conv_op(ctx);
  // the vector: fine-precision compact state of the FFT operator, FP64 for the convolution one
  const int pf = conv ? KD_C128 : ctx->p.prec_fine;
  const long len = compact_len(n);
  const int S = steps_for(tau, ctx->p.dt_fine);
  const double dt = tau / S;
  kd_status s;
  if ((s = ensure_ws(ctx, ctx->ws_f, n, ctx->p.prec_fine, 1)) != KD_OK) return s;
  if ((s = ensure_full_tmp(ctx, 3UL * n * n * 16)) != KD_OK) return s;
  if (conv && (s = ensure_conv_tmp(ctx, (size_t)len * 16)) != KD_OK) return s;
  void* X = conv ? ctx->conv_tmp : ctx->ws_f.X;
  KD_CUDA(cudaMemcpyAsync(ctx->full_tmp, b0, 3UL * n * n * 16, cudaMemcpyDefault, ctx->st), "copy b0");
  KD_LAUNCH(full_to_compact(KD_C128, ctx->full_tmp, pf, X, 1, n, ctx->st), "pack");
  // scal[8] = |b|^2, scal[9] = |M b|^2; partials in ctx->partials; t0 of the field in scal[10]
  double* n0 = ctx->scal + 8;
  double* n1 = ctx->scal + 9;
  double* tdev = ctx->scal + 10;
  KD_CUDA(cudaMemcpyAsync(tdev, &t0, 8, cudaMemcpyHostToDevice, ctx->st), "t0");
  KD_LAUNCH(norm2(pf, X, len, ctx->partials, n0, ctx->st), "norm");
  KD_LAUNCH(normalise(pf, X, len, n0, ctx->st), "normalise");
  FineArgs a = fine_args(ctx, ctx->ws_f, ctx->tab_f, n, 1, dt, tdev);
  if ((s = with_phases(ctx, ctx->ws_f, a, S)) != KD_OK) return s;
  double prev = NAN, cur = NAN;
  int it = 0;
  for (it = 1; it <= max_iter; ++it) {
    KD_LAUNCH(norm2(pf, X, len, ctx->partials, n0, ctx->st), "norm");
    if (conv) {
      if ((s = conv_fine(ctx, (const double*)X, (double*)X, 1, S, dt, tdev)) != KD_OK) return s;
    } else {
      KD_LAUNCH(run_fine(ctx, 0, pf, a, S, true, false), "fine steps");
    }
    KD_LAUNCH(norm2(pf, X, len, ctx->partials, n1, ctx->st), "norm");
    KD_CUDA(cudaMemcpyAsync(ctx->host_scal, n0, 16, cudaMemcpyDeviceToHost, ctx->st), "norm copy");
    KD_LAUNCH(normalise(pf, X, len, n1, ctx->st), "normalise");
    KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
    const double a0 = ctx->host_scal[0], a1 = ctx->host_scal[1];
    if (!(a0 > 0) || !(a1 > 0) || !isfinite(a0) || !isfinite(a1))
      return fail(ctx, KD_ENONFINITE, "kd_growth_power: zero or non-finite norm");
    prev = cur;
    cur = 0.5 * log(a1 / a0) / tau;
    if (it > 1 && fabs(cur - prev) <= tol) break;
  }
  if (it > max_iter) it = max_iter;
  *rate = cur;
  if (iters) *iters = it;
  if (b_out) {
    KD_LAUNCH(compact_to_full(pf, X, KD_C128, ctx->full_tmp, 1, n, ctx->st), "unpack");
    KD_CUDA(cudaMemcpyAsync(b_out, ctx->full_tmp, 3UL * n * n * 16, cudaMemcpyDefault, ctx->st), "copy out");
    KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
  }
  return (it >= max_iter && !(fabs(cur - prev) <= tol)) ? fail(ctx, KD_ENOTCONV, "kd_growth_power: tol not reached")
                                                        : KD_OK;
}
