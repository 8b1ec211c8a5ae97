// Leading eigenvalues of the fine propagator by restarted Arnoldi (include/kd.h:
// kd_growth_arnoldi).
//
// The growth rate of a kinematic dynamo (Sec. 1) is the real part of the leading eigenvalue
// of the linear operator for a steady flow (Roberts) and ln|mu| / period for the leading
// Floquet multiplier mu of a time-periodic one (Galloway-Proctor).  Both are eigenvalues of
// the propagator M over an interval tau (M = exp(L tau), or the one-period map), which the
// fine propagator applies.  Arnoldi builds an orthonormal basis V of the Krylov space
// span{v, M v, ..., M^{m-1} v} with M V_m = V_{m+1} H (H upper Hessenberg, (m+1) x m); the
// eigenvalues of the leading m x m block of H (Ritz values) approximate the eigenvalues of
// M of largest modulus, also complex ones (oscillating modes), where power iteration
// oscillates.  The residual of a Ritz pair (theta, V y) is |H[m][m-1]| |y[m-1]|.  Restart:
// the next start vector is the sum of the wanted Ritz vectors.
//
// Device side: the basis vectors (FP64 compact fields), the propagator, and the
// inner products and linear combinations of classical Gram-Schmidt with one
// re-orthogonalisation, every reduction in a fixed order.  Host side: the small dense
// eigenproblem of H (complex Schur form by shifted QR, eigenvectors by back substitution).
#include <math.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "kd_ctx.h"
#include "kd_hess.h"

using namespace kd;
using namespace kdi;

namespace {

using cd = std::complex<double>;
using kd::hess::hessenberg_schur;
using kd::hess::schur_vector;

constexpr int kDotBlocks = 128;
constexpr int kDotThreads = 256;

// partial[i][blk] = sum over the block's share of conj(V_i[e]) w[e]  (fixed order)
__global__ void k_dots_partial(const double2* V, long len, const double2* w, double2* partial) {
  const int i = blockIdx.y;
  const double2* v = V + (long)i * len;
  double re = 0.0, im = 0.0;
  for (long e = blockIdx.x * (long)kDotThreads + threadIdx.x; e < len; e += (long)gridDim.x * kDotThreads) {
    const double2 a = v[e], b = w[e];
    re += a.x * b.x + a.y * b.y;
    im += a.x * b.y - a.y * b.x;
  }
  __shared__ double sr[kDotThreads], si[kDotThreads];
  sr[threadIdx.x] = re;
  si[threadIdx.x] = im;
  __syncthreads();
  for (int s = kDotThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sr[threadIdx.x] += sr[threadIdx.x + s];
      si[threadIdx.x] += si[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(long)i * gridDim.x + blockIdx.x] = make_double2(sr[0], si[0]);
}

__global__ void k_dots_finish(const double2* partial, int nb, int nv, double2* h) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nv) return;
  double re = 0.0, im = 0.0;
  for (int b = 0; b < nb; ++b) {
    re += partial[(long)i * nb + b].x;
    im += partial[(long)i * nb + b].y;
  }
  h[i] = make_double2(re, im);
}

// w = (keep ? w : 0) + sum_i V_i c_i
__global__ void k_combine(double2* w, int keep, const double2* V, int nv, long len, const double2* c) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < len; e += (long)gridDim.x * blockDim.x) {
    double re = 0.0, im = 0.0;
    if (keep) {
      re = w[e].x;
      im = w[e].y;
    }
    for (int i = 0; i < nv; ++i) {
      const double2 v = V[(long)i * len + e], k = c[i];
      re += v.x * k.x - v.y * k.y;
      im += v.x * k.y + v.y * k.x;
    }
    w[e] = make_double2(re, im);
  }
}

__global__ void k_scale(double2* w, long len, double s) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < len; e += (long)gridDim.x * blockDim.x)
    w[e] = make_double2(w[e].x * s, w[e].y * s);
}

unsigned grid_of(long len) {
  long g = (len + 255) / 256;
  return (unsigned)(g > 4096 ? 4096 : g);
}

struct Arnoldi {
  kd_ctx* ctx;
  long len;
  double2* V = nullptr;        // [m + 1][len]
  double2* partial = nullptr;  // [m + 1][kDotBlocks]
  double2* dev_h = nullptr;    // [m + 1]
  std::vector<double2> host_h;

  kd_status dots(int nv, const double2* w, std::vector<cd>& out) {
    k_dots_partial<<<dim3(kDotBlocks, nv), kDotThreads, 0, ctx->st>>>(V, len, w, partial);
    k_dots_finish<<<(nv + 63) / 64, 64, 0, ctx->st>>>(partial, kDotBlocks, nv, dev_h);
    KD_CUDA(cudaGetLastError(), "dots");
    KD_CUDA(cudaMemcpyAsync(host_h.data(), dev_h, nv * sizeof(double2), cudaMemcpyDeviceToHost, ctx->st), "dots");
    KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
    out.resize(nv);
    for (int i = 0; i < nv; ++i) out[i] = cd(host_h[i].x, host_h[i].y);
    return KD_OK;
  }
  // w = (keep ? w : 0) + sum_i V_i c_i
  kd_status combine(double2* w, bool keep, int nv, const std::vector<cd>& c) {
    for (int i = 0; i < nv; ++i) host_h[i] = make_double2(c[i].real(), c[i].imag());
    KD_CUDA(cudaMemcpyAsync(dev_h, host_h.data(), nv * sizeof(double2), cudaMemcpyHostToDevice, ctx->st), "coef");
    k_combine<<<grid_of(len), 256, 0, ctx->st>>>(w, keep ? 1 : 0, V, nv, len, dev_h);
    KD_CUDA(cudaGetLastError(), "combine");
    // host_h is reused by the next call: the copy must have left it
    KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
    return KD_OK;
  }
  kd_status norm(const double2* w, double* out) {
    k_dots_partial<<<dim3(kDotBlocks, 1), kDotThreads, 0, ctx->st>>>(w, len, w, partial);
    k_dots_finish<<<1, 64, 0, ctx->st>>>(partial, kDotBlocks, 1, dev_h);
    KD_CUDA(cudaGetLastError(), "norm");
    KD_CUDA(cudaMemcpyAsync(host_h.data(), dev_h, sizeof(double2), cudaMemcpyDeviceToHost, ctx->st), "norm");
    KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
    *out = sqrt(host_h[0].x);
    return KD_OK;
  }
};

}  // namespace

extern "C" kd_status kd_growth_arnoldi(kd_ctx* ctx, const double* b0, double t0, double tau, int m, int nev,
                                       int restarts, double tol, double* mu, double* rate, int* iters,
                                       double* b_out) {
  if (!ctx) return KD_EINVAL;
  if (!b0 || !mu) return fail(ctx, KD_EINVAL, "kd_growth_arnoldi: NULL buffer");
  if (!(tau > 0) || !isfinite(tau) || !isfinite(t0)) return fail(ctx, KD_EINVAL, "kd_growth_arnoldi: tau must be > 0");
  if (m < 2 || m > KD_ARNOLDI_MAX_M || nev < 1 || nev >= m || restarts < 1 || !(tol >= 0))
    return fail(ctx, KD_EINVAL, "kd_growth_arnoldi: need 2 <= m <= 64, 1 <= nev < m, restarts >= 1, tol >= 0");
  const int n = ctx->p.n;
  const bool conv = conv_op(ctx);
  const int pf = ctx->p.prec_fine;
  const long len = compact_len(n);
  const int S = steps_for(tau, ctx->p.dt_fine);
  const double dt = tau / S;
  kd_status s;
  if ((s = ensure_ws(ctx, ctx->ws_f, n, pf, 1)) != KD_OK) return s;
  if ((s = ensure_full_tmp(ctx, 3UL * n * n * 16)) != KD_OK) return s;
  Arnoldi ar;
  ar.ctx = ctx;
  ar.len = len;
  ar.host_h.resize(m + 1);
  if ((s = dalloc(ctx, (void**)&ar.V, (size_t)(m + 1) * len * 16, "Arnoldi basis")) != KD_OK) return s;
  struct Free {
    kd_ctx* c;
    Arnoldi* a;
    ~Free() {
      cudaStreamSynchronize(c->st);
      dfree(c, a->V);
      dfree(c, a->partial);
      dfree(c, a->dev_h);
    }
  } release{ctx, &ar};
  if ((s = dalloc(ctx, (void**)&ar.partial, (size_t)(m + 1) * kDotBlocks * 16, "Arnoldi partials")) != KD_OK ||
      (s = dalloc(ctx, (void**)&ar.dev_h, (size_t)(m + 1) * 16, "Arnoldi coefficients")) != KD_OK)
    return s;
  double* tdev = ctx->scal + 10;
  KD_CUDA(cudaMemcpyAsync(tdev, &t0, 8, cudaMemcpyHostToDevice, ctx->st), "t0");
  FineArgs a = fine_args(ctx, ctx->ws_f, ctx->tab_f, n, 1, dt, tdev);
  if ((s = with_phases(ctx, ctx->ws_f, a, S)) != KD_OK) return s;
  // start vector: the dealiased b0
  KD_CUDA(cudaMemcpyAsync(ctx->full_tmp, b0, 3UL * n * n * 16, cudaMemcpyDefault, ctx->st), "copy b0");
  KD_LAUNCH(full_to_compact(KD_C128, ctx->full_tmp, KD_C128, ar.V, 1, n, ctx->st), "pack");

  // w = M v (FP64 in and out; the propagator in the context's fine precision)
  auto apply = [&](const double2* v, double2* w) -> kd_status {
    if (conv) return conv_fine(ctx, (const double*)v, (double*)w, 1, S, dt, tdev);
    KD_LAUNCH(compact_resample(KD_C128, v, n, pf, ctx->ws_f.X, n, 1, ctx->st), "to fine precision");
    KD_LAUNCH(run_fine(ctx, 0, pf, a, S, true, false), "fine steps");
    KD_LAUNCH(compact_resample(pf, ctx->ws_f.X, n, KD_C128, w, n, 1, ctx->st), "to FP64");
    return KD_OK;
  };

  std::vector<cd> H, T, Q, h1, h2;
  std::vector<int> order;
  std::vector<std::vector<cd>> Y(nev);
  std::vector<double> res(nev);
  int used = 0;
  bool converged = false;
  for (int rs = 0; rs < restarts && !converged; ++rs) {
    used = rs + 1;
    double nrm;
    if ((s = ar.norm(ar.V, &nrm)) != KD_OK) return s;
    if (!(nrm > 0) || !isfinite(nrm)) return fail(ctx, KD_ENONFINITE, "kd_growth_arnoldi: zero or non-finite start vector");
    k_scale<<<grid_of(len), 256, 0, ctx->st>>>(ar.V, len, 1.0 / nrm);
    H.assign((size_t)(m + 1) * m, cd(0.0));
    int mm = m;   // Krylov dimension reached (smaller on an invariant subspace)
    double hnorm = 0.0;
    for (int j = 0; j < m; ++j) {
      double2* w = ar.V + (long)(j + 1) * len;
      if ((s = apply(ar.V + (long)j * len, w)) != KD_OK) return s;
      // classical Gram-Schmidt, twice
      if ((s = ar.dots(j + 1, w, h1)) != KD_OK) return s;
      std::vector<cd> neg(j + 1);
      for (int i = 0; i <= j; ++i) neg[i] = -h1[i];
      if ((s = ar.combine(w, true, j + 1, neg)) != KD_OK) return s;
      if ((s = ar.dots(j + 1, w, h2)) != KD_OK) return s;
      for (int i = 0; i <= j; ++i) neg[i] = -h2[i];
      if ((s = ar.combine(w, true, j + 1, neg)) != KD_OK) return s;
      double beta;
      if ((s = ar.norm(w, &beta)) != KD_OK) return s;
      if (!isfinite(beta)) return fail(ctx, KD_ENONFINITE, "kd_growth_arnoldi: non-finite Krylov vector");
      for (int i = 0; i <= j; ++i) {
        H[(size_t)i * m + j] = h1[i] + h2[i];
        hnorm = std::max(hnorm, std::abs(H[(size_t)i * m + j]));
      }
      H[(size_t)(j + 1) * m + j] = beta;
      if (beta <= 1e-13 * std::max(hnorm, 1e-300)) {   // invariant subspace: the Ritz values are exact
        mm = j + 1;
        break;
      }
      k_scale<<<grid_of(len), 256, 0, ctx->st>>>(w, len, 1.0 / beta);
    }
    if (mm <= nev) return fail(ctx, KD_ENOTCONV, "kd_growth_arnoldi: the Krylov space closed before nev vectors");
    // Ritz values and vectors of the leading mm x mm block
    T.assign((size_t)mm * mm, cd(0.0));
    for (int i = 0; i < mm; ++i)
      for (int j = 0; j < mm; ++j) T[(size_t)i * mm + j] = H[(size_t)i * m + j];
    if (!hessenberg_schur(T, Q, mm)) return fail(ctx, KD_ENOTCONV, "kd_growth_arnoldi: Hessenberg QR did not converge");
    order.resize(mm);
    for (int i = 0; i < mm; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
      return std::abs(T[(size_t)x * mm + x]) > std::abs(T[(size_t)y * mm + y]);
    });
    const double beta_m = mm < m ? 0.0 : std::abs(H[(size_t)m * m + (m - 1)]);
    converged = true;
    for (int q = 0; q < nev; ++q) {
      const int p = order[q];
      Y[q] = schur_vector(T, Q, mm, p);
      const cd theta = T[(size_t)p * mm + p];
      res[q] = beta_m * std::abs(Y[q][mm - 1]) / std::max(std::abs(theta), 1e-300);
      mu[2 * q] = theta.real();
      mu[2 * q + 1] = theta.imag();
      if (rate) rate[q] = log(std::abs(theta)) / tau;
      if (!(res[q] <= tol)) converged = false;
    }
    // next start vector (or the output): the sum of the wanted Ritz vectors, into V[m]
    // (no longer needed as a basis vector), then V[0]
    std::vector<cd> c(mm, cd(0.0));
    for (int q = 0; q < nev; ++q)
      for (int i = 0; i < mm; ++i) c[i] += Y[q][i];
    double2* x = ar.V + (long)m * len;
    if ((s = ar.combine(x, false, mm, c)) != KD_OK) return s;
    KD_CUDA(cudaMemcpyAsync(ar.V, x, (size_t)len * 16, cudaMemcpyDeviceToDevice, ctx->st), "restart");
    if (b_out && (converged || rs + 1 == restarts)) {
      // the leading Ritz vector, unit norm
      if ((s = ar.combine(x, false, mm, Y[0])) != KD_OK) return s;
      KD_LAUNCH(compact_to_full(KD_C128, x, KD_C128, ctx->full_tmp, 1, n, ctx->st), "unpack");
      KD_CUDA(cudaMemcpyAsync(b_out, ctx->full_tmp, 3UL * n * n * 16, cudaMemcpyDefault, ctx->st), "copy out");
      KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
    }
  }
  if (iters) *iters = used;
  return converged ? KD_OK : fail(ctx, KD_ENOTCONV, "kd_growth_arnoldi: tol not reached");
}

extern "C" kd_status kd_hessenberg_eig(int m, const double* h, double* eig, double* vec) {
  if (m < 1 || m > 4096 || !h || !eig) return KD_EINVAL;
  std::vector<cd> T((size_t)m * m), Q;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      if (i > j + 1 && (h[2 * ((size_t)i * m + j)] != 0.0 || h[2 * ((size_t)i * m + j) + 1] != 0.0)) return KD_EINVAL;
      T[(size_t)i * m + j] = cd(h[2 * ((size_t)i * m + j)], h[2 * ((size_t)i * m + j) + 1]);
    }
  if (!hessenberg_schur(T, Q, m)) return KD_ENOTCONV;
  for (int p = 0; p < m; ++p) {
    eig[2 * p] = T[(size_t)p * m + p].real();
    eig[2 * p + 1] = T[(size_t)p * m + p].imag();
    if (vec) {
      const std::vector<cd> y = schur_vector(T, Q, m, p);
      for (int i = 0; i < m; ++i) {
        vec[2 * ((size_t)i * m + p)] = y[i].real();
        vec[2 * ((size_t)i * m + p) + 1] = y[i].imag();
      }
    }
  }
  return KD_OK;
}
