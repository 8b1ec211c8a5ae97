// C ABI (include/kd.h): context, workspaces, the fine / coarse propagators and the
// one-GPU Parareal driver (Sec. 3, Eq. 8 and Eq. 9; Algorithms of Sec. 4.1).
//
// Parareal on one GPU keeps every slice state on the device in FP64 compact form:
//   U  [N+1][3][P][P]   current iterate at the slice boundaries
//   Fv [N][3][P][P]     fine values F(U_n) of the last parallel step
//   Gv [N][3][Pc][Pc]   coarse values G(U_n) of the last serial sweep
// The parallel step converts U_n to the fine precision, advances all active slices
// in one batched propagation and converts back.  The serial sweep restricts U_n to
// the coarse grid, takes the coarse steps and applies the FP64 update
// U_{n+1} = F + (G_new - G_old) in one kernel.  Slices that are already exact are
// skipped (after k iterations U_0..U_k equal the serial fine solution and their
// coarse terms cancel exactly); this changes no value.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <complex>
#include <string>
#include <vector>

#include "../../include/kd.h"
#include "kd_coarse.h"
#include "kd_ctx.h"
#include "kd_fine.h"
#include "kd_learned.h"

using namespace kd;
using namespace kdi;

namespace kdi {

kd_status fail(kd_ctx* c, kd_status s, const std::string& m) {
  if (c) c->err = m;
  return s;
}

kd_status cuda_fail(kd_ctx* c, cudaError_t e, const char* where) {
  return fail(c, e == cudaErrorMemoryAllocation ? KD_ENOMEM : KD_ECUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

bool valid_n(int n) {
  return n == 16 || n == 32 || n == 64 || n == 128 || n == 256 || n == 512 || n == 1024;
}

kd_status dalloc(kd_ctx* ctx, void** p, size_t bytes, const char* what) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  // the context's allocation limit refuses the buffer as a failed cudaMalloc would
  if (ctx->alloc_limit && (bytes > ctx->alloc_limit || ctx->alloc_held > ctx->alloc_limit - bytes))
    return fail(ctx, KD_ENOMEM, std::string("allocation limit: ") + what + " (" + std::to_string(bytes) +
                                    " B) with " + std::to_string(ctx->alloc_held) + " B held exceeds the limit of " +
                                    std::to_string(ctx->alloc_limit) + " B");
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, KD_ENOMEM, std::string("cudaMalloc ") + what + " (" + std::to_string(bytes) + " B): " +
                                    cudaGetErrorString(e));
  }
  size_t i = 0;
  while (i < ctx->allocs.size() && ctx->allocs[i]) ++i;   // reuse a freed entry
  if (i == ctx->allocs.size()) {
    ctx->allocs.push_back(nullptr);
    ctx->alloc_sizes.push_back(0);
  }
  ctx->allocs[i] = *p;
  ctx->alloc_sizes[i] = bytes;
  ctx->alloc_held += bytes;
  ++ctx->alloc_gen;
  return KD_OK;
}

// Release a live buffer of this context; any other pointer (NULL, one already released)
// is left alone.
void dfree(kd_ctx* ctx, void* p) {
  if (!p) return;
  for (size_t i = 0; i < ctx->allocs.size(); ++i)
    if (ctx->allocs[i] == p) {
      cudaFree(p);
      ctx->allocs[i] = nullptr;
      ctx->alloc_held -= ctx->alloc_sizes[i];
      ctx->alloc_sizes[i] = 0;
      return;
    }
}

kd_status make_tables(kd_ctx* ctx, Tables& t, int n, int prec) {
  if (t.n == n && t.prec == prec) return KD_OK;
  std::vector<double> tw(2 * n), cg(n), sg(n);
  for (int e = 0; e < n; ++e) {
    // exp(-2 pi i e / n) and the collocation points 2 pi e / n, in double
    const double a = 2.0 * M_PI * (double)e / (double)n;
    tw[2 * e] = cos(a);
    tw[2 * e + 1] = -sin(a);
    cg[e] = cos(a);
    sg[e] = sin(a);
  }
  // exact values where the angle is a multiple of pi/2 (sides divisible by 4)
  for (int e = 0; n % 4 == 0 && e < n; e += n / 4) {
    const int q = (e / (n / 4)) & 3;
    const double c = q == 0 ? 1.0 : q == 2 ? -1.0 : 0.0;
    const double s = q == 1 ? 1.0 : q == 3 ? -1.0 : 0.0;
    tw[2 * e] = c;
    tw[2 * e + 1] = -s;
    cg[e] = c;
    sg[e] = s;
  }
  const size_t es = prec == KD_C128 ? 8 : 4;
  kd_status s;
  if ((s = dalloc(ctx, &t.tw, 2 * n * es, "twiddles")) != KD_OK) return s;
  if ((s = dalloc(ctx, &t.cosg, n * es, "cos table")) != KD_OK) return s;
  if ((s = dalloc(ctx, &t.sing, n * es, "sin table")) != KD_OK) return s;
  if (prec == KD_C128) {
    KD_CUDA(cudaMemcpy(t.tw, tw.data(), 2 * n * 8, cudaMemcpyHostToDevice), "tables");
    KD_CUDA(cudaMemcpy(t.cosg, cg.data(), n * 8, cudaMemcpyHostToDevice), "tables");
    KD_CUDA(cudaMemcpy(t.sing, sg.data(), n * 8, cudaMemcpyHostToDevice), "tables");
  } else {
    std::vector<float> a(2 * n), b(n), c(n);
    for (int i = 0; i < 2 * n; ++i) a[i] = (float)tw[i];
    for (int i = 0; i < n; ++i) {
      b[i] = (float)cg[i];
      c[i] = (float)sg[i];
    }
    KD_CUDA(cudaMemcpy(t.tw, a.data(), 2 * n * 4, cudaMemcpyHostToDevice), "tables");
    KD_CUDA(cudaMemcpy(t.cosg, b.data(), n * 4, cudaMemcpyHostToDevice), "tables");
    KD_CUDA(cudaMemcpy(t.sing, c.data(), n * 4, cudaMemcpyHostToDevice), "tables");
  }
  t.n = n;
  t.prec = prec;
  return KD_OK;
}

kd_status ensure_ws(kd_ctx* ctx, FineWs& w, int n, int prec, long batch) {
  if (w.cap >= batch && w.n == n && w.prec == prec) return KD_OK;
  dfree(ctx, w.X);
  dfree(ctx, w.R2);
  dfree(ctx, w.R3);
  dfree(ctx, w.R4);
  dfree(ctx, w.Xlo);
  dfree(ctx, w.M);
  dfree(ctx, w.W);
  dfree(ctx, w.ph);
  w = FineWs();
  const size_t es = csize(prec);
  const size_t spec = (size_t)batch * compact_len(n) * es;
  const size_t mixed = (size_t)batch * 3 * kept(n) * fine_fft_grid(n) * es;   // x on the transform's grid
  kd_status s;
  if ((s = dalloc(ctx, &w.X, spec, "state")) != KD_OK) return s;
  if ((s = dalloc(ctx, &w.R2, spec, "R2")) != KD_OK) return s;
  if ((s = dalloc(ctx, &w.R3, spec, "R3")) != KD_OK) return s;
  if ((s = dalloc(ctx, &w.R4, spec, "R4")) != KD_OK) return s;
  // complex64 state: its low part within a propagation call (kd_stage.cuh)
  if (prec == KD_C64 && (s = dalloc(ctx, &w.Xlo, spec, "state low part")) != KD_OK) return s;
  if ((s = dalloc(ctx, &w.M, mixed, "mixed M")) != KD_OK) return s;
  if ((s = dalloc(ctx, &w.W, mixed, "mixed W")) != KD_OK) return s;
  w.cap = batch;
  w.n = n;
  w.prec = prec;
  return KD_OK;
}

FineArgs fine_args(const kd_ctx* ctx, const FineWs& w, const Tables& t, int n, long batch, double dt,
                   const double* t0) {
  FineArgs a;
  a.n = fine_fft_grid(n);   // the transforms' side; the kept set is that of n
  a.K = n / 3;
  a.P = kept(n);
  a.batch = (int)batch;
  a.flow = ctx->p.flow;
  a.amp = ctx->p.flow == KD_FLOW_ROBERTS ? 1.0 : ctx->p.flow == KD_FLOW_GALLOWAY_PROCTOR ? sqrt(1.5) : 0.0;
  a.kz = ctx->p.kz;
  a.Rm = ctx->p.Rm;
  a.dt = dt;
  a.t0 = t0;
  a.X = w.X;
  a.R2 = w.R2;
  a.R3 = w.R3;
  a.R4 = w.R4;
  a.Xlo = w.Xlo;
  a.lo_valid = 0;
  a.M = w.M;
  a.W = w.W;
  a.tw = t.tw;
  a.cosg = t.cosg;
  a.sing = t.sing;
  a.phases = nullptr;
  a.phase_steps = 0;
  a.sp = nullptr;
  // the fine workspace steps with the fine scheme; the coarse propagator is RK443
  a.scheme = &w == &ctx->ws_f ? ctx->p.fine_scheme : SCHEME_RK443;
  return a;
}

constexpr size_t PROF_EVENTS = 16384;

void prof_flush(kd_ctx* ctx) {
  if (ctx->pev_used == 0) return;
  cudaEventSynchronize(ctx->pev[ctx->pev_used - 1]);
  for (size_t i = 0; i + 1 < ctx->pev_used; i += 2) {
    float m = 0.f;
    if (cudaEventElapsedTime(&m, ctx->pev[i], ctx->pev[i + 1]) == cudaSuccess) {
      ctx->prof_ms[ctx->pkid[i / 2]] += m;
      ctx->prof_n[ctx->pkid[i / 2]] += 1;
    }
  }
  ctx->pev_used = 0;
  ctx->pkid.clear();
}

void probe_before(void* u, int kid) {
  kd_ctx* ctx = (kd_ctx*)u;
  if (ctx->pev_used + 2 > PROF_EVENTS) prof_flush(ctx);
  while (ctx->pev.size() < ctx->pev_used + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    ctx->pev.push_back(e);
  }
  cudaEventRecord(ctx->pev[ctx->pev_used], ctx->st);
  ctx->pkid.push_back(kid);
}

void probe_after(void* u, int) {
  kd_ctx* ctx = (kd_ctx*)u;
  cudaEventRecord(ctx->pev[ctx->pev_used + 1], ctx->st);
  ctx->pev_used += 2;
}

LaunchProbe probe_of(kd_ctx* ctx) {
  LaunchProbe p;
  p.before = probe_before;
  p.after = probe_after;
  p.user = ctx;
  return p;
}

// Make room for the flow-phase table of `nsteps` steps and point the arguments at it.
kd_status with_phases(kd_ctx* ctx, FineWs& w, FineArgs& a, int nsteps) {
  a.phase_steps = nsteps;
  a.phases = nullptr;
  if (a.flow != KD_FLOW_GALLOWAY_PROCTOR || nsteps <= 0) return KD_OK;
  const size_t need = phase_table_bytes(w.prec, a.batch, nsteps);
  if (w.ph_bytes < need) {
    dfree(ctx, w.ph);
    w.ph = nullptr;
    w.ph_bytes = 0;
    kd_status s = dalloc(ctx, &w.ph, need, "phase table");
    if (s != KD_OK) return s;
    w.ph_bytes = need;
  }
  a.phases = w.ph;
  return KD_OK;
}

int run_fine(kd_ctx* ctx, int g, int prec, const FineArgs& a, int nsteps, bool prologue, bool store_last,
             const LaunchProbe* probe, const int* active) {
  StepCfg cfg;
  cfg.nsteps = nsteps;
  cfg.prologue = prologue;
  cfg.store_last = store_last;
  cfg.active = active;
  cfg.probe = probe;
  cfg.plan = ctx->plan[g];
  cfg.pdl = ctx->pdl != 0;
  cfg.st = ctx->st;
  return fine_run(prec, a, cfg);
}

kd_status ensure_full_tmp(kd_ctx* ctx, size_t bytes) {
  if (ctx->full_tmp_bytes >= bytes) return KD_OK;
  dfree(ctx, ctx->full_tmp);
  ctx->full_tmp = nullptr;
  ctx->full_tmp_bytes = 0;
  kd_status s = dalloc(ctx, &ctx->full_tmp, bytes, "staging");
  if (s == KD_OK) ctx->full_tmp_bytes = bytes;
  return s;
}

kd_status ensure_slices(kd_ctx* ctx, long N) {
  if (ctx->cap_slices >= N) return KD_OK;
  dfree(ctx, ctx->U);
  dfree(ctx, ctx->Fv);
  dfree(ctx, ctx->Gv);
  dfree(ctx, ctx->t0f);
  dfree(ctx, ctx->t0c);
  dfree(ctx, ctx->Uprev);
  // no stale pointer survives a failed allocation below
  ctx->U = ctx->Fv = ctx->Gv = ctx->t0f = ctx->t0c = ctx->Uprev = nullptr;
  ctx->cap_slices = 0;
  const int n = ctx->p.n;
  kd_status s;
  if ((s = dalloc(ctx, (void**)&ctx->U, (N + 1) * compact_len(n) * 16, "U")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&ctx->Fv, N * compact_len(n) * 16, "F values")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&ctx->Gv, N * 3L * ctx->cP * ctx->cP * 16, "G values")) != KD_OK) return s;
  if (ctx->p.fine_form == KD_FINE_INCREMENT &&
      (s = dalloc(ctx, (void**)&ctx->Uprev, N * compact_len(n) * 16, "previous iterate")) != KD_OK)
    return s;
  if ((s = dalloc(ctx, (void**)&ctx->t0f, (N + 1) * 8, "t0")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&ctx->t0c, (N + 1) * 8, "t0")) != KD_OK) return s;
  ctx->cap_slices = N;
  return KD_OK;
}

int steps_for(double dT, double dt) {
  double q = dT / dt;
  int s = (int)ceil(q - 1e-9 * (q > 1 ? q : 1));
  return s < 1 ? 1 : s;
}

kd_status check_params(const kd_params* p, std::string& why) {
  if (!p) return why = "params is NULL", KD_EINVAL;
  if (p->flow < 0 || p->flow > 2) return why = "flow must be 0, 1 or 2", KD_EINVAL;
  // the convolution operator's limit is checked in kd_create against the cluster solver
  if (p->n < 16 || p->n > 1024 || (p->n & 1)) return why = "n must be even and in [16, 1024]", KD_EINVAL;
  if (p->n_coarse < 16 || p->n_coarse > p->n || (p->n_coarse & 1))
    return why = "n_coarse must be even and in [16, n]", KD_EINVAL;
  if (p->fine_operator == KD_FINE_FFT && fine_fft_grid(p->n) == 0)
    return why = "n must be a power of two or an even side <= 286 (fine_operator KD_FINE_FFT)", KD_EINVAL;
  if (!(p->Rm > 0) || !isfinite(p->Rm)) return why = "Rm must be finite and > 0", KD_EINVAL;
  if (!isfinite(p->kz)) return why = "kz must be finite", KD_EINVAL;
  if (!(p->dt_fine > 0) || !(p->dt_coarse > 0)) return why = "time steps must be > 0", KD_EINVAL;
  if ((p->prec_fine != KD_C64 && p->prec_fine != KD_C128) || (p->prec_coarse != KD_C64 && p->prec_coarse != KD_C128))
    return why = "precision must be KD_C64 or KD_C128", KD_EINVAL;
  if (p->coarse_kind != KD_COARSE_CLASSICAL && p->coarse_kind != KD_COARSE_LEARNED) return why = "bad coarse_kind", KD_EINVAL;
  if (p->learned_modes < 0 || p->learned_modes == 1 || p->learned_modes / 2 > p->n / 3 ||
      p->learned_modes - p->learned_modes / 2 - 1 > p->n / 3 || p->learned_modes > 64)
    return why = "learned_modes: the set [-m/2, m - m/2) must lie in |k| <= n/3, m <= 64", KD_EINVAL;
  if (p->coarse_kind == KD_COARSE_LEARNED && (p->learned_modes == 0 || p->fine_form != KD_FINE_INCREMENT))
    return why = "the learned coarse propagator needs learned_modes > 0 and fine_form KD_FINE_INCREMENT", KD_EINVAL;
  if (p->fine_form != KD_FINE_DIRECT && p->fine_form != KD_FINE_INCREMENT) return why = "bad fine_form", KD_EINVAL;
  if (p->fine_operator != KD_FINE_FFT && p->fine_operator != KD_FINE_CONV) return why = "bad fine_operator", KD_EINVAL;

  if (p->fine_scheme != KD_RK443 && p->fine_scheme != KD_RK222 && p->fine_scheme != KD_RK111)
    return why = "bad fine_scheme", KD_EINVAL;
  if (p->fine_operator == KD_FINE_CONV && p->fine_scheme != KD_RK443)
    return why = "fine_operator KD_FINE_CONV steps with RK443 only", KD_EINVAL;
  return KD_OK;
}

// Coarse flow phases of every slice: [N][Sc][4][4] in the coarse precision.
kd_status coarse_phases(kd_ctx* ctx, int N, int Sc, double dtc) {
  if (ctx->p.flow != KD_FLOW_GALLOWAY_PROCTOR) return KD_OK;
  const size_t need = phase_table_bytes(ctx->p.prec_coarse, N, Sc);
  if (ctx->ph_c_bytes < need) {
    dfree(ctx, ctx->ph_c);
    ctx->ph_c = nullptr;
    ctx->ph_c_bytes = 0;
    kd_status s = dalloc(ctx, &ctx->ph_c, need, "coarse phase table");
    if (s != KD_OK) return s;
    ctx->ph_c_bytes = need;
  }
  FineArgs a = fine_args(ctx, ctx->ws_c, ctx->tab_c, ctx->p.n_coarse, N, dtc, ctx->t0c);
  a.phases = ctx->ph_c;
  KD_LAUNCH(launch_phases(ctx->p.prec_coarse, a, Sc, ctx->st), "coarse phases");
  return KD_OK;
}

CoarseArgs coarse_args(const kd_ctx* ctx, int steps, double dtc) {
  CoarseArgs c;
  memset(&c, 0, sizeof(c));
  c.Kc = ctx->cK;
  c.Pc = ctx->cP;
  c.Kf = ctx->p.n / 3;
  c.Pf = 2 * c.Kf + 1;
  c.flow = ctx->p.flow;
  c.amp = ctx->p.flow == KD_FLOW_ROBERTS ? 1.0 : ctx->p.flow == KD_FLOW_GALLOWAY_PROCTOR ? sqrt(1.5) : 0.0;
  c.kz = ctx->p.kz;
  c.Rm = ctx->p.Rm;
  c.dt = dtc;
  c.nsteps = steps;
  c.cluster = ctx->coarse_cluster;
  c.halo = ctx->coarse_sync == KD_SYNC_P2P ? 1 : ctx->coarse_sync == KD_SYNC_PULL ? 2 : 0;
  return c;
}

// Serial-sweep step of slice i with a coarse solve:
//   init:      U_{i+1} = G(U_i),                        Gv_i = G(U_i)
//   direct:    U_{i+1} = Fv_i + (G(U_i) - Gv_i),         Gv_i = G(U_i)
//   increment: U_{i+1} = Fv_i + G(U_i - Uprev_i)   (G linear; Uprev_i = previous iterate)
// (+ sigma of U_{i+1} when `last`).
kd_status coarse_step(kd_ctx* ctx, int i, int Sc, double dtc, bool init, bool last) {
  const int n = ctx->p.n, nc = ctx->p.n_coarse, pc = ctx->p.prec_coarse;
  const long len = compact_len(n), lenc = 3L * ctx->cP * ctx->cP;
  const bool incr = !init && ctx->p.fine_form == KD_FINE_INCREMENT;
  if (coarse_conv_supported(ctx->cP)) {
    CoarseArgs c = coarse_args(ctx, Sc, dtc);
    c.phases = ctx->ph_c ? (const char*)ctx->ph_c + (size_t)i * Sc * 16 * (pc == KD_C64 ? 4 : 8) : nullptr;
    if (ctx->p.flow != KD_FLOW_GALLOWAY_PROCTOR) c.phases = nullptr;
    c.Un = ctx->U + 2 * i * len;
    c.Uprev = incr ? ctx->Uprev + 2 * i * len : nullptr;
    c.mode = init ? COARSE_INIT : (incr ? COARSE_INCR : COARSE_UPDATE);
    c.Fv = init ? nullptr : ctx->Fv + 2 * i * len;
    c.Gold = ctx->Gv + 2 * i * lenc;
    c.Unext = ctx->U + 2 * (i + 1) * len;
    c.sigma_out = last ? ctx->scal : nullptr;
    KD_LAUNCH(coarse_conv_launch(pc, c, 1, ctx->st), "coarse solve");
    return KD_OK;
  }
  // general grids: restrict, multi-kernel RK443 steps, separate update
  const double* src = ctx->U + 2 * i * len;
  if (incr) {
    kd_status s0 = ensure_full_tmp(ctx, (size_t)len * 16);
    if (s0 != KD_OK) return s0;
    KD_LAUNCH(diff_kernel(src, ctx->Uprev + 2 * i * len, (double*)ctx->full_tmp, len, ctx->st), "increment");
    src = (const double*)ctx->full_tmp;
  }
  KD_LAUNCH(compact_resample(KD_C128, src, n, pc, ctx->ws_c.X, nc, 1, ctx->st), "restrict");
  FineArgs a = fine_args(ctx, ctx->ws_c, ctx->tab_c, nc, 1, dtc, ctx->t0c + i);
  kd_status s = with_phases(ctx, ctx->ws_c, a, Sc);
  if (s != KD_OK) return s;
  KD_LAUNCH(run_fine(ctx, 1, pc, a, Sc, true, false), "coarse steps");
  int nb = parareal_update(init ? nullptr : ctx->Fv + 2 * i * len, ctx->ws_c.X, pc, ctx->Gv + 2 * i * lenc,
                           ctx->U + 2 * (i + 1) * len, n, nc / 3, 2 * (nc / 3) + 1, init ? 1 : (incr ? 2 : 0),
                           last ? ctx->partials : nullptr, ctx->st);
  if (nb < 0) return fail(ctx, KD_ECUDA, "parareal update launch failed");
  ctx->launches += 1;
  if (last) KD_LAUNCH(finish_sigma(ctx->partials, nb, ctx->scal, ctx->st), "sigma");
  return KD_OK;
}

// Serial-sweep step of slice i with the learned coarse operator of phase i mod n_phase:
//   init:      U_{i+1} = P W R U_i
//   increment: U_{i+1} = Fv_i + P W R (U_i - Uprev_i)
kd_status learned_step(kd_ctx* ctx, int i, bool init, bool last) {
  const int n = ctx->p.n, Kf = n / 3, Pf = 2 * Kf + 1;
  const int K = ctx->cK, P = ctx->cP, nc = 3 * P * P;
  const long len = compact_len(n);
  const int ph = (ctx->blk_lo + i) % ctx->l_nphase;   // phase of the global slice index
  float* x = ctx->l_x;
  float* y = ctx->l_x + 2 * nc;
  KD_LAUNCH(learned_gather(ctx->U + 2 * i * len, init ? nullptr : ctx->Uprev + 2 * i * len, Kf, Pf, x, K, P, 1,
                           ctx->st),
            "learned gather");
  const int ld = (nc + 7) & ~7;
  KD_LAUNCH(learned_gemv(ctx->l_W + (size_t)ph * 2 * nc * ld, x, y, nc, ld, 1, ctx->st), "learned gemv");
  int nb = learned_update(init ? nullptr : ctx->Fv + 2 * i * len, y, K, P, ctx->U + 2 * (i + 1) * len, Kf, Pf,
                          init ? 1 : 0, last ? ctx->partials : nullptr, ctx->st);
  if (nb < 0) return fail(ctx, KD_ECUDA, "learned update launch failed");
  ctx->launches += 1;
  if (last) KD_LAUNCH(finish_sigma(ctx->partials, nb, ctx->scal, ctx->st), "sigma");
  return KD_OK;
}

bool use_learned(const kd_ctx* ctx, int i) {
  return ctx->p.coarse_kind == KD_COARSE_LEARNED && !ctx->fallback && ctx->l_nphase > 0 &&
         ctx->l_valid[(ctx->blk_lo + i) % ctx->l_nphase];
}

// Fine propagator in the spectral-convolution form (KD_FINE_CONV): `batch` FP64 compact
// fields `in` (fine set) -> `out` (may alias), nsteps steps of dt from t0[b], all in one
// persistent cluster launch with arithmetic in the fine precision.
kd_status conv_fine(kd_ctx* ctx, const double* in, double* out, long batch, int nsteps, double dt, const double* t0) {
  const int n = ctx->p.n, pf = ctx->p.prec_fine;
  // the fine workspace only carries the flow-phase table here
  kd_status s = ensure_ws(ctx, ctx->ws_f, n, pf, 1);
  if (s != KD_OK) return s;
  FineArgs a = fine_args(ctx, ctx->ws_f, ctx->tab_f, n, batch, dt, t0);
  if ((s = with_phases(ctx, ctx->ws_f, a, nsteps)) != KD_OK) return s;
  KD_LAUNCH(launch_phases(pf, a, nsteps, ctx->st), "fine phases");
  CoarseArgs c = coarse_args(ctx, nsteps, dt);
  c.Kc = n / 3;
  c.Pc = kept(n);
  c.phases = ctx->p.flow == KD_FLOW_GALLOWAY_PROCTOR ? a.phases : nullptr;
  c.Un = in;
  c.mode = COARSE_OUT;
  c.g64 = out;
  KD_LAUNCH(coarse_conv_launch(pf, c, (int)batch, ctx->st), "fine convolution steps");
  return KD_OK;
}

bool conv_op(const kd_ctx* ctx) { return ctx->p.fine_operator == KD_FINE_CONV; }

kd_status ensure_conv_tmp(kd_ctx* ctx, size_t bytes) {
  if (ctx->conv_tmp_bytes >= bytes) return KD_OK;
  dfree(ctx, ctx->conv_tmp);
  ctx->conv_tmp = nullptr;
  ctx->conv_tmp_bytes = 0;
  kd_status s = dalloc(ctx, &ctx->conv_tmp, bytes, "convolution staging");
  if (s == KD_OK) ctx->conv_tmp_bytes = bytes;
  return s;
}

// Parallel fine step over slices [first, N): Fv[n] = F(U[n]), directly or in the
// increment form Fv[n] += F(U[n] - Uprev[n]) (iter > 1).
static kd_status fine_sweep_launches(kd_ctx* ctx, int first, int N, int S, double dt, int iter);

kd_status run_graph(kd_ctx* ctx, const std::string& key, const std::function<kd_status()>& launches) {
  // the graph runs on the context's own capturable stream, ordered after the work
  // enqueued on ctx->st and before what follows there
  if (!ctx->st_g) {
    KD_CUDA(cudaStreamCreateWithFlags(&ctx->st_g, cudaStreamNonBlocking), "graph stream");
    for (cudaEvent_t& e : ctx->gev) KD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "graph event");
  }
  auto it = ctx->gcache.find(key);
  if (it == ctx->gcache.end()) {
    const long long l0 = ctx->launches;
    cudaGraph_t g = nullptr;
    cudaStream_t user = ctx->st;
    KD_CUDA(cudaStreamBeginCapture(ctx->st_g, cudaStreamCaptureModeThreadLocal), "begin capture");
    ctx->st = ctx->st_g;
    const kd_status s = launches();
    ctx->st = user;
    const cudaError_t e = cudaStreamEndCapture(ctx->st_g, &g);
    if (s != KD_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    KD_CUDA(e, "end capture");
    cudaGraphExec_t ge = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    KD_CUDA(ei, "graph instantiate");
    it = ctx->gcache.emplace(key, kd_ctx::GraphEntry{ge, ctx->launches - l0}).first;
    ctx->launches = l0;
  }
  KD_CUDA(cudaEventRecord(ctx->gev[0], ctx->st), "graph fence");
  KD_CUDA(cudaStreamWaitEvent(ctx->st_g, ctx->gev[0], 0), "graph fence");
  KD_CUDA(cudaGraphLaunch(it->second.exec, ctx->st_g), "graph launch");
  KD_CUDA(cudaEventRecord(ctx->gev[1], ctx->st_g), "graph fence");
  KD_CUDA(cudaStreamWaitEvent(ctx->st, ctx->gev[1], 0), "graph fence");
  ctx->launches += it->second.launches;
  return KD_OK;
}

// The FFT operator's fine sweep is ~8 S + 3 launches; with graphs on, the launches of
// one sweep shape are captured once into a CUDA graph (programmatic dependent launches
// included) and replayed; the values are those of the direct launches.
kd_status fine_sweep(kd_ctx* ctx, int first, int N, int S, double dt, int iter) {
  // (not for the pipelined iterations: their chunks already interleave with the serial
  // sweep on separate streams)
  if (!ctx->graphs || ctx->prof || ctx->overlap > 0 || conv_op(ctx) || N - first <= 0)
    return fine_sweep_launches(ctx, first, N, S, dt, iter);
  // the allocations the sweep may make happen before the capture
  {
    FineArgs a0 = fine_args(ctx, ctx->ws_f, ctx->tab_f, ctx->p.n, N - first, dt, ctx->t0f + first);
    kd_status s0 = with_phases(ctx, ctx->ws_f, a0, S);
    if (s0 != KD_OK) return s0;
  }
  long long dbits;
  memcpy(&dbits, &dt, 8);
  char key[192];
  snprintf(key, sizeof(key), "parareal %d %d %d %lld %d %d %d %d %d %llu", first, N, S, dbits, iter == 1 ? 1 : 0,
           ctx->plan[0].col, ctx->plan[0].row, ctx->pdl, ctx->p.fine_form, ctx->alloc_gen);
  return run_graph(ctx, key, [&] { return fine_sweep_launches(ctx, first, N, S, dt, iter); });
}

static kd_status fine_sweep_launches(kd_ctx* ctx, int first, int N, int S, double dt, int iter) {
  const int n = ctx->p.n, pf = ctx->p.prec_fine;
  const long b = N - first;
  if (b <= 0) return KD_OK;
  const long len = compact_len(n);
  const bool incr = ctx->p.fine_form == KD_FINE_INCREMENT;
  if (conv_op(ctx)) {
    if (!incr) return conv_fine(ctx, ctx->U + 2 * first * len, ctx->Fv + 2 * first * len, b, S, dt, ctx->t0f + first);
    kd_status s0 = ensure_conv_tmp(ctx, (size_t)b * len * 16);
    if (s0 != KD_OK) return s0;
    double* tmp = (double*)ctx->conv_tmp;
    KD_LAUNCH(delta_in(KD_C128, ctx->U + 2 * first * len, ctx->Uprev + 2 * first * len, tmp, b * len,
                       iter == 1 ? 1 : 0, ctx->st),
              "increment");
    if ((s0 = conv_fine(ctx, tmp, tmp, b, S, dt, ctx->t0f + first)) != KD_OK) return s0;
    KD_LAUNCH(accum_out(KD_C128, tmp, ctx->Fv + 2 * first * len, b * len, iter == 1 ? 1 : 0, ctx->st), "accumulate");
    return KD_OK;
  }
  if (incr)
    KD_LAUNCH(delta_in(pf, ctx->U + 2 * first * len, ctx->Uprev + 2 * first * len, ctx->ws_f.X, b * len,
                       iter == 1 ? 1 : 0, ctx->st),
              "increment to fine");
  else
    KD_LAUNCH(compact_resample(KD_C128, ctx->U + 2 * first * len, n, pf, ctx->ws_f.X, n, b, ctx->st), "to fine");
  FineArgs a = fine_args(ctx, ctx->ws_f, ctx->tab_f, n, b, dt, ctx->t0f + first);
  kd_status s = with_phases(ctx, ctx->ws_f, a, S);
  if (s != KD_OK) return s;
  LaunchProbe pr = probe_of(ctx);
  KD_LAUNCH(run_fine(ctx, 0, pf, a, S, true, false, ctx->prof ? &pr : nullptr), "fine steps");
  if (incr)
    KD_LAUNCH(accum_out(pf, ctx->ws_f.X, ctx->Fv + 2 * first * len, b * len, iter == 1 ? 1 : 0, ctx->st),
              "accumulate fine");
  else
    KD_LAUNCH(compact_resample(pf, ctx->ws_f.X, n, KD_C128, ctx->Fv + 2 * first * len, n, b, ctx->st), "from fine");
  return KD_OK;
}

kd_status copy_in_b0(kd_ctx* ctx, const double* b0) {
  const int n = ctx->p.n;
  const size_t fb = 3UL * n * n * 16;
  kd_status s = ensure_full_tmp(ctx, fb);
  if (s != KD_OK) return s;
  KD_CUDA(cudaMemcpyAsync(ctx->full_tmp, b0, fb, cudaMemcpyDefault, ctx->st), "copy b0");
  KD_LAUNCH(full_to_compact(KD_C128, ctx->full_tmp, KD_C128, ctx->U, 1, n, ctx->st), "b0 to compact");
  return KD_OK;
}

kd_status copy_out_slices(kd_ctx* ctx, double* u_slices, int N) {
  if (!u_slices) return KD_OK;
  const int n = ctx->p.n;
  const size_t fb = 3UL * n * n * 16;
  kd_status s = ensure_full_tmp(ctx, fb * (N + 1));
  if (s != KD_OK) return s;
  KD_LAUNCH(compact_to_full(KD_C128, ctx->U, KD_C128, ctx->full_tmp, N + 1, n, ctx->st), "slices to full");
  KD_CUDA(cudaMemcpyAsync(u_slices, ctx->full_tmp, fb * (N + 1), cudaMemcpyDefault, ctx->st), "copy slices");
  return KD_OK;
}

// ---------------------------------------------------------------- pipelined Parareal
struct Chunk {
  int lo, hi;
};

// [first, N) split into at most m nearly equal chunks
std::vector<Chunk> chunks_of(int first, int N, int m) {
  std::vector<Chunk> out;
  const int total = N - first;
  const int c = total < m ? total : m;
  for (int j = 0; j < c; ++j) out.push_back({first + j * total / c, first + (j + 1) * total / c});
  return out;
}

// One serial sweep of iteration k on ctx->st.  Before slice i it waits for the fine chunk
// of iteration k holding i (events F, in the order of `wait`); after slice i it releases
// the chunks of iteration k + 1 whose last slice is i (events E, order of `rel`): from
// then on the sweep no longer reads their U / Uprev / Fv, and their U_n^k are final.
kd_status pipelined_sweep(kd_ctx* ctx, int k, int N, int Sc, double dtc, const std::vector<Chunk>& wait,
                          const std::vector<Chunk>& rel) {
  cudaEvent_t* E = &ctx->pev2[0];
  cudaEvent_t* F = &ctx->pev2[kMaxChunks];
  const int n = ctx->p.n;
  const long len = compact_len(n), lenc = 3L * ctx->cP * ctx->cP;
  const int first = k == 0 ? 0 : (k - 1 < N - 1 ? k - 1 : N - 1);
  size_t wj = 0, rj = 0;
  kd_status s;
  for (int i = first; i < N; ++i) {
    while (wj < wait.size() && wait[wj].lo <= i) KD_CUDA(cudaStreamWaitEvent(ctx->st, F[wj++], 0), "wait fine");
    const bool last = k >= 1 && i == N - 1;
    if (k == 0) {
      if ((s = use_learned(ctx, i) ? learned_step(ctx, i, true, false) : coarse_step(ctx, i, Sc, dtc, true, false)) !=
          KD_OK)
        return s;
    } else if (i == first) {
      int nb = parareal_update(ctx->Fv + 2 * i * len, ctx->Gv + 2 * i * lenc, KD_C128, ctx->Gv + 2 * i * lenc,
                               ctx->U + 2 * (i + 1) * len, n, ctx->cK, ctx->cP, 0, last ? ctx->partials : nullptr,
                               ctx->st);
      if (nb < 0) return fail(ctx, KD_ECUDA, "parareal update launch failed");
      ctx->launches += 1;
      if (last) KD_LAUNCH(finish_sigma(ctx->partials, nb, ctx->scal, ctx->st), "sigma");
    } else if ((s = use_learned(ctx, i) ? learned_step(ctx, i, false, last)
                                        : coarse_step(ctx, i, Sc, dtc, false, last)) != KD_OK) {
      return s;
    }
    while (rj < rel.size() && rel[rj].hi - 1 <= i) KD_CUDA(cudaEventRecord(E[rj++], ctx->st), "release");
  }
  while (rj < rel.size()) KD_CUDA(cudaEventRecord(E[rj++], ctx->st), "release");
  return KD_OK;
}

// The fine chunks of iteration k on st2, each after its release event; records F per chunk
// and the span events ts / te.
kd_status pipelined_fine(kd_ctx* ctx, int k, int S, double dt, const std::vector<Chunk>& ck, cudaEvent_t ts,
                         cudaEvent_t te) {
  cudaEvent_t* E = &ctx->pev2[0];
  cudaEvent_t* F = &ctx->pev2[kMaxChunks];
  cudaStream_t saved = ctx->st;
  ctx->st = ctx->st2;
  kd_status s = KD_OK;
  for (size_t j = 0; j < ck.size() && s == KD_OK; ++j) {
    cudaError_t e = cudaStreamWaitEvent(ctx->st2, E[j], 0);
    if (e == cudaSuccess && j == 0) e = cudaEventRecord(ts, ctx->st2);
    if (e != cudaSuccess) {
      s = cuda_fail(ctx, e, "fine chunk wait");
      break;
    }
    s = fine_sweep(ctx, ck[j].lo, ck[j].hi, S, dt, k);
    if (s == KD_OK && (e = cudaEventRecord(F[j], ctx->st2)) != cudaSuccess) s = cuda_fail(ctx, e, "fine chunk done");
  }
  if (s == KD_OK) {
    cudaError_t e = cudaEventRecord(te, ctx->st2);
    if (e != cudaSuccess) s = cuda_fail(ctx, e, "fine span");
  }
  ctx->st = saved;
  return s;
}

// Iterations of kd_parareal_run with the fine sweep of iteration k + 1 overlapping the
// serial sweep of iteration k (speculatively: it only writes Fv / Uprev, which a stop
// after iteration k leaves unused).  Same values as the unpipelined order.
kd_status parareal_pipelined(kd_ctx* ctx, int N, int S, int Sc, double dt, double dtc, int k_max, double tol,
                             std::vector<double>& sig, int& k_done, int& conv, float& ms_fine, float& ms_coarse) {
  const int m = ctx->overlap < kMaxChunks ? ctx->overlap : kMaxChunks;
  cudaEvent_t fs[2] = {ctx->pev2[2 * kMaxChunks], ctx->pev2[2 * kMaxChunks + 1]};
  cudaEvent_t fe[2] = {ctx->pev2[2 * kMaxChunks + 2], ctx->pev2[2 * kMaxChunks + 3]};
  cudaEvent_t cs = ctx->pev2[2 * kMaxChunks + 4], ce = ctx->pev2[2 * kMaxChunks + 5];
  kd_status s;
  auto first_of = [&](int k) { return k - 1 < N - 1 ? k - 1 : N - 1; };
  // size the buffers both streams use for the largest chunk now: a reallocation later
  // would free memory the other stream may still be using
  {
    const int n = ctx->p.n;
    FineArgs a = fine_args(ctx, ctx->ws_f, ctx->tab_f, n, N, dt, ctx->t0f);
    if ((s = with_phases(ctx, ctx->ws_f, a, S)) != KD_OK) return s;
    if (conv_op(ctx) && (s = ensure_conv_tmp(ctx, (size_t)N * compact_len(n) * 16)) != KD_OK) return s;
    if (!coarse_conv_supported(ctx->cP) && (s = ensure_full_tmp(ctx, (size_t)compact_len(n) * 16)) != KD_OK) return s;
  }
  std::vector<Chunk> cur = chunks_of(0, N, m);
  // iterate 0 releases the chunks of iteration 1
  KD_CUDA(cudaEventRecord(cs, ctx->st), "event");
  if ((s = pipelined_sweep(ctx, 0, N, Sc, dtc, {}, k_max >= 1 ? cur : std::vector<Chunk>())) != KD_OK) return s;
  KD_CUDA(cudaEventRecord(ce, ctx->st), "event");
  if (k_max >= 1 && (s = pipelined_fine(ctx, 1, S, dt, cur, fs[1], fe[1])) != KD_OK) return s;
  KD_CUDA(cudaEventSynchronize(ce), "sync");
  {
    float m0 = 0.f;
    cudaEventElapsedTime(&m0, cs, ce);
    ms_coarse += m0;
  }
  for (int k = 1; k <= k_max; ++k) {
    const std::vector<Chunk> next = k < k_max ? chunks_of(first_of(k + 1), N, m) : std::vector<Chunk>();
    KD_CUDA(cudaEventRecord(cs, ctx->st), "event");
    if ((s = pipelined_sweep(ctx, k, N, Sc, dtc, cur, next)) != KD_OK) return s;
    KD_CUDA(cudaMemcpyAsync(ctx->host_scal, ctx->scal, 8, cudaMemcpyDeviceToHost, ctx->st), "sigma copy");
    KD_CUDA(cudaEventRecord(ce, ctx->st), "event");
    if (k < k_max && (s = pipelined_fine(ctx, k + 1, S, dt, next, fs[(k + 1) & 1], fe[(k + 1) & 1])) != KD_OK)
      return s;
    KD_CUDA(cudaEventSynchronize(ce), "sync");
    float m1 = 0.f, m2 = 0.f;
    cudaEventElapsedTime(&m1, fs[k & 1], fe[k & 1]);
    cudaEventElapsedTime(&m2, cs, ce);
    ms_fine += m1;
    ms_coarse += m2;
    cur = next;
    const double sigma = ctx->host_scal[0];
    sig.push_back(sigma);
    k_done = k;
    if (!isfinite(sigma)) return fail(ctx, KD_ENONFINITE, "kd_parareal_run: non-finite defect");
    if (sigma <= tol) {
      conv = 1;
      break;
    }
    if (ctx->p.coarse_kind == KD_COARSE_LEARNED && !ctx->fallback &&
        ((k >= 2 && sigma > sig[k - 2]) || (k_max > 1 && k >= k_max / 2)))
      ctx->fallback = 1;
  }
  KD_CUDA(cudaStreamSynchronize(ctx->st2), "sync");   // speculative fine chunks finished
  if (ctx->prof) prof_flush(ctx);
  return KD_OK;
}

}  // namespace kdi

extern "C" {

const char* kd_version(void) { return "kd 0.1 (sm_103a)"; }

const char* kd_last_error(kd_ctx* ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

kd_status kd_create(const kd_params* params, void* cuda_stream, kd_ctx** out) {
  if (!out) return KD_EINVAL;
  *out = nullptr;
  std::string why;
  kd_status s = check_params(params, why);
  if (s != KD_OK) {
    fprintf(stderr, "kd_create: %s\n", why.c_str());
    return s;
  }
  kd_ctx* ctx = new kd_ctx();
  ctx->p = *params;
  ctx->plan[0] = fine_default_plan(params->n, params->prec_fine);
  ctx->plan[1] = fine_default_plan(params->n_coarse, params->prec_coarse);
  if (params->learned_modes > 0) {
    ctx->cK = params->learned_modes / 2;
    ctx->cP = params->learned_modes;
  } else {
    ctx->cK = params->n_coarse / 3;
    ctx->cP = 2 * ctx->cK + 1;
  }
  ctx->st = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = fine_prepare(params->prec_fine);
  if (e == cudaSuccess) e = fine_prepare(params->prec_coarse);
  if (e == cudaSuccess) e = coarse_prepare(params->prec_coarse);
  if (e == cudaSuccess && params->fine_operator == KD_FINE_CONV) e = coarse_prepare(params->prec_fine);
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&ctx->ev[i]);
  int prio_lo = 0, prio_hi = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ctx->st2, cudaStreamNonBlocking, prio_lo);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ctx->st_hi, cudaStreamNonBlocking, prio_hi);
  for (int i = 0; i < 2 * kMaxChunks + 6 && e == cudaSuccess; ++i) {
    cudaEvent_t ev;
    e = cudaEventCreate(&ev);
    if (e == cudaSuccess) ctx->pev2.push_back(ev);
  }
  if (e != cudaSuccess) {
    fprintf(stderr, "kd_create: %s\n", cudaGetErrorString(e));
    delete ctx;
    return KD_ECUDA;
  }
  // the kept set the convolution operator's cluster solver must hold (known once its
  // kernels are set up)
  {
    std::string bad;
    if (params->fine_operator == KD_FINE_CONV && !coarse_conv_supported(kept(params->n)))
      bad = "fine_operator KD_FINE_CONV: the kept set of n does not fit the cluster solver (n <= 192)";
    else if (fine_fft_grid(params->n_coarse) == 0 && !coarse_conv_supported(ctx->cP))
      bad = "n_coarse: neither a power of two, nor <= 286, nor a coarse set the cluster solver holds";
    if (!bad.empty()) {
      fprintf(stderr, "kd_create: %s\n", bad.c_str());
      kd_destroy(ctx);
      return KD_EINVAL;
    }
  }
  if ((s = make_tables(ctx, ctx->tab_f, fine_fft_grid(params->n), params->prec_fine)) != KD_OK ||
      (s = make_tables(ctx, ctx->tab_c, fine_fft_grid(params->n_coarse), params->prec_coarse)) != KD_OK ||
      (s = dalloc(ctx, (void**)&ctx->partials, 2 * 1024 * 8, "partials")) != KD_OK ||
      (s = dalloc(ctx, (void**)&ctx->scal, 32 * 8, "scalars")) != KD_OK ||
      (s = dalloc(ctx, (void**)&ctx->Ebuf, (KD_MAX_SLICES + 1) * 8, "energies")) != KD_OK) {
    fprintf(stderr, "kd_create: %s\n", ctx->err.c_str());
    kd_destroy(ctx);
    return s;
  }
  if (cudaMallocHost((void**)&ctx->host_scal, 32 * 8) != cudaSuccess) {
    kd_destroy(ctx);
    return KD_ENOMEM;
  }
  *out = ctx;
  return KD_OK;
}

kd_status kd_destroy(kd_ctx* ctx) {
  if (!ctx) return KD_OK;
  cudaStreamSynchronize(ctx->st);
  for (cudaEvent_t e : ctx->pev) cudaEventDestroy(e);
  for (void* p : ctx->allocs)
    if (p) cudaFree(p);
  for (int i = 0; i < 4; ++i)
    if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
  if (ctx->st2) {
    cudaStreamSynchronize(ctx->st2);
    cudaStreamDestroy(ctx->st2);
  }
  if (ctx->st_hi) {
    cudaStreamSynchronize(ctx->st_hi);
    cudaStreamDestroy(ctx->st_hi);
  }
  for (cudaEvent_t e : ctx->pev2) cudaEventDestroy(e);
  for (cudaStream_t q : {ctx->st_h2d, ctx->st_d2h})
    if (q) {
      cudaStreamSynchronize(q);
      cudaStreamDestroy(q);
    }
  for (cudaEvent_t e : ctx->hev)
    if (e) cudaEventDestroy(e);
  if (ctx->host_scal) cudaFreeHost(ctx->host_scal);
  for (auto& g : ctx->gcache) cudaGraphExecDestroy(g.second.exec);
  if (ctx->st_g) {
    cudaStreamSynchronize(ctx->st_g);
    cudaStreamDestroy(ctx->st_g);
  }
  for (cudaEvent_t e : ctx->gev)
    if (e) cudaEventDestroy(e);
  delete ctx;
  return KD_OK;
}

kd_status kd_fine_batched(kd_ctx* ctx, const void* b_in, void* b_out, const double* t0, int nsteps, int batch) {
  if (!ctx) return KD_EINVAL;
  if (!b_in || !b_out || !t0) return fail(ctx, KD_EINVAL, "kd_fine_batched: NULL buffer");
  if (batch < 0 || nsteps < 0) return fail(ctx, KD_EINVAL, "kd_fine_batched: negative batch or nsteps");
  if (batch == 0) return KD_OK;
  const int n = ctx->p.n, pf = ctx->p.prec_fine;
  kd_status s = ensure_ws(ctx, ctx->ws_f, n, pf, batch);
  if (s != KD_OK) return s;
  if (conv_op(ctx)) {
    if ((s = ensure_conv_tmp(ctx, (size_t)batch * compact_len(n) * 16)) != KD_OK) return s;
    double* tmp = (double*)ctx->conv_tmp;
    KD_LAUNCH(full_to_compact(pf, b_in, KD_C128, tmp, batch, n, ctx->st), "pack");
    if (nsteps > 0 && (s = conv_fine(ctx, tmp, tmp, batch, nsteps, ctx->p.dt_fine, t0)) != KD_OK) return s;
    KD_LAUNCH(compact_to_full(KD_C128, tmp, pf, b_out, batch, n, ctx->st), "unpack");
    return KD_OK;
  }
  // kernels that take the state in the caller's layout skip the pack and unpack passes:
  // the first step reads b_in, the last writes the kept entries of b_out, and the rest of
  // b_out is zeroed (b_in == b_out is fine: a row is read before it is written)
  const bool full_io = nsteps > 0 && fine_full_io(n, pf, ctx->plan[0], ctx->p.fine_scheme);
  if (!full_io) KD_LAUNCH(full_to_compact(pf, b_in, pf, ctx->ws_f.X, batch, n, ctx->st), "pack");
  FineArgs a = fine_args(ctx, ctx->ws_f, ctx->tab_f, n, batch, ctx->p.dt_fine, t0);
  if (full_io) {
    a.x_in_full = b_in;
    a.x_out_full = b_out;
  }
  if ((s = with_phases(ctx, ctx->ws_f, a, nsteps)) != KD_OK) return s;
  LaunchProbe pr = probe_of(ctx);
  if (nsteps > 0)
    KD_LAUNCH(run_fine(ctx, 0, pf, a, nsteps, true, false, ctx->prof ? &pr : nullptr), "fine steps");
  if (full_io)
    KD_LAUNCH(zero_outside_kept(pf, b_out, batch, n, ctx->st), "zero fill");
  else
    KD_LAUNCH(compact_to_full(pf, ctx->ws_f.X, pf, b_out, batch, n, ctx->st), "unpack");
  return KD_OK;
}

kd_status kd_fine_batched_kept(kd_ctx* ctx, const void* c_in, void* c_out, const double* t0, int nsteps,
                               int batch) {
  if (!ctx) return KD_EINVAL;
  if (!c_in || !c_out || !t0) return fail(ctx, KD_EINVAL, "kd_fine_batched_kept: NULL buffer");
  if (batch < 0 || nsteps < 0) return fail(ctx, KD_EINVAL, "kd_fine_batched_kept: negative batch or nsteps");
  const int n = ctx->p.n, pf = ctx->p.prec_fine;
  const size_t es = csize(pf);
  if ((uintptr_t)c_in % es || (uintptr_t)c_out % es)
    return fail(ctx, KD_EINVAL, "kd_fine_batched_kept: buffers not aligned to the complex element");
  if (batch == 0) return KD_OK;
  const size_t bytes = (size_t)batch * compact_len(n) * es;
  kd_status s = ensure_ws(ctx, ctx->ws_f, n, pf, batch);
  if (s != KD_OK) return s;
  if (conv_op(ctx)) {
    if ((s = ensure_conv_tmp(ctx, (size_t)batch * compact_len(n) * 16)) != KD_OK) return s;
    double* tmp = (double*)ctx->conv_tmp;
    KD_LAUNCH(compact_resample(pf, c_in, n, KD_C128, tmp, n, batch, ctx->st), "widen");
    if (nsteps > 0 && (s = conv_fine(ctx, tmp, tmp, batch, nsteps, ctx->p.dt_fine, t0)) != KD_OK) return s;
    KD_LAUNCH(compact_resample(KD_C128, tmp, n, pf, c_out, n, batch, ctx->st), "narrow");
    return KD_OK;
  }
  // the kept-mode layout is the step's own state array: the steps run in place on c_out
  if (c_in != c_out) KD_CUDA(cudaMemcpyAsync(c_out, c_in, bytes, cudaMemcpyDeviceToDevice, ctx->st), "copy");
  if (nsteps == 0) return KD_OK;
  FineArgs a = fine_args(ctx, ctx->ws_f, ctx->tab_f, n, batch, ctx->p.dt_fine, t0);
  a.X = c_out;
  if ((s = with_phases(ctx, ctx->ws_f, a, nsteps)) != KD_OK) return s;
  LaunchProbe pr = probe_of(ctx);
  KD_LAUNCH(run_fine(ctx, 0, pf, a, nsteps, true, false, ctx->prof ? &pr : nullptr), "fine steps");
  return KD_OK;
}

// Chunk sizes of a host-buffer call.  chunk > 0: equal chunks (the last one ragged).
// chunk = 0: sizes that double from base = ceil(batch / 32) up to below cap = batch / 4,
// then equal chunks of at most cap, then the same ramp down: the first copy in and the
// last copy out (the pipeline's fill and drain) move base fields, while the steps in
// between run on batches large enough to fill the GPU; every chunk's copies fit under
// its neighbour's steps.
static std::vector<int> chunk_plan(int batch, int chunk) {
  std::vector<int> out;
  if (chunk > 0) {
    for (int f = 0; f < batch; f += chunk) out.push_back(batch - f < chunk ? batch - f : chunk);
    return out;
  }
  const int base = (batch + 31) / 32, cap = batch / 4 > base ? batch / 4 : base;
  std::vector<int> up;
  int ramp = 0;
  for (int c = base; c < cap; c *= 2) {
    up.push_back(c);
    ramp += c;
  }
  if (2 * ramp >= batch) return chunk_plan(batch, base);
  const int middle = batch - 2 * ramp, m = (middle + cap - 1) / cap;
  out = up;
  for (int i = 0; i < m; ++i) out.push_back(middle / m + (i < middle % m ? 1 : 0));
  out.insert(out.end(), up.rbegin(), up.rend());
  return out;
}

// The chunk pipeline of kd_fine_batched_host (slots and streams set up by the caller);
// enqueues everything and returns without waiting.
static kd_status host_chunks(kd_ctx* ctx, const void* h_in, void* h_out, const double* t0, int nsteps, int batch,
                             const std::vector<int>& plan, size_t fb) {
  kd_status s;
  // events per slot q: hev[q] input copied in, hev[2 + q] computed, hev[4 + q] output copied out
  KD_CUDA(cudaMemcpyAsync(ctx->hio_t0, t0, (size_t)batch * 8, cudaMemcpyHostToDevice, ctx->st), "times");
  for (int q = 2; q < 6; ++q) KD_CUDA(cudaEventRecord(ctx->hev[q], ctx->st), "event");
  int f0 = 0;
  for (int c = 0; c < (int)plan.size(); f0 += plan[c], ++c) {
    const int q = c & 1, nb = plan[c];
    void *din = ctx->hio[q], *dout = ctx->hio[2 + q];
    // input slot q is free once chunk c - 2 has been computed
    KD_CUDA(cudaStreamWaitEvent(ctx->st_h2d, ctx->hev[2 + q], 0), "wait");
    KD_CUDA(cudaMemcpyAsync(din, (const char*)h_in + f0 * fb, nb * fb, cudaMemcpyHostToDevice, ctx->st_h2d), "copy in");
    KD_CUDA(cudaEventRecord(ctx->hev[q], ctx->st_h2d), "event");
    // compute after the copy in, into an output slot that chunk c - 2 has left
    KD_CUDA(cudaStreamWaitEvent(ctx->st, ctx->hev[q], 0), "wait");
    KD_CUDA(cudaStreamWaitEvent(ctx->st, ctx->hev[4 + q], 0), "wait");
    if ((s = kd_fine_batched(ctx, din, dout, ctx->hio_t0 + f0, nsteps, nb)) != KD_OK) return s;
    KD_CUDA(cudaEventRecord(ctx->hev[2 + q], ctx->st), "event");
    KD_CUDA(cudaStreamWaitEvent(ctx->st_d2h, ctx->hev[2 + q], 0), "wait");
    KD_CUDA(cudaMemcpyAsync((char*)h_out + f0 * fb, dout, nb * fb, cudaMemcpyDeviceToHost, ctx->st_d2h), "copy out");
    KD_CUDA(cudaEventRecord(ctx->hev[4 + q], ctx->st_d2h), "event");
  }
  return KD_OK;
}

// The chunk pipeline of kd_fine_batched_host_kept: chunk c stays in device slot c mod 4
// from its copy in to its copy out and is stepped in place there.
static kd_status host_chunks_kept(kd_ctx* ctx, const void* h_in, void* h_out, const double* t0, int nsteps,
                                  int batch, const std::vector<int>& plan, size_t fb) {
  kd_status s;
  // events per slot q: hev[q] copied in, hev[4 + q] computed, hev[8 + q] copied out
  KD_CUDA(cudaMemcpyAsync(ctx->hio_t0, t0, (size_t)batch * 8, cudaMemcpyHostToDevice, ctx->st), "times");
  for (int q = 0; q < 4; ++q) KD_CUDA(cudaEventRecord(ctx->hev[8 + q], ctx->st), "event");
  int f0 = 0;
  for (int c = 0; c < (int)plan.size(); f0 += plan[c], ++c) {
    const int q = c & 3, nb = plan[c];
    void* slot = ctx->hio[q];
    // slot q is free once chunk c - 4 has been copied out
    KD_CUDA(cudaStreamWaitEvent(ctx->st_h2d, ctx->hev[8 + q], 0), "wait");
    KD_CUDA(cudaMemcpyAsync(slot, (const char*)h_in + f0 * fb, nb * fb, cudaMemcpyHostToDevice, ctx->st_h2d), "copy in");
    KD_CUDA(cudaEventRecord(ctx->hev[q], ctx->st_h2d), "event");
    KD_CUDA(cudaStreamWaitEvent(ctx->st, ctx->hev[q], 0), "wait");
    if ((s = kd_fine_batched_kept(ctx, slot, slot, ctx->hio_t0 + f0, nsteps, nb)) != KD_OK) return s;
    KD_CUDA(cudaEventRecord(ctx->hev[4 + q], ctx->st), "event");
    KD_CUDA(cudaStreamWaitEvent(ctx->st_d2h, ctx->hev[4 + q], 0), "wait");
    KD_CUDA(cudaMemcpyAsync((char*)h_out + f0 * fb, slot, nb * fb, cudaMemcpyDeviceToHost, ctx->st_d2h), "copy out");
    KD_CUDA(cudaEventRecord(ctx->hev[8 + q], ctx->st_d2h), "event");
  }
  return KD_OK;
}

// Set-up shared by the host-buffer calls: the four device slots for the largest chunk of
// `plan` at `slot_field` bytes a field, the start-time array and the copy streams.
static kd_status host_setup(kd_ctx* ctx, int batch, const std::vector<int>& plan, size_t slot_field) {
  int most = 0;
  for (int c : plan) most = c > most ? c : most;
  const size_t slot = slot_field * most;
  kd_status s;
  if (ctx->hio_bytes < slot) {
    for (void*& q : ctx->hio) {
      dfree(ctx, q);
      q = nullptr;
    }
    ctx->hio_bytes = 0;
    for (void*& q : ctx->hio)
      if ((s = dalloc(ctx, &q, slot, "host-call chunk")) != KD_OK) return s;
    ctx->hio_bytes = slot;
  }
  if (ctx->hio_t0_cap < batch) {
    dfree(ctx, ctx->hio_t0);
    ctx->hio_t0 = nullptr;
    ctx->hio_t0_cap = 0;
    if ((s = dalloc(ctx, (void**)&ctx->hio_t0, (size_t)batch * 8, "host-call times")) != KD_OK) return s;
    ctx->hio_t0_cap = batch;
  }
  if (!ctx->st_h2d) {
    KD_CUDA(cudaStreamCreateWithFlags(&ctx->st_h2d, cudaStreamNonBlocking), "copy stream");
    KD_CUDA(cudaStreamCreateWithFlags(&ctx->st_d2h, cudaStreamNonBlocking), "copy stream");
    for (cudaEvent_t& e : ctx->hev) KD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
  }
  return KD_OK;
}

// Waits for the three streams of a host-buffer call: whatever happened, no copy of the
// caller's memory is left in flight on return.
static kd_status host_finish(kd_ctx* ctx, kd_status s, const char* what) {
  const cudaError_t e1 = cudaStreamSynchronize(ctx->st_h2d), e2 = cudaStreamSynchronize(ctx->st_d2h);
  const cudaError_t e3 = cudaStreamSynchronize(ctx->st);
  if (s != KD_OK) return s;
  for (cudaError_t e : {e1, e2, e3})
    if (e != cudaSuccess) return cuda_fail(ctx, e, what);
  return KD_OK;
}

kd_status kd_fine_batched_host(kd_ctx* ctx, const void* h_in, void* h_out, const double* t0, int nsteps, int batch,
                               int chunk) {
  if (!ctx) return KD_EINVAL;
  if (!h_in || !h_out || !t0) return fail(ctx, KD_EINVAL, "kd_fine_batched_host: NULL buffer");
  if (batch < 0 || nsteps < 0 || chunk < 0) return fail(ctx, KD_EINVAL, "kd_fine_batched_host: negative argument");
  if (batch == 0) return KD_OK;
  const int n = ctx->p.n;
  const size_t fb = 3 * (size_t)n * n * csize(ctx->p.prec_fine);   // bytes of one field
  const std::vector<int> plan = chunk_plan(batch, chunk);
  kd_status s = host_setup(ctx, batch, plan, fb);
  if (s != KD_OK) return s;
  return host_finish(ctx, host_chunks(ctx, h_in, h_out, t0, nsteps, batch, plan, fb), "kd_fine_batched_host");
}

kd_status kd_fine_batched_host_kept(kd_ctx* ctx, const void* h_in, void* h_out, const double* t0, int nsteps,
                                    int batch, int chunk) {
  if (!ctx) return KD_EINVAL;
  if (!h_in || !h_out || !t0) return fail(ctx, KD_EINVAL, "kd_fine_batched_host_kept: NULL buffer");
  if (batch < 0 || nsteps < 0 || chunk < 0)
    return fail(ctx, KD_EINVAL, "kd_fine_batched_host_kept: negative argument");
  if (batch == 0) return KD_OK;
  const size_t fb = compact_len(ctx->p.n) * csize(ctx->p.prec_fine);   // bytes of one field
  const std::vector<int> plan = chunk_plan(batch, chunk);
  kd_status s = host_setup(ctx, batch, plan, fb);
  if (s != KD_OK) return s;
  return host_finish(ctx, host_chunks_kept(ctx, h_in, h_out, t0, nsteps, batch, plan, fb),
                     "kd_fine_batched_host_kept");
}

kd_status kd_coarse(kd_ctx* ctx, const double* b_in, double* b_out, const double* t0, int nsteps, int batch) {
  if (!ctx) return KD_EINVAL;
  if (!b_in || !b_out || !t0) return fail(ctx, KD_EINVAL, "kd_coarse: NULL buffer");
  if (batch < 0 || nsteps < 0) return fail(ctx, KD_EINVAL, "kd_coarse: negative batch or nsteps");
  if (batch == 0) return KD_OK;
  const int n = ctx->p.n, nc = ctx->p.n_coarse, pc = ctx->p.prec_coarse;
  kd_status s = ensure_ws(ctx, ctx->ws_c, nc, pc, batch);
  if (s != KD_OK) return s;
  // full (n) -> coarse compact via the staging buffer holding the fine compact form
  const size_t fcb = (size_t)batch * compact_len(n) * 16;
  if ((s = ensure_full_tmp(ctx, fcb)) != KD_OK) return s;
  KD_LAUNCH(full_to_compact(KD_C128, b_in, KD_C128, ctx->full_tmp, batch, n, ctx->st), "pack");
  if (coarse_conv_supported(ctx->cP) && nsteps > 0) {
    // persistent convolution-form solve, one block per field; result in ws_c.X as FP64
    if ((s = ensure_ws(ctx, ctx->ws_c, nc, KD_C128, batch)) != KD_OK) return s;
    FineArgs pa = fine_args(ctx, ctx->ws_c, ctx->tab_c, nc, batch, ctx->p.dt_coarse, t0);
    const size_t need = phase_table_bytes(pc, batch, nsteps);
    if (ctx->p.flow == KD_FLOW_GALLOWAY_PROCTOR && ctx->ph_c_bytes < need) {
      dfree(ctx, ctx->ph_c);
      ctx->ph_c = nullptr;
      ctx->ph_c_bytes = 0;
      if ((s = dalloc(ctx, &ctx->ph_c, need, "coarse phase table")) != KD_OK) return s;
      ctx->ph_c_bytes = need;
    }
    pa.phases = ctx->ph_c;
    KD_LAUNCH(launch_phases(pc, pa, nsteps, ctx->st), "coarse phases");
    CoarseArgs c = coarse_args(ctx, nsteps, ctx->p.dt_coarse);
    c.phases = ctx->p.flow == KD_FLOW_GALLOWAY_PROCTOR ? ctx->ph_c : nullptr;
    c.Un = (const double*)ctx->full_tmp;
    c.mode = COARSE_OUT;
    c.g64 = (double*)ctx->ws_c.X;
    KD_LAUNCH(coarse_conv_launch(pc, c, batch, ctx->st), "coarse solve");
    KD_LAUNCH(compact_resample(KD_C128, ctx->ws_c.X, nc, KD_C128, ctx->full_tmp, n, batch, ctx->st), "prolong");
    KD_LAUNCH(compact_to_full(KD_C128, ctx->full_tmp, KD_C128, b_out, batch, n, ctx->st), "unpack");
    return KD_OK;
  }
  KD_LAUNCH(compact_resample(KD_C128, ctx->full_tmp, n, pc, ctx->ws_c.X, nc, batch, ctx->st), "restrict");
  FineArgs a = fine_args(ctx, ctx->ws_c, ctx->tab_c, nc, batch, ctx->p.dt_coarse, t0);
  if ((s = with_phases(ctx, ctx->ws_c, a, nsteps)) != KD_OK) return s;
  if (nsteps > 0) KD_LAUNCH(run_fine(ctx, 1, pc, a, nsteps, true, false), "coarse steps");
  KD_LAUNCH(compact_resample(pc, ctx->ws_c.X, nc, KD_C128, ctx->full_tmp, n, batch, ctx->st), "prolong");
  KD_LAUNCH(compact_to_full(KD_C128, ctx->full_tmp, KD_C128, b_out, batch, n, ctx->st), "unpack");
  return KD_OK;
}

// Parareal from b0 (u_init NULL: iterate 0 is the serial coarse sweep), or resumed from
// the iterate u_init = U^{k0} of an earlier run (slices 0..k0 exact): the iterations
// k0 + 1, ... continue from it, the first fine sweep in direct form.
static kd_status parareal_core(kd_ctx* ctx, const double* b0, const double* u_init, int k0, double T, int N,
                               int k_max, double tol, double* u_slices, kd_parareal_stats* stats) {
  if (!ctx) return KD_EINVAL;
  NvtxRange range(u_init ? "kd_parareal_resume" : "kd_parareal_run");
  if (!b0 && !u_init) return fail(ctx, KD_EINVAL, "kd_parareal_run: b0 is NULL");
  if (N < 1 || N > KD_MAX_SLICES) return fail(ctx, KD_EINVAL, "kd_parareal_run: n_slices out of range");
  if (k_max < 0 || k_max > KD_MAX_ITERS) return fail(ctx, KD_EINVAL, "kd_parareal_run: k_max out of range");
  if (u_init && (k0 < 0 || k0 > k_max))
    return fail(ctx, KD_EINVAL, "kd_parareal_resume: need 0 <= k_done <= k_max");
  if (u_init && ctx->p.fine_form != KD_FINE_INCREMENT)
    return fail(ctx, KD_EUNSUPPORTED, "kd_parareal_resume: needs fine_form KD_FINE_INCREMENT");
  if (!(T > 0) || !isfinite(T)) return fail(ctx, KD_EINVAL, "kd_parareal_run: T must be > 0");
  const int n = ctx->p.n, nc = ctx->p.n_coarse;
  const double dT = T / N;
  const int S = steps_for(dT, ctx->p.dt_fine), Sc = steps_for(dT, ctx->p.dt_coarse);
  const double dt = dT / S, dtc = dT / Sc;
  kd_status s;
  const long long launches0 = ctx->launches;
  if ((s = ensure_slices(ctx, N)) != KD_OK) return s;
  if ((s = ensure_ws(ctx, ctx->ws_f, n, ctx->p.prec_fine, N)) != KD_OK) return s;
  if ((s = ensure_ws(ctx, ctx->ws_c, nc, ctx->p.prec_coarse, 1)) != KD_OK) return s;
  if (ctx->p.coarse_kind == KD_COARSE_LEARNED) {
    if (ctx->l_nphase == 0) return fail(ctx, KD_EINVAL, "kd_parareal_run: call kd_learned_init first");
    if (fabs(dT - ctx->l_sliceT) > 1e-9 * dT)
      return fail(ctx, KD_EINVAL, "kd_parareal_run: slice length differs from the learned operators' slice");
  }
  ctx->fallback = 0;
  ctx->blk_lo = 0;
  const long len = compact_len(n), lenc = 3L * ctx->cP * ctx->cP;
  KD_LAUNCH(fill_slice_times(ctx->t0f, N + 1, 0, dT, ctx->st), "times");
  KD_LAUNCH(fill_slice_times(ctx->t0c, N + 1, 0, dT, ctx->st), "times");

  KD_CUDA(cudaEventRecord(ctx->ev[0], ctx->st), "event");
  if (u_init) {
    const size_t fb = 3UL * n * n * 16;
    if ((s = ensure_full_tmp(ctx, fb * (N + 1))) != KD_OK) return s;
    KD_CUDA(cudaMemcpyAsync(ctx->full_tmp, u_init, fb * (N + 1), cudaMemcpyDefault, ctx->st), "copy iterate");
    KD_LAUNCH(full_to_compact(KD_C128, ctx->full_tmp, KD_C128, ctx->U, N + 1, n, ctx->st), "iterate to compact");
  } else if ((s = copy_in_b0(ctx, b0)) != KD_OK) {
    return s;
  }
  if ((s = coarse_phases(ctx, N, Sc, dtc)) != KD_OK) return s;
  float ms_fine = 0.f, ms_coarse = 0.f;
  int k_done = u_init ? k0 : 0, conv = 0;
  std::vector<double> sig(u_init ? k0 : 0, 0.0), terr(u_init ? k0 : 0, -1.0);
  if (ctx->overlap > 0 && N >= 2 && !u_init) {
    // the sweeps run on the high-priority stream, ordered after the caller's stream
    cudaStream_t user = ctx->st;
    KD_CUDA(cudaEventRecord(ctx->ev[1], user), "event");
    KD_CUDA(cudaStreamWaitEvent(ctx->st_hi, ctx->ev[1], 0), "event");
    ctx->st = ctx->st_hi;
    s = parareal_pipelined(ctx, N, S, Sc, dt, dtc, k_max, tol, sig, k_done, conv, ms_fine, ms_coarse);
    cudaEventRecord(ctx->ev[1], ctx->st_hi);
    ctx->st = user;
    cudaStreamWaitEvent(user, ctx->ev[1], 0);
    if (s != KD_OK) {
      cudaStreamSynchronize(ctx->st2);
      if (stats && s == KD_ENONFINITE) stats->k_con = k_done;
      return s;
    }
  } else {
  // iterate 0: serial coarse sweep (none when resuming)
  KD_CUDA(cudaEventRecord(ctx->ev[2], ctx->st), "event");
  if (!u_init) {
    NvtxRange r0("serial sweep 0");
    for (int i = 0; i < N; ++i)
      if ((s = use_learned(ctx, i) ? learned_step(ctx, i, true, false) : coarse_step(ctx, i, Sc, dtc, true, false)) !=
          KD_OK)
        return s;
  }
  KD_CUDA(cudaEventRecord(ctx->ev[3], ctx->st), "event");
  KD_CUDA(cudaEventSynchronize(ctx->ev[3]), "sync");
  {
    float m = 0.f;
    cudaEventElapsedTime(&m, ctx->ev[2], ctx->ev[3]);
    ms_coarse += m;
  }
  for (int k = k_done + 1; k <= k_max; ++k) {
    // parallel step over the slices that can still change: n >= k - 1
    // (the last slice is always swept so that sigma is measured)
    const int first = k - 1 < N - 1 ? k - 1 : N - 1;
    KD_CUDA(cudaEventRecord(ctx->ev[1], ctx->st), "event");
    {
      NvtxRange rf("fine sweep");
      // the first iteration of a run, or of a resumed run, is in direct form
      if ((s = fine_sweep(ctx, first, N, S, dt, (u_init && k == k0 + 1) ? 1 : k)) != KD_OK) return s;
    }
    KD_CUDA(cudaEventRecord(ctx->ev[2], ctx->st), "event");
    NvtxRange rs("serial sweep");
    // serial step; slice `first` has U_first unchanged, so G(U_first) is the stored
    // coarse value bit for bit and the coarse terms cancel without a coarse solve
    {
      const bool last = (first == N - 1);
      int nb = parareal_update(ctx->Fv + 2 * first * len, ctx->Gv + 2 * first * lenc, KD_C128,
                               ctx->Gv + 2 * first * lenc, ctx->U + 2 * (first + 1) * len, n, ctx->cK, ctx->cP, 0,
                               last ? ctx->partials : nullptr, ctx->st);
      if (nb < 0) return fail(ctx, KD_ECUDA, "parareal update launch failed");
      ctx->launches += 1;
      if (last) KD_LAUNCH(finish_sigma(ctx->partials, nb, ctx->scal, ctx->st), "sigma");
    }
    for (int i = first + 1; i < N; ++i)
      if ((s = use_learned(ctx, i) ? learned_step(ctx, i, false, i == N - 1)
                                   : coarse_step(ctx, i, Sc, dtc, false, i == N - 1)) != KD_OK)
        return s;
    if (ctx->ref_T) {
      // error of the last slice against the reference (scal[16])
      const int nbr = rel_error_partials(ctx->U + 2 * (long)N * len, ctx->ref_T, len, ctx->partials, ctx->st);
      if (nbr < 0) return fail(ctx, KD_ECUDA, "reference error launch failed");
      KD_LAUNCH(finish_sigma(ctx->partials, nbr, ctx->scal + 16, ctx->st), "reference error");
      KD_CUDA(cudaMemcpyAsync(ctx->host_scal + 16, ctx->scal + 16, 8, cudaMemcpyDeviceToHost, ctx->st), "error copy");
    }
    KD_CUDA(cudaMemcpyAsync(ctx->host_scal, ctx->scal, 8, cudaMemcpyDeviceToHost, ctx->st), "sigma copy");
    KD_CUDA(cudaEventRecord(ctx->ev[3], ctx->st), "event");
    KD_CUDA(cudaEventSynchronize(ctx->ev[3]), "sync");
    if (ctx->ref_T) terr.push_back(ctx->host_scal[16]);
    if (ctx->prof) prof_flush(ctx);
    float m1 = 0.f, m2 = 0.f;
    cudaEventElapsedTime(&m1, ctx->ev[1], ctx->ev[2]);
    cudaEventElapsedTime(&m2, ctx->ev[2], ctx->ev[3]);
    ms_fine += m1;
    ms_coarse += m2;
    const double sigma = ctx->host_scal[0];
    sig.push_back(sigma);
    k_done = k;
    if (!isfinite(sigma)) {
      if (stats) stats->k_con = k;
      return fail(ctx, KD_ENONFINITE, "kd_parareal_run: non-finite defect");
    }
    if (sigma <= tol) {
      conv = 1;
      break;
    }
    // fallback to the classical coarse propagator: the defect grew, or half of the
    // iteration budget is spent (the increment form needs no stored coarse values, so
    // the switch keeps the iteration consistent)
    if (ctx->p.coarse_kind == KD_COARSE_LEARNED && !ctx->fallback &&
        ((k >= k0 + 2 && sigma > sig[k - 2]) || (k_max > 1 && k >= k_max / 2)))
      ctx->fallback = 1;
  }
  }
  // energies and growth rate of the final iterate
  KD_LAUNCH(energy_kernel(ctx->U, len, N + 1, ctx->Ebuf, ctx->st), "energy");
  KD_LAUNCH(growth_fit(ctx->Ebuf, N + 1, dT, 0.5 * T, ctx->scal + 4, ctx->st), "growth fit");
  if ((s = copy_out_slices(ctx, u_slices, N)) != KD_OK) return s;
  KD_CUDA(cudaEventRecord(ctx->ev[3], ctx->st), "event");
  KD_CUDA(cudaEventSynchronize(ctx->ev[3]), "sync");
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->k_con = k_done;
    stats->converged = conv;
    stats->n_fine_steps = S;
    stats->n_coarse_steps = Sc;
    stats->dt_fine_used = dt;
    stats->dt_coarse_used = dtc;
    for (size_t i = 0; i < sig.size() && i < KD_MAX_ITERS; ++i) stats->sigma[i] = sig[i];
    for (int i = 0; i < KD_MAX_ITERS; ++i) stats->true_err[i] = i < (int)terr.size() ? terr[i] : -1.0;
    KD_CUDA(cudaMemcpy(stats->energy, ctx->Ebuf, (N + 1) * 8, cudaMemcpyDeviceToHost), "energy copy");
    double fit[2];
    KD_CUDA(cudaMemcpy(fit, ctx->scal + 4, 16, cudaMemcpyDeviceToHost), "fit copy");
    stats->growth_rate = fit[0];
    float mt = 0.f;
    cudaEventElapsedTime(&mt, ctx->ev[0], ctx->ev[3]);
    stats->ms_total = mt;
    stats->ms_fine = ms_fine;
    stats->ms_coarse = ms_coarse;
    stats->n_launches = ctx->launches - launches0;
    stats->fallback_used = ctx->fallback;
  }
  if (!conv && k_max > k0) return fail(ctx, KD_ENOTCONV, "kd_parareal_run: tol not reached within k_max");
  return KD_OK;
}

kd_status kd_set_reference(kd_ctx* ctx, const double* b_ref) {
  if (!ctx) return KD_EINVAL;
  if (!b_ref) {
    dfree(ctx, ctx->ref_T);
    ctx->ref_T = nullptr;
    return KD_OK;
  }
  const int n = ctx->p.n;
  const size_t fb = 3UL * n * n * 16;
  kd_status s;
  if (!ctx->ref_T && (s = dalloc(ctx, (void**)&ctx->ref_T, (size_t)compact_len(n) * 16, "reference")) != KD_OK) return s;
  if ((s = ensure_full_tmp(ctx, fb)) != KD_OK) return s;
  KD_CUDA(cudaMemcpyAsync(ctx->full_tmp, b_ref, fb, cudaMemcpyDefault, ctx->st), "copy reference");
  KD_LAUNCH(full_to_compact(KD_C128, ctx->full_tmp, KD_C128, ctx->ref_T, 1, n, ctx->st), "reference to compact");
  KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
  return KD_OK;
}

kd_status kd_parareal_run(kd_ctx* ctx, const double* b0, double T, int N, int k_max, double tol, double* u_slices,
                          kd_parareal_stats* stats) {
  return parareal_core(ctx, b0, nullptr, 0, T, N, k_max, tol, u_slices, stats);
}

kd_status kd_parareal_resume(kd_ctx* ctx, const double* u_init, int k_done, double T, int N, int k_max, double tol,
                             double* u_slices, kd_parareal_stats* stats) {
  if (!ctx) return KD_EINVAL;
  if (!u_init) return fail(ctx, KD_EINVAL, "kd_parareal_resume: u_init is NULL");
  return parareal_core(ctx, nullptr, u_init, k_done, T, N, k_max, tol, u_slices, stats);
}

kd_status kd_fine_serial(kd_ctx* ctx, const double* b0, double T, int N, double* u_slices) {
  if (!ctx) return KD_EINVAL;
  if (!b0) return fail(ctx, KD_EINVAL, "kd_fine_serial: b0 is NULL");
  if (N < 1 || N > KD_MAX_SLICES) return fail(ctx, KD_EINVAL, "kd_fine_serial: n_slices out of range");
  if (!(T > 0) || !isfinite(T)) return fail(ctx, KD_EINVAL, "kd_fine_serial: T must be > 0");
  const int n = ctx->p.n, pf = ctx->p.prec_fine;
  const double dT = T / N;
  const int S = steps_for(dT, ctx->p.dt_fine);
  const double dt = dT / S;
  kd_status s;
  if ((s = ensure_slices(ctx, N)) != KD_OK) return s;
  if ((s = ensure_ws(ctx, ctx->ws_f, n, pf, 1)) != KD_OK) return s;
  const long len = compact_len(n);
  // one field at a time is a different launch shape from the batched sweeps: tune it once
  if (!conv_op(ctx) && !ctx->plan_serial_ok) {
    const FinePlan saved = ctx->plan[0];
    if ((s = kd_autotune(ctx, KD_GRID_FINE, 1, 2, nullptr, nullptr)) != KD_OK) return s;
    ctx->plan_serial = ctx->plan[0];
    ctx->plan[0] = saved;
    ctx->plan_serial_ok = 1;
  }
  const FinePlan batched = ctx->plan[0];
  ctx->plan[0] = ctx->plan_serial;
  KD_LAUNCH(fill_slice_times(ctx->t0f, N + 1, 0, dT, ctx->st), "times");
  if ((s = copy_in_b0(ctx, b0)) != KD_OK) return s;
  for (int i = 0; i < N; ++i) {
    if (conv_op(ctx)) {
      if ((s = conv_fine(ctx, ctx->U + 2 * i * len, ctx->U + 2 * (i + 1) * len, 1, S, dt, ctx->t0f + i)) != KD_OK)
        return s;
      continue;
    }
    KD_LAUNCH(compact_resample(KD_C128, ctx->U + 2 * i * len, n, pf, ctx->ws_f.X, n, 1, ctx->st), "to fine");
    FineArgs a = fine_args(ctx, ctx->ws_f, ctx->tab_f, n, 1, dt, ctx->t0f + i);
    if ((s = with_phases(ctx, ctx->ws_f, a, S)) != KD_OK) return s;
    KD_LAUNCH(run_fine(ctx, 0, pf, a, S, true, false), "fine steps");
    KD_LAUNCH(compact_resample(pf, ctx->ws_f.X, n, KD_C128, ctx->U + 2 * (i + 1) * len, n, 1, ctx->st), "from fine");
  }
  ctx->plan[0] = batched;
  if ((s = copy_out_slices(ctx, u_slices, N)) != KD_OK) return s;
  KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
  return KD_OK;
}


// ----------------------------------------------------------- learned coarse G
static size_t roundup4(size_t m) { return (m + 3) & ~(size_t)3; }

kd_status kd_learned_init(kd_ctx* ctx, int n_phase, double slice_T) {
  if (!ctx) return KD_EINVAL;
  if (ctx->p.learned_modes <= 0) return fail(ctx, KD_EINVAL, "kd_learned_init: params.learned_modes is 0");
  if (n_phase < 1 || n_phase > 64 || !(slice_T > 0)) return fail(ctx, KD_EINVAL, "kd_learned_init: bad arguments");
  const int K = ctx->cK, P = ctx->cP, nc = 3 * P * P, pc = ctx->p.prec_coarse;
  const int ld = (nc + 7) & ~7;
  const size_t wcount = (size_t)2 * nc * ld;
  kd_status s;
  dfree(ctx, ctx->l_W);
  dfree(ctx, ctx->l_W0);
  ctx->l_W = nullptr;
  ctx->l_W0 = nullptr;
  ctx->l_nphase = 0;
  if ((s = dalloc(ctx, (void**)&ctx->l_W, n_phase * wcount * 2, "learned operators")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&ctx->l_W0, n_phase * wcount * 4, "classical operators")) != KD_OK) return s;
  if (!ctx->l_x && (s = dalloc(ctx, (void**)&ctx->l_x, 4 * (size_t)nc * 4, "learned vectors")) != KD_OK) return s;
  KD_CUDA(learned_gemv_prepare(ld), "gemv set-up");
  KD_CUDA(cudaMemsetAsync(ctx->l_W0, 0, n_phase * wcount * 4, ctx->st), "memset");
  // the classical coarse propagator on the learned set, applied to every unit vector
  const int Sc = steps_for(slice_T, ctx->p.dt_coarse);
  const double dtc = slice_T / Sc;
  const int chunk = nc < 1152 ? nc : 1152;
  double *d64 = nullptr, *g64 = nullptr, *t0 = nullptr;
  void* ph = nullptr;
  if ((s = dalloc(ctx, (void**)&d64, (size_t)chunk * nc * 16, "unit vectors")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&g64, (size_t)chunk * nc * 16, "classical columns")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&t0, (size_t)chunk * 8, "times")) != KD_OK) return s;
  if ((s = dalloc(ctx, &ph, phase_table_bytes(pc, chunk, Sc), "phases")) != KD_OK) return s;
  for (int p = 0; p < n_phase; ++p) {
    KD_LAUNCH(fill_times(t0, chunk, p * slice_T, 0.0, ctx->st), "times");
    FineArgs fa = fine_args(ctx, ctx->ws_c, ctx->tab_c, ctx->p.n_coarse, chunk, dtc, t0);
    fa.phases = ph;
    KD_LAUNCH(launch_phases(pc, fa, Sc, ctx->st), "phases");
    float* W0 = ctx->l_W0 + (size_t)p * wcount;
    for (int j0 = 0; j0 < nc; j0 += chunk) {
      const int cnt = nc - j0 < chunk ? nc - j0 : chunk;
      KD_LAUNCH(learned_unit_vectors(d64, nc, j0, cnt, ctx->st), "unit vectors");
      CoarseArgs c = coarse_args(ctx, Sc, dtc);
      c.Kf = K;
      c.Pf = P;
      c.phases = ctx->p.flow == KD_FLOW_GALLOWAY_PROCTOR ? ph : nullptr;
      c.Un = d64;
      c.mode = COARSE_OUT;
      c.g64 = g64;
      KD_LAUNCH(coarse_conv_launch(pc, c, cnt, ctx->st), "classical columns");
      KD_LAUNCH(learned_columns(g64, nc, ld, j0, cnt, W0, ctx->st), "columns");
    }
    KD_LAUNCH(f32_to_bf16(W0, ctx->l_W + (size_t)p * wcount, (long)wcount, ctx->st), "bf16");
  }
  KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
  dfree(ctx, d64);
  dfree(ctx, g64);
  dfree(ctx, t0);
  dfree(ctx, ph);
  ctx->l_nphase = n_phase;
  ctx->l_sliceT = slice_T;
  ctx->l_valid.assign(n_phase, 1);
  return KD_OK;
}

kd_status kd_learned_pairs(kd_ctx* ctx, const float* x, int n, const int* phase, float* y) {
  if (!ctx) return KD_EINVAL;
  if (ctx->l_nphase == 0) return fail(ctx, KD_EINVAL, "kd_learned_pairs: call kd_learned_init first");
  if (!x || !y || !phase || n < 0) return fail(ctx, KD_EINVAL, "kd_learned_pairs: bad arguments");
  const int nfine = ctx->p.n, Kf = nfine / 3, Pf = 2 * Kf + 1, pf = ctx->p.prec_fine;
  const int K = ctx->cK, P = ctx->cP, nc = 3 * P * P;
  const int S = steps_for(ctx->l_sliceT, ctx->p.dt_fine);
  const double dt = ctx->l_sliceT / S;
  const int chunk = 512;
  kd_status s;
  double* t0 = nullptr;
  if ((s = dalloc(ctx, (void**)&t0, chunk * 8, "times")) != KD_OK) return s;
  std::vector<double> th(chunk);
  for (int off = 0; off < n; off += chunk) {
    const int cnt = n - off < chunk ? n - off : chunk;
    for (int i = 0; i < cnt; ++i) {
      if (phase[off + i] < 0 || phase[off + i] >= ctx->l_nphase) return fail(ctx, KD_EINVAL, "bad phase index");
      th[i] = phase[off + i] * ctx->l_sliceT;
    }
    KD_CUDA(cudaMemcpyAsync(t0, th.data(), cnt * 8, cudaMemcpyHostToDevice, ctx->st), "times");
    if (conv_op(ctx)) {
      // the convolution operator on FP64 compact fields
      if ((s = ensure_conv_tmp(ctx, (size_t)cnt * compact_len(nfine) * 16)) != KD_OK) return s;
      KD_LAUNCH(learned_to_fine(x + 2L * off * nc, K, P, ctx->conv_tmp, KD_C128, Kf, Pf, cnt, ctx->st), "to fine");
      if ((s = conv_fine(ctx, (const double*)ctx->conv_tmp, (double*)ctx->conv_tmp, cnt, S, dt, t0)) != KD_OK)
        return s;
      KD_LAUNCH(fine_to_learned(ctx->conv_tmp, KD_C128, Kf, Pf, y + 2L * off * nc, K, P, cnt, ctx->st), "to learned");
      KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
      continue;
    }
    if ((s = ensure_ws(ctx, ctx->ws_f, nfine, pf, cnt)) != KD_OK) return s;
    KD_LAUNCH(learned_to_fine(x + 2L * off * nc, K, P, ctx->ws_f.X, pf, Kf, Pf, cnt, ctx->st), "to fine");
    FineArgs a = fine_args(ctx, ctx->ws_f, ctx->tab_f, nfine, cnt, dt, t0);
    if ((s = with_phases(ctx, ctx->ws_f, a, S)) != KD_OK) return s;
    KD_LAUNCH(run_fine(ctx, 0, pf, a, S, true, false), "fine steps");
    KD_LAUNCH(fine_to_learned(ctx->ws_f.X, pf, Kf, Pf, y + 2L * off * nc, K, P, cnt, ctx->st), "to learned");
    KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
  }
  dfree(ctx, t0);
  return KD_OK;
}

namespace {

// Device buffers of one training / gradient evaluation with m pairs (padded to mp).
struct TrainBufs {
  float *xp = nullptr, *yp = nullptr, *yT = nullptr, *C1 = nullptr, *C2 = nullptr;
  __nv_bfloat16 *Xs = nullptr, *XtT = nullptr, *A2 = nullptr, *Wbf = nullptr;
  int* err = nullptr;   // set by the tensor-core GEMM if one of its bounded waits ran out
};

kd_status train_bufs(kd_ctx* ctx, TrainBufs& b, int mp, int nc) {
  kd_status s;
  const size_t m2 = 2 * (size_t)mp;
  const size_t ld = (nc + 7) & ~7;
  if ((s = dalloc(ctx, (void**)&b.xp, m2 * nc * 4, "pairs x")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&b.yp, m2 * nc * 4, "pairs y")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&b.yT, m2 * nc * 4, "y transposed")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&b.C1, 2 * (size_t)nc * m2 * 4, "forward product")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&b.C2, 2 * (size_t)nc * ld * 4, "gradient product")) != KD_OK) return s;
  KD_CUDA(cudaMemsetAsync(b.C2, 0, 2 * (size_t)nc * ld * 4, ctx->st), "memset");   // padding columns stay 0
  if ((s = dalloc(ctx, (void**)&b.Xs, m2 * ld * 2, "x operand")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&b.XtT, m2 * nc * 2, "x^T operand")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&b.A2, 2 * (size_t)nc * m2 * 2, "residual operand")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&b.Wbf, 2 * (size_t)nc * ld * 2, "bf16 weights")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&b.err, 16, "gemm status")) != KD_OK) return s;
  KD_CUDA(cudaMemsetAsync(b.err, 0, 16, ctx->st), "memset");
  return KD_OK;
}

// C = A Bt^T on the engine the context selects (kd_set_learned_gemm)
int train_gemm(const kd_ctx* ctx, const TrainBufs& b, const __nv_bfloat16* A, const __nv_bfloat16* Bt, float* C,
               int M, int N, int K, int ldc) {
  return ctx->gemm_engine == KD_GEMM_MMA_SYNC ? gemm_bf16_tn(A, Bt, C, M, N, K, ldc, ctx->st)
                                              : gemm_bf16_tn_tc(A, Bt, C, M, N, K, ldc, b.err, ctx->st);
}

// KD_ECUDA if a tensor-core GEMM of this training reported a timed-out wait
kd_status check_gemm(kd_ctx* ctx, const TrainBufs& b) {
  int e = 0;
  KD_CUDA(cudaMemcpyAsync(&e, b.err, 4, cudaMemcpyDeviceToHost, ctx->st), "gemm status");
  KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
  return e ? fail(ctx, KD_ECUDA, "tensor-core GEMM: a bounded wait ran out") : KD_OK;
}

void free_train_bufs(kd_ctx* ctx, TrainBufs& b) {
  void* all[] = {b.xp, b.yp, b.yT, b.C1, b.C2, b.Xs, b.XtT, b.A2, b.Wbf, b.err};
  for (void* p : all) dfree(ctx, p);
  b = TrainBufs();
}

// gather the pairs `idx` into contiguous zero-padded buffers and build the operands
kd_status load_pairs(kd_ctx* ctx, TrainBufs& b, const float* x, const float* y, const std::vector<int>& idx, int mp,
                     int nc) {
  const size_t vb = 2 * (size_t)nc * 4;
  KD_CUDA(cudaMemsetAsync(b.xp, 0, mp * vb, ctx->st), "memset");
  KD_CUDA(cudaMemsetAsync(b.yp, 0, mp * vb, ctx->st), "memset");
  for (size_t t = 0; t < idx.size(); ++t) {
    KD_CUDA(cudaMemcpyAsync((char*)b.xp + t * vb, (const char*)x + (size_t)idx[t] * vb, vb, cudaMemcpyDeviceToDevice,
                            ctx->st),
            "gather x");
    KD_CUDA(cudaMemcpyAsync((char*)b.yp + t * vb, (const char*)y + (size_t)idx[t] * vb, vb, cudaMemcpyDeviceToDevice,
                            ctx->st),
            "gather y");
  }
  KD_LAUNCH(learned_pack_x(b.xp, mp, nc, (nc + 7) & ~7, b.Xs, b.XtT, ctx->st), "pack x");
  KD_LAUNCH(learned_transpose_y(b.yp, mp, nc, b.yT, ctx->st), "transpose y");
  return KD_OK;
}

// forward GEMM, residual (loss sum -> out[0]) and gradient GEMM (-> b.C2) for W in b.Wbf
kd_status forward_backward(kd_ctx* ctx, TrainBufs& b, int mp, int nc, double* loss_dev) {
  const int ld = (nc + 7) & ~7;
  KD_LAUNCH(train_gemm(ctx, b, b.Wbf, b.Xs, b.C1, 2 * nc, 2 * mp, ld, 2 * mp), "forward gemm");
  const int nb = learned_residual(b.C1, b.yT, mp, nc, b.A2, ctx->partials, ctx->st);
  if (nb < 0) return fail(ctx, KD_ECUDA, "residual launch failed");
  ctx->launches += 1;
  KD_LAUNCH(sum_partials(ctx->partials, nb, loss_dev, ctx->st), "loss");
  KD_LAUNCH(train_gemm(ctx, b, b.A2, b.XtT, b.C2, 2 * nc, nc, 2 * mp, ld), "gradient gemm");
  return KD_OK;
}

// The classical coarse propagator over one slice of phase p applied to the m learned
// vectors xp (complex FP32 [m][nc]) in FP64: g64 [m][nc].  Scratch: d64 (m nc complex
// FP64), t0 (m doubles), ph (the coarse phase table of m fields).
kd_status classical_on_set(kd_ctx* ctx, const float* xp, int m, int p, double* d64, double* g64, double* t0,
                           void* ph) {
  const int K = ctx->cK, P = ctx->cP, nc = 3 * P * P, pc = ctx->p.prec_coarse;
  const int Sc = steps_for(ctx->l_sliceT, ctx->p.dt_coarse);
  const double dtc = ctx->l_sliceT / Sc;
  KD_LAUNCH(learned_f32_to_f64(xp, d64, (long)m * nc, ctx->st), "to f64");
  KD_LAUNCH(fill_times(t0, m, p * ctx->l_sliceT, 0.0, ctx->st), "times");
  FineArgs fa = fine_args(ctx, ctx->ws_c, ctx->tab_c, ctx->p.n_coarse, m, dtc, t0);
  fa.phases = ph;
  KD_LAUNCH(launch_phases(pc, fa, Sc, ctx->st), "phases");
  CoarseArgs c = coarse_args(ctx, Sc, dtc);
  c.Kf = K;
  c.Pf = P;
  c.phases = ctx->p.flow == KD_FLOW_GALLOWAY_PROCTOR ? ph : nullptr;
  c.Un = d64;
  c.mode = COARSE_OUT;
  c.g64 = g64;
  KD_LAUNCH(coarse_conv_launch(pc, c, m, ctx->st), "classical");
  return KD_OK;
}

// In-place inverse of the Hermitian positive definite m x m matrix A (row-major) by its
// Cholesky factor A = L L^H: A^-1 = L^-H L^-1.  False if A is not positive definite.
bool herm_inverse(std::vector<std::complex<double>>& A, int m) {
  using C = std::complex<double>;
  auto a = [&](int i, int j) -> C& { return A[(size_t)i * m + j]; };
  for (int j = 0; j < m; ++j) {            // L in the lower triangle
    double d = a(j, j).real();
    for (int k = 0; k < j; ++k) d -= std::norm(a(j, k));
    if (!(d > 0.0)) return false;
    const double l = sqrt(d);
    a(j, j) = l;
    for (int i = j + 1; i < m; ++i) {
      C t = a(i, j);
      for (int k = 0; k < j; ++k) t -= a(i, k) * std::conj(a(j, k));
      a(i, j) = t / l;
    }
  }
  std::vector<C> Li((size_t)m * m, C(0.0));   // L^-1, lower triangular
  for (int j = 0; j < m; ++j) {
    Li[(size_t)j * m + j] = 1.0 / a(j, j);
    for (int i = j + 1; i < m; ++i) {
      C t(0.0);
      for (int k = j; k < i; ++k) t -= a(i, k) * Li[(size_t)k * m + j];
      Li[(size_t)i * m + j] = t / a(i, i);
    }
  }
  for (int i = 0; i < m; ++i)                // (L^-H L^-1)[i][j] = sum_k conj(Li[k][i]) Li[k][j]
    for (int j = 0; j <= i; ++j) {
      C t(0.0);
      for (int k = i; k < m; ++k) t += std::conj(Li[(size_t)k * m + i]) * Li[(size_t)k * m + j];
      a(i, j) = t;
      a(j, i) = std::conj(t);
    }
  return true;
}

// KD_TRAIN_MINNORM for one phase whose m pairs are loaded in b: W = W0 + R (G + lambda I)^-1
// X^H with R = Y - W0 X (W0 X by the classical propagator in FP64), G = X^H X, lambda = m wd
// (the minimiser of the training objective, in the span of the inputs when wd = 0); the
// correction R G^-1 X^H is the gradient GEMM with R G^-1 in place of the residual.
struct MinnormBufs {
  double *d64 = nullptr, *g64 = nullptr, *t0 = nullptr, *G64 = nullptr;
  float *Rf = nullptr, *G32 = nullptr, *Cb = nullptr, *Cc = nullptr;
  __nv_bfloat16 *A2lo = nullptr, *XtTlo = nullptr;
  void* ph = nullptr;
};

kd_status minnorm_phase(kd_ctx* ctx, TrainBufs& b, MinnormBufs& q, int p, int m, int mp, int nc, float wd,
                        const float* W0) {
  double *d64 = q.d64, *g64 = q.g64, *t0 = q.t0, *G64 = q.G64;
  float *Rf = q.Rf, *G32 = q.G32;
  void* ph = q.ph;
  const int ld = (nc + 7) & ~7;
  kd_status s;
  if ((s = classical_on_set(ctx, b.xp, m, p, d64, g64, t0, ph)) != KD_OK) return s;
  KD_LAUNCH(learned_resid64(b.yp, g64, Rf, (long)m * nc, ctx->st), "residual");
  KD_LAUNCH(learned_gram(b.xp, m, nc, G64, ctx->st), "gram");
  std::vector<std::complex<double>> G((size_t)m * m);
  KD_CUDA(cudaMemcpyAsync(G.data(), G64, G.size() * 16, cudaMemcpyDeviceToHost, ctx->st), "gram");
  KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
  for (int i = 0; i < m; ++i) G[(size_t)i * m + i] += (double)m * wd;
  if (!herm_inverse(G, m))
    return fail(ctx, KD_EINVAL, "kd_learned_train: the pairs' inputs of phase " + std::to_string(p) +
                                    " are linearly dependent; use weight_decay > 0");
  std::vector<float> g32(2 * G.size());
  for (size_t i = 0; i < G.size(); ++i) {
    g32[2 * i] = (float)G[i].real();
    g32[2 * i + 1] = (float)G[i].imag();
  }
  KD_CUDA(cudaMemcpyAsync(G32, g32.data(), g32.size() * 4, cudaMemcpyHostToDevice, ctx->st), "inverse");
  // A X^H = A_hi X_hi + A_lo X_hi + A_hi X_lo (A_lo X_lo dropped): three BF16 GEMMs
  KD_LAUNCH(learned_minnorm_operand(Rf, G32, m, mp, nc, b.A2, q.A2lo, ctx->st), "operand");
  KD_LAUNCH(learned_pack_x_lo(b.xp, mp, nc, q.XtTlo, ctx->st), "x low part");
  KD_LAUNCH(train_gemm(ctx, b, b.A2, b.XtT, b.C2, 2 * nc, nc, 2 * mp, ld), "correction gemm");
  KD_LAUNCH(train_gemm(ctx, b, q.A2lo, b.XtT, q.Cb, 2 * nc, nc, 2 * mp, ld), "correction gemm");
  KD_LAUNCH(train_gemm(ctx, b, b.A2, q.XtTlo, q.Cc, 2 * nc, nc, 2 * mp, ld), "correction gemm");
  KD_LAUNCH(learned_add_bf16(W0, b.C2, q.Cb, q.Cc, ctx->l_W + (size_t)p * 2 * nc * ld, 2L * nc * ld, ctx->st),
            "store");
  KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");   // g32 is host memory of this frame
  return KD_OK;
}

}  // namespace

kd_status kd_learned_train(kd_ctx* ctx, const float* x, const float* y, const int* phase, int n, int epochs, float lr,
                           float weight_decay, int method, double* loss_out) {
  if (!ctx) return KD_EINVAL;
  if (ctx->l_nphase == 0) return fail(ctx, KD_EINVAL, "kd_learned_train: call kd_learned_init first");
  if (!x || !y || !phase || n <= 0 || epochs < 0 || !(lr >= 0) || !(weight_decay >= 0) ||
      (method != KD_TRAIN_ADAM && method != KD_TRAIN_MOMENTUM && method != KD_TRAIN_MINNORM))
    return fail(ctx, KD_EINVAL, "kd_learned_train: bad arguments");
  const int P = ctx->cP, nc = 3 * P * P, ld = (nc + 7) & ~7;
  const size_t wcount = (size_t)2 * nc * ld;
  std::vector<std::vector<int>> byp(ctx->l_nphase);
  for (int i = 0; i < n; ++i) {
    if (phase[i] < 0 || phase[i] >= ctx->l_nphase) return fail(ctx, KD_EINVAL, "kd_learned_train: bad phase index");
    byp[phase[i]].push_back(i);
  }
  size_t mmax = 0;
  for (auto& v : byp) mmax = v.size() > mmax ? v.size() : mmax;
  const int mp = (int)roundup4(mmax);
  kd_status s;
  TrainBufs b;
  if (method == KD_TRAIN_MINNORM) {
    if (mmax > 4096) return fail(ctx, KD_EINVAL, "kd_learned_train: KD_TRAIN_MINNORM takes at most 4096 pairs a phase");
    MinnormBufs q;
    if ((s = train_bufs(ctx, b, mp, nc)) != KD_OK) return s;
    const int Sc = steps_for(ctx->l_sliceT, ctx->p.dt_coarse);
    const size_t cbytes = 2 * (size_t)nc * ld * 4;
    if ((s = dalloc(ctx, (void**)&q.d64, (size_t)mp * nc * 16, "inputs")) != KD_OK) return s;
    if ((s = dalloc(ctx, (void**)&q.g64, (size_t)mp * nc * 16, "classical outputs")) != KD_OK) return s;
    if ((s = dalloc(ctx, (void**)&q.t0, (size_t)mp * 8, "times")) != KD_OK) return s;
    if ((s = dalloc(ctx, &q.ph, phase_table_bytes(ctx->p.prec_coarse, mp, Sc), "phases")) != KD_OK) return s;
    if ((s = dalloc(ctx, (void**)&q.Rf, (size_t)mp * nc * 8, "residual")) != KD_OK) return s;
    if ((s = dalloc(ctx, (void**)&q.G64, (size_t)mp * mp * 16, "gram")) != KD_OK) return s;
    if ((s = dalloc(ctx, (void**)&q.G32, (size_t)mp * mp * 8, "gram inverse")) != KD_OK) return s;
    if ((s = dalloc(ctx, (void**)&q.A2lo, 2 * (size_t)nc * 2 * mp * 2, "operand low part")) != KD_OK) return s;
    if ((s = dalloc(ctx, (void**)&q.XtTlo, (size_t)nc * 2 * mp * 2, "x low part")) != KD_OK) return s;
    if ((s = dalloc(ctx, (void**)&q.Cb, cbytes, "correction")) != KD_OK) return s;
    if ((s = dalloc(ctx, (void**)&q.Cc, cbytes, "correction")) != KD_OK) return s;
    KD_CUDA(cudaMemsetAsync(q.Cb, 0, cbytes, ctx->st), "memset");   // padding columns stay 0
    KD_CUDA(cudaMemsetAsync(q.Cc, 0, cbytes, ctx->st), "memset");
    for (int p = 0; p < ctx->l_nphase; ++p) {
      const int m = (int)byp[p].size();
      if (m == 0) continue;
      if ((s = load_pairs(ctx, b, x, y, byp[p], mp, nc)) != KD_OK) return s;
      if ((s = minnorm_phase(ctx, b, q, p, m, mp, nc, weight_decay, ctx->l_W0 + (size_t)p * wcount)) != KD_OK)
        return s;
    }
    if ((s = check_gemm(ctx, b)) != KD_OK) return s;
    free_train_bufs(ctx, b);
    for (void* v : {(void*)q.d64, (void*)q.g64, (void*)q.t0, q.ph, (void*)q.Rf, (void*)q.G64, (void*)q.G32,
                    (void*)q.A2lo, (void*)q.XtTlo, (void*)q.Cb, (void*)q.Cc})
      dfree(ctx, v);
    return KD_OK;
  }
  float *Wm = nullptr, *m1 = nullptr, *v = nullptr;
  double* lossd = nullptr;
  if ((s = train_bufs(ctx, b, mp, nc)) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&Wm, wcount * 4, "master weights")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&m1, wcount * 4, "adam m")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&v, wcount * 4, "adam v")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&lossd, (size_t)ctx->l_nphase * (epochs > 0 ? epochs : 1) * 16, "losses")) != KD_OK)
    return s;
  for (int p = 0; p < ctx->l_nphase; ++p) {
    if (byp[p].empty()) continue;
    if ((s = load_pairs(ctx, b, x, y, byp[p], mp, nc)) != KD_OK) return s;
    const float* W0 = ctx->l_W0 + (size_t)p * wcount;
    KD_CUDA(cudaMemcpyAsync(Wm, W0, wcount * 4, cudaMemcpyDeviceToDevice, ctx->st), "init");
    KD_CUDA(cudaMemsetAsync(m1, 0, wcount * 4, ctx->st), "memset");
    KD_CUDA(cudaMemsetAsync(v, 0, wcount * 4, ctx->st), "memset");
    KD_LAUNCH(f32_to_bf16(Wm, b.Wbf, (long)wcount, ctx->st), "bf16");
    const float scale = 2.f / (float)byp[p].size();
    float eta = 0.f;
    if (method == KD_TRAIN_MOMENTUM) {
      // step size lr / lambda, lambda = (2/m) sum |x_i|^2 bounds the Hessian (2/m) X^H X
      const int nb = diff_norms(b.xp, b.xp, 2L * mp * nc, ctx->partials, ctx->st);
      if (nb < 0) return fail(ctx, KD_ECUDA, "norm launch failed");
      KD_LAUNCH(sum_partials(ctx->partials, nb, ctx->scal + 12, ctx->st), "norm");
      double h[2];
      KD_CUDA(cudaMemcpyAsync(h, ctx->scal + 12, 16, cudaMemcpyDeviceToHost, ctx->st), "norm");
      KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
      eta = (float)(lr / (scale * h[1] + 2.0 * weight_decay));
    }
    for (int e = 0; e < epochs; ++e) {
      if ((s = forward_backward(ctx, b, mp, nc, lossd + 2 * ((size_t)p * epochs + e))) != KD_OK) return s;
      if (method == KD_TRAIN_ADAM) {
        // cosine decay of the step size to zero over the epochs
        const float lr_e = (float)(0.5 * lr * (1.0 + cos(M_PI * e / (double)epochs)));
        const int nb = learned_adam(Wm, W0, b.C2, m1, v, b.Wbf, (long)wcount, scale, weight_decay, lr_e, 0.9f,
                                    0.999f, 1e-8f, e + 1, nullptr, ctx->st);
        if (nb < 0) return fail(ctx, KD_ECUDA, "adam launch failed");
        ctx->launches += 1;
      } else {
        KD_LAUNCH(learned_momentum(Wm, W0, b.C2, v, b.Wbf, (long)wcount, scale, weight_decay, eta, 0.9f, ctx->st),
                  "momentum");
      }
    }
    KD_CUDA(cudaMemcpyAsync(ctx->l_W + (size_t)p * wcount, b.Wbf, wcount * 2, cudaMemcpyDeviceToDevice, ctx->st),
            "store");
  }
  if (loss_out && epochs > 0) {
    std::vector<double> h((size_t)ctx->l_nphase * epochs * 2);
    KD_CUDA(cudaMemcpyAsync(h.data(), lossd, h.size() * 8, cudaMemcpyDeviceToHost, ctx->st), "losses");
    KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
    for (int p = 0; p < ctx->l_nphase; ++p)
      for (int e = 0; e < epochs; ++e)
        loss_out[(size_t)p * epochs + e] = byp[p].empty() ? 0.0 : h[2 * ((size_t)p * epochs + e)] / byp[p].size();
  }
  KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
  if ((s = check_gemm(ctx, b)) != KD_OK) return s;
  free_train_bufs(ctx, b);
  dfree(ctx, Wm);
  dfree(ctx, m1);
  dfree(ctx, v);
  dfree(ctx, lossd);
  return KD_OK;
}

kd_status kd_learned_loss_grad(kd_ctx* ctx, const float* W, const float* W0, float weight_decay, const float* x,
                               const float* y, int n, double* loss_out, float* grad_out) {
  if (!ctx) return KD_EINVAL;
  if (ctx->p.learned_modes <= 0 || !W || !x || !y || n <= 0 || !loss_out || !grad_out)
    return fail(ctx, KD_EINVAL, "kd_learned_loss_grad: bad arguments");
  const int P = ctx->cP, nc = 3 * P * P, ld = (nc + 7) & ~7;
  const size_t wcount = (size_t)2 * nc * ld;
  const int mp = (int)roundup4(n);
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  kd_status s;
  TrainBufs b;
  float *Wp = nullptr, *W0p = nullptr, *gp = nullptr;
  if ((s = train_bufs(ctx, b, mp, nc)) != KD_OK) return s;
  // the caller's [2 nc][nc] matrices in the padded [2 nc][ld] layout
  if ((s = dalloc(ctx, (void**)&Wp, wcount * 4, "weights")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&W0p, wcount * 4, "centre")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&gp, wcount * 4, "gradient")) != KD_OK) return s;
  KD_CUDA(cudaMemsetAsync(Wp, 0, wcount * 4, ctx->st), "memset");
  KD_CUDA(cudaMemsetAsync(W0p, 0, wcount * 4, ctx->st), "memset");
  KD_CUDA(cudaMemcpy2DAsync(Wp, ld * 4, W, nc * 4, nc * 4, 2 * nc, cudaMemcpyDeviceToDevice, ctx->st), "repack");
  if (W0)
    KD_CUDA(cudaMemcpy2DAsync(W0p, ld * 4, W0, nc * 4, nc * 4, 2 * nc, cudaMemcpyDeviceToDevice, ctx->st), "repack");
  if ((s = load_pairs(ctx, b, x, y, idx, mp, nc)) != KD_OK) return s;
  KD_LAUNCH(f32_to_bf16(Wp, b.Wbf, (long)wcount, ctx->st), "bf16");
  if ((s = forward_backward(ctx, b, mp, nc, ctx->scal + 8)) != KD_OK) return s;
  KD_LAUNCH(learned_grad(Wp, W0p, b.C2, gp, (long)wcount, 2.f / n, weight_decay, ctx->st), "gradient");
  KD_CUDA(cudaMemcpy2DAsync(grad_out, nc * 4, gp, ld * 4, nc * 4, 2 * nc, cudaMemcpyDeviceToDevice, ctx->st), "unpack");
  const int nb = diff_norms(Wp, W0p, (long)wcount, ctx->partials, ctx->st);
  if (nb < 0) return fail(ctx, KD_ECUDA, "norm launch failed");
  KD_LAUNCH(sum_partials(ctx->partials, nb, ctx->scal + 10, ctx->st), "norm");
  double h[4];
  KD_CUDA(cudaMemcpyAsync(h, ctx->scal + 8, 32, cudaMemcpyDeviceToHost, ctx->st), "loss");
  KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
  *loss_out = h[0] / n + weight_decay * h[2];
  if ((s = check_gemm(ctx, b)) != KD_OK) return s;
  free_train_bufs(ctx, b);
  dfree(ctx, Wp);
  dfree(ctx, W0p);
  dfree(ctx, gp);
  return KD_OK;
}

kd_status kd_learned_apply(kd_ctx* ctx, const float* x, float* y, int phase, int n) {
  if (!ctx) return KD_EINVAL;
  if (ctx->l_nphase == 0 || phase < 0 || phase >= ctx->l_nphase || !x || !y || n < 0)
    return fail(ctx, KD_EINVAL, "kd_learned_apply: bad arguments");
  if (n == 0) return KD_OK;
  const int P = ctx->cP, nc = 3 * P * P, ld = (nc + 7) & ~7;
  KD_LAUNCH(learned_gemv(ctx->l_W + (size_t)phase * 2 * nc * ld, x, y, nc, ld, n, ctx->st), "learned gemv");
  return KD_OK;
}

kd_status kd_learned_get(kd_ctx* ctx, int phase, void* W, int* valid) {
  if (!ctx) return KD_EINVAL;
  if (ctx->l_nphase == 0 || phase < 0 || phase >= ctx->l_nphase || !W)
    return fail(ctx, KD_EINVAL, "kd_learned_get: bad arguments");
  const int P = ctx->cP, nc = 3 * P * P, ld = (nc + 7) & ~7;
  KD_CUDA(cudaMemcpy2DAsync(W, (size_t)nc * 2, ctx->l_W + (size_t)phase * 2 * nc * ld, (size_t)ld * 2, (size_t)nc * 2,
                            2 * (size_t)nc, cudaMemcpyDefault, ctx->st),
          "operator out");
  KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
  if (valid) *valid = ctx->l_valid[phase];
  return KD_OK;
}

kd_status kd_learned_set(kd_ctx* ctx, int phase, const void* W, int valid) {
  if (!ctx) return KD_EINVAL;
  if (ctx->l_nphase == 0 || phase < 0 || phase >= ctx->l_nphase || !W)
    return fail(ctx, KD_EINVAL, "kd_learned_set: bad arguments");
  const int P = ctx->cP, nc = 3 * P * P, ld = (nc + 7) & ~7;
  KD_CUDA(cudaMemcpy2DAsync(ctx->l_W + (size_t)phase * 2 * nc * ld, (size_t)ld * 2, W, (size_t)nc * 2, (size_t)nc * 2,
                            2 * (size_t)nc, cudaMemcpyDefault, ctx->st),
          "operator in");
  KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
  ctx->l_valid[phase] = valid ? 1 : 0;
  return KD_OK;
}

kd_status kd_learned_eval(kd_ctx* ctx, const float* x, const float* y, const int* phase, int n, double* err_learned,
                          double* err_classical) {
  if (!ctx) return KD_EINVAL;
  if (ctx->l_nphase == 0 || !x || !y || !phase || n <= 0 || !err_learned || !err_classical)
    return fail(ctx, KD_EINVAL, "kd_learned_eval: bad arguments");
  const int P = ctx->cP, nc = 3 * P * P, pc = ctx->p.prec_coarse;
  const int Sc = steps_for(ctx->l_sliceT, ctx->p.dt_coarse);
  std::vector<std::vector<int>> byp(ctx->l_nphase);
  for (int i = 0; i < n; ++i) {
    if (phase[i] < 0 || phase[i] >= ctx->l_nphase) return fail(ctx, KD_EINVAL, "kd_learned_eval: bad phase index");
    byp[phase[i]].push_back(i);
  }
  size_t mmax = 0;
  for (auto& v : byp) mmax = v.size() > mmax ? v.size() : mmax;
  const int mp = (int)roundup4(mmax);
  kd_status s;
  TrainBufs b;
  double *d64 = nullptr, *g64 = nullptr, *t0 = nullptr;
  float* pred = nullptr;
  void* ph = nullptr;
  if ((s = train_bufs(ctx, b, mp, nc)) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&d64, (size_t)mp * nc * 16, "inputs")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&g64, (size_t)mp * nc * 16, "outputs")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&pred, (size_t)mp * nc * 8, "prediction")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&t0, (size_t)mp * 8, "times")) != KD_OK) return s;
  if ((s = dalloc(ctx, &ph, phase_table_bytes(pc, mp, Sc), "phases")) != KD_OK) return s;
  for (int p = 0; p < ctx->l_nphase; ++p) {
    err_learned[p] = err_classical[p] = -1.0;
    const int m = (int)byp[p].size();
    if (m == 0) continue;
    if ((s = load_pairs(ctx, b, x, y, byp[p], mp, nc)) != KD_OK) return s;
    // learned
    const int ld = (nc + 7) & ~7;
    KD_LAUNCH(learned_gemv(ctx->l_W + (size_t)p * 2 * nc * ld, b.xp, pred, nc, ld, m, ctx->st), "gemv");
    int nb = diff_norms(pred, b.yp, 2L * m * nc, ctx->partials, ctx->st);
    if (nb < 0) return fail(ctx, KD_ECUDA, "norm launch failed");
    KD_LAUNCH(sum_partials(ctx->partials, nb, ctx->scal + 8, ctx->st), "norm");
    // classical coarse propagator on the same set
    if ((s = classical_on_set(ctx, b.xp, m, p, d64, g64, t0, ph)) != KD_OK) return s;
    KD_LAUNCH(learned_f64_to_f32(g64, pred, (long)m * nc, ctx->st), "to f32");
    nb = diff_norms(pred, b.yp, 2L * m * nc, ctx->partials, ctx->st);
    if (nb < 0) return fail(ctx, KD_ECUDA, "norm launch failed");
    KD_LAUNCH(sum_partials(ctx->partials, nb, ctx->scal + 10, ctx->st), "norm");
    double h[4];
    KD_CUDA(cudaMemcpyAsync(h, ctx->scal + 8, 32, cudaMemcpyDeviceToHost, ctx->st), "errors");
    KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
    err_learned[p] = sqrt(h[0] / h[1]);
    err_classical[p] = sqrt(h[2] / h[3]);
    ctx->l_valid[p] = err_learned[p] <= err_classical[p] ? 1 : 0;
  }
  free_train_bufs(ctx, b);
  dfree(ctx, d64);
  dfree(ctx, g64);
  dfree(ctx, pred);
  dfree(ctx, t0);
  dfree(ctx, ph);
  return KD_OK;
}

long long kd_launch_count(kd_ctx* ctx) { return ctx ? ctx->launches : -1; }

kd_status kd_set_alloc_limit(kd_ctx* ctx, size_t max_bytes) {
  if (!ctx) return KD_EINVAL;
  ctx->alloc_limit = max_bytes;
  return KD_OK;
}

kd_status kd_get_alloc_bytes(kd_ctx* ctx, size_t* held, size_t* limit) {
  if (!ctx) return KD_EINVAL;
  if (held) *held = ctx->alloc_held;
  if (limit) *limit = ctx->alloc_limit;
  return KD_OK;
}

kd_status kd_profile(kd_ctx* ctx, int enable) {
  if (!ctx) return KD_EINVAL;
  prof_flush(ctx);
  ctx->prof = enable ? 1 : 0;
  ctx->prof_ms[0] = ctx->prof_ms[1] = 0.0;
  ctx->prof_n[0] = ctx->prof_n[1] = 0;
  return KD_OK;
}

kd_status kd_profile_read(kd_ctx* ctx, double* ms, long long* launches) {
  if (!ctx || !ms || !launches) return KD_EINVAL;
  prof_flush(ctx);
  for (int i = 0; i < 2; ++i) {
    ms[i] = ctx->prof_ms[i];
    launches[i] = ctx->prof_n[i];
  }
  return KD_OK;
}

kd_status kd_energy(kd_ctx* ctx, const double* fields, int count, double* energy_out) {
  if (!ctx) return KD_EINVAL;
  if (!fields || !energy_out || count < 0) return fail(ctx, KD_EINVAL, "kd_energy: bad argument");
  const long len = 3L * ctx->p.n * ctx->p.n;
  KD_LAUNCH(energy_kernel(fields, len, count, energy_out, ctx->st), "energy");
  return KD_OK;
}

kd_status kd_growth_rate(kd_ctx* ctx, const double* u_slices, int n_samples, double T, double fit_from,
                         double* rate_out) {
  if (!ctx) return KD_EINVAL;
  if (!u_slices || !rate_out || n_samples < 2 || !(T > 0))
    return fail(ctx, KD_EINVAL, "kd_growth_rate: bad argument");
  if (n_samples > KD_MAX_SLICES + 1) return fail(ctx, KD_EINVAL, "kd_growth_rate: too many samples");
  const long len = 3L * ctx->p.n * ctx->p.n;
  KD_LAUNCH(energy_kernel(u_slices, len, n_samples, ctx->Ebuf, ctx->st), "energy");
  KD_LAUNCH(growth_fit(ctx->Ebuf, n_samples, T / (n_samples - 1), fit_from, ctx->scal + 4, ctx->st), "fit");
  KD_CUDA(cudaMemcpyAsync(ctx->host_scal, ctx->scal + 4, 16, cudaMemcpyDeviceToHost, ctx->st), "fit copy");
  KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
  if (ctx->host_scal[1] != 1.0) return fail(ctx, KD_ENONFINITE, "kd_growth_rate: non-finite or zero energy");
  *rate_out = ctx->host_scal[0];
  return KD_OK;
}

}  // extern "C"
