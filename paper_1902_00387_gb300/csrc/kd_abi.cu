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
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/kd.h"
#include "kd_coarse.h"
#include "kd_fine.h"

using namespace kd;

namespace {

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
  void* M = nullptr;
  void* W = nullptr;
  void* ph = nullptr;      // flow-phase table
  size_t ph_bytes = 0;
};

size_t csize(int prec) { return prec == KD_C128 ? 16 : 8; }

}  // namespace

struct kd_ctx {
  kd_params p;
  cudaStream_t st = nullptr;
  int device = 0;
  Tables tab_f, tab_c;
  FineWs ws_f, ws_c;
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
  std::vector<void*> allocs;
  std::string err;
  long long launches = 0;     // kernels launched by this context
  // optional event timing of the fine column / row kernels
  int prof = 0;
  std::vector<cudaEvent_t> pev;
  std::vector<int> pkid;
  size_t pev_used = 0;
  double prof_ms[2] = {0.0, 0.0};
  long long prof_n[2] = {0, 0};
};

namespace {

kd_status fail(kd_ctx* c, kd_status s, const std::string& m) {
  if (c) c->err = m;
  return s;
}

kd_status cuda_fail(kd_ctx* c, cudaError_t e, const char* where) {
  return fail(c, e == cudaErrorMemoryAllocation ? KD_ENOMEM : KD_ECUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define KD_CUDA(call, where)                           \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

#define KD_LAUNCH(expr, where)                                        \
  do {                                                                \
    int r_ = (expr);                                                  \
    if (r_ < 0) return fail(ctx, KD_ECUDA, std::string(where) + ": launch failed"); \
    ctx->launches += r_ > 0 ? r_ : 1;                                 \
    cudaError_t e_ = cudaGetLastError();                              \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where);          \
  } while (0)

bool valid_n(int n) {
  return n == 16 || n == 32 || n == 64 || n == 128 || n == 256 || n == 512 || n == 1024;
}
int kept(int n) { return 2 * (n / 3) + 1; }
long compact_len(int n) { return 3L * kept(n) * kept(n); }  // complex entries per field

kd_status dalloc(kd_ctx* ctx, void** p, size_t bytes, const char* what) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, KD_ENOMEM, std::string("cudaMalloc ") + what + " (" + std::to_string(bytes) + " B): " +
                                    cudaGetErrorString(e));
  }
  ctx->allocs.push_back(*p);
  return KD_OK;
}

void dfree(kd_ctx* ctx, void* p) {
  if (!p) return;
  cudaFree(p);
  for (auto& a : ctx->allocs)
    if (a == p) a = nullptr;
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
  // exact values where the angle is a multiple of pi/2
  for (int e = 0; e < n; e += n / 4) {
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
  dfree(ctx, w.M);
  dfree(ctx, w.W);
  dfree(ctx, w.ph);
  w = FineWs();
  const size_t es = csize(prec);
  const size_t spec = (size_t)batch * compact_len(n) * es;
  const size_t mixed = (size_t)batch * 3 * kept(n) * n * es;
  kd_status s;
  if ((s = dalloc(ctx, &w.X, spec, "state")) != KD_OK) return s;
  if ((s = dalloc(ctx, &w.R2, spec, "R2")) != KD_OK) return s;
  if ((s = dalloc(ctx, &w.R3, spec, "R3")) != KD_OK) return s;
  if ((s = dalloc(ctx, &w.R4, spec, "R4")) != KD_OK) return s;
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
  a.n = n;
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
  a.M = w.M;
  a.W = w.W;
  a.tw = t.tw;
  a.cosg = t.cosg;
  a.sing = t.sing;
  a.phases = nullptr;
  a.phase_steps = 0;
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
  ctx->cap_slices = 0;
  const int n = ctx->p.n, nc = ctx->p.n_coarse;
  kd_status s;
  if ((s = dalloc(ctx, (void**)&ctx->U, (N + 1) * compact_len(n) * 16, "U")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&ctx->Fv, N * compact_len(n) * 16, "F values")) != KD_OK) return s;
  if ((s = dalloc(ctx, (void**)&ctx->Gv, N * compact_len(nc) * 16, "G values")) != KD_OK) return s;
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
  if (!valid_n(p->n)) return why = "n must be a power of two in [16, 1024]", KD_EINVAL;
  if (!valid_n(p->n_coarse) || p->n_coarse > p->n) return why = "n_coarse must be a power of two in [16, n]", KD_EINVAL;
  if (!(p->Rm > 0) || !isfinite(p->Rm)) return why = "Rm must be finite and > 0", KD_EINVAL;
  if (!isfinite(p->kz)) return why = "kz must be finite", KD_EINVAL;
  if (!(p->dt_fine > 0) || !(p->dt_coarse > 0)) return why = "time steps must be > 0", KD_EINVAL;
  if ((p->prec_fine != KD_C64 && p->prec_fine != KD_C128) || (p->prec_coarse != KD_C64 && p->prec_coarse != KD_C128))
    return why = "precision must be KD_C64 or KD_C128", KD_EINVAL;
  if (p->coarse_kind != KD_COARSE_CLASSICAL) return why = "only the classical coarse propagator is built", KD_EUNSUPPORTED;
  if (p->fine_form != KD_FINE_DIRECT && p->fine_form != KD_FINE_INCREMENT) return why = "bad fine_form", KD_EINVAL;
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
  c.Kc = ctx->p.n_coarse / 3;
  c.Kf = ctx->p.n / 3;
  c.flow = ctx->p.flow;
  c.amp = ctx->p.flow == KD_FLOW_ROBERTS ? 1.0 : ctx->p.flow == KD_FLOW_GALLOWAY_PROCTOR ? sqrt(1.5) : 0.0;
  c.kz = ctx->p.kz;
  c.Rm = ctx->p.Rm;
  c.dt = dtc;
  c.nsteps = steps;
  return c;
}

// Serial-sweep step of slice i with a coarse solve:
//   init:      U_{i+1} = G(U_i),                        Gv_i = G(U_i)
//   direct:    U_{i+1} = Fv_i + (G(U_i) - Gv_i),         Gv_i = G(U_i)
//   increment: U_{i+1} = Fv_i + G(U_i - Uprev_i)   (G linear; Uprev_i = previous iterate)
// (+ sigma of U_{i+1} when `last`).
kd_status coarse_step(kd_ctx* ctx, int i, int Sc, double dtc, bool init, bool last) {
  const int n = ctx->p.n, nc = ctx->p.n_coarse, pc = ctx->p.prec_coarse;
  const long len = compact_len(n), lenc = compact_len(nc);
  const bool incr = !init && ctx->p.fine_form == KD_FINE_INCREMENT;
  if (coarse_conv_supported(nc)) {
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
    KD_LAUNCH(coarse_conv_launch(pc, c, 1, nc, ctx->st), "coarse solve");
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
  KD_LAUNCH(fine_launch_steps(pc, a, Sc, true, false, ctx->st), "coarse steps");
  int nb = parareal_update(init ? nullptr : ctx->Fv + 2 * i * len, ctx->ws_c.X, pc, ctx->Gv + 2 * i * lenc,
                           ctx->U + 2 * (i + 1) * len, n, nc, init ? 1 : (incr ? 2 : 0),
                           last ? ctx->partials : nullptr, ctx->st);
  if (nb < 0) return fail(ctx, KD_ECUDA, "parareal update launch failed");
  ctx->launches += 1;
  if (last) KD_LAUNCH(finish_sigma(ctx->partials, nb, ctx->scal, ctx->st), "sigma");
  return KD_OK;
}

// Parallel fine step over slices [first, N): Fv[n] = F(U[n]), directly or in the
// increment form Fv[n] += F(U[n] - Uprev[n]) (iter > 1).
kd_status fine_sweep(kd_ctx* ctx, int first, int N, int S, double dt, int iter) {
  const int n = ctx->p.n, pf = ctx->p.prec_fine;
  const long b = N - first;
  if (b <= 0) return KD_OK;
  const long len = compact_len(n);
  const bool incr = ctx->p.fine_form == KD_FINE_INCREMENT;
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
  KD_LAUNCH(fine_launch_steps(pf, a, S, true, false, ctx->st, ctx->prof ? &pr : nullptr), "fine steps");
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

}  // namespace

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
  ctx->st = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = fine_prepare(params->prec_fine);
  if (e == cudaSuccess) e = fine_prepare(params->prec_coarse);
  if (e == cudaSuccess) e = coarse_prepare(params->prec_coarse);
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&ctx->ev[i]);
  if (e != cudaSuccess) {
    fprintf(stderr, "kd_create: %s\n", cudaGetErrorString(e));
    delete ctx;
    return KD_ECUDA;
  }
  if ((s = make_tables(ctx, ctx->tab_f, params->n, params->prec_fine)) != KD_OK ||
      (s = make_tables(ctx, ctx->tab_c, params->n_coarse, params->prec_coarse)) != KD_OK ||
      (s = dalloc(ctx, (void**)&ctx->partials, 2 * 1024 * 8, "partials")) != KD_OK ||
      (s = dalloc(ctx, (void**)&ctx->scal, 16 * 8, "scalars")) != KD_OK ||
      (s = dalloc(ctx, (void**)&ctx->Ebuf, (KD_MAX_SLICES + 1) * 8, "energies")) != KD_OK) {
    fprintf(stderr, "kd_create: %s\n", ctx->err.c_str());
    kd_destroy(ctx);
    return s;
  }
  if (cudaMallocHost((void**)&ctx->host_scal, 16 * 8) != cudaSuccess) {
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
  if (ctx->host_scal) cudaFreeHost(ctx->host_scal);
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
  KD_LAUNCH(full_to_compact(pf, b_in, pf, ctx->ws_f.X, batch, n, ctx->st), "pack");
  FineArgs a = fine_args(ctx, ctx->ws_f, ctx->tab_f, n, batch, ctx->p.dt_fine, t0);
  if ((s = with_phases(ctx, ctx->ws_f, a, nsteps)) != KD_OK) return s;
  LaunchProbe pr = probe_of(ctx);
  if (nsteps > 0)
    KD_LAUNCH(fine_launch_steps(pf, a, nsteps, true, false, ctx->st, ctx->prof ? &pr : nullptr), "fine steps");
  KD_LAUNCH(compact_to_full(pf, ctx->ws_f.X, pf, b_out, batch, n, ctx->st), "unpack");
  return KD_OK;
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
  if (coarse_conv_supported(nc) && nsteps > 0) {
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
    KD_LAUNCH(coarse_conv_launch(pc, c, batch, nc, ctx->st), "coarse solve");
    KD_LAUNCH(compact_resample(KD_C128, ctx->ws_c.X, nc, KD_C128, ctx->full_tmp, n, batch, ctx->st), "prolong");
    KD_LAUNCH(compact_to_full(KD_C128, ctx->full_tmp, KD_C128, b_out, batch, n, ctx->st), "unpack");
    return KD_OK;
  }
  KD_LAUNCH(compact_resample(KD_C128, ctx->full_tmp, n, pc, ctx->ws_c.X, nc, batch, ctx->st), "restrict");
  FineArgs a = fine_args(ctx, ctx->ws_c, ctx->tab_c, nc, batch, ctx->p.dt_coarse, t0);
  if ((s = with_phases(ctx, ctx->ws_c, a, nsteps)) != KD_OK) return s;
  if (nsteps > 0) KD_LAUNCH(fine_launch_steps(pc, a, nsteps, true, false, ctx->st), "coarse steps");
  KD_LAUNCH(compact_resample(pc, ctx->ws_c.X, nc, KD_C128, ctx->full_tmp, n, batch, ctx->st), "prolong");
  KD_LAUNCH(compact_to_full(KD_C128, ctx->full_tmp, KD_C128, b_out, batch, n, ctx->st), "unpack");
  return KD_OK;
}

kd_status kd_parareal_run(kd_ctx* ctx, const double* b0, double T, int N, int k_max, double tol, double* u_slices,
                          kd_parareal_stats* stats) {
  if (!ctx) return KD_EINVAL;
  if (!b0) return fail(ctx, KD_EINVAL, "kd_parareal_run: b0 is NULL");
  if (N < 1 || N > KD_MAX_SLICES) return fail(ctx, KD_EINVAL, "kd_parareal_run: n_slices out of range");
  if (k_max < 0 || k_max > KD_MAX_ITERS) return fail(ctx, KD_EINVAL, "kd_parareal_run: k_max out of range");
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
  const long len = compact_len(n), lenc = compact_len(nc);
  KD_LAUNCH(fill_times(ctx->t0f, N + 1, 0.0, dT, ctx->st), "times");
  KD_LAUNCH(fill_times(ctx->t0c, N + 1, 0.0, dT, ctx->st), "times");

  KD_CUDA(cudaEventRecord(ctx->ev[0], ctx->st), "event");
  if ((s = copy_in_b0(ctx, b0)) != KD_OK) return s;
  if ((s = coarse_phases(ctx, N, Sc, dtc)) != KD_OK) return s;
  float ms_fine = 0.f, ms_coarse = 0.f;
  // iterate 0: serial coarse sweep
  KD_CUDA(cudaEventRecord(ctx->ev[2], ctx->st), "event");
  for (int i = 0; i < N; ++i)
    if ((s = coarse_step(ctx, i, Sc, dtc, true, false)) != KD_OK) return s;
  KD_CUDA(cudaEventRecord(ctx->ev[3], ctx->st), "event");
  KD_CUDA(cudaEventSynchronize(ctx->ev[3]), "sync");
  {
    float m = 0.f;
    cudaEventElapsedTime(&m, ctx->ev[2], ctx->ev[3]);
    ms_coarse += m;
  }
  int k_done = 0, conv = 0;
  std::vector<double> sig;
  for (int k = 1; k <= k_max; ++k) {
    // parallel step over the slices that can still change: n >= k - 1
    // (the last slice is always swept so that sigma is measured)
    const int first = k - 1 < N - 1 ? k - 1 : N - 1;
    KD_CUDA(cudaEventRecord(ctx->ev[1], ctx->st), "event");
    if ((s = fine_sweep(ctx, first, N, S, dt, k)) != KD_OK) return s;
    KD_CUDA(cudaEventRecord(ctx->ev[2], ctx->st), "event");
    // serial step; slice `first` has U_first unchanged, so G(U_first) is the stored
    // coarse value bit for bit and the coarse terms cancel without a coarse solve
    {
      const bool last = (first == N - 1);
      int nb = parareal_update(ctx->Fv + 2 * first * len, ctx->Gv + 2 * first * lenc, KD_C128,
                               ctx->Gv + 2 * first * lenc, ctx->U + 2 * (first + 1) * len, n, nc, 0,
                               last ? ctx->partials : nullptr, ctx->st);
      if (nb < 0) return fail(ctx, KD_ECUDA, "parareal update launch failed");
      ctx->launches += 1;
      if (last) KD_LAUNCH(finish_sigma(ctx->partials, nb, ctx->scal, ctx->st), "sigma");
    }
    for (int i = first + 1; i < N; ++i)
      if ((s = coarse_step(ctx, i, Sc, dtc, false, i == N - 1)) != KD_OK) return s;
    KD_CUDA(cudaMemcpyAsync(ctx->host_scal, ctx->scal, 8, cudaMemcpyDeviceToHost, ctx->st), "sigma copy");
    KD_CUDA(cudaEventRecord(ctx->ev[3], ctx->st), "event");
    KD_CUDA(cudaEventSynchronize(ctx->ev[3]), "sync");
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
  }
  if (!conv && k_max > 0) return fail(ctx, KD_ENOTCONV, "kd_parareal_run: tol not reached within k_max");
  return KD_OK;
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
  KD_LAUNCH(fill_times(ctx->t0f, N + 1, 0.0, dT, ctx->st), "times");
  if ((s = copy_in_b0(ctx, b0)) != KD_OK) return s;
  for (int i = 0; i < N; ++i) {
    KD_LAUNCH(compact_resample(KD_C128, ctx->U + 2 * i * len, n, pf, ctx->ws_f.X, n, 1, ctx->st), "to fine");
    FineArgs a = fine_args(ctx, ctx->ws_f, ctx->tab_f, n, 1, dt, ctx->t0f + i);
    if ((s = with_phases(ctx, ctx->ws_f, a, S)) != KD_OK) return s;
    KD_LAUNCH(fine_launch_steps(pf, a, S, true, false, ctx->st), "fine steps");
    KD_LAUNCH(compact_resample(pf, ctx->ws_f.X, n, KD_C128, ctx->U + 2 * (i + 1) * len, n, 1, ctx->st), "from fine");
  }
  if ((s = copy_out_slices(ctx, u_slices, N)) != KD_OK) return s;
  KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
  return KD_OK;
}

long long kd_launch_count(kd_ctx* ctx) { return ctx ? ctx->launches : -1; }

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
  kd_status s;
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
