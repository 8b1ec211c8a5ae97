// kd_sweep_run: many independent Parareal problems (Sec. 3, Eq. 8 / Eq. 9 applied to each
// instance) batched on one GPU.
//
// Instances are grouped by (n, n_coarse).  A group keeps every instance's slice states on
// the device in FP64 compact form, U / Fv / Uprev [member][N + 1][3][P][P], and iterates
// all its unconverged members together:
//  - parallel step: the active (member, slice) pairs form one fine batch ordered by
//    decreasing fine step count, each field with its own dt, kz, Rm and flow
//    (FineArgs::sp); at step s only the prefix of fields that still have steps is
//    launched.  Increment form: the batch holds U - Uprev and Fv accumulates F of it.
//  - serial step: slice by slice, the restricted increments of all active members form
//    one coarse batch, U_{n+1} = Fv_n + prolong(G(restrict(U_n - Uprev_n))): for coarse
//    sets of side <= 88 one persistent cluster launch per slice (restriction, every
//    coarse step and the FP64 update fused, each field with its own step count),
//    otherwise the fine-step kernels on the coarse grid (fields ordered by decreasing
//    coarse step count, launched as a shrinking prefix) between a restriction and an
//    update kernel.
//  - defect (Eq. 9) per member from deterministic per-block partial sums.
// Members leave the iteration when their defect reaches tol.  Slices n < k - 1 are exact
// after k iterations and are skipped, as in kd_parareal_run.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <string>
#include <vector>

#include "kd_coarse.h"
#include "kd_ctx.h"

using namespace kd;
using namespace kdi;

namespace {

constexpr int kUpdBlocks = 64;   // blocks per field of the update / defect kernels

unsigned grid1(long total) {
  long g = (total + 255) / 256;
  if (g > 65535L * 8) g = 65535L * 8;
  return (unsigned)(g < 1 ? 1 : g);
}

// X[e] = U[slot_e] - Uprev[slot_e] (U[slot_e] on the first iteration), Uprev[slot_e] = U[slot_e]
template <typename To>
__global__ void k_delta_in_map(const cx<double>* U, cx<double>* Uprev, cx<To>* X, const int* emap, long len,
                               long nE, int first_iter) {
  const long total = nE * len;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const long e = t / len, i = t - e * len;
    const long g = (long)emap[e] * len + i;
    const cx<double> u = U[g];
    const cx<double> d = first_iter ? u : u - Uprev[g];
    Uprev[g] = u;
    X[t] = mk((To)d.x, (To)d.y);
  }
}

// Fv[slot_e] = X[e] (first iteration) or Fv[slot_e] + X[e]
template <typename Ti>
__global__ void k_accum_out_map(const cx<Ti>* X, cx<double>* Fv, const int* emap, long len, long nE,
                                int first_iter) {
  const long total = nE * len;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const long e = t / len, i = t - e * len;
    const long g = (long)emap[e] * len + i;
    const cx<double> x = mk((double)X[t].x, (double)X[t].y);
    Fv[g] = first_iter ? x : Fv[g] + x;
  }
}

// Xc[j] = restriction to |k| <= Kc of U[slot_j] - Uprev[slot_j] (Uprev may be NULL)
template <typename To>
__global__ void k_restrict_map(const cx<double>* U, const cx<double>* Uprev, const int* cmap, int Kf, int Pf,
                               cx<To>* Xc, int Kc, int Pc, long nC) {
  const long lenc = 3L * Pc * Pc, lenf = 3L * Pf * Pf;
  const long total = nC * lenc;
  const int off = Kf - Kc;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const long j = t / lenc;
    long r = t - j * lenc;
    const int c = (int)(r / ((long)Pc * Pc));
    r -= (long)c * Pc * Pc;
    const int iy = (int)(r / Pc), ix = (int)(r - (long)iy * Pc);
    const long g = (long)cmap[j] * lenf + ((long)c * Pf + iy + off) * Pf + ix + off;
    cx<double> d = U[g];
    if (Uprev) d = d - Uprev[g];
    Xc[t] = mk((To)d.x, (To)d.y);
  }
}

// U[slot_j + 1] = Fv[slot_j] (or 0 when Fv is NULL) + prolong(Xc[j]) (Xc may be NULL);
// with partials: per-block sums of |new - old|^2 and |new|^2 for the defect.
template <typename Ti>
__global__ void k_update_map(const cx<double>* Fv, const cx<Ti>* Xc, const int* cmap, cx<double>* U, int Kf, int Pf,
                             int Kc, int Pc, double* partials) {
  const long lenf = 3L * Pf * Pf;
  const int j = blockIdx.y;
  const long base = (long)cmap[j] * lenf;
  const cx<double>* F = Fv ? Fv + base : nullptr;
  cx<double>* Un = U + base + lenf;
  const cx<Ti>* G = Xc ? Xc + (long)j * 3 * Pc * Pc : nullptr;
  const int off = Kf - Kc;
  double dsum = 0.0, nsum = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < lenf; i += (long)gridDim.x * blockDim.x) {
    cx<double> v = F ? F[i] : mk(0.0, 0.0);
    if (G) {
      long r = i;
      const int c = (int)(r / ((long)Pf * Pf));
      r -= (long)c * Pf * Pf;
      const int iy = (int)(r / Pf) - off, ix = (int)(r % Pf) - off;
      if (iy >= 0 && iy < Pc && ix >= 0 && ix < Pc) {
        const cx<Ti> gv = G[((long)c * Pc + iy) * Pc + ix];
        v = v + mk((double)gv.x, (double)gv.y);
      }
    }
    if (partials) {
      const cx<double> o = Un[i];
      const double dx = v.x - o.x, dy = v.y - o.y;
      dsum += dx * dx + dy * dy;
      nsum += v.x * v.x + v.y * v.y;
    }
    Un[i] = v;
  }
  if (!partials) return;
  __shared__ double sd[256], sn[256];
  sd[threadIdx.x] = dsum;
  sn[threadIdx.x] = nsum;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sd[threadIdx.x] += sd[threadIdx.x + w];
      sn[threadIdx.x] += sn[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[((long)j * gridDim.x + blockIdx.x) * 2 + 0] = sd[0];
    partials[((long)j * gridDim.x + blockIdx.x) * 2 + 1] = sn[0];
  }
}

// sigma[j] = sqrt(sum diff / sum norm) over the nb partial pairs of member j (fixed order)
__global__ void k_sigma_map(const double* partials, int nb, double* sigma, int nC) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nC) return;
  double d = 0.0, s = 0.0;
  for (int b = 0; b < nb; ++b) {
    d += partials[((long)j * nb + b) * 2 + 0];
    s += partials[((long)j * nb + b) * 2 + 1];
  }
  sigma[j] = s > 0.0 ? sqrt(d / s) : (d > 0.0 ? INFINITY : 0.0);
}

struct Member {
  int idx = 0;           // instance index in the caller's arrays
  kd_instance in;
  int S = 0, Sc = 0;
  double dt = 0, dtc = 0;
  bool active = true;
  int status = KD_OK;
  int k = 0;
  std::vector<double> sigma;
  double growth = 0.0;
};

SliceParams slice_params(const kd_instance& in, double dt) {
  SliceParams p;
  p.amp = in.flow == KD_FLOW_ROBERTS ? 1.0 : in.flow == KD_FLOW_GALLOWAY_PROCTOR ? sqrt(1.5) : 0.0;
  p.kz = in.kz;
  p.Rm = in.Rm;
  p.dt = dt;
  p.flow = in.flow;
  p.pad = 0;
  return p;
}

struct GroupTimes {
  double fine = 0, coarse = 0, dof = 0;
  long long launches = 0;
};

// Device buffers of one group (owned by the group's context).
struct GroupBufs {
  double *U = nullptr, *Fv = nullptr, *Up = nullptr;
  SliceParams *spf = nullptr, *spc = nullptr;
  double *t0f = nullptr, *t0c = nullptr;
  int *emap = nullptr, *cmap = nullptr;
  double *partials = nullptr, *sigma = nullptr, *E = nullptr, *fit = nullptr;
  double* sig3 = nullptr;      // cluster path: (sigma, diff, norm) per field
  int* stepsc = nullptr;       // cluster path: coarse steps per field
  void* phc = nullptr;         // cluster path: coarse phase table of every slice
  size_t phc_bytes = 0;
};

// Device buffers of a group and the workspaces its launches use (made once per sweep
// object, before any launch is captured).
kd_status alloc_group(kd_ctx* ctx, const std::vector<Member>& mem, int N, GroupBufs& g) {
  const int m = (int)mem.size();
  const int n = mem[0].in.n, nc = mem[0].in.n_coarse;
  const long len = compact_len(n);
  const long slots = (long)m * (N + 1);
  kd_status s;
  if ((s = dalloc(ctx, (void**)&g.U, slots * len * 16, "sweep U")) != KD_OK ||
      (s = dalloc(ctx, (void**)&g.Fv, slots * len * 16, "sweep F values")) != KD_OK ||
      (s = dalloc(ctx, (void**)&g.Up, slots * len * 16, "sweep previous iterate")) != KD_OK ||
      (s = dalloc(ctx, (void**)&g.spf, (size_t)m * N * sizeof(SliceParams), "slice params")) != KD_OK ||
      (s = dalloc(ctx, (void**)&g.spc, (size_t)m * N * sizeof(SliceParams), "coarse params")) != KD_OK ||
      (s = dalloc(ctx, (void**)&g.sig3, (size_t)m * 3 * 8, "cluster defects")) != KD_OK ||
      (s = dalloc(ctx, (void**)&g.stepsc, (size_t)m * 4, "coarse steps")) != KD_OK ||
      (s = dalloc(ctx, (void**)&g.t0f, (size_t)m * N * 8, "slice times")) != KD_OK ||
      (s = dalloc(ctx, (void**)&g.t0c, (size_t)m * N * 8, "coarse times")) != KD_OK ||
      (s = dalloc(ctx, (void**)&g.emap, (size_t)m * N * 4, "fine map")) != KD_OK ||
      (s = dalloc(ctx, (void**)&g.cmap, (size_t)m * N * 4, "coarse map")) != KD_OK ||
      (s = dalloc(ctx, (void**)&g.partials, (size_t)m * kUpdBlocks * 2 * 8, "partials")) != KD_OK ||
      (s = dalloc(ctx, (void**)&g.sigma, (size_t)m * 8, "defects")) != KD_OK ||
      (s = dalloc(ctx, (void**)&g.E, (size_t)slots * 8, "energies")) != KD_OK ||
      (s = dalloc(ctx, (void**)&g.fit, (size_t)m * 2 * 8, "fits")) != KD_OK)
    return s;
  if ((s = ensure_ws(ctx, ctx->ws_f, n, KD_C64, (long)m * N)) != KD_OK) return s;
  if ((s = ensure_ws(ctx, ctx->ws_c, nc, KD_C64, m)) != KD_OK) return s;
  const size_t fb = 3UL * n * n * 16;
  const size_t need = fb > (size_t)len * 16 ? fb : (size_t)len * 16;
  if (ctx->full_tmp_bytes < need) {
    dfree(ctx, ctx->full_tmp);
    ctx->full_tmp = nullptr;
    ctx->full_tmp_bytes = 0;
    if ((s = dalloc(ctx, &ctx->full_tmp, need, "staging")) != KD_OK) return s;
    ctx->full_tmp_bytes = need;
  }
  return KD_OK;
}

// One solve of every member of a group from its initial field (the Parareal iterations of
// Eq. 8 with the defect of Eq. 9 per member).
kd_status exec_group(kd_ctx* ctx, std::vector<Member>& mem, GroupBufs& g, double T, int N, int k_max, double tol,
                     const double* const* b0, double* const* u_final, GroupTimes& gt) {
  const int m = (int)mem.size();
  const int n = mem[0].in.n, nc = mem[0].in.n_coarse;
  const int Kf = n / 3, Pf = kept(n), Kc = nc / 3, Pc = kept(nc);
  const long len = compact_len(n), lenc = compact_len(nc);
  const double dT = T / N;
  const long slots = (long)m * (N + 1);
  const size_t fb = 3UL * n * n * 16;
  kd_status s;
  const long long launches0 = ctx->launches;
  for (Member& mb : mem) {
    mb.active = true;
    mb.status = KD_OK;
    mb.k = 0;
    mb.sigma.clear();
    mb.growth = 0.0;
  }
  // initial fields -> U[member][0]
  for (int r = 0; r < m; ++r) {
    KD_CUDA(cudaMemcpyAsync(ctx->full_tmp, b0[mem[r].idx], fb, cudaMemcpyDefault, ctx->st), "copy b0");
    KD_LAUNCH(full_to_compact(KD_C128, ctx->full_tmp, KD_C128, g.U + 2 * (long)r * (N + 1) * len, 1, n, ctx->st),
              "b0 to compact");
  }
  auto slot = [&](int r, int sl) { return r * (N + 1) + sl; };
  std::vector<int> emap, cmap, act_f, act_c;
  std::vector<SliceParams> spf, spc;
  std::vector<double> t0f, t0c;
  cudaEvent_t e0 = ctx->ev[0], e1 = ctx->ev[1], e2 = ctx->ev[2];

  for (int k = 0; k <= k_max; ++k) {
    std::vector<int> A;   // active members
    for (int r = 0; r < m; ++r)
      if (mem[r].active) A.push_back(r);
    if (A.empty()) break;
    std::vector<int> Af = A, Ac = A;
    std::stable_sort(Af.begin(), Af.end(), [&](int a, int b) { return mem[a].S > mem[b].S; });
    std::stable_sort(Ac.begin(), Ac.end(), [&](int a, int b) { return mem[a].Sc > mem[b].Sc; });
    const int na = (int)A.size();
    const int first = k == 0 ? 0 : (k - 1 < N - 1 ? k - 1 : N - 1);
    KD_CUDA(cudaEventRecord(e0, ctx->st), "event");
    // ---- parallel fine step over slices [first, N) of the active members
    if (k >= 1) {
      const int nS = N - first;
      const long nE = (long)na * nS;
      emap.assign(nE, 0);
      spf.resize(nE);
      t0f.assign(nE, 0.0);
      for (int q = 0; q < na; ++q)
        for (int sl = first; sl < N; ++sl) {
          const long e = (long)q * nS + (sl - first);
          emap[e] = slot(Af[q], sl);
          spf[e] = slice_params(mem[Af[q]].in, mem[Af[q]].dt);
          t0f[e] = sl * dT;
        }
      const int Smax = mem[Af[0]].S;
      act_f.assign(Smax, 0);
      for (int st = 0; st < Smax; ++st) {
        int c = 0;
        while (c < na && mem[Af[c]].S > st) ++c;
        act_f[st] = c * nS;
        gt.dof += 3.0 * n * n * act_f[st];
      }
      KD_CUDA(cudaMemcpyAsync(g.emap, emap.data(), nE * 4, cudaMemcpyHostToDevice, ctx->st), "fine map");
      KD_CUDA(cudaMemcpyAsync(g.spf, spf.data(), nE * sizeof(SliceParams), cudaMemcpyHostToDevice, ctx->st),
              "slice params");
      KD_CUDA(cudaMemcpyAsync(g.t0f, t0f.data(), nE * 8, cudaMemcpyHostToDevice, ctx->st), "slice times");
      FineArgs a = fine_args(ctx, ctx->ws_f, ctx->tab_f, n, nE, mem[Af[0]].dt, g.t0f);
      a.flow = KD_FLOW_GALLOWAY_PROCTOR;   // the phase table holds every field's flow
      a.sp = g.spf;
      if ((s = with_phases(ctx, ctx->ws_f, a, Smax)) != KD_OK) return s;
      auto launches = [&]() -> kd_status {
        k_delta_in_map<float><<<grid1(nE * len), 256, 0, ctx->st>>>((const cx<double>*)g.U, (cx<double>*)g.Up,
                                                                      (cx<float>*)ctx->ws_f.X, g.emap, len, nE, k == 1);
        KD_LAUNCH(0, "increment to fine");
        KD_LAUNCH(run_fine(ctx, 0, KD_C64, a, Smax, true, false, nullptr, act_f.data()), "fine steps");
        k_accum_out_map<float><<<grid1(nE * len), 256, 0, ctx->st>>>((const cx<float>*)ctx->ws_f.X,
                                                                       (cx<double>*)g.Fv, g.emap, len, nE, k == 1);
        KD_LAUNCH(0, "accumulate fine");
        return KD_OK;
      };
      if (ctx->graphs && !ctx->prof) {
        // replayed when the same (iteration, active members, plan) recurs, e.g. in a
        // repeated kd_sweep_exec of the same instances
        std::string key = "sweep " + std::to_string(k == 1) + " " + std::to_string(first) + " " +
                          std::to_string(nE) + " " + std::to_string(Smax) + " " + std::to_string(ctx->plan[0].col) +
                          "," + std::to_string(ctx->plan[0].row) + " " + std::to_string(ctx->pdl) + " " +
                          std::to_string(ctx->alloc_gen) + " :";
        for (int r : Af) key += " " + std::to_string(r);
        if ((s = run_graph(ctx, key, launches)) != KD_OK) return s;
      } else if ((s = launches()) != KD_OK) {
        return s;
      }
    }
    KD_CUDA(cudaEventRecord(e1, ctx->st), "event");
    // ---- serial sweep
    int lo = first;
    if (k >= 1) {
      // slice `first` is unchanged since the last sweep: its coarse increment is zero
      cmap.assign(na, 0);
      for (int j = 0; j < na; ++j) cmap[j] = slot(Ac[j], first);
      KD_CUDA(cudaMemcpyAsync(g.cmap, cmap.data(), na * 4, cudaMemcpyHostToDevice, ctx->st), "coarse map");
      const bool last = first == N - 1;
      k_update_map<float><<<dim3(kUpdBlocks, na), 256, 0, ctx->st>>>((const cx<double>*)g.Fv, nullptr, g.cmap,
                                                                       (cx<double>*)g.U, Kf, Pf, Kc, Pc,
                                                                       last ? g.partials : nullptr);
      KD_LAUNCH(0, "update");
      lo = first + 1;
    }
    if (lo < N) {
      // per-slice copies of the members' coarse parameters, maps and start times ([slice][member])
      spc.resize((long)na * N);
      cmap.assign((long)na * N, 0);
      t0c.assign((long)na * N, 0.0);
      for (int sl = 0; sl < N; ++sl)
        for (int j = 0; j < na; ++j) {
          spc[(long)sl * na + j] = slice_params(mem[Ac[j]].in, mem[Ac[j]].dtc);
          cmap[(long)sl * na + j] = slot(Ac[j], sl);
          t0c[(long)sl * na + j] = sl * dT;
        }
      KD_CUDA(cudaMemcpyAsync(g.spc, spc.data(), (size_t)na * N * sizeof(SliceParams), cudaMemcpyHostToDevice,
                              ctx->st), "coarse params");
      KD_CUDA(cudaMemcpyAsync(g.cmap, cmap.data(), (size_t)na * N * 4, cudaMemcpyHostToDevice, ctx->st), "coarse map");
      KD_CUDA(cudaMemcpyAsync(g.t0c, t0c.data(), (size_t)na * N * 8, cudaMemcpyHostToDevice, ctx->st), "coarse times");
      const int Scmax = mem[Ac[0]].Sc;
      if (coarse_conv_supported(Pc)) {
        std::vector<int> stc(na);
        for (int j = 0; j < na; ++j) stc[j] = mem[Ac[j]].Sc;
        KD_CUDA(cudaMemcpyAsync(g.stepsc, stc.data(), na * 4, cudaMemcpyHostToDevice, ctx->st), "coarse steps");
        const size_t need = phase_table_bytes(KD_C64, (long)na * N, Scmax);
        if (g.phc_bytes < need) {
          dfree(ctx, g.phc);
          g.phc = nullptr;
          g.phc_bytes = 0;
          if ((s = dalloc(ctx, &g.phc, need, "coarse phase table")) != KD_OK) return s;
          g.phc_bytes = need;
        }
        FineArgs pa = fine_args(ctx, ctx->ws_c, ctx->tab_c, nc, (long)na * N, mem[Ac[0]].dtc, g.t0c);
        pa.flow = KD_FLOW_GALLOWAY_PROCTOR;
        pa.sp = g.spc;
        pa.phases = g.phc;
        KD_LAUNCH(launch_phases(KD_C64, pa, Scmax, ctx->st), "coarse phases");
        for (int sl = lo; sl < N; ++sl) {
          CoarseArgs c;
          memset(&c, 0, sizeof(c));
          c.Kc = Kc;
          c.Pc = Pc;
          c.Kf = Kf;
          c.Pf = Pf;
          c.flow = KD_FLOW_GALLOWAY_PROCTOR;
          c.nsteps = Scmax;
          c.phases = (const float*)g.phc + (size_t)sl * na * Scmax * 16;
          c.Un = g.U;
          c.Uprev = k >= 1 ? g.Up : nullptr;
          c.Fv = k >= 1 ? g.Fv : nullptr;
          c.Unext = g.U;
          c.mode = k >= 1 ? COARSE_INCR : COARSE_INIT;
          c.sigma_out = (k >= 1 && sl == N - 1) ? g.sig3 : nullptr;
          c.sp = g.spc + (long)sl * na;
          c.steps = g.stepsc;
          c.map = g.cmap + (long)sl * na;
          KD_LAUNCH(coarse_conv_launch(KD_C64, c, na, ctx->st), "coarse solve");
        }
      } else {
        act_c.assign(Scmax, 0);
        for (int st = 0; st < Scmax; ++st) {
          int c = 0;
          while (c < na && mem[Ac[c]].Sc > st) ++c;
          act_c[st] = c;
        }
        for (int sl = lo; sl < N; ++sl) {
          const int* cm = g.cmap + (long)sl * na;
          k_restrict_map<float><<<grid1((long)na * lenc), 256, 0, ctx->st>>>(
              (const cx<double>*)g.U, k >= 1 ? (const cx<double>*)g.Up : nullptr, cm, Kf, Pf,
              (cx<float>*)ctx->ws_c.X, Kc, Pc, na);
          KD_LAUNCH(0, "restrict");
          FineArgs ac = fine_args(ctx, ctx->ws_c, ctx->tab_c, nc, na, mem[Ac[0]].dtc, g.t0c + (long)sl * na);
          ac.flow = KD_FLOW_GALLOWAY_PROCTOR;
          ac.sp = g.spc + (long)sl * na;
          if ((s = with_phases(ctx, ctx->ws_c, ac, Scmax)) != KD_OK) return s;
          KD_LAUNCH(run_fine(ctx, 1, KD_C64, ac, Scmax, true, false, nullptr, act_c.data()), "coarse steps");
          const bool last = k >= 1 && sl == N - 1;
          k_update_map<float><<<dim3(kUpdBlocks, na), 256, 0, ctx->st>>>(
              k >= 1 ? (const cx<double>*)g.Fv : nullptr, (const cx<float>*)ctx->ws_c.X, cm, (cx<double>*)g.U, Kf,
              Pf, Kc, Pc, last ? g.partials : nullptr);
          KD_LAUNCH(0, "update");
        }
      }
    }
    KD_CUDA(cudaEventRecord(e2, ctx->st), "event");
    std::vector<double> sig(na, 0.0), sig3(3 * na, 0.0);
    const bool from_cluster = k >= 1 && first < N - 1 && coarse_conv_supported(Pc);
    if (k >= 1 && !from_cluster) {
      k_sigma_map<<<(na + 127) / 128, 128, 0, ctx->st>>>(g.partials, kUpdBlocks, g.sigma, na);
      KD_LAUNCH(0, "defect");
      KD_CUDA(cudaMemcpyAsync(sig.data(), g.sigma, na * 8, cudaMemcpyDeviceToHost, ctx->st), "defect copy");
    }
    if (from_cluster)
      KD_CUDA(cudaMemcpyAsync(sig3.data(), g.sig3, 3 * na * 8, cudaMemcpyDeviceToHost, ctx->st), "defect copy");
    KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
    float mf = 0.f, mc = 0.f;
    cudaEventElapsedTime(&mf, e0, e1);
    cudaEventElapsedTime(&mc, e1, e2);
    gt.fine += mf;
    gt.coarse += mc;
    if (k == 0) continue;
    if (from_cluster)
      for (int j = 0; j < na; ++j) sig[j] = sig3[3 * j];
    for (int j = 0; j < na; ++j) {
      Member& mb = mem[Ac[j]];
      mb.k = k;
      mb.sigma.push_back(sig[j]);
      if (!isfinite(sig[j])) {
        mb.status = KD_ENONFINITE;
        mb.active = false;
      } else if (sig[j] <= tol) {
        mb.status = KD_OK;
        mb.active = false;
      } else if (k == k_max) {
        mb.status = KD_ENOTCONV;
        mb.active = false;
      }
    }
  }
  for (Member& mb : mem)
    if (mb.active) {   // k_max == 0
      mb.status = k_max == 0 ? KD_ENOTCONV : mb.status;
      mb.active = false;
    }
  // energies, growth rates and final states
  KD_LAUNCH(energy_kernel(g.U, len, (int)slots, g.E, ctx->st), "energy");
  for (int r = 0; r < m; ++r)
    KD_LAUNCH(growth_fit(g.E + (long)r * (N + 1), N + 1, dT, 0.5 * T, g.fit + 2 * r, ctx->st), "growth fit");
  std::vector<double> fit(2 * m);
  KD_CUDA(cudaMemcpyAsync(fit.data(), g.fit, 2 * m * 8, cudaMemcpyDeviceToHost, ctx->st), "fit copy");
  for (int r = 0; r < m; ++r) {
    double* dst = u_final ? u_final[mem[r].idx] : nullptr;
    if (!dst) continue;
    KD_LAUNCH(compact_to_full(KD_C128, g.U + 2 * (long)slot(r, N) * len, KD_C128, ctx->full_tmp, 1, n, ctx->st),
              "final to full");
    KD_CUDA(cudaMemcpyAsync(dst, ctx->full_tmp, fb, cudaMemcpyDefault, ctx->st), "final copy");
  }
  KD_CUDA(cudaStreamSynchronize(ctx->st), "sync");
  for (int r = 0; r < m; ++r) mem[r].growth = fit[2 * r];
  gt.launches = ctx->launches - launches0;
  return KD_OK;
}

bool check_instance(const kd_instance& in, std::string& why) {
  if (in.flow < 0 || in.flow > 2) return why = "flow must be 0, 1 or 2", false;
  if (!valid_n(in.n)) return why = "n must be a power of two in [16, 1024]", false;
  if (!valid_n(in.n_coarse) || in.n_coarse > in.n) return why = "n_coarse must be a power of two in [16, n]", false;
  if (!(in.Rm > 0) || !isfinite(in.Rm) || !isfinite(in.kz)) return why = "Rm must be > 0, kz finite", false;
  if (!(in.dt_fine > 0) || !(in.dt_coarse > 0)) return why = "time steps must be > 0", false;
  return true;
}

void set_err(char* err, const std::string& m) {
  if (!err) return;
  snprintf(err, 256, "%s", m.c_str());
}

}  // namespace

// A prepared sweep: the instances grouped by (n, n_coarse), each group with its context,
// device buffers and workspaces, kept across kd_sweep_exec calls.
struct kd_sweep {
  double T = 0.0;
  int N = 0;
  int n_inst = 0;
  struct Group {
    kd_ctx* ctx = nullptr;
    std::vector<Member> mem;
    GroupBufs g;
    bool tuned = false;
  };
  std::vector<Group> groups;
};

extern "C" kd_status kd_sweep_destroy(kd_sweep* sw) {
  if (!sw) return KD_OK;
  for (auto& gr : sw->groups)
    if (gr.ctx) kd_destroy(gr.ctx);   // frees the group's buffers with the context's allocations
  delete sw;
  return KD_OK;
}

extern "C" kd_status kd_sweep_create(const kd_instance* inst, int n_inst, double T, int n_slices, void* cuda_stream,
                                     kd_sweep** out, char* err) {
  set_err(err, "");
  if (!out) return set_err(err, "kd_sweep_create: out is NULL"), KD_EINVAL;
  *out = nullptr;
  if (!inst || n_inst < 1) return set_err(err, "kd_sweep_create: no instances"), KD_EINVAL;
  if (n_slices < 1 || n_slices > KD_MAX_SLICES) return set_err(err, "kd_sweep_create: n_slices out of range"), KD_EINVAL;
  if (!(T > 0) || !isfinite(T)) return set_err(err, "kd_sweep_create: T must be > 0"), KD_EINVAL;
  for (int i = 0; i < n_inst; ++i) {
    std::string why;
    if (!check_instance(inst[i], why))
      return set_err(err, "kd_sweep_create: instance " + std::to_string(i) + ": " + why), KD_EINVAL;
  }
  const double dT = T / n_slices;
  std::map<std::pair<int, int>, std::vector<Member>> by_grid;
  for (int i = 0; i < n_inst; ++i) {
    Member mb;
    mb.idx = i;
    mb.in = inst[i];
    mb.S = steps_for(dT, inst[i].dt_fine);
    mb.Sc = steps_for(dT, inst[i].dt_coarse);
    mb.dt = dT / mb.S;
    mb.dtc = dT / mb.Sc;
    by_grid[{inst[i].n, inst[i].n_coarse}].push_back(mb);
  }
  kd_sweep* sw = new kd_sweep();
  sw->T = T;
  sw->N = n_slices;
  sw->n_inst = n_inst;
  for (auto& kv : by_grid) {
    kd_sweep::Group gr;
    gr.mem = kv.second;
    const Member& m0 = gr.mem[0];
    kd_params p;
    memset(&p, 0, sizeof(p));
    p.flow = m0.in.flow;
    p.n = m0.in.n;
    p.kz = m0.in.kz;
    p.Rm = m0.in.Rm;
    p.dt_fine = m0.in.dt_fine;
    p.prec_fine = KD_C64;
    p.n_coarse = m0.in.n_coarse;
    p.dt_coarse = m0.in.dt_coarse;
    p.prec_coarse = KD_C64;
    p.coarse_kind = KD_COARSE_CLASSICAL;
    p.learned_modes = 0;
    p.fine_form = KD_FINE_INCREMENT;
    kd_status s = kd_create(&p, cuda_stream, &gr.ctx);
    if (s == KD_OK) s = alloc_group(gr.ctx, gr.mem, n_slices, gr.g);
    if (s != KD_OK) {
      set_err(err, std::string("kd_sweep_create: ") + (gr.ctx ? gr.ctx->err : std::string("context creation failed")));
      if (gr.ctx) kd_destroy(gr.ctx);
      kd_sweep_destroy(sw);
      return s;
    }
    sw->groups.push_back(std::move(gr));
  }
  *out = sw;
  return KD_OK;
}

extern "C" kd_status kd_sweep_set_graphs(kd_sweep* sw, int enable) {
  if (!sw) return KD_EINVAL;
  for (auto& gr : sw->groups) kd_set_graphs(gr.ctx, enable);
  return KD_OK;
}

extern "C" kd_status kd_sweep_exec(kd_sweep* sw, const double* const* b0, int k_max, double tol,
                                   const char* tune_cache, double* const* u_final, kd_instance_result* results,
                                   kd_sweep_stats* stats, char* err) {
  const auto t_start = std::chrono::steady_clock::now();
  set_err(err, "");
  if (!sw || !b0) return set_err(err, "kd_sweep_exec: NULL sweep or b0"), KD_EINVAL;
  if (k_max < 0 || k_max > KD_MAX_ITERS) return set_err(err, "kd_sweep_exec: k_max out of range"), KD_EINVAL;
  for (int i = 0; i < sw->n_inst; ++i)
    if (!b0[i]) return set_err(err, "kd_sweep_exec: b0[" + std::to_string(i) + "] is NULL"), KD_EINVAL;
  kd_status worst = KD_OK;
  GroupTimes total;
  long long launches = 0;
  for (auto& gr : sw->groups) {
    std::vector<Member>& mem = gr.mem;
    kd_ctx* ctx = gr.ctx;
    kd_status s = KD_OK;
    if (tune_cache && !gr.tuned) {
      s = kd_autotune(ctx, KD_GRID_FINE, (int)mem.size() * sw->N, 2, tune_cache, nullptr);
      gr.tuned = s == KD_OK;
    }
    GroupTimes gt;
    if (s == KD_OK) s = exec_group(ctx, mem, gr.g, sw->T, sw->N, k_max, tol, b0, u_final, gt);
    if (s != KD_OK) return set_err(err, "kd_sweep_exec: " + ctx->err), s;
    launches += gt.launches;
    total.fine += gt.fine;
    total.coarse += gt.coarse;
    total.dof += gt.dof;
    for (const Member& mb : mem) {
      if (mb.status == KD_ENONFINITE) worst = KD_ENONFINITE;
      else if (mb.status == KD_ENOTCONV && worst == KD_OK) worst = KD_ENOTCONV;
      if (!results) continue;
      kd_instance_result& r = results[mb.idx];
      memset(&r, 0, sizeof(r));
      r.status = mb.status;
      r.k_con = mb.k;
      r.n_fine_steps = mb.S;
      r.n_coarse_steps = mb.Sc;
      r.dt_fine_used = mb.dt;
      r.dt_coarse_used = mb.dtc;
      for (size_t q = 0; q < mb.sigma.size() && q < KD_MAX_ITERS; ++q) r.sigma[q] = mb.sigma[q];
      r.growth_rate = mb.growth;
    }
  }
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->n_groups = (int)sw->groups.size();
    stats->ms_fine = total.fine;
    stats->ms_coarse = total.coarse;
    stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    stats->n_launches = launches;
    stats->fine_dof_steps = total.dof;
  }
  if (worst == KD_ENONFINITE) set_err(err, "kd_sweep_exec: an instance's defect was not finite");
  if (worst == KD_ENOTCONV) set_err(err, "kd_sweep_exec: some instances did not reach tol within k_max");
  return worst;
}

extern "C" kd_status kd_sweep_run(const kd_instance* inst, int n_inst, const double* const* b0, double T,
                                  int n_slices, int k_max, double tol, const char* tune_cache, double* const* u_final,
                                  kd_instance_result* results, kd_sweep_stats* stats, void* cuda_stream, char* err) {
  const auto t_start = std::chrono::steady_clock::now();
  if (!b0 && inst && n_inst >= 1) return set_err(err, "kd_sweep_run: no instances"), KD_EINVAL;
  if (k_max < 0 || k_max > KD_MAX_ITERS) return set_err(err, "kd_sweep_run: k_max out of range"), KD_EINVAL;
  for (int i = 0; b0 && inst && i < n_inst; ++i)
    if (!b0[i]) return set_err(err, "kd_sweep_run: b0[" + std::to_string(i) + "] is NULL"), KD_EINVAL;
  kd_sweep* sw = nullptr;
  kd_status s = kd_sweep_create(inst, n_inst, T, n_slices, cuda_stream, &sw, err);
  if (s != KD_OK) return s;
  s = kd_sweep_exec(sw, b0, k_max, tol, tune_cache, u_final, results, stats, err);
  kd_sweep_destroy(sw);
  if (stats) stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  return s;
}
