// Launch plans of the fine kernels and their autotuner (include/kd.h: kd_plan_variants,
// kd_set_plan, kd_get_plan, kd_autotune).
//
// A plan picks one column-kernel and one row-kernel variant (tile shape, stage-update
// style) for a grid and precision.  The autotuner times every pair on the context's own
// workspace with CUDA events and keeps the fastest; results persist in a small JSON file
// keyed by (device name, n, precision, batch rounded up to a power of two):
//
//   {"kd_autotune": 1, "entries": [
//     {"device": "...", "n": 128, "prec": 0, "batch": 64, "col": 0, "row": 2, "ms_per_step": 0.187}
//   ]}
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "kd_coarse.h"
#include "kd_ctx.h"

using namespace kd;
using namespace kdi;

namespace {

struct TuneEntry {
  std::string device;
  int n = 0, prec = 0, batch = 0, col = 0, row = 0;
  double ms = 0.0;
};

// Value of "key": in one entry object (string or number text), "" if absent.
std::string field(const std::string& obj, const char* key) {
  const std::string k = std::string("\"") + key + "\"";
  size_t p = obj.find(k);
  if (p == std::string::npos) return "";
  p = obj.find(':', p + k.size());
  if (p == std::string::npos) return "";
  ++p;
  while (p < obj.size() && (obj[p] == ' ' || obj[p] == '\t' || obj[p] == '\n' || obj[p] == '\r')) ++p;
  if (p < obj.size() && obj[p] == '"') {
    std::string out;
    for (++p; p < obj.size() && obj[p] != '"'; ++p) {
      if (obj[p] == '\\' && p + 1 < obj.size()) ++p;
      out.push_back(obj[p]);
    }
    return out;
  }
  size_t e = p;
  while (e < obj.size() && obj[e] != ',' && obj[e] != '}' && obj[e] != '\n') ++e;
  return obj.substr(p, e - p);
}

// Entries of a cache file; a missing or malformed file gives none.
std::vector<TuneEntry> read_cache(const char* path) {
  std::vector<TuneEntry> out;
  std::ifstream f(path);
  if (!f) return out;
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string s = ss.str();
  size_t p = s.find("\"entries\"");
  if (p == std::string::npos) return out;
  while (true) {
    const size_t a = s.find('{', p);
    if (a == std::string::npos) break;
    const size_t b = s.find('}', a);
    if (b == std::string::npos) break;
    const std::string obj = s.substr(a, b - a + 1);
    TuneEntry e;
    e.device = field(obj, "device");
    const std::string n = field(obj, "n"), pr = field(obj, "prec"), bt = field(obj, "batch"), c = field(obj, "col"),
                      r = field(obj, "row"), ms = field(obj, "ms_per_step");
    if (!e.device.empty() && !n.empty() && !pr.empty() && !bt.empty() && !c.empty() && !r.empty()) {
      e.n = atoi(n.c_str());
      e.prec = atoi(pr.c_str());
      e.batch = atoi(bt.c_str());
      e.col = atoi(c.c_str());
      e.row = atoi(r.c_str());
      e.ms = ms.empty() ? 0.0 : atof(ms.c_str());
      out.push_back(e);
    }
    p = b + 1;
  }
  return out;
}

std::string json_escape(const std::string& s) {
  std::string o;
  for (char ch : s) {
    if (ch == '"' || ch == '\\') o.push_back('\\');
    if ((unsigned char)ch >= 0x20) o.push_back(ch);
  }
  return o;
}

bool write_cache(const char* path, const std::vector<TuneEntry>& es) {
  const std::string tmp = std::string(path) + ".tmp";
  {
    std::ofstream f(tmp);
    if (!f) return false;
    f << "{\"kd_autotune\": 1, \"entries\": [\n";
    for (size_t i = 0; i < es.size(); ++i) {
      const TuneEntry& e = es[i];
      char buf[512];
      snprintf(buf, sizeof(buf),
               "  {\"device\": \"%s\", \"n\": %d, \"prec\": %d, \"batch\": %d, \"col\": %d, \"row\": %d, "
               "\"ms_per_step\": %.6g}%s\n",
               json_escape(e.device).c_str(), e.n, e.prec, e.batch, e.col, e.row, e.ms,
               i + 1 < es.size() ? "," : "");
      f << buf;
    }
    f << "]}\n";
    if (!f) return false;
  }
  return rename(tmp.c_str(), path) == 0;
}

int pow2_at_least(int b) {
  int p = 1;
  while (p < b && p < (1 << 30)) p <<= 1;
  return p;
}

// Seeded tuning data: a counter-based hash per complex entry, values in [-1e-3, 1e-3].
template <typename T>
__global__ void k_fill_hash(cx<T>* x, long total, unsigned seed) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    unsigned h = (unsigned)i * 2654435761u ^ seed;
    h ^= h >> 16;
    h *= 2246822519u;
    h ^= h >> 13;
    const unsigned h2 = h * 3266489917u ^ (h >> 15);
    x[i] = mk(T(1e-3) * (T((h & 0xffff) / 32767.5) - T(1)), T(1e-3) * (T((h2 & 0xffff) / 32767.5) - T(1)));
  }
}

int fill_hash(int prec, void* x, long total, unsigned seed, cudaStream_t st) {
  long g = (total + 255) / 256;
  if (g > 65535L * 8) g = 65535L * 8;
  if (prec == KD_C64)
    k_fill_hash<float><<<(unsigned)g, 256, 0, st>>>((cx<float>*)x, total, seed);
  else
    k_fill_hash<double><<<(unsigned)g, 256, 0, st>>>((cx<double>*)x, total, seed);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

bool grid_of(kd_ctx* ctx, int grid, int* n, int* prec) {
  if (grid == KD_GRID_FINE) {
    *n = ctx->p.n;
    *prec = ctx->p.prec_fine;
  } else if (grid == KD_GRID_COARSE) {
    *n = ctx->p.n_coarse;
    *prec = ctx->p.prec_coarse;
  } else {
    return false;
  }
  return true;
}

}  // namespace

extern "C" {

kd_status kd_plan_variants(kd_ctx* ctx, int grid, int* n_col, int* n_row) {
  if (!ctx) return KD_EINVAL;
  int n, prec;
  if (!grid_of(ctx, grid, &n, &prec) || !n_col || !n_row) return fail(ctx, KD_EINVAL, "kd_plan_variants: bad argument");
  if (!fine_variants(n, prec, n_col, n_row)) return fail(ctx, KD_EINVAL, "kd_plan_variants: unsupported grid");
  return KD_OK;
}

kd_status kd_set_plan(kd_ctx* ctx, int grid, int col, int row) {
  if (!ctx) return KD_EINVAL;
  int nc = 0, nr = 0;
  kd_status s = kd_plan_variants(ctx, grid, &nc, &nr);
  if (s != KD_OK) return s;
  if (col < 0 || col >= nc || row < 0 || row >= nr) return fail(ctx, KD_EINVAL, "kd_set_plan: variant out of range");
  ctx->plan[grid].col = col;
  ctx->plan[grid].row = row;
  return KD_OK;
}

kd_status kd_get_plan(kd_ctx* ctx, int grid, int* col, int* row) {
  if (!ctx) return KD_EINVAL;
  if ((grid != KD_GRID_FINE && grid != KD_GRID_COARSE) || !col || !row)
    return fail(ctx, KD_EINVAL, "kd_get_plan: bad argument");
  *col = ctx->plan[grid].col;
  *row = ctx->plan[grid].row;
  return KD_OK;
}

kd_status kd_set_coarse_cluster(kd_ctx* ctx, int blocks) {
  if (!ctx) return KD_EINVAL;
  if (!coarse_cluster_fits(ctx->cP, blocks))
    return fail(ctx, KD_EINVAL, "kd_set_coarse_cluster: the coarse set does not fit clusters of that size");
  ctx->coarse_cluster = blocks;
  return KD_OK;
}

kd_status kd_set_graphs(kd_ctx* ctx, int enable) {
  if (!ctx) return KD_EINVAL;
  ctx->graphs = enable ? 1 : 0;
  return KD_OK;
}

kd_status kd_set_learned_gemm(kd_ctx* ctx, int engine) {
  if (!ctx) return KD_EINVAL;
  if (engine != KD_GEMM_TCGEN05 && engine != KD_GEMM_MMA_SYNC)
    return fail(ctx, KD_EINVAL, "kd_set_learned_gemm: engine must be KD_GEMM_TCGEN05 or KD_GEMM_MMA_SYNC");
  ctx->gemm_engine = engine;
  return KD_OK;
}

kd_status kd_set_coarse_sync(kd_ctx* ctx, int mode) {
  if (!ctx) return KD_EINVAL;
  if (mode != KD_SYNC_CLUSTER && mode != KD_SYNC_P2P && mode != KD_SYNC_PULL)
    return fail(ctx, KD_EINVAL, "kd_set_coarse_sync: mode must be KD_SYNC_CLUSTER, KD_SYNC_P2P or KD_SYNC_PULL");
  ctx->coarse_sync = mode;
  return KD_OK;
}

kd_status kd_set_overlap(kd_ctx* ctx, int chunks) {
  if (!ctx) return KD_EINVAL;
  if (chunks < 0 || chunks > kMaxChunks) return fail(ctx, KD_EINVAL, "kd_set_overlap: chunks must be in [0, 16]");
  ctx->overlap = chunks;
  return KD_OK;
}

kd_status kd_set_dependent_launch(kd_ctx* ctx, int enable) {
  if (!ctx) return KD_EINVAL;
  ctx->pdl = enable ? 1 : 0;
  return KD_OK;
}

kd_status kd_autotune(kd_ctx* ctx, int grid, int batch, int nsteps, const char* cache_path, double* ms_per_step) {
  if (!ctx) return KD_EINVAL;
  int n, prec;
  if (!grid_of(ctx, grid, &n, &prec)) return fail(ctx, KD_EINVAL, "kd_autotune: bad grid");
  if (batch < 1 || nsteps < 1) return fail(ctx, KD_EINVAL, "kd_autotune: batch and nsteps must be >= 1");
  int nc = 0, nr = 0;
  if (!fine_variants(n, prec, &nc, &nr)) return fail(ctx, KD_EINVAL, "kd_autotune: unsupported grid");
  cudaDeviceProp prop;
  KD_CUDA(cudaGetDeviceProperties(&prop, ctx->device), "device properties");
  const std::string dev = prop.name;
  const int key = pow2_at_least(batch);
  std::vector<TuneEntry> cache;
  if (cache_path) {
    cache = read_cache(cache_path);
    for (const TuneEntry& e : cache)
      if (e.device == dev && e.n == n && e.prec == prec && e.batch == key && e.col >= 0 && e.col < nc && e.row >= 0 &&
          e.row < nr) {
        ctx->plan[grid].col = e.col;
        ctx->plan[grid].row = e.row;
        if (ms_per_step) *ms_per_step = -1.0;
        return KD_OK;
      }
  }
  FineWs& w = grid == KD_GRID_FINE ? ctx->ws_f : ctx->ws_c;
  Tables& t = grid == KD_GRID_FINE ? ctx->tab_f : ctx->tab_c;
  kd_status s = ensure_ws(ctx, w, n, prec, batch);
  if (s != KD_OK) return s;
  double* t0 = nullptr;
  if ((s = dalloc(ctx, (void**)&t0, (size_t)batch * 8, "tuning times")) != KD_OK) return s;
  s = KD_OK;
  KD_CUDA(cudaMemsetAsync(t0, 0, (size_t)batch * 8, ctx->st), "tuning times");
  const double dt = grid == KD_GRID_FINE ? ctx->p.dt_fine : ctx->p.dt_coarse;
  FineArgs a = fine_args(ctx, w, t, n, batch, dt, t0);
  if ((s = with_phases(ctx, w, a, nsteps)) != KD_OK) {
    dfree(ctx, t0);
    return s;
  }
  const FinePlan saved = ctx->plan[grid];
  double best = INFINITY;
  FinePlan best_plan = saved;
  for (int c = 0; c < nc && s == KD_OK; ++c)
    for (int r = 0; r < nr && s == KD_OK; ++r) {
      ctx->plan[grid].col = c;
      ctx->plan[grid].row = r;
      if (fill_hash(prec, w.X, (long)batch * compact_len(n), 12345u, ctx->st) < 0 ||
          run_fine(ctx, grid, prec, a, 1, true, false) < 0 || cudaEventRecord(ctx->ev[0], ctx->st) != cudaSuccess ||
          run_fine(ctx, grid, prec, a, nsteps, true, false) < 0 || cudaEventRecord(ctx->ev[1], ctx->st) != cudaSuccess ||
          cudaEventSynchronize(ctx->ev[1]) != cudaSuccess) {
        s = cuda_fail(ctx, cudaGetLastError(), "kd_autotune: timing run");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
      const double per = ms / nsteps;
      if (per < best) {
        best = per;
        best_plan = ctx->plan[grid];
      }
    }
  dfree(ctx, t0);
  if (s != KD_OK) {
    ctx->plan[grid] = saved;
    return s;
  }
  ctx->plan[grid] = best_plan;
  if (ms_per_step) *ms_per_step = best;
  if (cache_path) {
    TuneEntry e;
    e.device = dev;
    e.n = n;
    e.prec = prec;
    e.batch = key;
    e.col = best_plan.col;
    e.row = best_plan.row;
    e.ms = best;
    std::vector<TuneEntry> out;
    for (const TuneEntry& o : cache)
      if (!(o.device == dev && o.n == n && o.prec == prec && o.batch == key)) out.push_back(o);
    out.push_back(e);
    if (!write_cache(cache_path, out)) return fail(ctx, KD_EINVAL, std::string("kd_autotune: cannot write ") + cache_path);
  }
  return KD_OK;
}

}  // extern "C"
