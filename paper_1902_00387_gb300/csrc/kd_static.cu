// kd_fine_batched_static: the fine propagator of kd_fine_batched for callers that
// cannot allocate device memory.  Its workspace (grid tables, compact state, stage
// accumulators, mixed fields, flow phases) lives in one file-scope __device__ array of
// KD_STATIC_SCRATCH_BYTES; the call performs no cudaMalloc / cudaFree and no other
// allocating call, and creates no context object.
//
// Host code cannot use the array's name as a device address, so every call looks the
// address up with cudaGetSymbolAddress (with the caller's device current; a host-side
// lookup, no allocation).  The kernels' shared-memory opt-in is set on the first call on
// a device and again whenever that address changes, i.e. after cudaDeviceReset gave the
// device a new context, so that nothing cached from an earlier context is used.
#include <math.h>
#include <mutex>
#include <stdio.h>

#include "../../include/kd.h"
#include "kd_fine.h"

namespace {

__device__ __align__(256) unsigned char g_static_scratch[KD_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};   // address the kernels were set up for
bool g_prepared[kMaxDevices][2] = {{false}};

// Grid tables into the scratch: tw[e] = exp(-2 pi i e / n), cos / sin of 2 pi e / n,
// computed in double and rounded to T (multiples of pi / 2 exact).
template <typename T>
__global__ void k_static_tables(int n, T* tw, T* cg, T* sg) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  double c, s;
  if (e % (n / 4) == 0) {
    const int q = (e / (n / 4)) & 3;
    c = q == 0 ? 1.0 : q == 2 ? -1.0 : 0.0;
    s = q == 1 ? 1.0 : q == 3 ? -1.0 : 0.0;
  } else {
    const double a = 2.0 * 3.14159265358979323846 * (double)e / (double)n;
    c = cos(a);
    s = sin(a);
  }
  tw[2 * e] = (T)c;
  tw[2 * e + 1] = (T)(-s);
  cg[e] = (T)c;
  sg[e] = (T)s;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" kd_status kd_fine_batched_static(const kd_params* p, const void* b_in, void* b_out, const double* t0,
                                            int nsteps, int batch, void* cuda_stream) {
  using namespace kd;
  if (!p || !b_in || !b_out || !t0 || nsteps < 0 || batch < 0) {
    fprintf(stderr, "kd_fine_batched_static: NULL buffer or negative size\n");
    return KD_EINVAL;
  }
  const int n = p->n, prec = p->prec_fine;
  if (n < 16 || n > 1024 || (n & 1) || fine_fft_grid(n) == 0 || p->flow < 0 || p->flow > 2 ||
      (prec != KD_C64 && prec != KD_C128) || !(p->Rm > 0) ||
      !(p->dt_fine > 0) || !isfinite(p->kz) || p->fine_scheme < KD_RK443 || p->fine_scheme > KD_RK111) {
    fprintf(stderr, "kd_fine_batched_static: invalid parameters\n");
    return KD_EINVAL;
  }
  if (batch == 0) return KD_OK;
  // workspace carve-out (all offsets 256-byte aligned)
  const size_t rs = prec == KD_C64 ? 4 : 8, cs = 2 * rs;
  const int K = n / 3, P = 2 * K + 1;
  const int m = fine_fft_grid(n);   // the transforms' side (n itself for the FFT sides)
  // the per-field terms are bounded one by one first, so that their sum below cannot wrap
  // around for any int batch and nsteps
  const size_t lim = (size_t)KD_STATIC_SCRATCH_BYTES;
  const bool gp = p->flow == KD_FLOW_GALLOWAY_PROCTOR;
  if ((size_t)batch > lim / (3 * (size_t)P * P * cs) ||
      (gp && nsteps > 0 && (size_t)batch > lim / ((size_t)nsteps * 16 * rs))) {
    fprintf(stderr,
            "kd_fine_batched_static: %d fields of %d steps need more than the %d bytes of the static scratch; "
            "use a smaller batch or nsteps, or kd_fine_batched\n",
            batch, nsteps, KD_STATIC_SCRATCH_BYTES);
    return KD_EINVAL;
  }
  const size_t tab = align256(m * cs) + 2 * align256(m * rs);
  const size_t spec = align256((size_t)batch * 3 * P * P * cs);
  const size_t mixed = align256((size_t)batch * 3 * P * m * cs);
  const size_t phase = gp ? align256(phase_table_bytes(prec, batch, nsteps)) : 0;
  const int nspec = prec == KD_C64 ? 5 : 4;   // X, R2, R3, R4 (+ the state's low part, complex64)
  const size_t need = tab + nspec * spec + 2 * mixed + phase;
  if (need > (size_t)KD_STATIC_SCRATCH_BYTES) {
    fprintf(stderr,
            "kd_fine_batched_static: this request needs %zu bytes of workspace, more than the %d bytes of the "
            "static scratch; use a smaller batch or nsteps, or kd_fine_batched\n",
            need, KD_STATIC_SCRATCH_BYTES);
    return KD_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return KD_ECUDA;
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess || !ptr) {
      fprintf(stderr, "kd_fine_batched_static: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
      return KD_ECUDA;
    }
    if (ptr != g_scratch_addr[dev]) {   // first call on this device, or a new context
      g_scratch_addr[dev] = ptr;
      g_prepared[dev][0] = g_prepared[dev][1] = false;
    }
    if (!g_prepared[dev][prec]) {
      cudaError_t e = fine_prepare(prec);
      if (e != cudaSuccess) {
        fprintf(stderr, "kd_fine_batched_static: kernel set-up failed: %s\n", cudaGetErrorString(e));
        return KD_ECUDA;
      }
      g_prepared[dev][prec] = true;
    }
    base = (unsigned char*)g_scratch_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  unsigned char* q = base;
  void* tw = q;
  q += align256(m * cs);
  void* cg = q;
  q += align256(m * rs);
  void* sg = q;
  q += align256(m * rs);
  FineArgs a;
  a.n = m;
  a.K = K;
  a.P = P;
  a.batch = batch;
  a.flow = p->flow;
  a.amp = p->flow == KD_FLOW_ROBERTS ? 1.0 : p->flow == KD_FLOW_GALLOWAY_PROCTOR ? sqrt(1.5) : 0.0;
  a.kz = p->kz;
  a.Rm = p->Rm;
  a.dt = p->dt_fine;
  a.t0 = t0;
  a.X = q;
  a.R2 = q + spec;
  a.R3 = q + 2 * spec;
  a.R4 = q + 3 * spec;
  a.Xlo = prec == KD_C64 ? q + 4 * spec : nullptr;
  a.lo_valid = 0;
  q += nspec * spec;
  a.M = q;
  a.W = q + mixed;
  q += 2 * mixed;
  a.phases = phase ? q : nullptr;
  a.phase_steps = nsteps;
  a.sp = nullptr;
  a.scheme = p->fine_scheme;
  a.tw = tw;
  a.cosg = cg;
  a.sing = sg;
  // Every scratch region is written before it is read in this call (tables, packed
  // state, prologue mixed field, column output, stage-0 accumulators, phases, and the
  // state's low part, written by the first step's last stage and read from the second
  // step on), so no region has to be cleared.
  const unsigned tb = (unsigned)((m + 255) / 256);
  if (prec == KD_C64)
    k_static_tables<float><<<tb, 256, 0, st>>>(m, (float*)tw, (float*)cg, (float*)sg);
  else
    k_static_tables<double><<<tb, 256, 0, st>>>(m, (double*)tw, (double*)cg, (double*)sg);
  if (cudaGetLastError() != cudaSuccess) return KD_ECUDA;
  if (full_to_compact(prec, b_in, prec, a.X, batch, n, st) < 0) return KD_ECUDA;
  if (nsteps > 0 && fine_launch_steps(prec, a, nsteps, true, false, st) < 0) return KD_ECUDA;
  if (compact_to_full(prec, a.X, prec, b_out, batch, n, st) < 0) return KD_ECUDA;
  return cudaGetLastError() == cudaSuccess ? KD_OK : KD_ECUDA;
}
