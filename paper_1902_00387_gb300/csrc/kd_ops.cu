// Layout conversions, Fourier restriction / prolongation, the FP64 Parareal update
// (Sec. 3, Eq. 8), the convergence defect (Eq. 9), energies and the growth-rate fit.
// All reductions run in a fixed order so that results are bitwise reproducible.
#include <math.h>

#include "kd_fine.h"

namespace kd {

static inline unsigned nblk(long total, int threads) {
  long b = (total + threads - 1) / threads;
  return (unsigned)(b < 1 ? 1 : b);
}

template <typename T>
__device__ __forceinline__ cx<double> to_d(cx<T> v) {
  return mk((double)v.x, (double)v.y);
}
template <typename T>
__device__ __forceinline__ cx<T> from_d(cx<double> v) {
  return mk((T)v.x, (T)v.y);
}

// ------------------------------------------------------------------ layouts
template <typename Ti, typename To>
__global__ void k_full_to_compact(const cx<Ti>* full, cx<To>* comp, long total, int n, int K, int P) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long bc = i / ((long)P * P);
    const int r = (int)(i - bc * P * P);
    const int iy = r / P, ix = r - iy * P;
    // FFT order: wavenumber k < 0 sits at index k + n (any even n)
    const int y = iy >= K ? iy - K : iy - K + n, x = ix >= K ? ix - K : ix - K + n;
    comp[i] = from_d<To>(to_d(full[(bc * n + y) * n + x]));
  }
}

template <typename Ti, typename To>
__global__ void k_compact_to_full(const cx<Ti>* comp, cx<To>* full, long total, int n, int K, int P) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long bc = i / ((long)n * n);
    const int r = (int)(i - bc * n * n);
    const int y = r / n, x = r - y * n;
    const int ky = y < n / 2 ? y : y - n, kx = x < n / 2 ? x : x - n;
    cx<To> v = mk(To(0), To(0));
    if (ky >= -K && ky <= K && kx >= -K && kx <= K) v = from_d<To>(to_d(comp[(bc * P + ky + K) * P + kx + K]));
    full[i] = v;
  }
}

template <typename Ti, typename To>
__global__ void k_resample(const cx<Ti>* src, int Ks, int Ps, cx<To>* dst, int Kd, int Pd, long total) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long bc = i / ((long)Pd * Pd);
    const int r = (int)(i - bc * Pd * Pd);
    const int ky = r / Pd - Kd, kx = r % Pd - Kd;
    cx<To> v = mk(To(0), To(0));
    if (ky >= -Ks && ky <= Ks && kx >= -Ks && kx <= Ks) v = from_d<To>(to_d(src[(bc * Ps + ky + Ks) * Ps + kx + Ks]));
    dst[i] = v;
  }
}

static unsigned grid_for(long total) {
  unsigned g = nblk(total, 256);
  return g > 65535u * 8u ? 65535u * 8u : g;
}

template <typename Ti, typename To>
static int f2c(const void* full, void* comp, long batch, int n, cudaStream_t st) {
  const int K = n / 3, P = 2 * K + 1;
  const long total = batch * 3 * (long)P * P;
  k_full_to_compact<Ti, To><<<grid_for(total), 256, 0, st>>>((const cx<Ti>*)full, (cx<To>*)comp, total, n, K, P);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}
template <typename Ti, typename To>
static int c2f(const void* comp, void* full, long batch, int n, cudaStream_t st) {
  const int K = n / 3, P = 2 * K + 1;
  const long total = batch * 3 * (long)n * n;
  k_compact_to_full<Ti, To><<<grid_for(total), 256, 0, st>>>((const cx<Ti>*)comp, (cx<To>*)full, total, n, K, P);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}
template <typename Ti, typename To>
static int rs(const void* src, int ns, void* dst, int nd, long batch, cudaStream_t st) {
  const int Ks = ns / 3, Kd = nd / 3;
  const long total = batch * 3 * (long)(2 * Kd + 1) * (2 * Kd + 1);
  k_resample<Ti, To><<<grid_for(total), 256, 0, st>>>((const cx<Ti>*)src, Ks, 2 * Ks + 1, (cx<To>*)dst, Kd, 2 * Kd + 1, total);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int full_to_compact(int pin, const void* full, int pout, void* comp, long batch, int n, cudaStream_t st) {
  if (pin == 1 && pout == 1) return f2c<double, double>(full, comp, batch, n, st);
  if (pin == 1 && pout == 0) return f2c<double, float>(full, comp, batch, n, st);
  if (pin == 0 && pout == 1) return f2c<float, double>(full, comp, batch, n, st);
  return f2c<float, float>(full, comp, batch, n, st);
}
int compact_to_full(int pin, const void* comp, int pout, void* full, long batch, int n, cudaStream_t st) {
  if (pin == 1 && pout == 1) return c2f<double, double>(comp, full, batch, n, st);
  if (pin == 1 && pout == 0) return c2f<double, float>(comp, full, batch, n, st);
  if (pin == 0 && pout == 1) return c2f<float, double>(comp, full, batch, n, st);
  return c2f<float, float>(comp, full, batch, n, st);
}
// Zeros of the full layout outside the kept square: whole rows |ky| > K, and the columns
// |kx| > K of the other rows (a row of the full layout in 16-byte pieces where aligned).
template <typename T>
__global__ void k_zero_unkept(cx<T>* full, long rows, int n, int K) {
  const int w = n - (2 * K + 1);            // unkept columns K + 1 .. n - K - 1 of a kept row
  for (long r = blockIdx.x; r < rows; r += gridDim.x) {
    const int y = (int)(r % n);
    const bool kept = y <= K || y >= n - K;
    cx<T>* row = full + r * (long)n;
    const int c0 = kept ? K + 1 : 0, cnt = kept ? w : n;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) row[c0 + i] = mk(T(0), T(0));
  }
}

int zero_outside_kept(int prec, void* full, long batch, int n, cudaStream_t st) {
  const long rows = batch * 3L * n;
  const unsigned g = rows < 65535L * 8 ? (unsigned)rows : 65535u * 8;
  if (prec == 1)
    k_zero_unkept<double><<<g, 256, 0, st>>>((cx<double>*)full, rows, n, n / 3);
  else
    k_zero_unkept<float><<<g, 256, 0, st>>>((cx<float>*)full, rows, n, n / 3);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int compact_resample(int pin, const void* src, int ns, int pout, void* dst, int nd, long batch, cudaStream_t st) {
  if (pin == 1 && pout == 1) return rs<double, double>(src, ns, dst, nd, batch, st);
  if (pin == 1 && pout == 0) return rs<double, float>(src, ns, dst, nd, batch, st);
  if (pin == 0 && pout == 1) return rs<float, double>(src, ns, dst, nd, batch, st);
  return rs<float, float>(src, ns, dst, nd, batch, st);
}

// ------------------------------------------------- increment form of the fine step
// F is linear in b, so F(U^k) = F(U^{k-1}) + F(U^k - U^{k-1}).  The fine sweep then
// rounds only the increment to the fine precision and accumulates in FP64.
template <typename To>
__global__ void k_delta_in(const cx<double>* U, cx<double>* Uprev, cx<To>* X, long total, int first) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const cx<double> u = U[i];
    const cx<double> d = first ? u : u - Uprev[i];
    X[i] = from_d<To>(d);
    Uprev[i] = u;
  }
}

template <typename Ti>
__global__ void k_accum_out(const cx<Ti>* X, cx<double>* Fv, long total, int first) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const cx<double> x = to_d(X[i]);
    Fv[i] = first ? x : Fv[i] + x;
  }
}

int delta_in(int pout, const double* U, double* Uprev, void* X, long total, int first, cudaStream_t st) {
  if (pout == 0)
    k_delta_in<float><<<grid_for(total), 256, 0, st>>>((const cx<double>*)U, (cx<double>*)Uprev, (cx<float>*)X, total, first);
  else
    k_delta_in<double><<<grid_for(total), 256, 0, st>>>((const cx<double>*)U, (cx<double>*)Uprev, (cx<double>*)X, total, first);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int accum_out(int pin, const void* X, double* Fv, long total, int first, cudaStream_t st) {
  if (pin == 0)
    k_accum_out<float><<<grid_for(total), 256, 0, st>>>((const cx<float>*)X, (cx<double>*)Fv, total, first);
  else
    k_accum_out<double><<<grid_for(total), 256, 0, st>>>((const cx<double>*)X, (cx<double>*)Fv, total, first);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

__global__ void k_diff(const double* U, const double* Uprev, double* d, long total) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < 2 * total; i += (long)gridDim.x * blockDim.x)
    d[i] = U[i] - Uprev[i];
}

int diff_kernel(const double* U, const double* Uprev, double* d, long total, cudaStream_t st) {
  k_diff<<<grid_for(2 * total), 256, 0, st>>>(U, Uprev, d, total);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

// ------------------------------------------------------------ parareal update
constexpr int UPD_THREADS = 256;

template <typename Tg>
__global__ void __launch_bounds__(UPD_THREADS)
k_update(const cx<double>* F, const cx<Tg>* g, cx<double>* Gold, cx<double>* U, int Kf, int Pf, int Kc, int Pc,
         long total, int init, double* partials) {
  __shared__ double s_d[UPD_THREADS], s_n[UPD_THREADS];
  double acc_d = 0.0, acc_n = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i / ((long)Pf * Pf));
    const int r = (int)(i - (long)c * Pf * Pf);
    const int ky = r / Pf - Kf, kx = r % Pf - Kf;
    cx<double> gv = mk(0.0, 0.0), go = mk(0.0, 0.0);
    long ic = -1;
    if (ky >= -Kc && ky < Pc - Kc && kx >= -Kc && kx < Pc - Kc) {
      ic = ((long)c * Pc + ky + Kc) * Pc + kx + Kc;
      gv = to_d(g[ic]);
      go = Gold[ic];
    }
    cx<double> u;
    if (init == 1) {
      u = gv;                       // initial coarse sweep
    } else if (init == 2) {
      u = F[i] + gv;                // increment form: F(U^k) + G(U^{k+1} - U^k)
    } else {
      u = F[i] + (gv - go);         // F(U^k) + (G(U^{k+1}) - G(U^k))
    }
    if (ic >= 0 && init != 2) Gold[ic] = gv;
    if (partials) {
      const cx<double> old = U[i];
      const cx<double> d = u - old;
      acc_d += d.x * d.x + d.y * d.y;
      acc_n += u.x * u.x + u.y * u.y;
    }
    U[i] = u;
  }
  if (partials) {
    s_d[threadIdx.x] = acc_d;
    s_n[threadIdx.x] = acc_n;
    __syncthreads();
    for (int s = UPD_THREADS / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        s_d[threadIdx.x] += s_d[threadIdx.x + s];
        s_n[threadIdx.x] += s_n[threadIdx.x + s];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      partials[2 * blockIdx.x] = s_d[0];
      partials[2 * blockIdx.x + 1] = s_n[0];
    }
  }
}

int parareal_update(const double* F, const void* g, int pg, double* Gold, double* U_next, int n, int Kc, int Pc,
                    int init, double* partials, cudaStream_t st) {
  const int Kf = n / 3, Pf = 2 * Kf + 1;
  const long total = 3L * Pf * Pf;
  unsigned grid = nblk(total, UPD_THREADS);
  if (grid > 1024) grid = 1024;
  if (pg == 1)
    k_update<double><<<grid, UPD_THREADS, 0, st>>>((const cx<double>*)F, (const cx<double>*)g, (cx<double>*)Gold,
                                                   (cx<double>*)U_next, Kf, Pf, Kc, Pc, total, init, partials);
  else
    k_update<float><<<grid, UPD_THREADS, 0, st>>>((const cx<double>*)F, (const cx<float>*)g, (cx<double>*)Gold,
                                                  (cx<double>*)U_next, Kf, Pf, Kc, Pc, total, init, partials);
  cudaError_t e = cudaGetLastError();
  return e != cudaSuccess ? -(int)e : (int)grid;
}

__global__ void k_finish_sigma(const double* partials, int nb, double* out) {
  __shared__ double s_d[256], s_n[256];
  double d = 0.0, nn = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    d += partials[2 * i];
    nn += partials[2 * i + 1];
  }
  s_d[threadIdx.x] = d;
  s_n[threadIdx.x] = nn;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      s_d[threadIdx.x] += s_d[threadIdx.x + s];
      s_n[threadIdx.x] += s_n[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sqrt(s_d[0]) / sqrt(s_n[0]);
    out[1] = s_d[0];
    out[2] = s_n[0];
  }
}

// per block: partial sums of |a - r|^2 and |r|^2 (fixed order), for finish_sigma
__global__ void k_rel_error(const cx<double>* a, const cx<double>* r, long len, double* partials) {
  __shared__ double s_d[256], s_n[256];
  double d = 0.0, nn = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < len; i += (long)gridDim.x * blockDim.x) {
    const cx<double> x = a[i], y = r[i];
    const double dx = x.x - y.x, dy = x.y - y.y;
    d += dx * dx + dy * dy;
    nn += y.x * y.x + y.y * y.y;
  }
  s_d[threadIdx.x] = d;
  s_n[threadIdx.x] = nn;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      s_d[threadIdx.x] += s_d[threadIdx.x + s];
      s_n[threadIdx.x] += s_n[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = s_d[0];
    partials[2 * blockIdx.x + 1] = s_n[0];
  }
}

int rel_error_partials(const double* a, const double* ref, long len, double* partials, cudaStream_t st) {
  long nb = (len + 255) / 256;
  if (nb > 256) nb = 256;
  if (nb < 1) nb = 1;
  k_rel_error<<<(unsigned)nb, 256, 0, st>>>((const cx<double>*)a, (const cx<double>*)ref, len, partials);
  return cudaPeekAtLastError() == cudaSuccess ? (int)nb : -1;
}

int finish_sigma(const double* partials, int nblocks, double* out, cudaStream_t st) {
  k_finish_sigma<<<1, 256, 0, st>>>(partials, nblocks, out);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

// ---------------------------------------------------------------- energies
__global__ void k_energy(const cx<double>* f, long len, double* E) {
  __shared__ double s[256];
  const cx<double>* p = f + (long)blockIdx.x * len;
  double acc = 0.0;
  for (long i = threadIdx.x; i < len; i += blockDim.x) acc += p[i].x * p[i].x + p[i].y * p[i].y;
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) E[blockIdx.x] = s[0];
}

int energy_kernel(const double* fields, long len, int count, double* E, cudaStream_t st) {
  if (count <= 0) return 0;
  k_energy<<<count, 256, 0, st>>>((const cx<double>*)fields, len, E);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

__global__ void k_growth_fit(const double* E, int count, double dt, double fit_from, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double st = 0.0, sy = 0.0;
  int m = 0, ok = 1;
  for (int i = 0; i < count; ++i) {
    const double t = i * dt;
    if (t < fit_from - 1e-12) continue;
    const double e = E[i];
    if (!(e > 0.0) || !isfinite(e)) ok = 0;
    st += t;
    sy += 0.5 * log(e);
    ++m;
  }
  const double tm = st / m, ym = sy / m;
  double num = 0.0, den = 0.0;
  for (int i = 0; i < count; ++i) {
    const double t = i * dt;
    if (t < fit_from - 1e-12) continue;
    const double y = 0.5 * log(E[i]);
    num += (t - tm) * (y - ym);
    den += (t - tm) * (t - tm);
  }
  out[0] = num / den;
  out[1] = (ok && m >= 2 && isfinite(out[0])) ? 1.0 : 0.0;
}

int growth_fit(const double* E, int count, double dt, double fit_from, double* out, cudaStream_t st) {
  k_growth_fit<<<1, 32, 0, st>>>(E, count, dt, fit_from, out);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

__global__ void k_fill_times(double* dst, int count, double t0, double dT) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) dst[i] = t0 + i * dT;
}

__global__ void k_fill_slice_times(double* dst, int count, int first, double dT) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) dst[i] = (double)(first + i) * dT;
}

int fill_slice_times(double* dst, int count, int first, double dT, cudaStream_t st) {
  k_fill_slice_times<<<nblk(count, 256), 256, 0, st>>>(dst, count, first, dT);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int fill_times(double* dst, int count, double t0, double dT, cudaStream_t st) {
  if (count <= 0) return 0;
  k_fill_times<<<nblk(count, 256), 256, 0, st>>>(dst, count, t0, dT);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace kd
