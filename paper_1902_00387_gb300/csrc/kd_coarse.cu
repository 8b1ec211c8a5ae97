// Classical coarse propagator G (Sec. 3.2, Sec. 5.2: the same equations on the coarse
// N_C grid with the coarse step) as one persistent thread-block cluster per field for
// coarse sets of side <= 88 (coarse grids up to 128) with portable clusters, and up to
// 127 (grids up to 190) with 16-block clusters,
// fused with the Fourier restriction of the fine input and, in the Parareal sweep,
// with the FP64 update U_{n+1} = F + (G_new - G_old) and the defect of Eq. 9.
//
// The explicit term is evaluated as the exact spectral convolution
//     w_hat(k) = sum_q u_hat(q, t) x b_hat(k - q),   q in {(+-1, 0), (0, +-1)},
// followed by the curl i k3 x w_hat on the dealiased set.  The flow has only those
// four Fourier modes and n/3 + 1 < n/2, so the pseudo-spectral product of the fine
// kernels has no aliasing and this is the same discrete operator (equal to round-off).
//
// Layout: the stage values live in shared memory with a one-mode ring of zeros around
// the kept square; the IMEX RK443 state X0 and accumulators R2..R4 of each mode live in
// the registers of the thread that owns the mode.
#include <cooperative_groups.h>

#include "kd_coarse.h"
#include "kd_stage.cuh"

namespace cgrp = cooperative_groups;

namespace kd {

template <typename T>
struct UHat {
  cx<T> py[2], pz[2];   // q = (+1, 0), (-1, 0): u_hat = (0, py, pz)
  cx<T> qx[2], qz[2];   // q = (0, +1), (0, -1): u_hat = (qx, 0, qz)
};

// u_hat of u = A (cos(y + py), sin(x + px), cos(x + px) + sin(y + py)) with
// ex = exp(i px), ey = exp(i py):  sin a = (e^{ia} - e^{-ia}) / 2i, cos a = (e^{ia} + e^{-ia}) / 2.
template <typename T>
__device__ __forceinline__ UHat<T> uhat(T A, const Phase<T>& p) {
  const T h = T(0.5) * A;
  const cx<T> ex = mk(p.cpx, p.spx), ey = mk(p.cpy, p.spy);
  UHat<T> u;
  // x-modes: u_y = A sin(x + px) -> (+1): A ex / 2i = -i h ex, (-1): -A conj(ex) / 2i = i h conj(ex)
  u.py[0] = mk(h * ex.y, -h * ex.x);
  u.py[1] = mk(h * ex.y, h * ex.x);
  u.pz[0] = mk(h * ex.x, h * ex.y);       // u_z: A cos(x + px) -> h ex, h conj(ex)
  u.pz[1] = mk(h * ex.x, -h * ex.y);
  // y-modes: u_x = A cos(y + py) -> h ey, h conj(ey); u_z: A sin(y + py) -> -i h ey, i h conj(ey)
  u.qx[0] = mk(h * ey.x, h * ey.y);
  u.qx[1] = mk(h * ey.x, -h * ey.y);
  u.qz[0] = mk(h * ey.y, -h * ey.x);
  u.qz[1] = mk(h * ey.y, h * ey.x);
  return u;
}

// ---------------------------------------------------------------------------
// Cluster version: the coarse square is split into row stripes over the CS blocks of
// a thread-block cluster.  Each block keeps its stripe plus one halo row above and
// below, double-buffered: a stage reads buffer `cur`, writes its new rows into `nxt`
// locally and its first / last row into the neighbours' halo rows of `nxt` through
// distributed shared memory, then one cluster barrier makes `nxt` current.
constexpr int CCB = 256;   // threads per block of the cluster kernel (MPT = 2, 4)
constexpr int CCB1 = 512;  // threads per block with one mode per thread

template <typename T, int MPT, int NT = CCB>
__global__ void __launch_bounds__(NT) coarse_cluster_kernel(CoarseArgs a, int CS, int H) {
  cgrp::cluster_group cluster = cgrp::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int K = a.Kc, P = a.Pc, L = P + 2, LH = H + 2;
  const int Kf = a.Kf, Pf = a.Pf;
  const int rank = (int)cluster.block_rank();
  const int b = blockIdx.x / CS;                  // field of this cluster
  const int y0 = rank * H;                        // first global row of the stripe
  const int hr = max(0, min(H, P - y0));          // rows owned
  cx<T>* buf = (cx<T>*)smem_raw;                  // [2][3][LH][L]
  T* s_ph = (T*)(buf + 2 * 3 * LH * L);           // [nsteps][4][4] when staged
  const int bufsz = 3 * LH * L;
  const long lenf2 = 2L * 3 * Pf * Pf;            // doubles per fine compact field
  const long slot = a.map ? (long)a.map[b] : (long)b;
  const double* Un = a.Un + slot * lenf2;
  const double* Uprev = a.Uprev ? a.Uprev + (a.map ? slot * lenf2 : 0) : nullptr;
  const double* Fv = a.Fv ? a.Fv + (a.map ? slot * lenf2 : 0) : nullptr;
  double* Unext = a.Unext ? a.Unext + (a.map ? (slot + 1) * lenf2 : 0) : nullptr;
  double* sig = a.sigma_out ? a.sigma_out + (a.map ? 3L * b : 0) : nullptr;
  const int nsteps = a.steps ? a.steps[b] : a.nsteps;
  for (int i = threadIdx.x; i < 2 * bufsz; i += NT) buf[i] = mk(T(0), T(0));
  const bool stage_ph = a.phases && a.nsteps * 16 <= a.phase_smem;
  const T* ph_g = a.phases ? (const T*)a.phases + (long)b * a.nsteps * 16 : nullptr;
  if (stage_ph)
    for (int i = threadIdx.x; i < a.nsteps * 16; i += NT) s_ph[i] = ph_g[i];
  __syncthreads();

  const int M = hr * P;
  cx<T> x0[MPT][3], r2[MPT][3], r3[MPT][3], r4[MPT][3];
  T lam_dt[MPT], inv_d[MPT], fkx[MPT], fky[MPT];
  const T kz = a.sp ? (T)a.sp[b].kz : (T)a.kz, dt = a.sp ? (T)a.sp[b].dt : (T)a.dt;
  const T inv_rm = T(1) / (a.sp ? (T)a.sp[b].Rm : (T)a.Rm);
#pragma unroll
  for (int i = 0; i < MPT; ++i) {
    const int m = threadIdx.x + NT * i;
    const int ly = m < M ? m / P : 0, ix = m < M ? m % P : 0;
    const int iy = y0 + ly;
    fkx[i] = (T)(ix - K);
    fky[i] = (T)(iy - K);
    const T lam = (fkx[i] * fkx[i] + fky[i] * fky[i] + kz * kz) * inv_rm;
    lam_dt[i] = dt * lam;
    inv_d[i] = T(1) / (T(1) + dt * T(0.5) * lam);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      cx<T> v = mk(T(0), T(0));
      if (m < M) {
        const long src = ((long)c * Pf + (iy + Kf - K)) * Pf + (ix + Kf - K);
        if (Uprev)
          v = mk((T)(Un[2 * src] - Uprev[2 * src]), (T)(Un[2 * src + 1] - Uprev[2 * src + 1]));
        else
          v = mk((T)Un[2 * src], (T)Un[2 * src + 1]);
      }
      x0[i][c] = v;
    }
  }
  // initial stage value into buffer 0: own rows and the neighbours' halos
  auto put = [&](int bsel, int ly, int ix, int c, cx<T> v) {
    buf[bsel * bufsz + (c * LH + ly + 1) * L + ix + 1] = v;
    if (ly == 0 && rank > 0) {
      cx<T>* peer = cluster.map_shared_rank(buf, rank - 1);
      peer[bsel * bufsz + (c * LH + H + 1) * L + ix + 1] = v;
    }
    if (ly == hr - 1 && rank < CS - 1 && y0 + hr < P) {
      cx<T>* peer = cluster.map_shared_rank(buf, rank + 1);
      peer[bsel * bufsz + (c * LH + 0) * L + ix + 1] = v;
    }
  };
  cluster.sync();   // every block has zeroed its buffers before peers write halos
#pragma unroll
  for (int i = 0; i < MPT; ++i) {
    const int m = threadIdx.x + NT * i;
    if (m < M)
#pragma unroll
      for (int c = 0; c < 3; ++c) put(0, m / P, m % P, c, x0[i][c]);
  }
  cluster.sync();

  const T A = a.sp ? (T)a.sp[b].amp : (T)a.amp;
  int cur = 0;
  for (int s = 0; s < nsteps; ++s) {
#pragma unroll 1
    for (int j = 0; j < 4; ++j) {
      Phase<T> ph;
      if (ph_g) {
        const T* p = stage_ph ? s_ph + (s * 4 + j) * 4 : ph_g + (s * 4 + j) * 4;
        ph.cpx = p[0];
        ph.spx = p[1];
        ph.cpy = p[2];
        ph.spy = p[3];
      } else {
        ph.cpx = T(1);
        ph.spx = T(0);
        ph.cpy = T(1);
        ph.spy = T(0);
      }
      const UHat<T> u = uhat<T>(A, ph);
      const cx<T>* Xs = buf + cur * bufsz;
#pragma unroll
      for (int i = 0; i < MPT; ++i) {
        const int m = threadIdx.x + NT * i;
        if (m >= M) continue;
        const int ly = m / P + 1, ix = m % P + 1;
        cx<T> w[3] = {mk(T(0), T(0)), mk(T(0), T(0)), mk(T(0), T(0))};
#pragma unroll
        for (int sgn = 0; sgn < 2; ++sgn) {
          const int sx = ix - (sgn == 0 ? 1 : -1);
          const cx<T> bx = Xs[(0 * LH + ly) * L + sx], by = Xs[(1 * LH + ly) * L + sx], bz = Xs[(2 * LH + ly) * L + sx];
          const cx<T> uy = u.py[sgn], uz = u.pz[sgn];
          w[0] = w[0] + cmul(uy, bz) - cmul(uz, by);
          w[1] = w[1] + cmul(uz, bx);
          w[2] = w[2] - cmul(uy, bx);
          const int sy = ly - (sgn == 0 ? 1 : -1);
          const cx<T> cxv = Xs[(0 * LH + sy) * L + ix], cyv = Xs[(1 * LH + sy) * L + ix], czv = Xs[(2 * LH + sy) * L + ix];
          const cx<T> ux = u.qx[sgn], uz2 = u.qz[sgn];
          w[0] = w[0] - cmul(uz2, cyv);
          w[1] = w[1] + cmul(uz2, cxv) - cmul(ux, czv);
          w[2] = w[2] + cmul(ux, cyv);
        }
        cx<T> F[3];
        F[0] = mul_i(w[2] * fky[i] - w[1] * kz);
        F[1] = mul_i(w[0] * kz - w[2] * fkx[i]);
        F[2] = mul_i(w[1] * fkx[i] - w[0] * fky[i]);
        const T dl = lam_dt[i], id = inv_d[i];
        cx<T> xn[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const cx<T> f = F[c];
          if (j == 0) {
            const cx<T> x1 = (x0[i][c] + f * (dt * T(0.5))) * id;
            r2[i][c] = x0[i][c] + f * (dt * T(11.0 / 18.0)) - x1 * (dl * T(1.0 / 6.0));
            r3[i][c] = x0[i][c] + f * (dt * T(5.0 / 6.0)) + x1 * (dl * T(0.5));
            r4[i][c] = x0[i][c] + f * (dt * T(0.25)) - x1 * (dl * T(1.5));
            xn[c] = x1;
          } else if (j == 1) {
            const cx<T> x2 = (r2[i][c] + f * (dt * T(1.0 / 18.0))) * id;
            r3[i][c] = r3[i][c] - f * (dt * T(5.0 / 6.0)) - x2 * (dl * T(0.5));
            r4[i][c] = r4[i][c] + f * (dt * T(1.75)) + x2 * (dl * T(1.5));
            xn[c] = x2;
          } else if (j == 2) {
            const cx<T> x3 = (r3[i][c] + f * (dt * T(0.5))) * id;
            r4[i][c] = r4[i][c] + f * (dt * T(0.75)) - x3 * (dl * T(0.5));
            xn[c] = x3;
          } else {
            const cx<T> x4 = (r4[i][c] - f * (dt * T(1.75))) * id;
            x0[i][c] = x4;
            xn[c] = x4;
          }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) put(cur ^ 1, ly - 1, ix - 1, c, xn[c]);
      }
      cluster.sync();   // new stage values (own rows and halos) are complete everywhere
      cur ^= 1;
    }
  }

  // outputs from the final stage value (buffer `cur`), by stripe
  const cx<T>* Xf = buf + cur * bufsz;
  if (a.mode == COARSE_OUT) {
    double* g = a.g64 + (long)b * 2 * 3 * P * P;
    for (int i = threadIdx.x; i < 3 * M; i += NT) {
      const int c = i / M, r = i - c * M;
      const int ly = r / P, ix = r % P;
      const cx<T> v = Xf[(c * LH + ly + 1) * L + ix + 1];
      const long o = ((long)c * P + y0 + ly) * P + ix;
      g[2 * o] = (double)v.x;
      g[2 * o + 1] = (double)v.y;
    }
    cluster.sync();
    return;
  }
  // fused Parareal update over the fine rows ky in this block's share of [-Kf, Kf]
  __shared__ double red_d[NT / 32], red_n[NT / 32];
  __shared__ double cl_d[16], cl_n[16];
  const int fr0 = (Pf * rank) / CS, fr1 = (Pf * (rank + 1)) / CS;   // fine rows of this block
  const int Mf = (fr1 - fr0) * Pf;
  double acc_d = 0.0, acc_n = 0.0;
  for (int i = threadIdx.x; i < 3 * Mf; i += NT) {
    const int c = i / Mf, r = i - c * Mf;
    const int fy = fr0 + r / Pf, fx = r % Pf;
    const int ky = fy - Kf, kx = fx - Kf;
    const long fi = ((long)c * Pf + fy) * Pf + fx;
    double gx = 0.0, gy = 0.0, ox = 0.0, oy = 0.0;
    long ic = -1;
    if (ky >= -K && ky < P - K && kx >= -K && kx < P - K) {
      ic = ((long)c * P + ky + K) * P + kx + K;
      // the coarse value of row ky + K lives in the block owning that row
      const int iy = ky + K, owner = iy / H;
      const cx<T>* src = owner == rank ? Xf : cluster.map_shared_rank(Xf, owner);
      const cx<T> v = src[(c * LH + iy - owner * H + 1) * L + kx + K + 1];
      gx = (double)v.x;
      gy = (double)v.y;
      if (a.mode == COARSE_UPDATE) {
        ox = a.Gold[2 * ic];
        oy = a.Gold[2 * ic + 1];
      }
    }
    double ux, uy;
    if (a.mode == COARSE_INIT) {
      ux = gx;
      uy = gy;
    } else {
      ux = Fv[2 * fi] + (gx - ox);
      uy = Fv[2 * fi + 1] + (gy - oy);
    }
    if (ic >= 0 && a.mode != COARSE_INCR && a.Gold) {
      a.Gold[2 * ic] = gx;
      a.Gold[2 * ic + 1] = gy;
    }
    if (sig) {
      const double dx = ux - Unext[2 * fi], dy = uy - Unext[2 * fi + 1];
      acc_d += dx * dx + dy * dy;
      acc_n += ux * ux + uy * uy;
    }
    Unext[2 * fi] = ux;
    Unext[2 * fi + 1] = uy;
  }
  if (sig) {
    for (int o = 16; o > 0; o >>= 1) {
      acc_d += __shfl_down_sync(0xffffffffu, acc_d, o);
      acc_n += __shfl_down_sync(0xffffffffu, acc_n, o);
    }
    if ((threadIdx.x & 31) == 0) {
      red_d[threadIdx.x >> 5] = acc_d;
      red_n[threadIdx.x >> 5] = acc_n;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double d = 0.0, n = 0.0;
      for (int w = 0; w < NT / 32; ++w) {
        d += red_d[w];
        n += red_n[w];
      }
      double* pd = cluster.map_shared_rank(cl_d, 0);
      double* pn = cluster.map_shared_rank(cl_n, 0);
      pd[rank] = d;
      pn[rank] = n;
    }
  }
  cluster.sync();   // partial sums delivered; peers' buffers no longer read
  if (sig && rank == 0 && threadIdx.x == 0) {
    double d = 0.0, n = 0.0;
    for (int r = 0; r < CS; ++r) {
      d += cl_d[r];
      n += cl_n[r];
    }
    sig[0] = sqrt(d) / sqrt(n);
    sig[1] = d;
    sig[2] = n;
  }
}

// cluster split of a P-row coarse square: CS blocks of H rows (H <= 8 for P <= 64,
// H <= 11 for P <= 88; 16 blocks of H <= 8 rows for P <= 127)
// clusters of more than 8 blocks need the non-portable size opt-in (granted in prepare)
static int g_max_cluster = 8;

static void cluster_shape(int P, int* CS, int* H, int req = 0) {
  int cs = req > 0 ? req : (P + 5) / 6;
  if (cs > g_max_cluster) cs = g_max_cluster;
  if (req == 0 && cs > 8) cs = 8;
  if (cs < 1) cs = 1;
  *H = (P + cs - 1) / cs;
  *CS = cs;
}

constexpr int kMaxPhaseSlots = 8192;   // staged flow phases (512 steps x 4 stages x 4)

static size_t cluster_smem(int prec, int P, int nsteps, int* phase_slots, int req = 0) {
  const int L = P + 2;
  int CS, H;
  cluster_shape(P, &CS, &H, req);
  const size_t es = prec == 0 ? 4 : 8;
  const size_t base = (size_t)2 * 3 * (H + 2) * L * 2 * es;
  const int slots = nsteps * 16 <= kMaxPhaseSlots ? nsteps * 16 : 0;
  *phase_slots = slots;
  return base + (size_t)slots * es;
}

// modes per thread needed for a P-row square (0: unsupported)
// modes per thread of a block (1: CCB1 threads; 2, 4: CCB threads); 0 if the rows of a
// block do not fit
static int modes_per_thread(int P, int req = 0) {
  int CS, H;
  cluster_shape(P, &CS, &H, req);
  if (H * P <= CCB) return 2;
  if (H * P <= CCB1) return 1;
  if (H * P <= 2 * CCB) return 2;
  if (H * P <= 4 * CCB) return 4;
  return 0;
}

bool coarse_cluster_fits(int P, int cs) {
  return P >= 1 && cs >= 0 && cs <= g_max_cluster && (cs == 0 || cs <= P) && modes_per_thread(P, cs) > 0;
}

// smallest cluster larger than the default that holds a P-row square (0: none)
static int min_fitting_cluster(int P) {
  for (int cs = 9; cs <= g_max_cluster; ++cs)
    if (coarse_cluster_fits(P, cs)) return cs;
  return 0;
}

// the default shape, or (squares above 88 rows) the smallest larger cluster that holds them
bool coarse_conv_supported(int P) { return P >= 1 && (modes_per_thread(P) > 0 || min_fitting_cluster(P) > 0); }

template <typename T>
static cudaError_t prepare_T() {
  // 16-block clusters where the device grants them
  if (cudaFuncSetAttribute(coarse_cluster_kernel<T, 2>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
          cudaSuccess &&
      cudaFuncSetAttribute(coarse_cluster_kernel<T, 4>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
          cudaSuccess &&
      cudaFuncSetAttribute(coarse_cluster_kernel<T, 1, CCB1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
          cudaSuccess)
    g_max_cluster = 16;
  cudaGetLastError();
  int slots = 0;
  const int prec = sizeof(T) == 4 ? 0 : 1;
  int bytes = 0;   // the largest shared-memory need over every supported square and cluster size
  for (int P = 1; P <= 128; ++P)
    for (int cs = 0; cs <= g_max_cluster; ++cs)
      if (coarse_cluster_fits(P, cs)) {
        const int b = (int)cluster_smem(prec, P, 512, &slots, cs);
        if (b > bytes) bytes = b;
      }
  cudaError_t e = cudaFuncSetAttribute(coarse_cluster_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(coarse_cluster_kernel<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(coarse_cluster_kernel<T, 1, CCB1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t coarse_prepare(int prec) { return prec == 0 ? prepare_T<float>() : prepare_T<double>(); }

static int sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 132;
  }
  return sms;
}

// Default cluster size: the per-stage time is a fixed barrier / latency part plus a part
// proportional to the rows of a block, so a few fields take the largest clusters that all
// fit on the GPU at once (~3 rows per block, up to 16 blocks); larger batches keep ~6 rows
// per block (at most 8) so that more clusters run concurrently.
static int auto_cluster(int P, int batch) {
  if (g_max_cluster >= 16 && batch * 16 <= sm_count()) {
    const int cs = (P + 2) / 3 < 16 ? (P + 2) / 3 : 16;
    if (cs > 8 && coarse_cluster_fits(P, cs)) return cs;
  }
  return modes_per_thread(P) > 0 ? 0 : min_fitting_cluster(P);
}

template <typename T>
static int launch_cluster(const CoarseArgs& a0, int batch, cudaStream_t st) {
  CoarseArgs a = a0;
  const int req = a.cluster > 0 && coarse_cluster_fits(a.Pc, a.cluster) ? a.cluster : auto_cluster(a.Pc, batch);
  int CS, H, slots;
  cluster_shape(a.Pc, &CS, &H, req);
  const size_t sm = cluster_smem(sizeof(T) == 4 ? 0 : 1, a.Pc, a.nsteps, &slots, req);
  a.phase_smem = slots;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(CS * batch), 1, 1);
  const int mpt = modes_per_thread(a.Pc, req);
  cfg.blockDim = dim3(mpt == 1 ? CCB1 : CCB, 1, 1);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = mpt == 1   ? cudaLaunchKernelEx(&cfg, coarse_cluster_kernel<T, 1, CCB1>, a, CS, H)
                       : mpt == 2 ? cudaLaunchKernelEx(&cfg, coarse_cluster_kernel<T, 2>, a, CS, H)
                                  : cudaLaunchKernelEx(&cfg, coarse_cluster_kernel<T, 4>, a, CS, H);
  return e == cudaSuccess ? 1 : -1;
}

int coarse_conv_launch(int prec, const CoarseArgs& a, int batch, cudaStream_t st) {
  if (!coarse_conv_supported(a.Pc) || batch <= 0) return -1;
  return prec == 0 ? launch_cluster<float>(a, batch, st) : launch_cluster<double>(a, batch, st);
}

}  // namespace kd
