// Persistent thread-block-cluster kernel of the classical coarse propagator and of the
// convolution-form fine operator (Sec. 3.2, Sec. 5.2); host code in kd_coarse.cu.  The
// halo-exchange variant is a template parameter (CoarseArgs::halo selects it at launch);
// the default variant is instantiated in kd_coarse.cu, the others in kd_coarse_alt.cu.
#pragma once

#include <cooperative_groups.h>

#include "kd_coarse.h"
#include "kd_stage.cuh"
#include "kd_wait.cuh"

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

// Halo exchange after each stage (CoarseArgs::halo).  0 (default): the first and last rows
// are stored into the neighbours' halo rows through distributed shared memory, then one
// cluster barrier.  2 (pull): no halo copies; after a split cluster barrier (arrive after
// the stage's own stores, wait before the first / last rows of the next stage, the rows
// between computed meanwhile) a block reads the neighbours' edge rows in place.
// 1 (point-to-point, measured slower on GB300: 1.57 vs 1.29 us per stage at 16 blocks): a block
// pushes its first and last rows into the neighbours' halo rows with st.async, which
// counts the bytes on the receiver's mbarrier (complete_tx); the receiver waits on its own
// mbarrier instead of a cluster-wide barrier.  Stage g's halos arrive on mbarrier g mod 4;
// the expected byte count of stage g + 3 is posted during stage g, after every thread of
// the block has passed the wait of stage g - 1 on the same mbarrier (the block barrier at
// the top of stage g) and before any push of stage g + 1 (which the data of stage g + 3
// depends on), so no phase is skipped and no byte is counted in the wrong phase.
constexpr long long kHaloWaitCycles = 4000000;   // ~2 ms at 2 GHz; then the outputs are NaN

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t peer_addr(uint32_t a, int rank) {
  uint32_t o;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(o) : "r"(a), "r"(rank));
  return o;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect(uint32_t bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// bounded wait for the phase of the given parity; false after kHaloWaitCycles
__device__ __forceinline__ bool mbar_wait(uint32_t bar, unsigned parity) {
  return mbar_wait_bounded<true>(bar, parity, kHaloWaitCycles);
}

__device__ __forceinline__ void push(uint32_t dst, cx<float> v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(dst),
               "f"(v.x), "f"(v.y), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void push(uint32_t dst, cx<double> v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];" ::"r"(dst),
               "d"(v.x), "d"(v.y), "r"(bar)
               : "memory");
}

template <typename T, int MPT, int NT, int HALO>
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
  T lam_dt[MPT], gain[MPT], fkx[MPT], fky[MPT];
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
    gain[i] = implicit_gain(dt * T(0.5) * lam);
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
  constexpr bool p2p = HALO == 1;      // push with st.async + mbarrier
  constexpr bool pull = HALO == 2;     // read the neighbours' rows, split cluster barrier
  constexpr bool split = p2p || pull;  // interior rows before, first / last rows after the wait
  // halo rows this block receives: the last row of rank - 1 (into row 0 of the halo ring)
  // and the first row of rank + 1 (into row H + 1)
  const bool from_up = hr > 0 && rank > 0;
  const bool from_dn = rank < CS - 1 && y0 + H < P;
  const unsigned halo_bytes = (unsigned)((from_up ? 1 : 0) + (from_dn ? 1 : 0)) * 3u * (unsigned)P * sizeof(cx<T>);
  __shared__ __align__(8) unsigned long long hbar[4];
  __shared__ int s_bad;
  const int G = 4 * nsteps;   // stages
  if (threadIdx.x == 0) {
    s_bad = 0;
    if (p2p) {
      for (int q = 0; q < 4; ++q) mbar_init(smem_addr(&hbar[q]), 1);
      for (int g = 0; g < 3 && g < G; ++g) mbar_expect(smem_addr(&hbar[g]), halo_bytes);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  // per-thread mode layout, fixed for the whole solve: offset ly L + ix of mode i in the
  // haloed stripe (ly, ix from 1), and whether it lies in the first / last row; threads
  // owning a mode of the first or last row wait for the halos (point-to-point exchange)
  int off[MPT];
  unsigned first_mask = 0, last_mask = 0;
#pragma unroll
  for (int i = 0; i < MPT; ++i) {
    const int m = threadIdx.x + NT * i;
    const int ly = m < M ? m / P : 0, ix = m < M ? m % P : 0;
    off[i] = m < M ? (ly + 1) * L + ix + 1 : -1;
    if (m < M && ly == 0) first_mask |= 1u << i;
    if (m < M && ly == hr - 1) last_mask |= 1u << i;
  }
  const bool has_edge = (first_mask | last_mask) != 0;
  const uint32_t buf_s = smem_addr(buf), hbar_s = smem_addr(hbar);
  const uint32_t up_buf = rank > 0 ? peer_addr(buf_s, rank - 1) : 0u, up_bar = rank > 0 ? peer_addr(hbar_s, rank - 1) : 0u;
  const uint32_t dn_buf = rank < CS - 1 ? peer_addr(buf_s, rank + 1) : 0u;
  const uint32_t dn_bar = rank < CS - 1 ? peer_addr(hbar_s, rank + 1) : 0u;
  // stage value of mode i into buffer bsel; the first / last row also into the
  // neighbours' halo rows H + 1 / 0 (st.async counted on their mbarrier q when p2p, plain
  // distributed-shared stores otherwise)
  auto put = [&](int bsel, int q, bool remote, int i, int c, cx<T> v) {
    const int o = bsel * bufsz + c * LH * L + off[i];
    buf[o] = v;
    if (!remote) return;
    if ((first_mask >> i) & 1u && rank > 0) {
      const int o_up = o + H * L;
      if (p2p) {
        push(up_buf + (uint32_t)(o_up * sizeof(cx<T>)), v, up_bar + (uint32_t)(q * 8));
      } else {
        cx<T>* peer = cluster.map_shared_rank(buf, rank - 1);
        peer[o_up] = v;
      }
    }
    if ((last_mask >> i) & 1u && rank < CS - 1 && y0 + hr < P) {
      const int o_dn = o - hr * L;
      if (p2p) {
        push(dn_buf + (uint32_t)(o_dn * sizeof(cx<T>)), v, dn_bar + (uint32_t)(q * 8));
      } else {
        cx<T>* peer = cluster.map_shared_rank(buf, rank + 1);
        peer[o_dn] = v;
      }
    }
  };
  cluster.sync();   // every block has zeroed its buffers (and set up its mbarriers) before peers write halos
#pragma unroll
  for (int i = 0; i < MPT; ++i) {
    const int m = threadIdx.x + NT * i;
    if (m < M)
#pragma unroll
      for (int c = 0; c < 3; ++c) put(0, 0, G > 0, i, c, x0[i][c]);
  }
  if (pull) {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  } else if (!p2p) {
    cluster.sync();
  }
  // pull: the first row's upper neighbour row is the last row H of rank - 1, the last row's
  // lower neighbour the first row of rank + 1 (zero rows of the own ring at the edges)
  const bool has_next = rank < CS - 1 && y0 + hr < P;
  const cx<T>* up_peer = pull && rank > 0 ? cluster.map_shared_rank(buf, rank - 1) : nullptr;
  const cx<T>* dn_peer = pull && has_next ? cluster.map_shared_rank(buf, rank + 1) : nullptr;

  const T A = a.sp ? (T)a.sp[b].amp : (T)a.amp;
  int cur = 0;
  for (int s = 0; s < nsteps; ++s) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int g = 4 * s + j;
      if (split) __syncthreads();   // own rows of the current buffer are complete in this block
      if (p2p && threadIdx.x == 0 && g + 3 < G) mbar_expect(hbar_s + (uint32_t)(((g + 3) & 3) * 8), halo_bytes);
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
      // rows above the first and below the last row: the own halo ring, or the neighbours'
      // rows themselves (pull; offset o of a first-row mode maps to o + (H - 1) L in rank - 1,
      // of a last-row mode to o + (1 - hr) L in rank + 1)
      const cx<T>* Xup = up_peer ? up_peer + cur * bufsz + (H - 1) * L : Xs - L;
      const cx<T>* Xdn = dn_peer ? dn_peer + cur * bufsz + (1 - hr) * L : Xs + L;

      // one mode's stage: convolution, curl, IMEX update, store (pass 0: rows that need no
      // halo; pass 1: the first and last rows, after the halos have arrived)
      auto stage_pass = [&](int pass) {
#pragma unroll
        for (int i = 0; i < MPT; ++i) {
          const int o = off[i];
          if (o < 0) continue;
          const bool edge = ((first_mask | last_mask) >> i) & 1u;
          if (split && (edge ? 0 : 1) != (pass == 0 ? 1 : 0)) continue;
          // u_hat of the flows of Sec. 2 (see uhat): u_y(+-x) = -+ i u_z(+-x) and
          // u_z(+-y) = -+ i u_x(+-y), so each neighbour's cross product takes two complex
          // products: with z = u_z(q), x neighbour b = b_hat(k - q), q = +-x:
          //   w += (z (-b_y -+ i b_z), z b_x, +- i z b_x);
          // with v = u_x(q), y neighbour c = b_hat(k - q), q = +-y:
          //   w += (+- i v c_y, v (-c_z -+ i c_x), v c_y)
          cx<T> w[3] = {mk(T(0), T(0)), mk(T(0), T(0)), mk(T(0), T(0))};
#pragma unroll
          for (int sgn = 0; sgn < 2; ++sgn) {
            const int ox = o + (sgn == 0 ? -1 : 1);   // x neighbour ix -+ 1
            const cx<T> bx = Xs[ox], by = Xs[LH * L + ox], bz = Xs[2 * LH * L + ox];
            const cx<T> z = u.pz[sgn];
            const cx<T> p = cmul(z, bx);
            const cx<T> s0 = sgn == 0 ? mk(bz.y - by.x, -by.y - bz.x) : mk(-by.x - bz.y, bz.x - by.y);
            w[0] = w[0] + cmul(z, s0);
            w[1] = w[1] + p;
            w[2] = sgn == 0 ? w[2] + mul_i(p) : w[2] - mul_i(p);
            // y neighbour ly -+ 1 (in the neighbour block's rows when pulling them)
            cx<T> cxv, cyv, czv;
            const bool far = pull && (sgn == 0 ? ((first_mask >> i) & 1u) : ((last_mask >> i) & 1u));
            if (far) {
              const cx<T>* Y = sgn == 0 ? Xup : Xdn;
              cxv = Y[o];
              cyv = Y[LH * L + o];
              czv = Y[2 * LH * L + o];
            } else {
              const int oy = o + (sgn == 0 ? -L : L);
              cxv = Xs[oy];
              cyv = Xs[LH * L + oy];
              czv = Xs[2 * LH * L + oy];
            }
            const cx<T> v = u.qx[sgn];
            const cx<T> r = cmul(v, cyv);
            const cx<T> s1 = sgn == 0 ? mk(cxv.y - czv.x, -czv.y - cxv.x) : mk(-czv.x - cxv.y, cxv.x - czv.y);
            w[0] = sgn == 0 ? w[0] + mul_i(r) : w[0] - mul_i(r);
            w[1] = w[1] + cmul(v, s1);
            w[2] = w[2] + r;
          }
          cx<T> F[3];
          F[0] = mul_i(w[2] * fky[i] - w[1] * kz);
          F[1] = mul_i(w[0] * kz - w[2] * fkx[i]);
          F[2] = mul_i(w[1] * fkx[i] - w[0] * fky[i]);
          const T dl = lam_dt[i], gi = gain[i];
          cx<T> xn[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const cx<T> f = F[c];
            if (j == 0) {
              const cx<T> x1 = implicit_solve(x0[i][c] + f * (dt * T(0.5)), gi);
              r2[i][c] = x0[i][c] + f * (dt * T(11.0 / 18.0)) - x1 * (dl * T(1.0 / 6.0));
              r3[i][c] = x0[i][c] + f * (dt * T(5.0 / 6.0)) + x1 * (dl * T(0.5));
              r4[i][c] = x0[i][c] + f * (dt * T(0.25)) - x1 * (dl * T(1.5));
              xn[c] = x1;
            } else if (j == 1) {
              const cx<T> x2 = implicit_solve(r2[i][c] + f * (dt * T(1.0 / 18.0)), gi);
              r3[i][c] = r3[i][c] - f * (dt * T(5.0 / 6.0)) - x2 * (dl * T(0.5));
              r4[i][c] = r4[i][c] + f * (dt * T(1.75)) + x2 * (dl * T(1.5));
              xn[c] = x2;
            } else if (j == 2) {
              const cx<T> x3 = implicit_solve(r3[i][c] + f * (dt * T(0.5)), gi);
              r4[i][c] = r4[i][c] + f * (dt * T(0.75)) - x3 * (dl * T(0.5));
              xn[c] = x3;
            } else {
              const cx<T> x4 = implicit_solve(r4[i][c] - f * (dt * T(1.75)), gi);
              x0[i][c] = x4;
              xn[c] = x4;
            }
          }
          // no pushes after the last stage, nor once a halo wait of this block timed out
          const bool send = !pull && g + 1 < G && !*(volatile int*)&s_bad;
#pragma unroll
          for (int c = 0; c < 3; ++c) put(cur ^ 1, (g + 1) & 3, send, i, c, xn[c]);
        }
      };
      if (p2p) {
        stage_pass(0);
        if (has_edge && !*(volatile int*)&s_bad &&
            !mbar_wait(hbar_s + (uint32_t)((g & 3) * 8), (unsigned)((g >> 2) & 1)))
          *(volatile int*)&s_bad = 1;
        stage_pass(1);
      } else if (pull) {
        stage_pass(0);
        asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");   // previous stage everywhere
        stage_pass(1);
        asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
      } else {
        stage_pass(0);
        cluster.sync();   // new stage values (own rows and halos) are complete everywhere
      }
      cur ^= 1;
    }
  }
  if (p2p) {
    __syncthreads();
    if (s_bad) {
      // a halo never arrived: let stores still in flight land, then poison the outputs
      for (int w = 0; w < 100; ++w) __nanosleep(1000);
      for (int i = threadIdx.x; i < 2 * bufsz; i += NT) buf[i] = mk(T(NAN), T(NAN));
    }
    cluster.sync();   // the final stage values of every block are complete
  } else if (pull) {
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");   // the final stage everywhere
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


// the three modes-per-thread variants of one halo exchange
template <typename T, int HALO>
cudaError_t cluster_allow_nonportable() {
  cudaError_t e = cudaFuncSetAttribute(coarse_cluster_kernel<T, 1, CCB1, HALO>,
                                       cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(coarse_cluster_kernel<T, 2, CCB, HALO>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(coarse_cluster_kernel<T, 4, CCB, HALO>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

template <typename T, int HALO>
cudaError_t cluster_set_smem(int bytes) {
  cudaError_t e =
      cudaFuncSetAttribute(coarse_cluster_kernel<T, 1, CCB1, HALO>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(coarse_cluster_kernel<T, 2, CCB, HALO>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(coarse_cluster_kernel<T, 4, CCB, HALO>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

template <typename T, int HALO>
cudaError_t cluster_launch(const cudaLaunchConfig_t& cfg, int mpt, const CoarseArgs& a, int CS, int H) {
  return mpt == 1   ? cudaLaunchKernelEx(&cfg, coarse_cluster_kernel<T, 1, CCB1, HALO>, a, CS, H)
         : mpt == 2 ? cudaLaunchKernelEx(&cfg, coarse_cluster_kernel<T, 2, CCB, HALO>, a, CS, H)
                    : cudaLaunchKernelEx(&cfg, coarse_cluster_kernel<T, 4, CCB, HALO>, a, CS, H);
}

}  // namespace kd
