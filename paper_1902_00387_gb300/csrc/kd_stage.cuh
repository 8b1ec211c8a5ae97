// Pointwise pieces of the fine step shared by the kernel families: the flow
// u(x, y, t) (Sec. 2.1 / 2.2), the cross product u x b, the spectral curl
// i k3 x w_hat, and the IMEX RK443 stage update with diagonal implicit diffusion.
#pragma once
#include <type_traits>

#include "kd_common.cuh"

namespace kd {

// Flow phases of the Galloway-Proctor flow at the stage time t:
// (cos(cos t), sin(cos t), cos(sin t), sin(sin t)); Roberts: (1, 0, 1, 0).
template <typename T>
struct Phase {
  T cpx, spx, cpy, spy;
};

template <typename T>
__device__ __forceinline__ Phase<T> load_phase(const FineArgs& a, long b, int step, int stage) {
  Phase<T> p;
  if (a.flow == FLOW_GP) {
    const T* ph = (const T*)a.phases + (((long)b * a.phase_steps + step) * 4 + stage) * 4;
    p.cpx = ph[0];
    p.spx = ph[1];
    p.cpy = ph[2];
    p.spy = ph[3];
  } else {
    p.cpx = T(1);
    p.spx = T(0);
    p.cpy = T(1);
    p.spy = T(0);
  }
  return p;
}

// Flow amplitude of field b.
template <typename T>
__device__ __forceinline__ T flow_amp(const FineArgs& a, long b) {
  return a.sp ? (T)a.sp[b].amp : (T)a.amp;
}

// Per-field coefficients of the stage update: dt, kz and 1 / Rm in precision T.
template <typename T>
struct StageCoef {
  T dt, kz, inv_rm;
};

template <typename T>
__device__ __forceinline__ StageCoef<T> stage_coef(const FineArgs& a, long b) {
  StageCoef<T> q;
  if (a.sp) {
    const SliceParams& p = a.sp[b];
    q.dt = (T)p.dt;
    q.kz = (T)p.kz;
    q.inv_rm = T(1) / (T)p.Rm;
  } else {
    q.dt = (T)a.dt;
    q.kz = (T)a.kz;
    q.inv_rm = T(1) / (T)a.Rm;
  }
  return q;
}

// w = u x b at the grid point with cos/sin of x and y given;
// u = A (cos(y + py), sin(x + px), cos(x + px) + sin(y + py)).
template <typename T>
__device__ __forceinline__ void cross_u(T A, const Phase<T>& p, T cxg, T sxg, T cyg, T syg, cx<T>& bx, cx<T>& by,
                                        cx<T>& bz) {
  const T ux = A * (cyg * p.cpy - syg * p.spy);
  const T uy = A * (sxg * p.cpx + cxg * p.spx);
  const T uz = A * ((cxg * p.cpx - sxg * p.spx) + (syg * p.cpy + cyg * p.spy));
  const cx<T> vx = bx, vy = by, vz = bz;
  bx = vz * uy - vy * uz;
  by = vx * uz - vz * ux;
  bz = vy * ux - vx * uy;
}

// Stage arrays with no aliasing between them, so that loads of several points can be
// issued before the stores of earlier points.
template <typename T>
struct StageArrays {
  cx<T>* __restrict__ X;
  cx<T>* __restrict__ R2;
  cx<T>* __restrict__ R3;
  cx<T>* __restrict__ R4;
};

template <typename T>
__device__ __forceinline__ StageArrays<T> stage_arrays(const FineArgs& a) {
  StageArrays<T> s;
  s.X = (cx<T>*)a.X;
  s.R2 = (cx<T>*)a.R2;
  s.R3 = (cx<T>*)a.R3;
  s.R4 = (cx<T>*)a.R4;
  return s;
}

// One IMEX RK443 stage at spectral point s (index into the compact arrays) for the
// three components: w_hat (already scaled by 1/n^2) -> F = i k3 x w_hat -> new stage
// value (returned in w).  MODE = stage 0..3.
template <int MODE, typename T>
__device__ __forceinline__ void stage_update(const StageCoef<T>& q, const StageArrays<T>& sa, long s0, long cstride,
                                             T fkx, T fky, cx<T>& w0, cx<T>& w1, cx<T>& w2) {
  const T dt = q.dt;
  const T kz = q.kz;
  cx<T> F[3];
  F[0] = mul_i(w2 * fky - w1 * kz);
  F[1] = mul_i(w0 * kz - w2 * fkx);
  F[2] = mul_i(w1 * fkx - w0 * fky);
  const T lam = (fkx * fkx + fky * fky + kz * kz) * q.inv_rm;
  const T inv_d = T(1) / (T(1) + dt * T(0.5) * lam);
  const T dl = dt * lam;
  cx<T>* __restrict__ X = sa.X;
  cx<T>* __restrict__ R2 = sa.R2;
  cx<T>* __restrict__ R3 = sa.R3;
  cx<T>* __restrict__ R4 = sa.R4;
  cx<T> out[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const long s = s0 + c * cstride;
    const cx<T> f = F[c];
    if (MODE == 0) {
      const cx<T> x0 = X[s];
      const cx<T> x1 = (x0 + f * (dt * T(0.5))) * inv_d;
      R2[s] = x0 + f * (dt * T(11.0 / 18.0)) - x1 * (dl * T(1.0 / 6.0));
      R3[s] = x0 + f * (dt * T(5.0 / 6.0)) + x1 * (dl * T(0.5));
      R4[s] = x0 + f * (dt * T(0.25)) - x1 * (dl * T(1.5));
      out[c] = x1;
    } else if (MODE == 1) {
      const cx<T> x2 = (R2[s] + f * (dt * T(1.0 / 18.0))) * inv_d;
      R3[s] = R3[s] - f * (dt * T(5.0 / 6.0)) - x2 * (dl * T(0.5));
      R4[s] = R4[s] + f * (dt * T(1.75)) + x2 * (dl * T(1.5));
      out[c] = x2;
    } else if (MODE == 2) {
      const cx<T> x3 = (R3[s] + f * (dt * T(0.5))) * inv_d;
      R4[s] = R4[s] + f * (dt * T(0.75)) - x3 * (dl * T(0.5));
      out[c] = x3;
    } else {
      const cx<T> x4 = (R4[s] - f * (dt * T(1.75))) * inv_d;
      X[s] = x4;
      out[c] = x4;
    }
  }
  w0 = out[0];
  w1 = out[1];
  w2 = out[2];
}

// Ascher-Ruuth-Spiteri (2,2,2) and (1,1,1) in the same accumulator form as RK443 above:
// stage j evaluates F_j at X_j, forms X_{j+1} = (Q_{j+1} + dt H_{j+1,j} F_j) / (1 + dt g lam)
// with Q_1 = X_0 and Q_i = R_i, and adds its terms to the later accumulators
// R_i += dt H_ij F_j - dt A_{i,j+1} lam X_{j+1} (R_i = X_0 + ... from stage 0).  Both are
// stiffly accurate: the last stage value is the new state.
//   RK222: g = 1 - 1/sqrt(2), d = 1 - 1/(2g); A = [[g], [1-g, g]], H = [[g], [d, 1-d]]
//   RK111: A = [[1]], H = [[1]]
struct Tab222 {
  static constexpr double g = 0.29289321881345247560;    // 1 - 1/sqrt(2)
  static constexpr double d = -0.70710678118654752440;   // 1 - 1/(2 g)
};

template <int SCH, int MODE, typename T>
__device__ __forceinline__ void stage_update_tab(const StageCoef<T>& q, const StageArrays<T>& sa, long s0,
                                                 long cstride, T fkx, T fky, cx<T>& w0, cx<T>& w1, cx<T>& w2) {
  const T dt = q.dt;
  const T kz = q.kz;
  cx<T> F[3];
  F[0] = mul_i(w2 * fky - w1 * kz);
  F[1] = mul_i(w0 * kz - w2 * fkx);
  F[2] = mul_i(w1 * fkx - w0 * fky);
  const T lam = (fkx * fkx + fky * fky + kz * kz) * q.inv_rm;
  const T gam = SCH == SCHEME_RK222 ? T(Tab222::g) : T(1);
  const T inv_d = T(1) / (T(1) + dt * gam * lam);
  const T dl = dt * lam;
  cx<T>* __restrict__ X = sa.X;
  cx<T>* __restrict__ R2 = sa.R2;
  cx<T> out[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const long s = s0 + c * cstride;
    const cx<T> f = F[c];
    if (SCH == SCHEME_RK111) {
      const cx<T> x1 = (X[s] + f * dt) * inv_d;
      X[s] = x1;
      out[c] = x1;
    } else if (MODE == 0) {
      const cx<T> x0 = X[s];
      const cx<T> x1 = (x0 + f * (dt * gam)) * inv_d;
      R2[s] = x0 + f * (dt * T(Tab222::d)) - x1 * (dl * (T(1) - gam));
      out[c] = x1;
    } else {
      const cx<T> x2 = (R2[s] + f * (dt * (T(1) - T(Tab222::d)))) * inv_d;
      X[s] = x2;
      out[c] = x2;
    }
  }
  w0 = out[0];
  w1 = out[1];
  w2 = out[2];
}

// Stage update of scheme SCH (RK443: stage_update above).
template <int SCH, int MODE, typename T>
__device__ __forceinline__ void stage_update_s(const StageCoef<T>& q, const StageArrays<T>& sa, long s0,
                                               long cstride, T fkx, T fky, cx<T>& w0, cx<T>& w1, cx<T>& w2) {
  if constexpr (SCH == SCHEME_RK443)
    stage_update<MODE, T>(q, sa, s0, cstride, fkx, fky, w0, w1, w2);
  else
    stage_update_tab<SCH, MODE, T>(q, sa, s0, cstride, fkx, fky, w0, w1, w2);
}

// Call f(std::integral_constant<int, m>) for the runtime stage index m = 0..3, so that
// the stage update of a loop body is specialised for its stage.
template <class F>
__device__ __forceinline__ void with_stage(int mode, F&& f) {
  switch (mode) {
    case 0: f(std::integral_constant<int, 0>()); break;
    case 1: f(std::integral_constant<int, 1>()); break;
    case 2: f(std::integral_constant<int, 2>()); break;
    default: f(std::integral_constant<int, 3>()); break;
  }
}

}  // namespace kd
