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

// The diagonal implicit solve X = t / (1 + h), h = dt A_ii lambda(k), written as
// X = t - t g with g = h / (1 + h): the same value in exact arithmetic, but the factor that
// multiplies the whole state at every stage is 1 - g with g small, so its rounding error is
// relative to g rather than to 1.  A once-rounded (1 + h)^-1 errs by the same fraction of
// an ulp at every stage of every step for a given mode, and that error accumulates over a
// slice (~3e-5 relative after 800 complex64 steps at 256^2, Rm 1000).
template <typename T>
__device__ __forceinline__ T implicit_gain(T h) {
  return h / (T(1) + h);
}
__device__ __forceinline__ cx<float> implicit_solve(cx<float> t, float g) {
  return mk(__fmaf_rn(-t.x, g, t.x), __fmaf_rn(-t.y, g, t.y));
}
__device__ __forceinline__ cx<double> implicit_solve(cx<double> t, double g) {
  return mk(__fma_rn(-t.x, g, t.x), __fma_rn(-t.y, g, t.y));
}

// Stage arrays with no aliasing between them, so that loads of several points can be
// issued before the stores of earlier points.
//
// Precision of the state between steps.  Over a slice the lowest modes change by only
// ~1e-7..1e-6 of their value per step (dt lambda is that small there), and a complex64
// state rounded to nearest after each step then errs in the same direction step after
// step: the relative error grows linearly, ~3.5e-8 per step at 256^2 (Rm 1000) and 1024^2
// (Rm 1e4).  So the state is carried as an unevaluated sum X + Xlo of two complex64
// numbers within a propagation call, and the last stage's accumulator holds the increment
// R4 - X0 instead of R4: the step's increment e is formed in complex64 (it is small, and
// its rounding is relative to it) and added to (X, Xlo) with an error-free sum.  The RHS,
// the transforms and the other accumulators stay complex64.  Xlo starts at zero (lo_valid
// false at the first step of a call) and is dropped at the end of the call, so the state
// that leaves the call is rounded once.  For complex128 Xlo is NULL and the same update
// is an ordinary sum.
template <typename T>
struct StageArrays {
  cx<T>* __restrict__ X;
  cx<T>* __restrict__ R2;
  cx<T>* __restrict__ R3;
  cx<T>* __restrict__ R4;
  cx<T>* __restrict__ Xlo;
  bool lo_valid;
};

template <typename T>
__device__ __forceinline__ StageArrays<T> stage_arrays(const FineArgs& a) {
  StageArrays<T> s;
  s.X = (cx<T>*)a.X;
  s.R2 = (cx<T>*)a.R2;
  s.R3 = (cx<T>*)a.R3;
  s.R4 = (cx<T>*)a.R4;
  s.Xlo = (cx<T>*)a.Xlo;
  s.lo_valid = a.lo_valid != 0;
  return s;
}

// Error-free sum of two reals: a + b = s + err exactly (Knuth's two-sum).
template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T& s, T& err) {
  s = a + b;
  const T bb = s - a;
  err = (a - (s - bb)) + (b - bb);
}

// State update of the last stage: X_new = x0 + e with x0 = X[s] (+ Xlo[s]); returns the new
// state rounded to precision T (the stage value the next transforms take).
template <typename T>
__device__ __forceinline__ cx<T> state_add(const StageArrays<T>& sa, long s, cx<T> x0, cx<T> e) {
  if (!sa.Xlo) {
    const cx<T> x = x0 + e;
    sa.X[s] = x;
    return x;
  }
  const cx<T> lo = sa.lo_valid ? sa.Xlo[s] : mk(T(0), T(0));
  T s0, e0, s1, e1;
  two_sum(x0.x, e.x, s0, e0);
  two_sum(x0.y, e.y, s1, e1);
  T h0, l0, h1, l1;
  two_sum(s0, lo.x + e0, h0, l0);
  two_sum(s1, lo.y + e1, h1, l1);
  sa.X[s] = mk(h0, h1);
  sa.Xlo[s] = mk(l0, l1);
  return mk(h0, h1);
}

// Increment of the last stage: x_new = (x0 + t) / (1 + h) = x0 + e, e = t - g (x0 + t).
template <typename T>
__device__ __forceinline__ cx<T> final_increment(cx<T> x0, cx<T> t, T g) {
  return t - (x0 + t) * g;
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
  const T g = implicit_gain(dt * T(0.5) * lam);
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
      const cx<T> x1 = implicit_solve(x0 + f * (dt * T(0.5)), g);
      R2[s] = x0 + f * (dt * T(11.0 / 18.0)) - x1 * (dl * T(1.0 / 6.0));
      R3[s] = x0 + f * (dt * T(5.0 / 6.0)) + x1 * (dl * T(0.5));
      R4[s] = f * (dt * T(0.25)) - x1 * (dl * T(1.5));
      out[c] = x1;
    } else if (MODE == 1) {
      const cx<T> x2 = implicit_solve(R2[s] + f * (dt * T(1.0 / 18.0)), g);
      R3[s] = R3[s] - f * (dt * T(5.0 / 6.0)) - x2 * (dl * T(0.5));
      R4[s] = R4[s] + f * (dt * T(1.75)) + x2 * (dl * T(1.5));
      out[c] = x2;
    } else if (MODE == 2) {
      const cx<T> x3 = implicit_solve(R3[s] + f * (dt * T(0.5)), g);
      R4[s] = R4[s] + f * (dt * T(0.75)) - x3 * (dl * T(0.5));
      out[c] = x3;
    } else {
      const cx<T> x0 = X[s];
      out[c] = state_add(sa, s, x0, final_increment(x0, R4[s] - f * (dt * T(1.75)), g));
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
// stiffly accurate: the last stage value is the new state, formed as X_0 plus its increment
// (the accumulator R2 of RK222 holds R2 - X0; state_add above).
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
  const T g = implicit_gain(dt * gam * lam);
  const T dl = dt * lam;
  cx<T>* __restrict__ X = sa.X;
  cx<T>* __restrict__ R2 = sa.R2;
  cx<T> out[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const long s = s0 + c * cstride;
    const cx<T> f = F[c];
    if (SCH == SCHEME_RK111) {
      const cx<T> x0 = X[s];
      out[c] = state_add(sa, s, x0, final_increment(x0, f * dt, g));
    } else if (MODE == 0) {
      const cx<T> x0 = X[s];
      const cx<T> x1 = implicit_solve(x0 + f * (dt * gam), g);
      R2[s] = f * (dt * T(Tab222::d)) - x1 * (dl * (T(1) - gam));    // R2 - X0
      out[c] = x1;
    } else {
      const cx<T> x0 = X[s];
      out[c] = state_add(sa, s, x0, final_increment(x0, R2[s] + f * (dt * (T(1) - T(Tab222::d))), g));
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
