// Pieces of the 2D stage shared by the split sweeps (stage2d.cu) and the
// fused stage kernel (stage2d_fused.cu): wave speeds, the characteristic
// system of the 2D Euler flux Jacobian, and the time step of a stage.
#pragma once

#include "flux2d.cuh"
#include "hweno_math.cuh"
#include "internal.h"

namespace hweno {
namespace {

template <int EQ, class Real>
__device__ __forceinline__ void speeds2(const Real* U, Real gam, Real& sx, Real& sy) {
  if constexpr (EQ == HWENO_BURGERS) {
    sx = sy = fabs(U[0]);
  } else {
    Real rr;
    const Prim2<Real> q = std::is_same<Real, double>::value ? prim2_rr(U, gam - Real(1), rr)
                                                            : prim2(U, gam - Real(1));
    const Real c = speed_from_sq(gam * q.p * q.ir);
    sx = fabs(q.u) + c;
    sy = fabs(q.v) + c;
  }
}

// Characteristic system of the 2D Euler flux Jacobian in direction DIR at
// velocity (u, v), enthalpy H, sound speed c. Rows of L and columns of R in
// the eigenvalue order un - c, un, shear, un + c; normal velocity un (slot
// kn = 1 + DIR), tangential ut (slot kt = 2 - DIR). Zeros are skipped.
template <class Real, int DIR>
struct Char2 {
  Real un, ut, H, c, q, b1, b2, ic;
  // sound speed from c^2 (one reciprocal square root gives c and 1/c)
  __device__ __forceinline__ void init(Real u, Real v, Real H_, Real c2, Real gm1) {
    un = DIR == 0 ? u : v;
    ut = DIR == 0 ? v : u;
    H = H_;
    sound_speed(c2, c, ic);
    q = Real(0.5) * (u * u + v * v);
    b1 = gm1 * ic * ic;
    b2 = b1 * q;
  }
  // row r of L applied to (x0, x1, x2, x3)
  __device__ __forceinline__ Real left(int r, Real x0, Real x1, Real x2, Real x3) const {
    const Real xn = DIR == 0 ? x1 : x2, xt = DIR == 0 ? x2 : x1;
    if (r == 2) return xt - ut * x0;
    const Real A = Real(0.5) * (b2 * x0 - b1 * un * xn - b1 * ut * xt + b1 * x3);
    if (r == 1) return x0 - Real(2) * A;
    const Real B = Real(0.5) * ic * (un * x0 - xn);
    return r == 0 ? A + B : A - B;
  }
  // R s
  __device__ __forceinline__ void right(const Real* s, Real* out) const {
    const Real sum = s[0] + s[1] + s[3], dif = s[3] - s[0];
    const Real on = un * sum + c * dif;
    const Real ot = ut * sum + s[2];
    out[0] = sum;
    out[DIR == 0 ? 1 : 2] = on;
    out[DIR == 0 ? 2 : 1] = ot;
    out[3] = H * (s[0] + s[3]) + q * s[1] + ut * s[2] + un * c * dif;
  }
};

__device__ __forceinline__ double time_step2(const Args2D& a, int& lands) {
  if (a.dt_in) {  // replay of a recorded step
    lands = 0;
    return a.dt_in[0];
  }
  double dt;
  if (a.sp.dt_mode == 2) {
    dt = a.sp.dt_fixed;
  } else {
    const double rate = __dadd_rn(__ddiv_rn(a.alpha_in[0], a.hx), __ddiv_rn(a.alpha_in[1], a.hy));
    dt = rate > 0.0 ? __ddiv_rn(a.sp.cfl, rate) : __longlong_as_double(0x7ff0000000000000LL);
  }
  const double rest = a.t_end - a.t[0];
  lands = dt >= rest;
  return lands ? rest : dt;
}

}  // namespace
}  // namespace hweno
