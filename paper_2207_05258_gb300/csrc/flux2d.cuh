// Point fluxes, flux Jacobian-vector products and boundary mappings of the
// 2D equations (Zhang & Zhao, arXiv:2207.05258, Eq. EQ3 and Sec. 3), shared by
// the 2D stage kernels and their adjoint. The arithmetic is templated on the
// scalar (FP64 and FP32 paths).
#pragma once

#include "hweno.h"
#include "hweno_math.cuh"
#include "internal.h"

namespace hweno {

template <int EQ>
struct Dim2 { static constexpr int M = EQ == HWENO_BURGERS ? 1 : 4; };

// Primitive quantities of a 2D Euler state.
template <class Real>
struct Prim2 {
  Real ir, u, v, p, Ep;
};

template <class Real>
__device__ __forceinline__ Prim2<Real> prim2_ir(const Real* U, Real gm1, Real ir) {
  Prim2<Real> q;
  q.ir = ir;
  q.u = U[1] * q.ir;
  q.v = U[2] * q.ir;
  q.p = gm1 * (U[3] - Real(0.5) * (U[1] * q.u + U[2] * q.v));
  q.Ep = U[3] + q.p;
  return q;
}

template <class Real>
__device__ __forceinline__ Prim2<Real> prim2(const Real* U, Real gm1) {
  return prim2_ir(U, gm1, recip(U[0]));
}

// The same with 1/rho as the square of rr = 1/sqrt(rho), which the caller
// also uses (sqrt(rho) = rho rr for the Roe average).
template <class Real>
__device__ __forceinline__ Prim2<Real> prim2_rr(const Real* U, Real gm1, Real& rr) {
  rr = rsq(U[0]);
  return prim2_ir(U, gm1, rr * rr);
}

// Flux in direction DIR and the Jacobian-vector product A_DIR D (Eq. EQ3:
// h = f'(u) u_x, xi = g'(u) u_x, eta = f'(u) u_y, theta = g'(u) u_y).
template <int EQ, int DIR, class Real>
__device__ __forceinline__ void flux2(const Real* U, const Prim2<Real>& q, Real* F) {
  if constexpr (EQ == HWENO_BURGERS) {
    F[0] = Real(0.5) * U[0] * U[0];
  } else if constexpr (DIR == 0) {
    F[0] = U[1]; F[1] = U[1] * q.u + q.p; F[2] = U[1] * q.v; F[3] = q.Ep * q.u;
  } else {
    F[0] = U[2]; F[1] = U[2] * q.u; F[2] = U[2] * q.v + q.p; F[3] = q.Ep * q.v;
  }
}

template <int EQ, int DIR, class Real>
__device__ __forceinline__ void jvp2(const Real* U, const Prim2<Real>& q, const Real* D, Real gm1,
                                     Real* out) {
  if constexpr (EQ == HWENO_BURGERS) {
    out[0] = U[0] * D[0];
  } else {
    const Real du = (D[1] - q.u * D[0]) * q.ir;
    const Real dv = (D[2] - q.v * D[0]) * q.ir;
    const Real dp = gm1 * (D[3] - (q.u * D[1] + q.v * D[2]) + Real(0.5) * (q.u * q.u + q.v * q.v) * D[0]);
    if constexpr (DIR == 0) {
      out[0] = D[1];
      out[1] = D[1] * q.u + U[1] * du + dp;
      out[2] = D[1] * q.v + U[1] * dv;
      out[3] = (D[3] + dp) * q.u + q.Ep * du;
    } else {
      out[0] = D[2];
      out[1] = D[2] * q.u + U[2] * du;
      out[2] = D[2] * q.v + U[2] * dv + dp;
      out[3] = (D[3] + dp) * q.v + q.Ep * dv;
    }
  }
}

// Ghost handling along one direction. kind: 0 copy, 1 mirror, 2 imposed
// state (pre = 0: sp.inflow, pre = 1: sp.pre).
struct Src {
  int idx;
  int kind;
  int pre;
};

__device__ __forceinline__ double imposed(const SchemeParams& sp, const Src& s, int c) {
  return s.pre ? sp.pre[c] : sp.inflow[c];
}

__device__ __forceinline__ Src map_x(int i, int n, const SchemeParams& sp) {
  Src r{i, 0, 0};
  if (i >= 0 && i < n) return r;
  const int b = i < 0 ? sp.bc[0] : sp.bc[1];
  if (b == HWENO_BC_PERIODIC) r.idx = i < 0 ? i + n : i - n;
  else if (b == HWENO_BC_OUTFLOW) r.idx = i < 0 ? 0 : n - 1;
  else if (b == HWENO_BC_REFLECTIVE) { r.kind = 1; r.idx = i < 0 ? -i - 1 : 2 * n - 1 - i; }
  else r.kind = 2;
  return r;
}

// y ghost rows that take an imposed state or, on the double-Mach bottom,
// depend on x: column i (cell centre x = x0 + (i + 1/2) dx) at stage time
// ts. Out of line, so that the FP64 arithmetic of the shock position runs
// for these ghosts only and not, speculated, for every loaded point.
static __device__ __noinline__ Src map_y_imposed(int j, int n, int b, int i, double x0, double dx,
                                          double y0, double dy, double ts,
                                          const SchemeParams& sp) {
  Src r{j, 0, 0};
  const double x = __dadd_rn(x0, __dmul_rn((double)i + 0.5, dx));
  if (b == HWENO_BC_DMR_BOTTOM && !(x < sp.dmr_x0)) {  // the wall
    r.kind = 1;
    r.idx = j < 0 ? -j - 1 : 2 * n - 1 - j;
  } else if (b == HWENO_BC_DMR_TOP) {  // the exact shock at the ghost's height
    const double yg = __dadd_rn(y0, __dmul_rn((double)j + 0.5, dy));
    const double xs = __dadd_rn(__dadd_rn(sp.dmr_x0, __ddiv_rn(yg, sp.dmr_tan)),
                                __ddiv_rn(__dmul_rn(sp.dmr_speed, ts), sp.dmr_sin));
    r.kind = 2;
    r.pre = x < xs ? 0 : 1;
  } else {
    r.kind = 2;  // inflow, or the DMR bottom left of the wall
  }
  return r;
}

// y ghosts of column i at stage time ts; the DMR bottom wall starts at
// dmr_x0 and the top carries the exact shock position at the ghost's height
// (reading of Example 3.11).
__device__ __forceinline__ Src map_y(int j, int n, int i, double x0, double dx, double y0,
                                     double dy, double ts, const SchemeParams& sp) {
  Src r{j, 0, 0};
  if (j >= 0 && j < n) return r;
  const int b = j < 0 ? sp.bc[2] : sp.bc[3];
  if (b == HWENO_BC_PERIODIC) r.idx = j < 0 ? j + n : j - n;
  else if (b == HWENO_BC_OUTFLOW) r.idx = j < 0 ? 0 : n - 1;
  else if (b == HWENO_BC_REFLECTIVE) {
    r.kind = 1;
    r.idx = j < 0 ? -j - 1 : 2 * n - 1 - j;
  } else {
    r = map_y_imposed(j, n, b, i, x0, dx, y0, dy, ts, sp);
  }
  return r;
}

// Reflection sign of component c through a wall normal to DIR (Burgers: u
// odd; Euler: the normal momentum odd).
template <int EQ, int DIR>
__device__ __forceinline__ float refl2(int c) {
  return EQ == HWENO_BURGERS ? -1.f : (c == 1 + DIR ? -1.f : 1.f);
}

}  // namespace hweno
