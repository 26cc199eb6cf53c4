// Implementation of the one-dimensional L-HWENO stage kernels, shared by the
// FP64 (stage1d.cu) and FP32 (stage1d_f32.cu) translation units; see
// stage1d.cu for the structure of a stage.
#pragma once

#include <cfloat>
#include <type_traits>

#include <cooperative_groups.h>
#include <cuda/atomic>

#include "hweno.h"
#include "hweno_math.cuh"
#include "internal.h"

namespace hweno {
namespace {


template <int EQ>
struct Dim1 { static constexpr int M = EQ == HWENO_EULER ? 3 : 1; };

// Source of point i (possibly a ghost) of an instance with n points.
// kind: 0 copy, 1 mirror (reflective wall), 2 imposed state.
__device__ __forceinline__ int map_1d(int i, int n, int bclo, int bchi, int& kind) {
  kind = 0;
  if (i >= 0 && i < n) return i;
  const int b = i < 0 ? bclo : bchi;
  if (b == HWENO_BC_PERIODIC) return i < 0 ? i + n : i - n;
  if (b == HWENO_BC_OUTFLOW) return i < 0 ? 0 : n - 1;
  if (b == HWENO_BC_REFLECTIVE) { kind = 1; return i < 0 ? -i - 1 : 2 * n - 1 - i; }
  kind = 2;
  return 0;
}

// Sign of component c of U under reflection (Burgers: u odd; Euler: momentum
// odd; a Buckley-Leverett saturation even, though the host rejects such
// walls). The normal derivative takes the opposite sign.
template <int EQ>
__device__ __forceinline__ float refl_sign(int c) {
  if (EQ == HWENO_BUCKLEY) return 1.f;
  return EQ == HWENO_BURGERS ? -1.f : (c == 1 ? -1.f : 1.f);
}

// Buckley-Leverett flux f = 4u^2/D and f' = 8u(1 - u)/D^2, D = 4u^2 + (1-u)^2.
template <class Real>
__device__ __forceinline__ void buckley_f(Real u, Real& f, Real& df) {
  const Real w = Real(1) - u;
  const Real iD = Real(1) / (Real(4) * u * u + w * w);
  f = Real(4) * u * u * iD;
  df = Real(8) * u * w * iD * iD;
}

// Per-point contribution to alpha; a01 = max |f'| over [0, 1] (Buckley-
// Leverett only).
template <int EQ, class Real>
__device__ __forceinline__ Real wave_speed(const Real* u, Real gam, Real a01) {
  if constexpr (EQ == HWENO_BURGERS) {
    return fabs(u[0]);
  } else if constexpr (EQ == HWENO_BUCKLEY) {
    Real f, df;
    buckley_f(u[0], f, df);
    return fmax(a01, fabs(df));
  } else {
    // FP64: 1/rho as the square of one reciprocal square root
    Real ir;
    if constexpr (std::is_same<Real, double>::value) {
      const Real rr = rsq(u[0]);
      ir = rr * rr;
    } else {
      ir = recip(u[0]);
    }
    const Real vel = u[1] * ir;
    const Real p = (gam - Real(1)) * (u[2] - Real(0.5) * u[1] * vel);
    return fabs(vel) + speed_from_sq(gam * p * ir);
  }
}

// Time step of an instance from the wave speed of u^n (dt_mode), clipped to
// land on t_end. Same expression order as the problem statement:
// dt = cfl / (alpha / h).
__device__ __forceinline__ double time_step(const SchemeParams& sp, double alpha, double h,
                                            double t, double t_end, int& lands) {
  double dt;
  if (sp.dt_mode == 2) {
    dt = sp.dt_fixed;
  } else {
    const double rate = alpha / h;
    dt = rate > 0.0 ? sp.cfl / rate : __longlong_as_double(0x7ff0000000000000LL);
  }
  const double rest = t_end - t;
  lands = dt >= rest;
  return lands ? rest : dt;
}

// Wave speed of the stage input, per instance (alpha of Sec. 2.1).
template <int EQ, class Real, int P>
__global__ void __launch_bounds__(kThreads1D) k_alpha_1d(const __grid_constant__ Args1D a) {
  constexpr int M = Dim1<EQ>::M;
  __shared__ Real red[kThreads1D / 32];
  const int b = blockIdx.x;
  const int k = a.tile_inst[b], s = a.tile_start[b], n = a.inst_n[k];
  if (a.skip_done && !(a.t[k] < a.t_end)) return;
  const int np = min(P, n - s);
  const Real* U = static_cast<const Real*>(a.U) + a.inst_off[k] * M;
  const Real gam = pick<Real>(a.sp.wd, a.sp.wf)[9];
  const Real a01 = pick<Real>(a.sp.wd, a.sp.wf)[10];
  Real amax = Real(0);
  bool bad = false;
  for (int j = threadIdx.x; j < np; j += blockDim.x) {
    Real u[M];
#pragma unroll
    for (int c = 0; c < M; ++c) u[c] = U[(long long)c * n + s + j];
    const Real sp = wave_speed<EQ>(u, gam, a01);
    bad |= !(sp <= real_max<Real>());
    amax = fmax(amax, sp);
  }
  if (bad) atomicOr(a.status, STATUS_NONFINITE);
  amax = block_max_t(amax, red);
  if (threadIdx.x == 0)
    atomicMax(&a.alpha_out[k], (unsigned long long)__double_as_longlong((double)amax));
}

// Shared-memory layout of one tile of NT * PPT points (P = NT * PPT - 4
// updated points, two ghosts per side, P + 1 interfaces).
template <int EQ, class Real, int NT, int PPT>
struct Layout1D {
  static constexpr int M = Dim1<EQ>::M;
  static constexpr bool EUL = EQ == HWENO_EULER;
  static constexpr int P = NT * PPT - 4;
  static constexpr int NP = P + 4;
  static constexpr int NF = P + 1;
  static constexpr int NE = EUL ? 4 : 0;  // sqrt(rho), u, H, c^2
  static constexpr size_t bytes = sizeof(Real) * ((size_t)(6 * M + NE) * NP + 2 * M * NF);
};

// Resident CTAs requested per SM for a variant: the per-precision setting for
// 128-thread CTAs, scaled to the variant's thread count.
template <class Real, int NT>
struct MinBlocks1D {
  static constexpr int base = MinBlocks<Real, HWENO_MINB_1D_F64, HWENO_MINB_1D_F32>::value;
  static constexpr int value = base * 128 / NT > 0 ? base * 128 / NT : 1;
};

// The persistent kernel's register budget (FP32: its own setting; the work
// queue and stage bookkeeping need registers the tiled kernel does not). At
// 8 CTAs per SM (64 registers) the FP32 persistent kernel spilled 80 bytes;
// requesting 6 lets it use the factored projections in 71 registers, which
// still leaves 7 resident: +3% for the FP32 persistent run (measured 6383
// against 6193 M point-updates/s on the 2048-instance batch).
#ifndef HWENO_MINB_RUN_F32
#define HWENO_MINB_RUN_F32 6
#endif
template <class Real, int NT>
struct MinBlocksRun {
  static constexpr int base = MinBlocks<Real, HWENO_MINB_1D_F64, HWENO_MINB_RUN_F32>::value;
  static constexpr int value = base * 128 / NT > 0 ? base * 128 / NT : 1;
};

// The arrays one stage reads and writes (the rest of Args1D is shared by
// every stage of a step).
struct StageIO {
  const void* U;
  const void* V;
  const void* U0;
  const void* Vt0;
  void* Uout;
  void* Vout;
  void* Vt0out;
  const double* alpha_in;
  unsigned long long* alpha_out;
};

__device__ __forceinline__ StageIO io_of(const Args1D& a) {
  return StageIO{a.U, a.V, a.U0, a.Vt0, a.Uout, a.Vout, a.Vt0out, a.alpha_in, a.alpha_out};
}

// Point g of a tile starting at s (instance point s - 2 + g; ghosts by the
// boundary conditions): stores u, dx v (the limiter's scaled derivative),
// the split fluxes f^+-, H^+- (H = dx h) and, for Euler, sqrt(rho), u, H and
// c^2 in shared memory.
template <int EQ, class Real, class TV>
__device__ __forceinline__ void tile_point(const Args1D& a, const Real* U, const Real* V, int n,
                                           int s, int g, Real ha, Real hda, Real dx, Real hdx,
                                           Real gam,
                                           Real gm1,
                                           const TV& sU, const TV& sV, const TV& sFp,
                                           const TV& sFm, const TV& sHp, const TV& sHm,
                                           const TV& sE) {
  constexpr int M = Dim1<EQ>::M;
  int kind;
  const int src = map_1d(s - 2 + g, n, a.sp.bc[0], a.sp.bc[1], kind);
  HWENO_CHECK(kind == 2 || (src >= 0 && src < n), a.status);
  Real u[M], v[M];
#pragma unroll
  for (int c = 0; c < M; ++c) {
    if (kind == 2) {
      u[c] = pick<Real>(a.sp.inflow, a.sp.inflowf)[c];
      v[c] = Real(0);
    } else {
      u[c] = U[(long long)c * n + src];
      v[c] = V[(long long)c * n + src];
      if (kind == 1) { const Real sg = Real(refl_sign<EQ>(c)); u[c] *= sg; v[c] *= -sg; }
    }
    sU[c][g] = u[c];
    sV[c][g] = dx * v[c];
  }
  Real F[M], H[M];
  if constexpr (EQ == HWENO_BURGERS) {
    F[0] = Real(0.5) * u[0] * u[0];
    H[0] = u[0] * v[0];
  } else if constexpr (EQ == HWENO_BUCKLEY) {
    Real df;
    buckley_f(u[0], F[0], df);
    H[0] = df * v[0];
  } else {
    // 1/rho and sqrt(rho) from one reciprocal square root
    const Real rr = rsq(u[0]);
    const Real ir = rr * rr;
    const Real vel = u[1] * ir;
    const Real p = gm1 * (u[2] - Real(0.5) * u[1] * vel);
    const Real Ep = u[2] + p;
    F[0] = u[1];
    F[1] = u[1] * vel + p;
    F[2] = Ep * vel;
    const Real dvel = (v[1] - vel * v[0]) * ir;
    const Real dp = gm1 * (v[2] - vel * v[1] + Real(0.5) * vel * vel * v[0]);
    H[0] = v[1];
    H[1] = v[1] * vel + u[1] * dvel + dp;
    H[2] = (v[2] + dp) * vel + Ep * dvel;
    sE[0][g] = u[0] * rr;
    sE[1][g] = vel;
    sE[2][g] = Ep * ir;
    sE[3][g] = gam * p * ir;
  }
#pragma unroll
  for (int c = 0; c < M; ++c)
    split_pm(F[c], u[c], H[c], v[c], ha, hda, hdx, sFp[c][g], sFm[c][g], sHp[c][g], sHm[c][g]);
}

// The limited derivative v~ at loaded point g (Sec. 2.2): v unchanged with
// the limiter off, component-wise, or (Euler) on the characteristic fields
// of the eigenvectors at U_g.
// Factored characteristic projections (Char1) in the tiled stage and
// persistent kernels in FP64 and in the FP32 persistent kernel; the FP32
// tiled kernel, capped at 64 registers, and the 124-point cluster step keep
// the rows of L applied one by one (the factored form's larger live set
// spills there).
template <class Real>
constexpr bool kFactored = std::is_same<Real, double>::value;
#ifndef HWENO_FAC_RUN_F32
#define HWENO_FAC_RUN_F32 1
#endif
template <class Real>
constexpr bool kFactoredRun = kFactored<Real> || HWENO_FAC_RUN_F32;

template <int EQ, class Real, class TV, bool FAC = true>
__device__ __forceinline__ void limited_point(const Args1D& a, int g, Real idx, Real gm1,
                                              const Weights<Real>& w, const TV& sU,
                                              const TV& sV, const TV& sE, Real* vt) {
  constexpr int M = Dim1<EQ>::M;
  constexpr bool EUL = EQ == HWENO_EULER;
  if (a.sp.limiter == 0) {
#pragma unroll
    for (int c = 0; c < M; ++c) vt[c] = sV[c][g] * idx;
  } else if (!EUL || a.sp.limiter == 2) {
#pragma unroll
    for (int c = 0; c < M; ++c)
      vt[c] = limited_derivative(sU[c][g - 1], sU[c][g], sU[c][g + 1], sV[c][g - 1],
                                 sV[c][g + 1], w) * idx;
  } else if constexpr (EUL && !FAC) {  // the rows of L applied one by one
    Real cg, icg;
    sound_speed(sE[3][g], cg, icg);
    Eigen<Real, 3> e;
    euler_eigen<Real, 3>(0, sE[1][g], Real(0), sE[2][g], cg, icg, gm1, e);
    Frac<Real> zr[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const Real l0 = e.L[q][0], l1q = e.L[q][1], l2q = e.L[q][2];
      auto pj = [&](const TV& A, int gg) { return l0 * A[0][gg] + l1q * A[1][gg] + l2q * A[2][gg]; };
      zr[q] = limited_derivative_frac(pj(sU, g - 1), pj(sU, g), pj(sU, g + 1),
                                      pj(sV, g - 1), pj(sV, g + 1), w);
    }
    Real z[3];
    resolve3(zr[0], zr[1], zr[2], z[0], z[1], z[2]);
#pragma unroll
    for (int c = 0; c < 3; ++c)
      vt[c] = (e.R[c][0] * z[0] + e.R[c][1] * z[1] + e.R[c][2] * z[2]) * idx;
  } else if constexpr (EUL) {  // factored projections (Char1)
    Real cg, icg;
    sound_speed(sE[3][g], cg, icg);
    const Char1<Real> ch(sE[1][g], sE[2][g], cg, icg, gm1);
    // the five projected vectors (u at g-1, g, g+1; dx v at g-1, g+1) as
    // (x0, A, B); each field's projection is then one operation
    Real x0[5], fa[5], fb[5];
    auto fac = [&](int k, const TV& X, int gg) {
      x0[k] = X[0][gg];
      ch.factors(X[0][gg], X[1][gg], X[2][gg], fa[k], fb[k]);
    };
    fac(0, sU, g - 1); fac(1, sU, g); fac(2, sU, g + 1); fac(3, sV, g - 1); fac(4, sV, g + 1);
    Frac<Real> zr[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      auto pj = [&](int k) { return ch.row(q, x0[k], fa[k], fb[k]); };
      zr[q] = limited_derivative_frac(pj(0), pj(1), pj(2), pj(3), pj(4), w);
    }
    Real z[3];
    resolve3(zr[0], zr[1], zr[2], z[0], z[1], z[2]);
    ch.right(z, vt);
#pragma unroll
    for (int c = 0; c < 3; ++c) vt[c] *= idx;
  }
}

// Factors of the SSP-RK3 combination of a stage: x_out = a x0 + b (x + dt L)
// with L^1 = -dF / dx, L^2 = -dD / dx^2 (dF, dD the flux differences), so
// x_out = a x0 + b x + k dF with k1 = -b dt / dx for U, k2 = -b dt / dx^2
// for V (one FMA per component on the difference; the same expression in
// exact arithmetic).
template <class Real, int MODE>
struct RKFactors {
  Real b, k1, k2;
  __device__ __forceinline__ RKFactors(Real rdt, Real idx, Real idx2) {
    b = MODE == MODE_STAGE1 ? Real(1) : MODE == MODE_STAGE2 ? Real(0.25) : Real(2.0 / 3.0);
    k1 = -(b * rdt) * idx;
    k2 = -(b * rdt) * idx2;
  }
};

// The SSP-RK3 combination of one stage at instance point q (component
// stride n) from the stage input u, the flux differences dF, dD and v~:
// writes U, V of the stage output (stage 1 also v~^n) and returns U in un.
template <int EQ, class Real, int MODE>
__device__ __forceinline__ void stage_update(const StageIO& io, long long base, long long n,
                                             const Real* u, const Real* dF, const Real* dD,
                                             const Real* vt, const RKFactors<Real, MODE>& f,
                                             Real* un) {
  constexpr int M = Dim1<EQ>::M;
#pragma unroll
  for (int c = 0; c < M; ++c) {
    const long long q = base + (long long)c * n;
    Real vn;
    if constexpr (MODE == MODE_STAGE1) {
      un[c] = u[c] + f.k1 * dF[c];
      vn = vt[c] + f.k2 * dD[c];
      static_cast<Real*>(io.Vt0out)[q] = vt[c];
    } else if constexpr (MODE == MODE_STAGE2) {
      const Real u0 = static_cast<const Real*>(io.U0)[q];
      const Real v0 = static_cast<const Real*>(io.Vt0)[q];
      un[c] = (Real(0.75) * u0 + Real(0.25) * u[c]) + f.k1 * dF[c];
      vn = (Real(0.75) * v0 + Real(0.25) * vt[c]) + f.k2 * dD[c];
    } else {
      const Real u0 = static_cast<const Real*>(io.U0)[q];
      const Real v0 = static_cast<const Real*>(io.Vt0)[q];
      un[c] = (Real(1.0 / 3.0) * u0 + Real(2.0 / 3.0) * u[c]) + f.k1 * dF[c];
      vn = (Real(1.0 / 3.0) * v0 + Real(2.0 / 3.0) * vt[c]) + f.k2 * dD[c];
    }
    static_cast<Real*>(io.Uout)[q] = un[c];
    static_cast<Real*>(io.Vout)[q] = vn;
  }
}

// One stage on the tile of instance k starting at point s (the whole CTA;
// contains barriers, so every thread calls it with the same k, s).
template <int EQ, class Real, int MODE, int NT, int PPT, bool FAC = false>
__device__ __forceinline__ void stage_tile(const Args1D& a, const StageIO& io, const int k,
                                           const int s) {
  using Lay = Layout1D<EQ, Real, NT, PPT>;
  constexpr int M = Lay::M;
  constexpr int NP = Lay::NP;
  constexpr int NF = Lay::NF;
  constexpr bool EUL = Lay::EUL;
  extern __shared__ __align__(16) unsigned char smem1d[];
  Real* base = reinterpret_cast<Real*>(smem1d);
  unsigned* const st = a.status;
  const auto sU = tile_view<NP>(base, M, st);
  const auto sV = tile_view<NP>(base + 1 * M * NP, M, st);
  const auto sFp = tile_view<NP>(base + 2 * M * NP, M, st);
  const auto sFm = tile_view<NP>(base + 3 * M * NP, M, st);
  const auto sHp = tile_view<NP>(base + 4 * M * NP, M, st);
  const auto sHm = tile_view<NP>(base + 5 * M * NP, M, st);
  const auto sE = tile_view<NP>(base + 6 * M * NP, Lay::NE, st);
  const auto sF = tile_view<NF>(base + (6 * M + Lay::NE) * NP, M, st);
  const auto sD = tile_view<NF>(base + (6 * M + Lay::NE) * NP + M * NF, M, st);
  using TV = std::remove_const_t<decltype(sU)>;
  __shared__ Real red[NT / 32];
  __shared__ double s_dt;

  const int n = a.inst_n[k];
  if (a.skip_done && !(a.t[k] < a.t_end)) return;
  const int np = min(Lay::P, n - s);
  HWENO_CHECK(s >= 0 && np >= 1, st);
  const long long off = a.inst_off[k] * M;
  const Real* geo = pick<Real>(a.inst_geo, a.inst_geof) + 3 * k;
  const Real dx = geo[0], idx = geo[1], idx2 = geo[2];
  const Real alpha = Real(io.alpha_in[k]);
  const Real gam = pick<Real>(a.sp.wd, a.sp.wf)[9];
  const Real gm1 = gam - Real(1);
  const Weights<Real> w = weights_from(pick<Real>(a.sp.wd, a.sp.wf));

  // time step: once per CTA (thread 0), read back after the barriers below
  if (threadIdx.x == 0) {
    double dt = 0.0;
    if constexpr (MODE == MODE_STAGE1) {
      int lands = 0;
      dt = a.dt_in ? a.dt_in[k]
                   : time_step(a.sp, io.alpha_in[k], a.inst_hx[k], a.t[k], a.t_end, lands);
      if (s == 0) { a.dt[k] = dt; a.lands[k] = lands; }
    } else if constexpr (MODE != MODE_RHS) {
      dt = a.dt[k];
    }
    s_dt = dt;
  }

  // 1-2: tile load with ghosts; point fluxes and splitting
  {
    const Real* U = static_cast<const Real*>(io.U) + off;
    const Real* V = static_cast<const Real*>(io.V) + off;
    const Real hdx = Real(0.5) * dx;
    const Real ha = Real(0.5) * alpha, hda = hdx * alpha;
    for (int g = threadIdx.x; g < np + 4; g += blockDim.x)
      tile_point<EQ, Real, TV>(a, U, V, n, s, g, ha, hda, dx, hdx, gam, gm1, sU, sV, sFp, sFm,
                               sHp, sHm, sE);
  }
  __syncthreads();

  // 3: interfaces x_{s+j-1/2}, j = 0..np; left point at shared index j + 1
  for (int j = threadIdx.x; j <= np; j += blockDim.x) {
    const int gl = j + 1;
    if constexpr (!EUL) {
      sF[0][j] = interface_flux(sFp[0][gl - 1], sFp[0][gl], sFp[0][gl + 1], sHp[0][gl - 1],
                                sHp[0][gl], sHp[0][gl + 1], sFm[0][gl], sFm[0][gl + 1],
                                sFm[0][gl + 2], sHm[0][gl], sHm[0][gl + 1], sHm[0][gl + 2], w);
    } else {
      Real uu, HH, cc;
      if (a.sp.eig_avg == 0) {  // Roe average of U_i, U_{i+1}
        const Real sl = sE[0][gl], sr = sE[0][gl + 1];
        const Real is = recip(sl + sr);
        uu = (sl * sE[1][gl] + sr * sE[1][gl + 1]) * is;
        HH = (sl * sE[2][gl] + sr * sE[2][gl + 1]) * is;
      } else {  // arithmetic mean state
        const Real r = Real(0.5) * (sU[0][gl] + sU[0][gl + 1]);
        const Real mo = Real(0.5) * (sU[1][gl] + sU[1][gl + 1]);
        const Real E = Real(0.5) * (sU[2][gl] + sU[2][gl + 1]);
        const Real ir = Real(1) / r;
        uu = mo * ir;
        HH = (E + gm1 * (E - Real(0.5) * mo * uu)) * ir;
      }
      Real ic;
      sound_speed(gm1 * (HH - Real(0.5) * uu * uu), cc, ic);
      if constexpr (!FAC) {  // the rows of L applied one by one
      Eigen<Real, 3> e;
      euler_eigen<Real, 3>(0, uu, Real(0), HH, cc, ic, gm1, e);
      Frac<Real> fr[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const Real l0 = e.L[q][0], l1 = e.L[q][1], l2 = e.L[q][2];
        auto pj = [&](const TV& A, int g) { return l0 * A[0][g] + l1 * A[1][g] + l2 * A[2][g]; };
        fr[q] = interface_flux_frac(pj(sFp, gl - 1), pj(sFp, gl), pj(sFp, gl + 1),
                                    pj(sHp, gl - 1), pj(sHp, gl), pj(sHp, gl + 1),
                                    pj(sFm, gl), pj(sFm, gl + 1), pj(sFm, gl + 2),
                                    pj(sHm, gl), pj(sHm, gl + 1), pj(sHm, gl + 2), w);
      }
      Real f[3];
      resolve3(fr[0], fr[1], fr[2], f[0], f[1], f[2]);
#pragma unroll
      for (int c = 0; c < 3; ++c)
        sF[c][j] = e.R[c][0] * f[0] + e.R[c][1] * f[1] + e.R[c][2] * f[2];
      } else {
      const Char1<Real> ch(uu, HH, cc, ic, gm1);
      // the twelve projected vectors (f^+, H^+ at gl-1..gl+1; f^-, H^- at
      // gl..gl+2) as (x0, A, B); each field's projection is one operation
      Real x0[12], fa[12], fb[12];
      auto fac = [&](int k, const TV& X, int g) {
        x0[k] = X[0][g];
        ch.factors(X[0][g], X[1][g], X[2][g], fa[k], fb[k]);
      };
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        fac(d, sFp, gl - 1 + d);
        fac(3 + d, sHp, gl - 1 + d);
        fac(6 + d, sFm, gl + d);
        fac(9 + d, sHm, gl + d);
      }
      Frac<Real> fr[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        auto pj = [&](int k) { return ch.row(q, x0[k], fa[k], fb[k]); };
        fr[q] = interface_flux_frac(pj(0), pj(1), pj(2), pj(3), pj(4), pj(5), pj(6), pj(7),
                                    pj(8), pj(9), pj(10), pj(11), w);
      }
      Real f[3], out[3];
      resolve3(fr[0], fr[1], fr[2], f[0], f[1], f[2]);
      ch.right(f, out);
#pragma unroll
      for (int c = 0; c < 3; ++c) sF[c][j] = out[c];
      }
    }
#pragma unroll
    for (int c = 0; c < M; ++c)
      sD[c][j] = derivative_flux(sFp[c][gl - 1], sFp[c][gl], sFp[c][gl + 1], sHp[c][gl - 1],
                                 sHp[c][gl], sHp[c][gl + 1], sFm[c][gl], sFm[c][gl + 1],
                                 sFm[c][gl + 2], sHm[c][gl], sHm[c][gl + 1], sHm[c][gl + 2]);
  }
  __syncthreads();

  // 4: points
  const RKFactors<Real, MODE> rk(Real(s_dt), idx, idx2);
  const bool want_alpha = MODE != MODE_RHS && io.alpha_out != nullptr;  // uniform
  Real amax = Real(0);
  bool bad = false;
  for (int j = threadIdx.x; j < np; j += blockDim.x) {
    const int g = j + 2;
    Real dF[M], dD[M], vt[M];
#pragma unroll
    for (int c = 0; c < M; ++c) {
      dF[c] = sF[c][j + 1] - sF[c][j];
      dD[c] = sD[c][j + 1] - sD[c][j];
    }
    limited_point<EQ, Real, TV, FAC>(a, g, idx, gm1, w, sU, sV, sE, vt);

    HWENO_CHECK(s + j < n, st);
    const long long base = off + s + j;
    if constexpr (MODE == MODE_RHS) {
#pragma unroll
      for (int c = 0; c < M; ++c) {
        static_cast<Real*>(a.L1)[base + (long long)c * n] = -dF[c] * idx;
        static_cast<Real*>(a.L2)[base + (long long)c * n] = -dD[c] * idx2;
        if (a.Vlim) static_cast<Real*>(a.Vlim)[base + (long long)c * n] = vt[c];
      }
    } else {
      Real u[M], un[M];
#pragma unroll
      for (int c = 0; c < M; ++c) u[c] = sU[c][g];
      stage_update<EQ, Real, MODE>(io, base, n, u, dF, dD, vt, rk, un);
      if (want_alpha) {
        const Real sp = wave_speed<EQ>(un, gam, pick<Real>(a.sp.wd, a.sp.wf)[10]);
        bad |= !(sp <= real_max<Real>());
        amax = fmax(amax, sp);
      }
    }
  }
  // the wave speed of the stage output (stages 1 and 2; stage 3 as well when
  // the persistent run asks for the next step's alpha)
  if (want_alpha) {
    if (bad) atomicOr(a.status, STATUS_NONFINITE);
    amax = block_max_t(amax, red);
    if (threadIdx.x == 0)
      atomicMax(&io.alpha_out[k], (unsigned long long)__double_as_longlong((double)amax));
  }
}

template <int EQ, class Real, int MODE, int NT, int PPT>
__global__ void __launch_bounds__(NT, (MinBlocks1D<Real, NT>::value))
k_stage_1d(const __grid_constant__ Args1D a) {
  stage_tile<EQ, Real, MODE, NT, PPT, kFactored<Real>>(a, io_of(a), a.tile_inst[blockIdx.x],
                                      a.tile_start[blockIdx.x]);
}

template <int EQ, class Real, int MODE, int NT, int PPT>
cudaError_t stage_launch(const Args1D& a, int ntiles, cudaStream_t s) {
  constexpr size_t bytes = Layout1D<EQ, Real, NT, PPT>::bytes;
  static unsigned configured = 0;  // devices whose limit is raised
  if (const cudaError_t e = ensure_smem_limit(k_stage_1d<EQ, Real, MODE, NT, PPT>, bytes, configured)) return e;
  k_stage_1d<EQ, Real, MODE, NT, PPT><<<ntiles, NT, bytes, s>>>(a);
  return cudaGetLastError();
}

template <int EQ, class Real, int NT, int PPT>
cudaError_t stage_modes(int mode, const Args1D& a, int ntiles, cudaStream_t s) {
  switch (mode) {
    case MODE_RHS: return stage_launch<EQ, Real, MODE_RHS, NT, PPT>(a, ntiles, s);
    case MODE_STAGE1: return stage_launch<EQ, Real, MODE_STAGE1, NT, PPT>(a, ntiles, s);
    case MODE_STAGE2: return stage_launch<EQ, Real, MODE_STAGE2, NT, PPT>(a, ntiles, s);
    default: return stage_launch<EQ, Real, MODE_STAGE3, NT, PPT>(a, ntiles, s);
  }
}

// Variants of kVariants1D: (threads, points per thread).
template <int EQ, class Real>
cudaError_t stage_variants(int variant, int mode, const Args1D& a, int ntiles, cudaStream_t s) {
  switch (variant) {
    case 1: return stage_modes<EQ, Real, 64, 1>(mode, a, ntiles, s);
    case 2: return stage_modes<EQ, Real, 256, 1>(mode, a, ntiles, s);
    case 3: return stage_modes<EQ, Real, 128, 2>(mode, a, ntiles, s);
    case 4: return stage_modes<EQ, Real, 64, 2>(mode, a, ntiles, s);
    default: return stage_modes<EQ, Real, 128, 1>(mode, a, ntiles, s);
  }
}

template <int EQ, class Real>
cudaError_t alpha_variants(int variant, const Args1D& a, int ntiles, cudaStream_t s) {
  switch (tile_points(variant)) {
    case 60: k_alpha_1d<EQ, Real, 60><<<ntiles, kThreads1D, 0, s>>>(a); break;
    case 252: k_alpha_1d<EQ, Real, 252><<<ntiles, kThreads1D, 0, s>>>(a); break;
    default: k_alpha_1d<EQ, Real, 124><<<ntiles, kThreads1D, 0, s>>>(a); break;
  }
  return cudaGetLastError();
}

template <class Real>
cudaError_t stage_prec(int eq, int variant, int mode, const Args1D& a, int ntiles, cudaStream_t s) {
  return eq == HWENO_BURGERS ? stage_variants<HWENO_BURGERS, Real>(variant, mode, a, ntiles, s)
                             : stage_variants<HWENO_EULER, Real>(variant, mode, a, ntiles, s);
}

template <class Real>
cudaError_t alpha_prec(int eq, int variant, const Args1D& a, int ntiles, cudaStream_t s) {
  return eq == HWENO_BURGERS ? alpha_variants<HWENO_BURGERS, Real>(variant, a, ntiles, s)
                             : alpha_variants<HWENO_EULER, Real>(variant, a, ntiles, s);
}


// ---------------------------------------------------------------------------
// Persistent run (PersistArgs): whole steps of a ragged batch in one launch.
// ---------------------------------------------------------------------------

// Bounded wait until *ctr >= target (acquire at device scope, so that the
// loads after the CTA barrier see the other CTAs' stores). Gives up after
// about two seconds, or as soon as another CTA has given up, and then sets
// STATUS_TIMEOUT.
__device__ __forceinline__ bool wait_count(unsigned* ctr, unsigned target, unsigned* status) {
  cuda::atomic_ref<unsigned, cuda::thread_scope_device> c(*ctr);
  cuda::atomic_ref<unsigned, cuda::thread_scope_device> st(*status);
  unsigned ns = 32;
  for (int it = 0; it < (1 << 23); ++it) {
    if (c.load(cuda::memory_order_acquire) >= target) return true;
    if (st.load(cuda::memory_order_relaxed) & STATUS_TIMEOUT) return false;
    __nanosleep(ns);
    if (ns < 256) ns <<= 1;
  }
  atomicOr(status, STATUS_TIMEOUT);
  return false;
}

__device__ __forceinline__ void release_add(unsigned* ctr, unsigned v) {
  cuda::atomic_ref<unsigned, cuda::thread_scope_device> c(*ctr);
  c.fetch_add(v, cuda::memory_order_release);
}

// Tickets t = (step n, stage, tile b) in lexicographic order. A tile of
// instance k in stage `stage` of step n needs all (3n + stage) * tiles(k)
// earlier tiles of k to be complete; they hold smaller tickets, so the CTAs
// that took them are resident: the waits always end. The last stage-3 tile of
// k does the time update (as k_finalize), clears the alpha slots the step
// after next accumulates into, and releases step n + 1 of k.
template <int EQ, class Real, int NT, int PPT>
__global__ void __launch_bounds__(NT, (MinBlocksRun<Real, NT>::value))
k_run_1d(const __grid_constant__ Args1D a, const __grid_constant__ PersistArgs p) {
  __shared__ long long s_ticket;
  __shared__ int s_stop, s_gave_up;
  const long long per_step = 3LL * p.ntiles;
  const long long total = per_step * p.steps;
  for (;;) {
    if (threadIdx.x == 0) {
      s_ticket = (long long)atomicAdd(p.next, 1ULL);
      cuda::atomic_ref<unsigned, cuda::thread_scope_device> st(*a.status);
      s_stop = (st.load(cuda::memory_order_relaxed) & STATUS_TIMEOUT) != 0;
    }
    __syncthreads();  // also separates this tile's shared-memory use from the last one's
    const long long tk = s_ticket;
    if (tk >= total || s_stop) break;
    const int n = (int)(tk / per_step);
    const int r = (int)(tk - (long long)n * per_step);
    const int stage = r / p.ntiles;
    const int b = r - stage * p.ntiles;
    const int k = a.tile_inst[b], s = a.tile_start[b];
    HWENO_CHECK(k >= 0 && k < p.batch, a.status);
    const unsigned ntk = (unsigned)p.inst_tiles[k];
    if (threadIdx.x == 0) {
      const unsigned need = (unsigned)(3 * n + stage) * ntk + (k == 0 ? p.wait_extra : 0u);
      s_gave_up = !wait_count(&p.done[k], need, a.status);
    }
    __syncthreads();
    if (s_gave_up) break;  // this tile's inputs are not ready: leave it untouched
    const int par = n & 1;
    unsigned long long* slot0 = p.alpha + (size_t)(par * 3) * p.batch;  // this step's slots
    StageIO io = io_of(a);
    if (stage == 0) {
      io.Uout = p.U1; io.Vout = p.V1; io.Vt0out = p.Vt0;
      io.alpha_in = reinterpret_cast<const double*>(slot0);
      io.alpha_out = slot0 + p.batch;
      stage_tile<EQ, Real, MODE_STAGE1, NT, PPT, kFactoredRun<Real>>(a, io, k, s);
    } else if (stage == 1) {
      io.U = p.U1; io.V = p.V1; io.U0 = a.U; io.Vt0 = p.Vt0;
      io.Uout = p.U2; io.Vout = p.V2; io.Vt0out = nullptr;
      io.alpha_in = reinterpret_cast<const double*>(slot0 + p.batch);
      io.alpha_out = slot0 + 2 * p.batch;
      stage_tile<EQ, Real, MODE_STAGE2, NT, PPT, kFactoredRun<Real>>(a, io, k, s);
    } else {
      io.U = p.U2; io.V = p.V2; io.U0 = a.U; io.Vt0 = p.Vt0;
      io.Uout = const_cast<void*>(a.U); io.Vout = const_cast<void*>(a.V); io.Vt0out = nullptr;
      io.alpha_in = reinterpret_cast<const double*>(slot0 + 2 * p.batch);
      io.alpha_out = p.alpha + (size_t)((par ^ 1) * 3) * p.batch;  // alpha(U^{n+1})
      stage_tile<EQ, Real, MODE_STAGE3, NT, PPT, kFactoredRun<Real>>(a, io, k, s);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      if (stage < 2) {
        release_add(&p.done[k], 1u);
      } else if (atomicAdd(&p.done3[k], 1u) + 1u == ntk) {
        // time update of instance k (as k_finalize)
        double tk_ = a.t[k];
        if (tk_ < a.t_end) {
          const double d = a.dt[k];
          tk_ = a.lands[k] ? a.t_end : tk_ + d;
          const_cast<double*>(a.t)[k] = tk_;
          const double al = __longlong_as_double((long long)slot0[k]);
          if (!(al <= DBL_MAX)) atomicOr(a.status, STATUS_NONFINITE);
          if (p.pu) atomicAdd(p.pu, (unsigned long long)a.inst_n[k]);
        }
        if (n == p.steps - 1 && tk_ < a.t_end) atomicAdd(p.active, 1);
        p.done3[k] = 0u;
        slot0[k] = 0ull;                 // accumulated again by stage 3 of step n + 1
        slot0[p.batch + k] = 0ull;       // and by stages 1, 2 of step n + 2
        slot0[2 * p.batch + k] = 0ull;
        __threadfence();
        release_add(&p.done[k], ntk);
      }
    }
  }
}

template <int EQ, class Real, int NT, int PPT>
cudaError_t run_launch(const Args1D& a, const PersistArgs& p, int ctas, cudaStream_t s) {
  constexpr size_t bytes = Layout1D<EQ, Real, NT, PPT>::bytes;
  static unsigned configured = 0;  // devices whose limit is raised
  if (const cudaError_t e = ensure_smem_limit(k_run_1d<EQ, Real, NT, PPT>, bytes, configured)) return e;
  k_run_1d<EQ, Real, NT, PPT><<<ctas, NT, bytes, s>>>(a, p);
  return cudaGetLastError();
}

template <int EQ, class Real, int NT, int PPT>
int run_occupancy() {
  constexpr size_t bytes = Layout1D<EQ, Real, NT, PPT>::bytes;
  if (cudaFuncSetAttribute(k_run_1d<EQ, Real, NT, PPT>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_run_1d<EQ, Real, NT, PPT>, NT,
                                                    bytes) != cudaSuccess)
    return 0;
  return nb;
}

template <int EQ, class Real>
cudaError_t run_variants(int variant, const Args1D& a, const PersistArgs& p, int ctas,
                         cudaStream_t s) {
  switch (variant) {
    case 1: return run_launch<EQ, Real, 64, 1>(a, p, ctas, s);
    case 2: return run_launch<EQ, Real, 256, 1>(a, p, ctas, s);
    case 3: return run_launch<EQ, Real, 128, 2>(a, p, ctas, s);
    case 4: return run_launch<EQ, Real, 64, 2>(a, p, ctas, s);
    default: return run_launch<EQ, Real, 128, 1>(a, p, ctas, s);
  }
}

template <int EQ, class Real>
int occupancy_variants(int variant) {
  switch (variant) {
    case 1: return run_occupancy<EQ, Real, 64, 1>();
    case 2: return run_occupancy<EQ, Real, 256, 1>();
    case 3: return run_occupancy<EQ, Real, 128, 2>();
    case 4: return run_occupancy<EQ, Real, 64, 2>();
    default: return run_occupancy<EQ, Real, 128, 1>();
  }
}

template <class Real>
cudaError_t run_prec(int eq, int variant, const Args1D& a, const PersistArgs& p, int ctas,
                     cudaStream_t s) {
  return eq == HWENO_BURGERS ? run_variants<HWENO_BURGERS, Real>(variant, a, p, ctas, s)
                             : run_variants<HWENO_EULER, Real>(variant, a, p, ctas, s);
}

template <class Real>
int occupancy_prec(int eq, int variant) {
  return eq == HWENO_BURGERS ? occupancy_variants<HWENO_BURGERS, Real>(variant)
                             : occupancy_variants<HWENO_EULER, Real>(variant);
}


// ---------------------------------------------------------------------------
// Fused step of small instances (FusedArgs): one CTA per instance.
// ---------------------------------------------------------------------------
template <int EQ, class Real>
__global__ void __launch_bounds__(kFusedThreads)
k_step_small_1d(const __grid_constant__ Args1D a, const __grid_constant__ FusedArgs f) {
  constexpr int M = Dim1<EQ>::M;
  __shared__ Real red[kFusedThreads / 32];
  const int k = blockIdx.x;
  const int n = a.inst_n[k];
  unsigned long long* s0 = f.alpha;
  unsigned long long* s1 = f.alpha + f.batch;
  unsigned long long* s2 = f.alpha + 2 * f.batch;
  if (!(a.t[k] < a.t_end)) {  // finished: nothing moves (as k_finalize)
    if (threadIdx.x == 0 && f.dt_used) f.dt_used[k] = 0.0;
    return;
  }
  // alpha(U^n) over the instance; the stage slots start from zero
  {
    const Real* U = static_cast<const Real*>(a.U) + a.inst_off[k] * M;
    const Real gam = pick<Real>(a.sp.wd, a.sp.wf)[9];
    const Real a01 = pick<Real>(a.sp.wd, a.sp.wf)[10];
    Real amax = Real(0);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      Real u[M];
#pragma unroll
      for (int c = 0; c < M; ++c) u[c] = U[(long long)c * n + j];
      amax = fmax(amax, wave_speed<EQ>(u, gam, a01));
    }
    amax = block_max_t(amax, red);
    if (threadIdx.x == 0) {
      s0[k] = (unsigned long long)__double_as_longlong((double)amax);
      s1[k] = 0ull;
      s2[k] = 0ull;
    }
    __syncthreads();
  }
  StageIO io = io_of(a);
  io.Uout = f.U1; io.Vout = f.V1; io.Vt0out = f.Vt0;
  io.alpha_in = reinterpret_cast<const double*>(s0); io.alpha_out = s1;
  stage_tile<EQ, Real, MODE_STAGE1, kFusedThreads, kFusedPPT>(a, io, k, 0);
  __syncthreads();
  io.U = f.U1; io.V = f.V1; io.U0 = a.U; io.Vt0 = f.Vt0; io.Uout = f.U2; io.Vout = f.V2;
  io.Vt0out = nullptr;
  io.alpha_in = reinterpret_cast<const double*>(s1); io.alpha_out = s2;
  stage_tile<EQ, Real, MODE_STAGE2, kFusedThreads, kFusedPPT>(a, io, k, 0);
  __syncthreads();
  io.U = f.U2; io.V = f.V2; io.Uout = const_cast<void*>(a.U); io.Vout = const_cast<void*>(a.V);
  io.alpha_in = reinterpret_cast<const double*>(s2); io.alpha_out = nullptr;
  stage_tile<EQ, Real, MODE_STAGE3, kFusedThreads, kFusedPPT>(a, io, k, 0);
  __syncthreads();
  if (threadIdx.x == 0) {  // time update (as k_finalize)
    double tk = a.t[k];
    const double d = a.dt[k];
    tk = a.lands[k] ? a.t_end : tk + d;
    const_cast<double*>(a.t)[k] = tk;
    if (!(__longlong_as_double((long long)s0[k]) <= DBL_MAX)) atomicOr(a.status, STATUS_NONFINITE);
    if (f.pu) atomicAdd(f.pu, (unsigned long long)n);
    if (f.dt_used) f.dt_used[k] = d;
    if (tk < a.t_end) atomicAdd(f.active, 1);
  }
}

template <int EQ, class Real>
cudaError_t step_small_launch(const Args1D& a, const FusedArgs& f, cudaStream_t s) {
  constexpr size_t bytes = Layout1D<EQ, Real, kFusedThreads, kFusedPPT>::bytes;
  static unsigned configured = 0;  // devices whose limit is raised
  if (const cudaError_t e = ensure_smem_limit(k_step_small_1d<EQ, Real>, bytes, configured)) return e;
  k_step_small_1d<EQ, Real><<<f.batch, kFusedThreads, bytes, s>>>(a, f);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Latency form of one stage for the cluster step: a kSplitTile-point tile
// (32 loaded points, one per lane) on four warps, which sit on the SM's four
// sub-partitions. The FP64 cost of a warp instruction does not depend on
// how many lanes are active, so a stage's time is set by the longest
// instruction stream of one warp; here the work of a point is divided over
// the warps instead of the points: warp 0 the "+" reconstructions of the
// interfaces, warp 1 the "-" ones, warp 2 the limiter, warp 3 the derivative
// fluxes; warp 0 then combines the sides and updates the points.
// ---------------------------------------------------------------------------
template <int EQ, class Real>
struct SplitLayout {
  static constexpr int M = Dim1<EQ>::M;
  static constexpr int P = kSplitTile;
  static constexpr int NP = P + 4;  // loaded points s-2 .. s+P+1
  static constexpr int NF = P + 1;  // interfaces
  static constexpr int NE = EQ == HWENO_EULER ? 4 : 0;
  // sU, sV, sFp, sFm, sHp, sHm [M][NP]; sE [NE][NP]; side numerators and
  // denominators [2][M][NF] each; sD, sF [M][NF]; sVt [M][P]
  static constexpr size_t bytes =
      sizeof(Real) * ((size_t)(6 * M + NE) * NP + (size_t)6 * M * NF + (size_t)M * P);
};
static_assert(kSplitTile + 4 == 32, "one loaded point per lane");

// One side of an interface flux as a deferred quotient: sd = 0 the "+"
// reconstruction from f^+, H^+ at i-1, i, i+1; sd = 1 the "-" one from
// f^-, H^- at i, i+1, i+2 (the mirror image: reversed, H negated).
template <class Real>
__device__ __forceinline__ Frac<Real> side_frac(int sd, Real f0, Real f1, Real f2, Real H0,
                                               Real H1, Real H2, const Weights<Real>& w) {
  const Cand<Real> c = candidates(sd ? f2 : f0, f1, sd ? f0 : f2, sd ? -H2 : H0, sd ? -H1 : H1,
                                  sd ? -H0 : H2, w);
  if constexpr (std::is_same<Real, double>::value) {
    Real n, d;
    combine_nd(c, w, n, d);
    return Frac<Real>{n, d};
  } else {
    return Frac<Real>{combine_direct(c, w), Real(1)};
  }
}

// The two sides of one field summed as in interface_flux_frac.
template <class Real>
__device__ __forceinline__ Frac<Real> sides_sum(Real na, Real da, Real nb, Real db) {
  return sum_frac(na, da, nb, db);
}

template <int EQ, class Real, int MODE>
__device__ __forceinline__ void stage_tile_split(const Args1D& a, const StageIO& io, const int k,
                                                 const int s, const double alpha_in,
                                                 const double dt, double* part_out) {
  using Lay = SplitLayout<EQ, Real>;
  constexpr int M = Lay::M;
  constexpr int NP = Lay::NP;
  constexpr int NF = Lay::NF;
  constexpr int P = Lay::P;
  constexpr bool EUL = EQ == HWENO_EULER;
  extern __shared__ __align__(16) unsigned char smem1d[];
  Real* base = reinterpret_cast<Real*>(smem1d);
  unsigned* const st = a.status;
  const auto sU = tile_view<NP>(base, M, st);
  const auto sV = tile_view<NP>(base + 1 * M * NP, M, st);
  const auto sFp = tile_view<NP>(base + 2 * M * NP, M, st);
  const auto sFm = tile_view<NP>(base + 3 * M * NP, M, st);
  const auto sHp = tile_view<NP>(base + 4 * M * NP, M, st);
  const auto sHm = tile_view<NP>(base + 5 * M * NP, M, st);
  const auto sE = tile_view<NP>(base + 6 * M * NP, Lay::NE, st);
  using TV = std::remove_const_t<decltype(sU)>;
  Real* const sides = base + (6 * M + Lay::NE) * NP;  // numerators, denominators [2][M][NF] each
  const auto sSn0 = tile_view<NF>(sides, M, st), sSn1 = tile_view<NF>(sides + M * NF, M, st);
  const auto sSd0 = tile_view<NF>(sides + 2 * M * NF, M, st);
  const auto sSd1 = tile_view<NF>(sides + 3 * M * NF, M, st);
  const auto sD = tile_view<NF>(sides + 4 * M * NF, M, st);
  const auto sF = tile_view<NF>(sides + 5 * M * NF, M, st);
  const auto sVt = tile_view<P>(sides + 6 * M * NF, M, st);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = a.inst_n[k];
  const int np = min(P, n - s);
  HWENO_CHECK(s >= 0 && np >= 1, st);
  const long long off = a.inst_off[k] * M;
  const Real* geo = pick<Real>(a.inst_geo, a.inst_geof) + 3 * k;
  const Real dx = geo[0], idx = geo[1], idx2 = geo[2];
  const Real alpha = Real(alpha_in);
  const Real gam = pick<Real>(a.sp.wd, a.sp.wf)[9];
  const Real gm1 = gam - Real(1);
  const Weights<Real> w = weights_from(pick<Real>(a.sp.wd, a.sp.wf));

  // A (warp 0): the tile with ghosts, point fluxes and splitting; lane g is
  // point s - 2 + g
  if (warp == 0 && lane < np + 4)
    tile_point<EQ, Real, TV>(a, static_cast<const Real*>(io.U) + off,
                             static_cast<const Real*>(io.V) + off, n, s, lane,
                             Real(0.5) * alpha, Real(0.5) * dx * alpha, dx, Real(0.5) * dx,
                             gam, gm1, sU, sV, sFp, sFm, sHp, sHm, sE);
  __syncthreads();

  // B: warps 0 / 1 the "+" / "-" side of interface x_{s+j-1/2}, j = lane
  // (left point at loaded index j + 1); warp 2 the limited derivative of
  // point j = lane; warp 3 the derivative flux of interface j = lane
  Char1<Real> ch{};  // Euler: characteristic system at the interface (warps 0, 1)
  if (warp < 2) {
    const int sd = warp, j = lane, gl = j + 1, b = gl - 1 + sd;  // first stencil point
    if (j <= np) {
      const TV SF = sd ? sFm : sFp;
      const TV SH = sd ? sHm : sHp;
      const auto sSn = sd ? sSn1 : sSn0;
      const auto sSd = sd ? sSd1 : sSd0;
      if constexpr (!EUL) {
        const Frac<Real> fr = side_frac(sd, SF[0][b], SF[0][b + 1], SF[0][b + 2], SH[0][b],
                                        SH[0][b + 1], SH[0][b + 2], w);
        sSn[0][j] = fr.n;
        sSd[0][j] = fr.d;
      } else {
        Real uu, HH, cc;
        if (a.sp.eig_avg == 0) {  // Roe average of U_i, U_{i+1}
          const Real sl = sE[0][gl], sr = sE[0][gl + 1];
          const Real is = recip(sl + sr);
          uu = (sl * sE[1][gl] + sr * sE[1][gl + 1]) * is;
          HH = (sl * sE[2][gl] + sr * sE[2][gl + 1]) * is;
        } else {  // arithmetic mean state
          const Real r = Real(0.5) * (sU[0][gl] + sU[0][gl + 1]);
          const Real mo = Real(0.5) * (sU[1][gl] + sU[1][gl + 1]);
          const Real E = Real(0.5) * (sU[2][gl] + sU[2][gl + 1]);
          const Real ir = Real(1) / r;
          uu = mo * ir;
          HH = (E + gm1 * (E - Real(0.5) * mo * uu)) * ir;
        }
        Real ic;
        sound_speed(gm1 * (HH - Real(0.5) * uu * uu), cc, ic);
        ch = Char1<Real>(uu, HH, cc, ic, gm1);
        // the side's six projected vectors as (x0, A, B)
        Real x0[6], fa[6], fb[6];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          x0[d] = SF[0][b + d];
          ch.factors(SF[0][b + d], SF[1][b + d], SF[2][b + d], fa[d], fb[d]);
          x0[3 + d] = SH[0][b + d];
          ch.factors(SH[0][b + d], SH[1][b + d], SH[2][b + d], fa[3 + d], fb[3 + d]);
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          auto pj = [&](int k) { return ch.row(q, x0[k], fa[k], fb[k]); };
          const Frac<Real> fr = side_frac(sd, pj(0), pj(1), pj(2), pj(3), pj(4), pj(5), w);
          sSn[q][j] = fr.n;
          sSd[q][j] = fr.d;
        }
      }
    }
  } else if (warp == 2) {
    const int j = lane, g = j + 2;
    if (j < np) {
      Real vt[M];
      limited_point<EQ, Real, TV>(a, g, idx, gm1, w, sU, sV, sE, vt);
#pragma unroll
      for (int c = 0; c < M; ++c) sVt[c][j] = vt[c];
    }
  } else {
    const int j = lane, gl = j + 1;
    if (j <= np)
#pragma unroll
      for (int c = 0; c < M; ++c)
        sD[c][j] = derivative_flux(sFp[c][gl - 1], sFp[c][gl], sFp[c][gl + 1], sHp[c][gl - 1],
                                   sHp[c][gl], sHp[c][gl + 1], sFm[c][gl], sFm[c][gl + 1],
                                   sFm[c][gl + 2], sHm[c][gl], sHm[c][gl + 1], sHm[c][gl + 2]);
  }
  __syncthreads();

  // C (warp 0): interface fluxes from the two sides, then the points
  if (warp != 0) return;
  {
    const int j = lane;
    if (j <= np) {
      if constexpr (!EUL) {
        sF[0][j] = resolve1(sides_sum(sSn0[0][j], sSd0[0][j], sSn1[0][j], sSd1[0][j]));
      } else {
        Frac<Real> fr[3];
#pragma unroll
        for (int q = 0; q < 3; ++q)
          fr[q] = sides_sum(sSn0[q][j], sSd0[q][j], sSn1[q][j], sSd1[q][j]);
        Real f[3], out[3];
        resolve3(fr[0], fr[1], fr[2], f[0], f[1], f[2]);
        ch.right(f, out);
#pragma unroll
        for (int c = 0; c < 3; ++c) sF[c][j] = out[c];
      }
    }
  }
  __syncwarp();
  const RKFactors<Real, MODE> rk(Real(dt), idx, idx2);
  const bool want_alpha = part_out != nullptr;  // uniform
  Real amax = Real(0);
  bool bad = false;
  const int j = lane;
  if (j < np) {
    const int g = j + 2;
    Real dF[M], dD[M];
#pragma unroll
    for (int c = 0; c < M; ++c) {
      dF[c] = sF[c][j + 1] - sF[c][j];
      dD[c] = sD[c][j + 1] - sD[c][j];
    }
    Real u[M], vt[M], un[M];
#pragma unroll
    for (int c = 0; c < M; ++c) { u[c] = sU[c][g]; vt[c] = sVt[c][j]; }
    stage_update<EQ, Real, MODE>(io, off + s + j, n, u, dF, dD, vt, rk, un);
    if (want_alpha) {
      const Real sp = wave_speed<EQ>(un, gam, pick<Real>(a.sp.wd, a.sp.wf)[10]);
      bad = !(sp <= real_max<Real>());
      amax = sp;
    }
  }
  if (want_alpha) {
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
      if (bad) atomicOr(a.status, STATUS_NONFINITE);
      *part_out = (double)amax;  // this CTA's share of the stage output's wave speed
    }
  }
}

// ---------------------------------------------------------------------------
// Fused step of small instances on thread-block clusters (fused_small = 2):
// one cluster of C CTAs per instance, CTA r of the cluster holding the
// kTile1D-point tile that starts at r * kTile1D, each CTA alone on its SM
// (its shared-memory request leaves no room for a second one). The wave
// speed of U^n is reduced through distributed shared memory; the stages are
// separated by cluster barriers, whose release / acquire order makes each
// stage's global writes (state, alpha slots) visible to the next. f.steps
// steps run in one launch (one from hweno_step, K from the persistent run).
// Every CTA passes the same six barriers per step whatever its share of the
// instance.
// ---------------------------------------------------------------------------
template <int EQ, class Real>
__global__ void __launch_bounds__(kThreads1D)
k_step_cluster_1d(const __grid_constant__ Args1D a, const __grid_constant__ FusedArgs f) {
  namespace cg = cooperative_groups;
  constexpr int M = Dim1<EQ>::M;
  constexpr int P = kTile1D;
  __shared__ Real red[kThreads1D / 32];
  __shared__ double part;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int k = blockIdx.x / C;
  const int n = a.inst_n[k];
  const int s = rank * P;
  unsigned long long* s0 = f.alpha;
  unsigned long long* s1 = f.alpha + f.batch;
  unsigned long long* s2 = f.alpha + 2 * f.batch;
  for (int step = 0; step < f.steps; ++step) {
    const bool live = a.t[k] < a.t_end;  // t[k] is written only after the fifth barrier
    const bool has = live && s < n;
    {  // alpha(U^n) of this tile's points
      Real amax = Real(0);
      if (has) {
        const Real* U = static_cast<const Real*>(a.U) + a.inst_off[k] * M;
        const Real gam = pick<Real>(a.sp.wd, a.sp.wf)[9];
        const Real a01 = pick<Real>(a.sp.wd, a.sp.wf)[10];
        const int e = min(s + P, n);
        for (int j = s + threadIdx.x; j < e; j += blockDim.x) {
          Real u[M];
#pragma unroll
          for (int c = 0; c < M; ++c) u[c] = U[(long long)c * n + j];
          amax = fmax(amax, wave_speed<EQ>(u, gam, a01));
        }
      }
      amax = block_max_t(amax, red);
      if (threadIdx.x == 0) part = (double)amax;
    }
    cl.sync();
    if (live && rank == 0 && threadIdx.x < 32) {  // the instance's alpha; stage slots from zero
      // one lane per CTA of the cluster (C <= 16) reads its partial, in parallel
      double m = (int)threadIdx.x < C ? *cl.map_shared_rank(&part, (int)threadIdx.x) : 0.0;
      for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (threadIdx.x == 0) {
        s0[k] = (unsigned long long)__double_as_longlong(m);
        s1[k] = 0ull;
        s2[k] = 0ull;
      }
    }
    cl.sync();
    StageIO io = io_of(a);
    io.Uout = f.U1; io.Vout = f.V1; io.Vt0out = f.Vt0;
    io.alpha_in = reinterpret_cast<const double*>(s0); io.alpha_out = s1;
    if (has) stage_tile<EQ, Real, MODE_STAGE1, kThreads1D, 1>(a, io, k, s);
    cl.sync();
    io.U = f.U1; io.V = f.V1; io.U0 = a.U; io.Vt0 = f.Vt0; io.Uout = f.U2; io.Vout = f.V2;
    io.Vt0out = nullptr;
    io.alpha_in = reinterpret_cast<const double*>(s1); io.alpha_out = s2;
    if (has) stage_tile<EQ, Real, MODE_STAGE2, kThreads1D, 1>(a, io, k, s);
    cl.sync();
    io.U = f.U2; io.V = f.V2; io.Uout = const_cast<void*>(a.U); io.Vout = const_cast<void*>(a.V);
    io.alpha_in = reinterpret_cast<const double*>(s2); io.alpha_out = nullptr;
    if (has) stage_tile<EQ, Real, MODE_STAGE3, kThreads1D, 1>(a, io, k, s);
    cl.sync();  // every CTA is past its reads of t[k]
    if (rank == 0 && threadIdx.x == 0) {
      if (!live) {  // finished: nothing moves (as k_finalize)
        if (f.dt_used) f.dt_used[k] = 0.0;
      } else {  // time update (as k_finalize); tile 0 wrote dt and lands
        double tk = a.t[k];
        const double d = a.dt[k];
        tk = a.lands[k] ? a.t_end : tk + d;
        const_cast<double*>(a.t)[k] = tk;
        if (!(__longlong_as_double((long long)s0[k]) <= DBL_MAX)) atomicOr(a.status, STATUS_NONFINITE);
        if (f.pu) atomicAdd(f.pu, (unsigned long long)n);
        if (f.dt_used) f.dt_used[k] = d;
        if (step == f.steps - 1 && tk < a.t_end) atomicAdd(f.active, 1);
      }
    }
    cl.sync();  // the new t[k] before the next step reads it
  }
}

// The latency form of the cluster step (instances of at most kSplitMax *
// kSplitTile points, stage_tile_split). Every CTA keeps the instance's time,
// wave speeds and time step itself (the same arithmetic on the same values in
// every CTA); each stage leaves its CTA's share of the output's wave speed in
// shared memory, and after the stage's cluster barrier every CTA reduces the
// shares through distributed shared memory. A step thus takes one cluster
// barrier per stage, and the K steps of a launch one more before the first.
// Rank 0 publishes t, dt, lands, the wave speeds (the alpha slots a step
// record copies), the counters and dt_used.
template <int EQ, class Real>
__global__ void __launch_bounds__(kThreads1D)
k_step_cluster_split_1d(const __grid_constant__ Args1D a, const __grid_constant__ FusedArgs f) {
  namespace cg = cooperative_groups;
  constexpr int M = Dim1<EQ>::M;
  constexpr int P = kSplitTile;
  __shared__ Real red[kThreads1D / 32];
  __shared__ double part[4];  // shares: alpha of U^n and of the three stage outputs
  __shared__ double s_alpha, s_dt;
  __shared__ int s_lands;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int k = blockIdx.x / C;
  const int n = a.inst_n[k];
  const int s = rank * P;
  const bool mine = s < n;
  if (threadIdx.x < 4) part[threadIdx.x] = 0.0;
  double t = a.t[k];  // rank 0 writes t[k] only after the first step's barriers
  // the cluster's maximum of share q (after a cluster barrier), to every thread
  auto cluster_alpha = [&](int q) -> double {
    if (threadIdx.x < 32) {
      double m = (int)threadIdx.x < C ? cl.map_shared_rank(part, (int)threadIdx.x)[q] : 0.0;
      for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (threadIdx.x == 0) s_alpha = m;
    }
    __syncthreads();
    return s_alpha;
  };
  {  // alpha(U^n) of this tile's points
    Real amax = Real(0);
    if (mine && t < a.t_end) {
      const Real* U = static_cast<const Real*>(a.U) + a.inst_off[k] * M;
      const Real gam = pick<Real>(a.sp.wd, a.sp.wf)[9];
      const Real a01 = pick<Real>(a.sp.wd, a.sp.wf)[10];
      const int e = min(s + P, n);
      for (int j = s + threadIdx.x; j < e; j += blockDim.x) {
        Real u[M];
#pragma unroll
        for (int c = 0; c < M; ++c) u[c] = U[(long long)c * n + j];
        amax = fmax(amax, wave_speed<EQ>(u, gam, a01));
      }
    }
    amax = block_max_t(amax, red);
    if (threadIdx.x == 0) part[0] = (double)amax;
  }
  cl.sync();
  double alpha = cluster_alpha(0);
  for (int step = 0; step < f.steps; ++step) {
    const bool live = t < a.t_end;  // the same in every CTA
    const bool has = live && mine;
    double dt = 0.0;
    int lands = 0;
    if (live) {
      if (threadIdx.x == 0) {
        s_dt = a.dt_in ? a.dt_in[k] : time_step(a.sp, alpha, a.inst_hx[k], t, a.t_end, s_lands);
        if (a.dt_in) s_lands = 0;
      }
      __syncthreads();
      dt = s_dt;
      lands = s_lands;
    }
    StageIO io = io_of(a);
    io.Uout = f.U1; io.Vout = f.V1; io.Vt0out = f.Vt0;
    if (has) stage_tile_split<EQ, Real, MODE_STAGE1>(a, io, k, s, alpha, dt, &part[1]);
    cl.sync();
    const double a1 = cluster_alpha(1);
    io.U = f.U1; io.V = f.V1; io.U0 = a.U; io.Vt0 = f.Vt0; io.Uout = f.U2; io.Vout = f.V2;
    io.Vt0out = nullptr;
    if (has) stage_tile_split<EQ, Real, MODE_STAGE2>(a, io, k, s, a1, dt, &part[2]);
    cl.sync();
    const double a2 = cluster_alpha(2);
    io.U = f.U2; io.V = f.V2; io.Uout = const_cast<void*>(a.U); io.Vout = const_cast<void*>(a.V);
    const bool more = step + 1 < f.steps;  // stage 3 also gives alpha of U^{n+1}
    if (has) stage_tile_split<EQ, Real, MODE_STAGE3>(a, io, k, s, a2, dt, more ? &part[3] : nullptr);
    cl.sync();
    if (live) {
      const double tn = lands ? a.t_end : t + dt;
      if (rank == 0 && threadIdx.x == 0) {
        const_cast<double*>(a.t)[k] = tn;
        a.dt[k] = dt;
        a.lands[k] = lands;
        f.alpha[k] = (unsigned long long)__double_as_longlong(alpha);
        f.alpha[f.batch + k] = (unsigned long long)__double_as_longlong(a1);
        f.alpha[2 * f.batch + k] = (unsigned long long)__double_as_longlong(a2);
        if (!(alpha <= DBL_MAX)) atomicOr(a.status, STATUS_NONFINITE);
        if (f.pu) atomicAdd(f.pu, (unsigned long long)n);
        if (f.dt_used) f.dt_used[k] = dt;
        if (!more && tn < a.t_end) atomicAdd(f.active, 1);
      }
      t = tn;
    } else if (rank == 0 && threadIdx.x == 0 && f.dt_used) {
      f.dt_used[k] = 0.0;  // finished: nothing moves
    }
    if (more) alpha = cluster_alpha(3);
  }
}

// Launch on clusters of C CTAs; returns cudaErrorNotSupported (nothing
// launched) when the device cannot hold such a cluster.
template <int EQ, class Real, bool SPLIT>
cudaError_t step_cluster_try(const Args1D& a, const FusedArgs& f, int C, cudaStream_t s) {
  constexpr size_t tile =
      SPLIT ? SplitLayout<EQ, Real>::bytes : Layout1D<EQ, Real, kThreads1D, 1>::bytes;
  constexpr size_t bytes = tile > kClusterSmem ? tile : kClusterSmem;
  auto kern = SPLIT ? k_step_cluster_split_1d<EQ, Real> : k_step_cluster_1d<EQ, Real>;
  static unsigned configured = 0;  // devices whose limit is raised
  if (const cudaError_t e = ensure_smem_limit(kern, bytes, configured)) return e;
  static unsigned nonportable = 0;  // devices allowed clusters above 8
  int dev = 0;
  if (const cudaError_t e = cudaGetDevice(&dev)) return e;
  const unsigned bit = dev < 32 ? 1u << dev : 0u;
  if (C > 8 && !(nonportable & bit)) {
    if (const cudaError_t e =
            cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1))
      return e;
    nonportable |= bit;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(f.batch * C));
  cfg.blockDim = dim3(kThreads1D);
  cfg.dynamicSmemBytes = bytes;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  // whether a cluster of this size fits, once per device and size
  static signed char fits[32][kSplitMax + 1] = {};  // 0 unknown, 1 yes, -1 no
  signed char& ok = fits[dev < 32 ? dev : 0][C];
  if (ok == 0) {
    int clusters = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg);
    if (e != cudaSuccess) { cudaGetLastError(); clusters = 0; }
    ok = clusters > 0 ? 1 : -1;
  }
  if (ok < 0) return cudaErrorNotSupported;
  return cudaLaunchKernelEx(&cfg, kern, a, f);
}

// The cluster step: for instances of at most kSplitMax * kSplitTile points
// the latency form (28-point tiles, the work of a point over four warps) when
// the device holds such clusters, else 124-point tiles.
template <int EQ, class Real>
cudaError_t step_cluster_launch(const Args1D& a, const FusedArgs& f, int max_n, cudaStream_t s) {
  const int Cs = (max_n + kSplitTile - 1) / kSplitTile;
  if (Cs <= kSplitMax) {
    const cudaError_t e = step_cluster_try<EQ, Real, true>(a, f, Cs, s);
    if (e != cudaErrorNotSupported) return e;
  }
  const int C = (max_n + kTile1D - 1) / kTile1D;
  return step_cluster_try<EQ, Real, false>(a, f, C, s);
}

template <class Real>
cudaError_t step_cluster_prec(int eq, const Args1D& a, const FusedArgs& f, int max_n,
                              cudaStream_t s) {
  return eq == HWENO_BURGERS ? step_cluster_launch<HWENO_BURGERS, Real>(a, f, max_n, s)
                             : step_cluster_launch<HWENO_EULER, Real>(a, f, max_n, s);
}

template <class Real>
cudaError_t step_small_prec(int eq, const Args1D& a, const FusedArgs& f, cudaStream_t s) {
  return eq == HWENO_BURGERS ? step_small_launch<HWENO_BURGERS, Real>(a, f, s)
                             : step_small_launch<HWENO_EULER, Real>(a, f, s);
}

}  // namespace
}  // namespace hweno
