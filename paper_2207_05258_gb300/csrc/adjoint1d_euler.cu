// Discrete adjoint of one SSP-RK3 stage of the 1D L-HWENO scheme for the
// Euler equations (Zhang & Zhao, arXiv:2207.05258, Sec. 2.1-2.2) in FP64: the
// characteristic-wise nonlinear fluxes with Roe-averaged eigenvectors, the
// linear derivative fluxes, the characteristic (or component-wise) HWENO
// limiter and the stage combination, with alpha and dt of the forward run
// frozen and the |.| branches of tau taken at the forward state.
//
// Reverse of the interface flux f-hat = R(U-bar) sum_sides side(L(U-bar) F):
// the cotangent of the characteristic flux is R^T mu; the sides are reversed
// by hand (side_vjp); the projections give the cotangents of the split point
// fluxes and of L, R; L, R are pulled back to the Roe state (u-bar, H-bar) by
// one reverse pass through the eigenvector formulas, and the Roe average to
// the two states by hand. The split point fluxes F^{+-}, H^{+-} are pulled
// back to (u, v) once per point by a reverse pass through the flux F(u) and
// H = F'(u) v.
//
// Tiling as the Burgers adjoint: one CTA per tile of P points, items
// (interfaces j = s-2 .. s+P, limited derivatives j = s-1 .. s+P) store their
// per-stencil-slot cotangents field-major in shared memory, every loaded
// point gathers its slots in a fixed order, and owned points add their ghost
// images at walls. No atomics.
#include "hweno.h"
#include "hweno_adjoint.cuh"
#include "internal.h"

namespace hweno {
namespace {

constexpr int P = kTile1D;  // owned points per tile (the default 1D tile)
constexpr int NT = 128;     // threads per CTA
constexpr int NL = P + 6;   // loaded points s-3 .. s+P+2
constexpr int NI = P + 3;   // interfaces j = s-2 .. s+P
constexpr int NV = P + 2;   // limited derivatives j = s-1 .. s+P
constexpr int NS = 12;      // per interface slot: gF[3], gH[3], gu[3], gv[3]
constexpr int NLS = 15;     // per limiter item: gu at j-1, j, j+1 [3 each], gv at j-1, j+1

// Point flux F(u) and H = F'(u) v of the 1D Euler equations.
template <class T>
__device__ __forceinline__ void euler_fh(const T* u, const T* v, double gm1, T* F, T* H) {
  const T ir = T(1.0) / u[0];
  const T vel = u[1] * ir;
  const T p = gm1 * (u[2] - 0.5 * u[1] * vel);
  const T Ep = u[2] + p;
  F[0] = u[1];
  F[1] = u[1] * vel + p;
  F[2] = Ep * vel;
  const T dvel = (v[1] - vel * v[0]) * ir;
  const T dp = gm1 * (v[2] - vel * v[1] + 0.5 * vel * vel * v[0]);
  H[0] = v[1];
  H[1] = v[1] * vel + u[1] * dvel + dp;
  H[2] = (v[2] + dp) * vel + Ep * dvel;
}

// gu += d(gF.F + gH.H)/du, gv += d(gH.H)/dv at (u, v): one reverse pass
// through euler_fh.
__device__ __forceinline__ void point_vjp(const double* u, const double* v, const double* gF,
                                          const double* gH, double gm1, double* gu, double* gv) {
  const double ir = 1.0 / u[0], vel = u[1] * ir;
  const double p = gm1 * (u[2] - 0.5 * u[1] * vel), Ep = u[2] + p;
  const double dvel = (v[1] - vel * v[0]) * ir;
  const double dp = gm1 * (v[2] - vel * v[1] + 0.5 * vel * vel * v[0]);
  // F = (u1, u1 vel + p, Ep vel); H = (v1, v1 vel + u1 dvel + dp, (v2 + dp) vel + Ep dvel)
  double a_vel = gF[1] * u[1] + gF[2] * Ep + gH[1] * v[1] + gH[2] * (v[2] + dp);
  double a_p = gF[1];
  double a_Ep = gF[2] * vel + gH[2] * dvel;
  const double a_dvel = gH[1] * u[1] + gH[2] * Ep;
  const double a_dp = gH[1] + gH[2] * vel;
  double a_u0 = 0.0, a_u1 = gF[0] + gF[1] * vel + gH[1] * dvel, a_u2 = 0.0;
  // dvel = (v1 - vel v0) / rho, dp = gm1 (v2 - vel v1 + vel^2 v0 / 2)
  a_vel += -a_dvel * v[0] * ir + a_dp * gm1 * (vel * v[0] - v[1]);
  double a_ir = a_dvel * (v[1] - vel * v[0]);
  gv[0] += 0.5 * gm1 * a_dp * vel * vel - a_dvel * vel * ir;
  gv[1] += gH[0] + gH[1] * vel + a_dvel * ir - gm1 * a_dp * vel;
  gv[2] += gH[2] * vel + gm1 * a_dp;
  // Ep = u2 + p, p = gm1 (u2 - u1 vel / 2), vel = u1 / rho
  a_p += a_Ep;
  a_u2 += a_Ep + gm1 * a_p;
  a_u1 -= 0.5 * gm1 * a_p * vel;
  a_vel -= 0.5 * gm1 * a_p * u[1];
  a_u1 += a_vel * ir;
  a_ir += a_vel * u[1];
  a_u0 -= a_ir * ir * ir;
  gu[0] += a_u0;
  gu[1] += a_u1;
  gu[2] += a_u2;
}

// Eigenvectors at velocity u and enthalpy H: returns them in e and the
// pullback (gu, gH) of sum gL.L + gR.R.
__device__ __forceinline__ void eigen_at(double u, double H, double gm1, Eigen<double, 3>& e) {
  const double c2 = gm1 * (H - 0.5 * u * u);
  const double c = ::sqrt(c2), ic = 1.0 / c;
  euler_eigen<double, 3>(0, u, 0.0, H, c, ic, gm1, e);
}

// One reverse pass through the formulas of euler_eigen (M = 3: q = u^2/2,
// b1 = (gamma-1)/c^2, b2 = b1 q, c^2 = (gamma-1)(H - q)).
__device__ __forceinline__ void eigen_vjp(double u, double H, double gm1, const double (*gL)[3],
                                          const double (*gR)[3], double& gu, double& gH) {
  const double q = 0.5 * u * u;
  const double c = ::sqrt(gm1 * (H - q)), ic = 1.0 / c;
  const double b1 = gm1 * ic * ic;
  const double sL1 = gL[0][1] + gL[2][1];
  const double a_b2 = 0.5 * (gL[0][0] + gL[2][0]) - gL[1][0];
  const double a_uc = 0.5 * (gL[0][0] - gL[2][0]);
  double a_b1 = -0.5 * u * sL1 + 0.5 * (gL[0][2] + gL[2][2]) + u * gL[1][1] - gL[1][2];
  double a_ic = 0.5 * (gL[2][1] - gL[0][1]);
  double a_u = b1 * (gL[1][1] - 0.5 * sL1) + gR[1][0] + gR[1][1] + gR[1][2] +
               c * (gR[2][2] - gR[2][0]);
  double a_c = gR[1][2] - gR[1][0] + u * (gR[2][2] - gR[2][0]);
  double a_H = gR[2][0] + gR[2][2];
  double a_q = gR[2][1];
  // b2 = b1 q, uc = u ic, b1 = gm1 ic^2, ic = 1/c, c = sqrt(gm1 (H - q))
  a_b1 += q * a_b2;
  a_q += b1 * a_b2;
  a_u += ic * a_uc;
  a_ic += u * a_uc + 2.0 * gm1 * ic * a_b1;
  a_c -= ic * ic * a_ic;
  const double a_in = 0.5 * gm1 * ic * a_c;  // d c / d (H - q) = gm1 / (2 c)
  a_H += a_in;
  a_q -= a_in;
  gu = a_u + u * a_q;
  gH = a_H;
}

// Velocity and total enthalpy of a conserved state, H = gamma E / rho -
// (gamma - 1) vel^2 / 2, and the pullback of (gvel, gH) onto (rho, m, E).
__device__ __forceinline__ void vel_enthalpy(const double* u, double gm1, double& vel, double& H) {
  const double ir = 1.0 / u[0];
  vel = u[1] * ir;
  H = (gm1 + 1.0) * u[2] * ir - 0.5 * gm1 * vel * vel;
}

__device__ __forceinline__ void vel_enthalpy_vjp(const double* u, double gm1, double gvel,
                                                 double gH, double* gu) {
  const double ir = 1.0 / u[0], vel = u[1] * ir;
  const double gv = gvel - gH * gm1 * vel;  // H depends on vel
  gu[0] += -gv * vel * ir - gH * (gm1 + 1.0) * u[2] * ir * ir;
  gu[1] += gv * ir;
  gu[2] += gH * (gm1 + 1.0) * ir;
}

__global__ void __launch_bounds__(NT, 2) k_adjoint_euler_1d(const __grid_constant__ AdjArgs1D a) {
  extern __shared__ double smem[];
  double (*su)[NL] = reinterpret_cast<double (*)[NL]>(smem);        // [3][NL]
  double (*sv)[NL] = su + 3;                                         // [3][NL]
  double (*sFp)[NL] = sv + 3;                                        // [3][NL] x 4
  double (*sFm)[NL] = sFp + 3;
  double (*sHp)[NL] = sFm + 3;
  double (*sHm)[NL] = sHp + 3;
  double (*tU)[NL] = sFp;  // phase C totals reuse the split fluxes' space
  double (*tV)[NL] = sFm;
  double (*mL1)[P + 4] = reinterpret_cast<double (*)[P + 4]>(&sHm[3][0]);  // [3][P+4]
  double (*mL2)[P + 4] = mL1 + 3;
  double (*mVt)[NV] = reinterpret_cast<double (*)[NV]>(&mL2[3][0]);        // [3][NV]
  double (*sIt)[NI] = reinterpret_cast<double (*)[NI]>(&mVt[3][0]);        // [4*NS][NI]
  double (*sLm)[NV] = reinterpret_cast<double (*)[NV]>(&sIt[4 * NS][0]);   // [NLS][NV]

  const int b = blockIdx.x;
  const int k = a.tile_inst[b], s = a.tile_start[b], n = a.inst_n[k];
  const int np = min(P, n - s);
  const long long off = a.inst_off[k] * 3;
  const double dt = a.dt[k];
  if (dt == 0.0) {  // the instance did not step: the stage is the identity
    for (int ip = threadIdx.x; ip < np; ip += blockDim.x)
      for (int c = 0; c < 3; ++c) {
        const long long q = off + (long long)c * n + s + ip;
        a.outU[q] = a.lamU[q];
        a.outV[q] = a.lamV[q];
        if (a.accOutU) { a.accOutU[q] = 0.0; a.accOutVt[q] = 0.0; }
      }
    return;
  }
  const double* geo = a.inst_geo + 3 * k;
  const double dx = geo[0], idx = geo[1], idx2 = geo[2];
  const double alpha = a.alpha[k];
  const double gm1 = a.sp.wd[9] - 1.0;
  const Weights<double> w = weights_from(a.sp.wd);
  const bool periodic = a.sp.bc[0] == HWENO_BC_PERIODIC;
  const int lim = a.sp.limiter;
  const double hdx = 0.5 * dx;
  const double sgn_u[3] = {1.0, -1.0, 1.0};  // reflection: momentum odd, v opposite

  // A: forward point data on s-3 .. s+np+2 (ghosts as the forward loads them)
  for (int g = threadIdx.x; g < np + 6; g += blockDim.x) {
    int kind;
    const int src = ghost_src(s - 3 + g, n, a.sp.bc[0], a.sp.bc[1], kind);
    HWENO_CHECK(kind == 2 || (src >= 0 && src < n), a.status);
    double u[3], v[3], F[3], H[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (kind == 2) { u[c] = a.sp.inflow[c]; v[c] = 0.0; }
      else {
        u[c] = a.U[off + (long long)c * n + src];
        v[c] = a.V[off + (long long)c * n + src];
        if (kind == 1) { u[c] *= sgn_u[c]; v[c] *= -sgn_u[c]; }
      }
      su[c][g] = u[c];
      sv[c][g] = v[c];
    }
    euler_fh(u, v, gm1, F, H);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      sFp[c][g] = 0.5 * (F[c] + alpha * u[c]);
      sFm[c][g] = 0.5 * (F[c] - alpha * u[c]);
      sHp[c][g] = hdx * (H[c] + alpha * v[c]);
      sHm[c][g] = hdx * (H[c] - alpha * v[c]);
    }
  }
  // cotangents of L^1, L^2 at s-2 .. s+np+1 and of v~ at s-1 .. s+np
  auto pt = [&](int p) { return periodic ? (p % n + n) % n : p; };
  for (int g = threadIdx.x; g < np + 4; g += blockDim.x) {
    const int p = pt(s - 2 + g);
    const bool in = p >= 0 && p < n;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long q = off + (long long)c * n + p;
      mL1[c][g] = in ? a.b * dt * a.lamU[q] : 0.0;
      mL2[c][g] = in ? a.b * dt * a.lamV[q] : 0.0;
    }
  }
  for (int g = threadIdx.x; g < np + 2; g += blockDim.x) {
    const int p = pt(s - 1 + g);
    const bool in = p >= 0 && p < n;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long q = off + (long long)c * n + p;
      mVt[c][g] = in ? a.b * a.lamV[q] + (a.accVt ? a.accVt[q] : 0.0) : 0.0;
    }
  }
  __syncthreads();

  // B1: interfaces j = s-2+jf; stencil points j-1..j+2 are loaded jf..jf+3
  // (slots 0..3); left and right states of the Roe average are slots 1, 2.
  for (int jf = threadIdx.x; jf < np + 3; jf += blockDim.x) {
    double mf[3], mD[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      mf[c] = (mL1[c][jf + 1] - mL1[c][jf]) * idx;
      mD[c] = (mL2[c][jf + 1] - mL2[c][jf]) * idx2;
    }
    // split-flux cotangents per slot, accumulated in this item's own column
    // of sIt: [slot * NS + f], f = gF^+ 0..2, gF^- 3..5, gH^+ 6..8, gH^- 9..11
    auto acc = [&](int kk, int f, double x) { sIt[kk * NS + f][jf] += x; };
#pragma unroll
    for (int f = 0; f < 4 * NS; ++f) sIt[f][jf] = 0.0;
    // linear derivative fluxes, component by component
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double gp[6] = {0, 0, 0, 0, 0, 0}, gm[6] = {0, 0, 0, 0, 0, 0};
      dflux_vjp(mD[c], gp, gm);
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) {
        acc(kk, c, gp[kk]); acc(kk, 6 + c, gp[3 + kk]);
        acc(kk + 1, 3 + c, gm[kk]); acc(kk + 1, 9 + c, gm[3 + kk]);
      }
    }
    // characteristic nonlinear fluxes
    const double uL[3] = {su[0][jf + 1], su[1][jf + 1], su[2][jf + 1]};
    const double uR[3] = {su[0][jf + 2], su[1][jf + 2], su[2][jf + 2]};
    const double sL = ::sqrt(uL[0]), sR = ::sqrt(uR[0]), iS = 1.0 / (sL + sR);
    double velL, HL, velR, HR;
    vel_enthalpy(uL, gm1, velL, HL);
    vel_enthalpy(uR, gm1, velR, HR);
    const double ub = (sL * velL + sR * velR) * iS, Hb = (sL * HL + sR * HR) * iS;
    Eigen<double, 3> e;
    eigen_at(ub, Hb, gm1, e);
    double gL[3][3], gR[3][3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const double gq = e.R[0][q] * mf[0] + e.R[1][q] * mf[1] + e.R[2][q] * mf[2];
      double pFp[3], pHp[3], pFm[3], pHm[3];
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) {
        pFp[kk] = e.L[q][0] * sFp[0][jf + kk] + e.L[q][1] * sFp[1][jf + kk] + e.L[q][2] * sFp[2][jf + kk];
        pHp[kk] = e.L[q][0] * sHp[0][jf + kk] + e.L[q][1] * sHp[1][jf + kk] + e.L[q][2] * sHp[2][jf + kk];
        pFm[kk] = e.L[q][0] * sFm[0][jf + 1 + kk] + e.L[q][1] * sFm[1][jf + 1 + kk] + e.L[q][2] * sFm[2][jf + 1 + kk];
        pHm[kk] = e.L[q][0] * sHm[0][jf + 1 + kk] + e.L[q][1] * sHm[1][jf + 1 + kk] + e.L[q][2] * sHm[2][jf + 1 + kk];
      }
      double gp[6] = {0, 0, 0, 0, 0, 0}, gm[6] = {0, 0, 0, 0, 0, 0};
      const double fq = flux_vjp(pFp, pHp, pFm, pHm, gq, w, gp, gm, a.sp.adj_frozen != 0);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        gR[c][q] = mf[c] * fq;
        double sl = 0.0;
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
          sl += gp[kk] * sFp[c][jf + kk] + gp[3 + kk] * sHp[c][jf + kk] +
                 gm[kk] * sFm[c][jf + 1 + kk] + gm[3 + kk] * sHm[c][jf + 1 + kk];
          acc(kk, c, e.L[q][c] * gp[kk]);
          acc(kk, 6 + c, e.L[q][c] * gp[3 + kk]);
          acc(kk + 1, 3 + c, e.L[q][c] * gm[kk]);
          acc(kk + 1, 9 + c, e.L[q][c] * gm[3 + kk]);
        }
        gL[q][c] = sl;
      }
    }
    // eigenvectors -> Roe state -> the two states
    double gub, gHb;
    eigen_vjp(ub, Hb, gm1, gL, gR, gub, gHb);
    double gUL[3] = {0, 0, 0}, gUR[3] = {0, 0, 0};
    const double gsL = (gub * (velL - ub) + gHb * (HL - Hb)) * iS;
    const double gsR = (gub * (velR - ub) + gHb * (HR - Hb)) * iS;
    gUL[0] += 0.5 * gsL / sL;
    gUR[0] += 0.5 * gsR / sR;
    vel_enthalpy_vjp(uL, gm1, gub * sL * iS, gHb * sL * iS, gUL);
    vel_enthalpy_vjp(uR, gm1, gub * sR * iS, gHb * sR * iS, gUR);
    // per slot, in place: gF, gH (through the point fluxes) and the direct
    // gu, gv (splitting terms and, at slots 1 and 2, the Roe average)
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double fp = sIt[kk * NS + c][jf], fm = sIt[kk * NS + 3 + c][jf];
        const double hp = sIt[kk * NS + 6 + c][jf], hm = sIt[kk * NS + 9 + c][jf];
        double du = 0.5 * alpha * (fp - fm);
        if (kk == 1) du += gUL[c];
        if (kk == 2) du += gUR[c];
        sIt[kk * NS + c][jf] = 0.5 * (fp + fm);
        sIt[kk * NS + 3 + c][jf] = hdx * (hp + hm);
        sIt[kk * NS + 6 + c][jf] = du;
        sIt[kk * NS + 9 + c][jf] = hdx * alpha * (hp - hm);
      }
  }

  // B2: limited derivatives j = s-1+jl; points j-1, j, j+1 are loaded jl+1..jl+3
  for (int jl = threadIdx.x; jl < np + 2; jl += blockDim.x) {
    double gu[3][3], gv[2][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) { gu[0][c] = gu[1][c] = gu[2][c] = 0.0; gv[0][c] = gv[1][c] = 0.0; }
    if (lim == 2) {  // component-wise
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double g5[5] = {0, 0, 0, 0, 0};
        limiter_vjp(su[c][jl + 1], su[c][jl + 2], su[c][jl + 3], dx * sv[c][jl + 1],
                    dx * sv[c][jl + 3], mVt[c][jl] * idx, w, g5, a.sp.adj_frozen != 0);
        gu[0][c] = g5[0]; gu[1][c] = g5[1]; gu[2][c] = g5[2];
        gv[0][c] = dx * g5[3]; gv[1][c] = dx * g5[4];
      }
    } else if (lim == 1) {  // characteristic, eigenvectors at U_j
      const double u0[3] = {su[0][jl + 2], su[1][jl + 2], su[2][jl + 2]};
      double vel, H;
      vel_enthalpy(u0, gm1, vel, H);
      Eigen<double, 3> e;
      eigen_at(vel, H, gm1, e);
      double gL[3][3], gR[3][3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const double gz = (e.R[0][q] * mVt[0][jl] + e.R[1][q] * mVt[1][jl] + e.R[2][q] * mVt[2][jl]) * idx;
        auto pj = [&](double (*A)[NL], int g) {
          return e.L[q][0] * A[0][g] + e.L[q][1] * A[1][g] + e.L[q][2] * A[2][g];
        };
        double g5[5] = {0, 0, 0, 0, 0};
        const double z = limiter_vjp(pj(su, jl + 1), pj(su, jl + 2), pj(su, jl + 3),
                                     dx * pj(sv, jl + 1), dx * pj(sv, jl + 3), gz, w, g5,
                                     a.sp.adj_frozen != 0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          gR[c][q] = mVt[c][jl] * idx * z;
          gL[q][c] = g5[0] * su[c][jl + 1] + g5[1] * su[c][jl + 2] + g5[2] * su[c][jl + 3] +
                     dx * (g5[3] * sv[c][jl + 1] + g5[4] * sv[c][jl + 3]);
          gu[0][c] += e.L[q][c] * g5[0];
          gu[1][c] += e.L[q][c] * g5[1];
          gu[2][c] += e.L[q][c] * g5[2];
          gv[0][c] += dx * e.L[q][c] * g5[3];
          gv[1][c] += dx * e.L[q][c] * g5[4];
        }
      }
      double gvel, gH;
      eigen_vjp(vel, H, gm1, gL, gR, gvel, gH);
      vel_enthalpy_vjp(u0, gm1, gvel, gH, gu[1]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      sLm[c][jl] = gu[0][c];
      sLm[3 + c][jl] = gu[1][c];
      sLm[6 + c][jl] = gu[2][c];
      sLm[9 + c][jl] = gv[0][c];
      sLm[12 + c][jl] = gv[1][c];
    }
  }
  __syncthreads();

  // C: per loaded point, gather the slots that refer to it (fixed order) and
  // pull the point-flux cotangents back to (u, v)
  for (int g = threadIdx.x; g < np + 6; g += blockDim.x) {
    double gF[3] = {0, 0, 0}, gH[3] = {0, 0, 0}, gu[3] = {0, 0, 0}, gv[3] = {0, 0, 0};
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const int jf = g - kk;
      if (jf < 0 || jf >= np + 3) continue;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        gF[c] += sIt[kk * NS + c][jf];
        gH[c] += sIt[kk * NS + 3 + c][jf];
        gu[c] += sIt[kk * NS + 6 + c][jf];
        gv[c] += sIt[kk * NS + 9 + c][jf];
      }
    }
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
      const int jl = g - 1 - kk;
      if (jl < 0 || jl >= np + 2) continue;
#pragma unroll
      for (int c = 0; c < 3; ++c) gu[c] += sLm[3 * kk + c][jl];
    }
    if (g - 1 >= 0 && g - 1 < np + 2)
#pragma unroll
      for (int c = 0; c < 3; ++c) gv[c] += sLm[9 + c][g - 1];
    if (g - 3 >= 0 && g - 3 < np + 2)
#pragma unroll
      for (int c = 0; c < 3; ++c) gv[c] += sLm[12 + c][g - 3];
    const double u[3] = {su[0][g], su[1][g], su[2][g]};
    const double v[3] = {sv[0][g], sv[1][g], sv[2][g]};
    point_vjp(u, v, gF, gH, gm1, gu, gv);
#pragma unroll
    for (int c = 0; c < 3; ++c) { tU[c][g] = gu[c]; tV[c][g] = gv[c]; }
  }
  __syncthreads();

  // D: owned points: stage terms, then ghost images at walls
  for (int ip = threadIdx.x; ip < np; ip += blockDim.x) {
    const int i = s + ip, g = ip + 3;
    double ru[3], rv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long q = off + (long long)c * n + i;
      ru[c] = a.b * a.lamU[q] + (a.accU ? a.accU[q] : 0.0) + tU[c][g];
      rv[c] = tV[c][g] + (lim == 0 ? mVt[c][ip + 1] : 0.0);
    }
    if (!periodic) {
#pragma unroll
      for (int e6 = 0; e6 < 6; ++e6) {
        const int gg = e6 < 3 ? e6 : np + e6;  // 0,1,2 and np+3..np+5
        const int p = s - 3 + gg;
        if (p >= 0 && p < n) continue;  // a halo point of another tile, not a ghost
        int kind;
        const int src = ghost_src(p, n, a.sp.bc[0], a.sp.bc[1], kind);
        HWENO_CHECK(kind == 2 || (src >= 0 && src < n), a.status);
        if (kind == 2 || src != i) continue;
#pragma unroll
        for (int c = 0; c < 3; ++c) {  // ghost u = S u_src, v = -S v_src (mirror) or copies
          ru[c] += (kind == 1 ? sgn_u[c] : 1.0) * tU[c][gg];
          rv[c] += (kind == 1 ? -sgn_u[c] : 1.0) * tV[c][gg];
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long q = off + (long long)c * n + i;
      a.outU[q] = ru[c];
      a.outV[q] = rv[c];
      if (a.accOutU) {
        a.accOutU[q] = a.cN * a.lamNU[q] + a.c2 * a.lamU[q];
        a.accOutVt[q] = a.cN * a.lamNV[q] + a.c2 * a.lamV[q];
      }
    }
  }
}

constexpr size_t kSmemEuler =
    sizeof(double) * (18 * NL + 6 * (P + 4) + 3 * NV + 4 * NS * NI + NLS * NV);

}  // namespace

cudaError_t launch_adjoint_1d_euler(const AdjArgs1D& a, int ntiles, cudaStream_t s) {
  static unsigned configured = 0;  // devices whose limit is raised
  if (const cudaError_t e = ensure_smem_limit(k_adjoint_euler_1d, kSmemEuler, configured)) return e;
  k_adjoint_euler_1d<<<ntiles, NT, kSmemEuler, s>>>(a);
  return cudaGetLastError();
}

}  // namespace hweno
