// Discrete adjoint of one SSP-RK3 stage of the 2D L-HWENO scheme (Zhang &
// Zhao, arXiv:2207.05258, Eq. ode2H with the mixed-derivative fluxes of Eq.
// mixed and the dimension-by-dimension limiter) in FP64, with the wave
// speeds alpha_x, alpha_y and dt of the forward run frozen and the |.|
// branches of tau taken at the forward state.
//
// The stage's right-hand side is a sum of line terms: along x, f-hat (U),
// h-hat (V, from h = A_x V) and the central eta-hat (W, from eta = A_x W)
// and the x-limited v~; along y, g-hat (U), theta-hat (W, from A_y W), the
// central xi-hat (V, from A_y V) and the y-limited w~. One kernel template
// reverses the terms of one direction over lines of that direction: with N
// the derivative normal to the line direction's faces (V in x, W in y) and T
// the other one, a line carries the flux F_d(U), H = A_d N (derivative
// flux), E = A_d T (central flux) and the limiter of N.
//
// Per tile of P points of one line (rows for x, columns for y; column
// accesses are strided, which costs little next to the FP64 arithmetic that
// bounds these kernels): interface items j = s-2 .. s+P and limiter items
// j = s-1 .. s+P store per-stencil-slot cotangents field-major in shared
// memory; every loaded point gathers its slots in a fixed order and pulls the
// point-flux cotangents back to (U, N, T) by forward-mode differentiation of
// the flux and Jacobian-vector products; owned points add their ghost images
// at walls. The characteristic pieces follow the 1D Euler adjoint with the
// 4x4 eigen-system of A_d at the Roe average (u, v, H). No atomics.
#include "flux2d.cuh"
#include "hweno.h"
#include "hweno_adjoint.cuh"
#include "internal.h"

namespace hweno {
namespace {

constexpr int P = kTile1D;  // owned points per tile
constexpr int NT = 128;
constexpr int NL = P + 6;   // loaded points s-3 .. s+P+2
constexpr int NI = P + 3;   // interfaces j = s-2 .. s+P
constexpr int NV = P + 2;   // limiter items j = s-1 .. s+P

template <int EQ>
struct AdjLayout2D {
  static constexpr int M = Dim2<EQ>::M;
  // loads: u, N, T, F+, F-, H+, H-, E (8M rows of NL); cotangent inputs m1,
  // mn, mt (3M rows of P + 4) and mlim (M rows of NV); interface slots (4
  // slots x 5M fields x NI); limiter items (5M fields x NV); per-thread
  // scratch for the eigenvector cotangents (Euler: 32 x NT)
  static constexpr size_t doubles = (size_t)8 * M * NL + 3 * M * (P + 4) + M * NV +
                                    (size_t)20 * M * NI + 5 * M * NV +
                                    (EQ == HWENO_EULER ? 32 * NT : 0);
  static constexpr size_t bytes = sizeof(double) * doubles;
};

// (u, v, H) of a conserved 2D Euler state, H = gamma E / rho - (gamma - 1)
// (u^2 + v^2) / 2, and the pullback of (gu, gv, gH) onto (rho, m, n, E).
__device__ __forceinline__ void velh2(const double* U, double gm1, double& u, double& v, double& H) {
  const double ir = 1.0 / U[0];
  u = U[1] * ir;
  v = U[2] * ir;
  H = (gm1 + 1.0) * U[3] * ir - 0.5 * gm1 * (u * u + v * v);
}

__device__ __forceinline__ void velh2_vjp(const double* U, double gm1, double gu, double gv,
                                          double gH, double* g) {
  const double ir = 1.0 / U[0], u = U[1] * ir, v = U[2] * ir;
  const double gu2 = gu - gH * gm1 * u, gv2 = gv - gH * gm1 * v;
  g[0] += -(gu2 * u + gv2 * v) * ir - gH * (gm1 + 1.0) * U[3] * ir * ir;
  g[1] += gu2 * ir;
  g[2] += gv2 * ir;
  g[3] += gH * (gm1 + 1.0) * ir;
}

// Eigen-system of A_DIR at (u, v, H).
template <int DIR>
__device__ __forceinline__ void eigen2(double u, double v, double H, double gm1,
                                       Eigen<double, 4>& e) {
  const double c = ::sqrt(gm1 * (H - 0.5 * (u * u + v * v))), ic = 1.0 / c;
  euler_eigen<double, 4>(DIR, u, v, H, c, ic, gm1, e);
}

// Pullback of sum gL.L + gR.R (gLR: 16 entries of gL then 16 of gR, stride
// NT in shared memory) onto (u, v, H).
template <int DIR>
__device__ __forceinline__ void eigen2_vjp(double u, double v, double H, double gm1,
                                           const double* gLR, double* g3) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const Dd uu(u, k == 0 ? 1.0 : 0.0), vv(v, k == 1 ? 1.0 : 0.0), HH(H, k == 2 ? 1.0 : 0.0);
    const Dd c = sqrt(Dd(gm1) * (HH - 0.5 * (uu * uu + vv * vv)));
    const Dd ic = Dd(1.0) / c;
    Eigen<Dd, 4> e;
    euler_eigen<Dd, 4>(DIR, uu, vv, HH, c, ic, Dd(gm1), e);
    double s = 0.0;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        s += gLR[(r * 4 + q) * NT] * e.L[r][q].d + gLR[(16 + r * 4 + q) * NT] * e.R[r][q].d;
    g3[k] = s;
  }
}

// Pullback of gF.F(u) + gH.A(u) N + gE.A(u) T onto u, N and T.
template <int EQ, int DIR>
__device__ __forceinline__ void point2_vjp(const double* u, const double* N, const double* T,
                                           const double* gF, const double* gH, const double* gE,
                                           double gm1, double* gu, double* gN, double* gT) {
  constexpr int M = Dim2<EQ>::M;
#pragma unroll
  for (int k = 0; k < M; ++k) {  // d/du_k by forward mode
    Dd uu[M], NN[M], TT[M], F[M], H[M], E[M];
#pragma unroll
    for (int c = 0; c < M; ++c) {
      uu[c] = Dd(u[c], k == c ? 1.0 : 0.0);
      NN[c] = Dd(N[c]);
      TT[c] = Dd(T[c]);
    }
    Prim2<Dd> q{};
    if constexpr (EQ == HWENO_EULER) q = prim2(uu, Dd(gm1));
    flux2<EQ, DIR>(uu, q, F);
    jvp2<EQ, DIR>(uu, q, NN, Dd(gm1), H);
    jvp2<EQ, DIR>(uu, q, TT, Dd(gm1), E);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < M; ++c) s += gF[c] * F[c].d + gH[c] * H[c].d + gE[c] * E[c].d;
    gu[k] += s;
  }
  // A^T gH and A^T gE from the columns A e_k (the products are linear in the
  // derivative argument)
  Prim2<double> q{};
  if constexpr (EQ == HWENO_EULER) q = prim2(u, gm1);
#pragma unroll
  for (int k = 0; k < M; ++k) {
    double ek[M], col[M];
#pragma unroll
    for (int c = 0; c < M; ++c) ek[c] = c == k ? 1.0 : 0.0;
    jvp2<EQ, DIR>(u, q, ek, gm1, col);
    double sH = 0.0, sE = 0.0;
#pragma unroll
    for (int c = 0; c < M; ++c) { sH += gH[c] * col[c]; sE += gE[c] * col[c]; }
    gN[k] += sH;
    gT[k] += sE;
  }
}

template <int EQ, int DIR>
__global__ void __launch_bounds__(NT, 1) k_adjoint_sweep_2d(const __grid_constant__ AdjArgs2D a) {
  constexpr int M = Dim2<EQ>::M;
  constexpr bool EUL = EQ == HWENO_EULER;
  constexpr int NS = 5 * M;  // per slot: F+, F-, H+, H- (then gF, gH, gu, gN), E
  extern __shared__ double smem[];
  double (*su)[NL] = reinterpret_cast<double (*)[NL]>(smem);  // [M]
  double (*sN)[NL] = su + M;
  double (*sT)[NL] = sN + M;
  double (*sFp)[NL] = sT + M;
  double (*sFm)[NL] = sFp + M;
  double (*sHp)[NL] = sFm + M;
  double (*sHm)[NL] = sHp + M;
  double (*sE)[NL] = sHm + M;
  double (*tU)[NL] = sFp;  // phase C totals reuse the split fluxes' space
  double (*tN)[NL] = sFm;
  double (*tT)[NL] = sHp;
  double (*m1)[P + 4] = reinterpret_cast<double (*)[P + 4]>(&sE[M][0]);
  double (*mn)[P + 4] = m1 + M;
  double (*mt)[P + 4] = mn + M;
  double (*ml)[NV] = reinterpret_cast<double (*)[NV]>(&mt[M][0]);
  double (*sIt)[NI] = reinterpret_cast<double (*)[NI]>(&ml[M][0]);   // [4 NS][NI]
  double (*sLm)[NV] = reinterpret_cast<double (*)[NV]>(&sIt[4 * NS][0]);  // [5M][NV]
  double* sG = &sLm[5 * M][0];  // [32][NT] (Euler)

  const int nx = a.nx, ny = a.ny;
  const long long Ntot = (long long)nx * ny;
  const int n = DIR == 0 ? nx : ny;
  const int line = blockIdx.y, s = blockIdx.x * P;
  const int np = min(P, n - s);
  auto at = [&](int p) -> long long {
    return DIR == 0 ? (long long)line * nx + p : (long long)p * nx + line;
  };
  const double dt = a.dt[0];
  if (dt == 0.0) {  // the step did not happen: the stage is the identity
    if (DIR == 1) {
      for (int ip = threadIdx.x; ip < np; ip += blockDim.x)
#pragma unroll
        for (int c = 0; c < M; ++c) {
          const long long q = c * Ntot + at(s + ip);
          a.outU[q] = a.lamU[q]; a.outV[q] = a.lamV[q]; a.outW[q] = a.lamW[q];
          if (a.accOutU) { a.accOutU[q] = 0.0; a.accOutVt[q] = 0.0; a.accOutWt[q] = 0.0; }
        }
    }
    return;
  }
  const double h = a.geod[3 * DIR], ih = a.geod[3 * DIR + 1], ih2 = a.geod[3 * DIR + 2];
  const double hh = 0.5 * h;
  const double alpha = a.alpha[DIR];
  const double gm1 = a.sp.wd[9] - 1.0;
  const Weights<double> w = weights_from(a.sp.wd);
  const bool periodic = a.sp.bc[2 * DIR] == HWENO_BC_PERIODIC;  // both ends (host checks)
  const int lim = a.sp.limiter;
  const double ts = __dadd_rn(a.t[0], __dmul_rn(a.stage_c, dt));
  const double xc = DIR == 1 ? __dadd_rn(a.x0, __dmul_rn((double)line + 0.5, a.dx)) : 0.0;
  auto src_of = [&](int p) {
    return DIR == 0 ? map_x(p, nx, a.sp) : map_y(p, ny, xc, a.y0, a.dy, ts, a.sp);
  };
  // the line's normal and tangential derivative fields and their cotangents
  const double* Nf = DIR == 0 ? a.V : a.W;
  const double* Tf = DIR == 0 ? a.W : a.V;
  const double* lamN = DIR == 0 ? a.lamV : a.lamW;
  const double* lamT = DIR == 0 ? a.lamW : a.lamV;
  const double* accN = DIR == 0 ? a.accVt : a.accWt;

  // A: forward point data on s-3 .. s+np+2 (ghosts as the forward loads them)
  for (int g = threadIdx.x; g < np + 6; g += blockDim.x) {
    const Src sr = src_of(s - 3 + g);
    double u[M], N[M], T[M];
#pragma unroll
    for (int c = 0; c < M; ++c) {
      if (sr.kind == 2) {
        u[c] = imposed(a.sp, sr, c); N[c] = 0.0; T[c] = 0.0;
      } else {
        const long long q = c * Ntot + at(sr.idx);
        u[c] = a.U[q]; N[c] = Nf[q]; T[c] = Tf[q];
        if (sr.kind == 1) {
          const double sg = refl2<EQ, DIR>(c);
          u[c] *= sg; N[c] *= -sg; T[c] *= sg;
        }
      }
      su[c][g] = u[c]; sN[c][g] = N[c]; sT[c][g] = T[c];
    }
    Prim2<double> pq{};
    if constexpr (EUL) pq = prim2(u, gm1);
    double F[M], H[M], E[M];
    flux2<EQ, DIR>(u, pq, F);
    jvp2<EQ, DIR>(u, pq, N, gm1, H);
    jvp2<EQ, DIR>(u, pq, T, gm1, E);
#pragma unroll
    for (int c = 0; c < M; ++c) {
      sFp[c][g] = 0.5 * (F[c] + alpha * u[c]);
      sFm[c][g] = 0.5 * (F[c] - alpha * u[c]);
      sHp[c][g] = hh * (H[c] + alpha * N[c]);
      sHm[c][g] = hh * (H[c] - alpha * N[c]);
      sE[c][g] = E[c];
    }
  }
  // cotangents of the line's parts of L^1, of the N and T equations, and of
  // the limited N, at s-2 .. s+np+1 (limiter: s-1 .. s+np)
  auto pt = [&](int p) { return periodic ? (p % n + n) % n : p; };
  const double bdt = a.b * dt;
  for (int g = threadIdx.x; g < np + 4; g += blockDim.x) {
    const int p = pt(s - 2 + g);
    const bool in = p >= 0 && p < n;
#pragma unroll
    for (int c = 0; c < M; ++c) {
      const long long q = c * Ntot + at(in ? p : 0);
      m1[c][g] = in ? bdt * a.lamU[q] : 0.0;
      mn[c][g] = in ? bdt * lamN[q] : 0.0;
      mt[c][g] = in ? bdt * lamT[q] : 0.0;
    }
  }
  for (int g = threadIdx.x; g < np + 2; g += blockDim.x) {
    const int p = pt(s - 1 + g);
    const bool in = p >= 0 && p < n;
#pragma unroll
    for (int c = 0; c < M; ++c) {
      const long long q = c * Ntot + at(in ? p : 0);
      ml[c][g] = in ? a.b * lamN[q] + (accN ? accN[q] : 0.0) : 0.0;
    }
  }
  __syncthreads();

  // B1: interfaces j = s-2+jf; stencil loaded jf..jf+3 (slots 0..3)
  for (int jf = threadIdx.x; jf < np + 3; jf += blockDim.x) {
    auto acc = [&](int kk, int f, double x) { sIt[kk * NS + f][jf] += x; };
#pragma unroll
    for (int f = 0; f < 4 * NS; ++f) sIt[f][jf] = 0.0;
    double mf[M];
#pragma unroll
    for (int c = 0; c < M; ++c) {
      mf[c] = (m1[c][jf + 1] - m1[c][jf]) * ih;
      const double mD = (mn[c][jf + 1] - mn[c][jf]) * ih2;
      const double mc = (mt[c][jf + 1] - mt[c][jf]) * ih;
      double gp[6] = {0, 0, 0, 0, 0, 0}, gm[6] = {0, 0, 0, 0, 0, 0};
      dflux_vjp(mD, gp, gm);
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) {
        acc(kk, c, gp[kk]); acc(kk, 2 * M + c, gp[3 + kk]);
        acc(kk + 1, M + c, gm[kk]); acc(kk + 1, 3 * M + c, gm[3 + kk]);
      }
      // central flux (Eq. mixed): -1/12, 7/12, 7/12, -1/12
      acc(0, 4 * M + c, -mc / 12.0);
      acc(1, 4 * M + c, 7.0 * mc / 12.0);
      acc(2, 4 * M + c, 7.0 * mc / 12.0);
      acc(3, 4 * M + c, -mc / 12.0);
    }
    if constexpr (!EUL) {
      double gp[6] = {0, 0, 0, 0, 0, 0}, gm[6] = {0, 0, 0, 0, 0, 0};
      flux_vjp(&sFp[0][jf], &sHp[0][jf], &sFm[0][jf + 1], &sHm[0][jf + 1], mf[0], w, gp, gm,
               a.sp.adj_frozen != 0);
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) {
        acc(kk, 0, gp[kk]); acc(kk, 2, gp[3 + kk]);
        acc(kk + 1, 1, gm[kk]); acc(kk + 1, 3, gm[3 + kk]);
      }
    } else {
      double UL[4], UR[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) { UL[c] = su[c][jf + 1]; UR[c] = su[c][jf + 2]; }
      double uL, vL, HL, uR, vR, HR;
      velh2(UL, gm1, uL, vL, HL);
      velh2(UR, gm1, uR, vR, HR);
      const double sL = ::sqrt(UL[0]), sR = ::sqrt(UR[0]), iS = 1.0 / (sL + sR);
      const double ub = (sL * uL + sR * uR) * iS, vb = (sL * vL + sR * vR) * iS;
      const double Hb = (sL * HL + sR * HR) * iS;
      Eigen<double, 4> e;
      eigen2<DIR>(ub, vb, Hb, gm1, e);
      double* gLR = sG + threadIdx.x;  // [32] stride NT
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        double gq = 0.0;
#pragma unroll
        for (int c = 0; c < 4; ++c) gq += e.R[c][q] * mf[c];
        double pFp[3], pHp[3], pFm[3], pHm[3];
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
          pFp[kk] = pHp[kk] = pFm[kk] = pHm[kk] = 0.0;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            pFp[kk] += e.L[q][c] * sFp[c][jf + kk];
            pHp[kk] += e.L[q][c] * sHp[c][jf + kk];
            pFm[kk] += e.L[q][c] * sFm[c][jf + 1 + kk];
            pHm[kk] += e.L[q][c] * sHm[c][jf + 1 + kk];
          }
        }
        double gp[6] = {0, 0, 0, 0, 0, 0}, gm[6] = {0, 0, 0, 0, 0, 0};
        const double fq = flux_vjp(pFp, pHp, pFm, pHm, gq, w, gp, gm, a.sp.adj_frozen != 0);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          gLR[(16 + c * 4 + q) * NT] = mf[c] * fq;  // gR[c][q]
          double sl = 0.0;
#pragma unroll
          for (int kk = 0; kk < 3; ++kk) {
            sl += gp[kk] * sFp[c][jf + kk] + gp[3 + kk] * sHp[c][jf + kk] +
                  gm[kk] * sFm[c][jf + 1 + kk] + gm[3 + kk] * sHm[c][jf + 1 + kk];
            acc(kk, c, e.L[q][c] * gp[kk]);
            acc(kk, 2 * M + c, e.L[q][c] * gp[3 + kk]);
            acc(kk + 1, M + c, e.L[q][c] * gm[kk]);
            acc(kk + 1, 3 * M + c, e.L[q][c] * gm[3 + kk]);
          }
          gLR[(q * 4 + c) * NT] = sl;  // gL[q][c]
        }
      }
      double g3[3];
      eigen2_vjp<DIR>(ub, vb, Hb, gm1, gLR, g3);
      // Roe average -> the two states (slots 1 and 2, direct u cotangents)
      const double gsL = (g3[0] * (uL - ub) + g3[1] * (vL - vb) + g3[2] * (HL - Hb)) * iS;
      const double gsR = (g3[0] * (uR - ub) + g3[1] * (vR - vb) + g3[2] * (HR - Hb)) * iS;
      double gUL[4] = {0.5 * gsL / sL, 0, 0, 0}, gUR[4] = {0.5 * gsR / sR, 0, 0, 0};
      velh2_vjp(UL, gm1, g3[0] * sL * iS, g3[1] * sL * iS, g3[2] * sL * iS, gUL);
      velh2_vjp(UR, gm1, g3[0] * sR * iS, g3[1] * sR * iS, g3[2] * sR * iS, gUR);
      // kept in this thread's scratch until the per-slot conversion below
#pragma unroll
      for (int c = 0; c < 4; ++c) { gLR[c * NT] = gUL[c]; gLR[(4 + c) * NT] = gUR[c]; }
    }
    // per slot, in place: gF, gH, direct gu (splitting, Roe), direct gN
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
#pragma unroll
      for (int c = 0; c < M; ++c) {
        const double fp = sIt[kk * NS + c][jf], fm = sIt[kk * NS + M + c][jf];
        const double hp = sIt[kk * NS + 2 * M + c][jf], hm = sIt[kk * NS + 3 * M + c][jf];
        double du = 0.5 * alpha * (fp - fm);
        if constexpr (EUL) {
          if (kk == 1) du += sG[c * NT + threadIdx.x];
          if (kk == 2) du += sG[(4 + c) * NT + threadIdx.x];
        }
        sIt[kk * NS + c][jf] = 0.5 * (fp + fm);
        sIt[kk * NS + M + c][jf] = hh * (hp + hm);
        sIt[kk * NS + 2 * M + c][jf] = du;
        sIt[kk * NS + 3 * M + c][jf] = hh * alpha * (hp - hm);
      }
  }

  // B2: limiter items j = s-1+jl; points j-1, j, j+1 loaded jl+1..jl+3
  for (int jl = threadIdx.x; jl < np + 2; jl += blockDim.x) {
#pragma unroll
    for (int f = 0; f < 5 * M; ++f) sLm[f][jl] = 0.0;
    if (lim == 2 || (lim == 1 && !EUL)) {  // component-wise
#pragma unroll
      for (int c = 0; c < M; ++c) {
        double g5[5] = {0, 0, 0, 0, 0};
        limiter_vjp(su[c][jl + 1], su[c][jl + 2], su[c][jl + 3], h * sN[c][jl + 1],
                    h * sN[c][jl + 3], ml[c][jl] * ih, w, g5, a.sp.adj_frozen != 0);
        sLm[c][jl] = g5[0]; sLm[M + c][jl] = g5[1]; sLm[2 * M + c][jl] = g5[2];
        sLm[3 * M + c][jl] = h * g5[3]; sLm[4 * M + c][jl] = h * g5[4];
      }
    } else if constexpr (EUL) {
      if (lim == 1) {  // characteristic, eigenvectors of A_d at U_j
        double U0[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) U0[c] = su[c][jl + 2];
        double u0, v0, H0;
        velh2(U0, gm1, u0, v0, H0);
        Eigen<double, 4> e;
        eigen2<DIR>(u0, v0, H0, gm1, e);
        double* gLR = sG + threadIdx.x;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          double gz = 0.0;
#pragma unroll
          for (int c = 0; c < 4; ++c) gz += e.R[c][q] * ml[c][jl];
          gz *= ih;
          double x[5] = {0, 0, 0, 0, 0};
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            x[0] += e.L[q][c] * su[c][jl + 1];
            x[1] += e.L[q][c] * su[c][jl + 2];
            x[2] += e.L[q][c] * su[c][jl + 3];
            x[3] += e.L[q][c] * sN[c][jl + 1];
            x[4] += e.L[q][c] * sN[c][jl + 3];
          }
          double g5[5] = {0, 0, 0, 0, 0};
          const double z = limiter_vjp(x[0], x[1], x[2], h * x[3], h * x[4], gz, w, g5,
                                       a.sp.adj_frozen != 0);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            gLR[(16 + c * 4 + q) * NT] = ml[c][jl] * ih * z;
            gLR[(q * 4 + c) * NT] = g5[0] * su[c][jl + 1] + g5[1] * su[c][jl + 2] +
                                    g5[2] * su[c][jl + 3] +
                                    h * (g5[3] * sN[c][jl + 1] + g5[4] * sN[c][jl + 3]);
            sLm[c][jl] += e.L[q][c] * g5[0];
            sLm[M + c][jl] += e.L[q][c] * g5[1];
            sLm[2 * M + c][jl] += e.L[q][c] * g5[2];
            sLm[3 * M + c][jl] += h * e.L[q][c] * g5[3];
            sLm[4 * M + c][jl] += h * e.L[q][c] * g5[4];
          }
        }
        double g3[3], gc[4] = {0, 0, 0, 0};
        eigen2_vjp<DIR>(u0, v0, H0, gm1, gLR, g3);
        velh2_vjp(U0, gm1, g3[0], g3[1], g3[2], gc);
#pragma unroll
        for (int c = 0; c < 4; ++c) sLm[M + c][jl] += gc[c];
      }
    }
  }
  __syncthreads();

  // C: per loaded point, gather the slots (fixed order) and pull the point
  // flux cotangents back to (u, N, T)
  for (int g = threadIdx.x; g < np + 6; g += blockDim.x) {
    double gF[M], gH[M], gE[M], gu[M], gN[M], gT[M];
#pragma unroll
    for (int c = 0; c < M; ++c) { gF[c] = gH[c] = gE[c] = gu[c] = gN[c] = gT[c] = 0.0; }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const int jf = g - kk;
      if (jf < 0 || jf >= np + 3) continue;
#pragma unroll
      for (int c = 0; c < M; ++c) {
        gF[c] += sIt[kk * NS + c][jf];
        gH[c] += sIt[kk * NS + M + c][jf];
        gu[c] += sIt[kk * NS + 2 * M + c][jf];
        gN[c] += sIt[kk * NS + 3 * M + c][jf];
        gE[c] += sIt[kk * NS + 4 * M + c][jf];
      }
    }
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
      const int jl = g - 1 - kk;
      if (jl < 0 || jl >= np + 2) continue;
#pragma unroll
      for (int c = 0; c < M; ++c) gu[c] += sLm[kk * M + c][jl];
    }
    if (g - 1 >= 0 && g - 1 < np + 2)
#pragma unroll
      for (int c = 0; c < M; ++c) gN[c] += sLm[3 * M + c][g - 1];
    if (g - 3 >= 0 && g - 3 < np + 2)
#pragma unroll
      for (int c = 0; c < M; ++c) gN[c] += sLm[4 * M + c][g - 3];
    double u[M], N[M], T[M];
#pragma unroll
    for (int c = 0; c < M; ++c) { u[c] = su[c][g]; N[c] = sN[c][g]; T[c] = sT[c][g]; }
    point2_vjp<EQ, DIR>(u, N, T, gF, gH, gE, gm1, gu, gN, gT);
#pragma unroll
    for (int c = 0; c < M; ++c) { tU[c][g] = gu[c]; tN[c][g] = gN[c]; tT[c][g] = gT[c]; }
  }
  __syncthreads();

  // D: owned points: ghost images at walls, then the output of the sweep
  for (int ip = threadIdx.x; ip < np; ip += blockDim.x) {
    const int g = ip + 3;
    double ru[M], rn[M], rt[M];
#pragma unroll
    for (int c = 0; c < M; ++c) {
      ru[c] = tU[c][g];
      rn[c] = tN[c][g] + (lim == 0 ? ml[c][ip + 1] : 0.0);
      rt[c] = tT[c][g];
    }
    if (!periodic) {
#pragma unroll
      for (int e6 = 0; e6 < 6; ++e6) {
        const int gg = e6 < 3 ? e6 : np + e6;  // 0,1,2 and np+3..np+5
        const int p = s - 3 + gg;
        if (p >= 0 && p < n) continue;  // a halo point of another tile
        const Src sr = src_of(p);
        if (sr.kind == 2 || sr.idx != s + ip) continue;
#pragma unroll
        for (int c = 0; c < M; ++c) {
          const double sg = sr.kind == 1 ? (double)refl2<EQ, DIR>(c) : 1.0;
          ru[c] += sg * tU[c][gg];
          rn[c] += (sr.kind == 1 ? -sg : 1.0) * tN[c][gg];
          rt[c] += sg * tT[c][gg];
        }
      }
    }
    const long long q0 = at(s + ip);
#pragma unroll
    for (int c = 0; c < M; ++c) {
      const long long q = c * Ntot + q0;
      if constexpr (DIR == 0) {
        a.part[q] = ru[c];
        a.part[(M + c) * Ntot + q0] = rn[c];      // V
        a.part[(2 * M + c) * Ntot + q0] = rt[c];  // W
      } else {
        a.outU[q] = a.part[q] + ru[c] + a.b * a.lamU[q] + (a.accU ? a.accU[q] : 0.0);
        a.outV[q] = a.part[(M + c) * Ntot + q0] + rt[c];
        a.outW[q] = a.part[(2 * M + c) * Ntot + q0] + rn[c];
        if (a.accOutU) {
          a.accOutU[q] = a.cN * a.lamNU[q] + a.c2 * a.lamU[q];
          a.accOutVt[q] = a.cN * a.lamNV[q] + a.c2 * a.lamV[q];
          a.accOutWt[q] = a.cN * a.lamNW[q] + a.c2 * a.lamW[q];
        }
      }
    }
  }
}

template <int EQ, int DIR>
cudaError_t sweep_launch(const AdjArgs2D& a, cudaStream_t s) {
  constexpr size_t bytes = AdjLayout2D<EQ>::bytes;
  static unsigned configured = 0;  // devices whose limit is raised
  if (const cudaError_t e = ensure_smem_limit(k_adjoint_sweep_2d<EQ, DIR>, bytes, configured)) return e;
  const int n = DIR == 0 ? a.nx : a.ny, lines = DIR == 0 ? a.ny : a.nx;
  const dim3 grid((n + P - 1) / P, lines);
  k_adjoint_sweep_2d<EQ, DIR><<<grid, NT, bytes, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_adjoint_2d(int eq, int dir, const AdjArgs2D& a, cudaStream_t s) {
  if (eq == HWENO_BURGERS)
    return dir == 0 ? sweep_launch<HWENO_BURGERS, 0>(a, s) : sweep_launch<HWENO_BURGERS, 1>(a, s);
  return dir == 0 ? sweep_launch<HWENO_EULER, 0>(a, s) : sweep_launch<HWENO_EULER, 1>(a, s);
}

}  // namespace hweno
