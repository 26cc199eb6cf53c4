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
// point-flux cotangents back to (U, N, T) by a reverse pass through the flux
// and Jacobian-vector products; owned points add their ghost images at walls.
// Two threads (in different warps) share each item. The characteristic pieces follow the 1D Euler adjoint with the
// 4x4 eigen-system of A_d at the Roe average (u, v, H). No atomics.
#include "flux2d.cuh"
#include "hweno.h"
#include "hweno_adjoint.cuh"
#include "internal.h"

namespace hweno {
namespace {

// 128 threads: two CTAs (2 x 99.5 KB of shared memory, 180 registers) per
// SM, whose barriers overlap; measured 3.7% faster per adjoint step than one
// CTA of 256 threads with 122-point tiles, despite the wider halo share.
#ifndef HWENO_ADJ2D_NT
#define HWENO_ADJ2D_NT 128
#endif
constexpr int NT = HWENO_ADJ2D_NT;  // threads: two per item (NT / 2 a power of two)
static_assert((NT & (NT - 1)) == 0 && NT >= 128, "NT / 2 indexes items with a mask");
constexpr int NH = NT / 2;  // items per pass
constexpr int P = NH - 6;   // owned points per tile (the loaded points fill one pass)
constexpr int NL = P + 6;   // loaded points s-3 .. s+P+2
constexpr int NI = P + 3;   // interfaces j = s-2 .. s+P
constexpr int NV = P + 2;   // limiter items j = s-1 .. s+P

template <int EQ>
struct AdjLayout2D {
  static constexpr int M = Dim2<EQ>::M;
  // loads: u, N, T, F+, F-, H+, H-, E (8M rows of NL); cotangent inputs m1,
  // mn, mt (3M rows of P + 4) and mlim (M rows of NV); interface slots (4
  // slots x 5M fields x NI); limiter items (5M fields x NV); per-item
  // scratch for the eigenvector cotangents and the second half's partial
  // sums (Euler: 32 + 20 rows of NH)
  static constexpr size_t doubles = (size_t)8 * M * NL + 3 * M * (P + 4) + M * NV +
                                    (size_t)20 * M * NI + 5 * M * NV +
                                    (EQ == HWENO_EULER ? 52 * NH : 0);
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

// Pullback of sum gL.L + gR.R (gLR: gL[r][k] at r*4+k, gR[r][k] at
// 16+r*4+k, stride NH in shared memory) onto (u, v, H): one reverse pass
// through the formulas of euler_eigen (b1 = (gamma-1)/c^2, b2 = b1 q,
// q = (u^2+v^2)/2, c^2 = (gamma-1)(H - q)).
template <int DIR>
__device__ __forceinline__ void eigen2_vjp(double u, double v, double H, double gm1,
                                           const double* gLR, double* g3) {
  constexpr int kn = DIR == 0 ? 1 : 2, kt = DIR == 0 ? 2 : 1;
  auto gL = [&](int r, int k) { return gLR[(r * 4 + k) * NH]; };
  auto gR = [&](int r, int k) { return gLR[(16 + r * 4 + k) * NH]; };
  const double un = DIR == 0 ? u : v, ut = DIR == 0 ? v : u;
  const double q = 0.5 * (u * u + v * v);
  const double c = ::sqrt(gm1 * (H - q)), ic = 1.0 / c;
  const double b1 = gm1 * ic * ic;
  // cotangents of the intermediate scalars, read off the entries
  const double sLn = gL(0, kn) + gL(3, kn), sLt = gL(0, kt) + gL(3, kt);
  const double a_b2 = 0.5 * (gL(0, 0) + gL(3, 0)) - gL(1, 0);
  const double a_unc = 0.5 * (gL(0, 0) - gL(3, 0));
  double a_b1 = -0.5 * (un * sLn + ut * sLt) + 0.5 * (gL(0, 3) + gL(3, 3)) + un * gL(1, kn) +
                ut * gL(1, kt) - gL(1, 3);
  double a_ic = 0.5 * (gL(3, kn) - gL(0, kn));
  double a_un = b1 * (gL(1, kn) - 0.5 * sLn) + gR(kn, 0) + gR(kn, 1) + gR(kn, 3) +
                c * (gR(3, 3) - gR(3, 0));
  const double a_ut = b1 * (gL(1, kt) - 0.5 * sLt) - gL(2, 0) + gR(kt, 0) + gR(kt, 1) +
                      gR(kt, 3) + gR(3, 2);
  double a_c = gR(kn, 3) - gR(kn, 0) + un * (gR(3, 3) - gR(3, 0));
  double a_H = gR(3, 0) + gR(3, 3);
  double a_q = gR(3, 1);
  // b2 = b1 q, unc = un ic, b1 = gm1 ic^2, ic = 1/c, c = sqrt(gm1 (H - q))
  a_b1 += q * a_b2;
  a_q += b1 * a_b2;
  a_un += ic * a_unc;
  a_ic += un * a_unc + 2.0 * gm1 * ic * a_b1;
  a_c -= ic * ic * a_ic;
  const double a_in = 0.5 * gm1 * ic * a_c;  // d c / d (H - q) = gm1 / (2 c)
  a_H += a_in;
  a_q -= a_in;
  g3[0] = u * a_q + (DIR == 0 ? a_un : a_ut);
  g3[1] = v * a_q + (DIR == 0 ? a_ut : a_un);
  g3[2] = a_H;
}

// Reverse pass through U -> gF.F(U) + gH.A(U)N + gE.A(U)T, with F the flux
// of direction DIR and A its Jacobian (the products of Eq. EQ3, computed by
// prim2 / flux2 / jvp2): adds the cotangent of U to gu.
template <int EQ, int DIR>
__device__ __forceinline__ void point2_vjp_u(const double* U, const double* N, const double* T,
                                             const double* gF, const double* gH,
                                             const double* gE, double gm1, double* gu) {
  if constexpr (EQ == HWENO_BURGERS) {
    gu[0] += gF[0] * U[0] + gH[0] * N[0] + gE[0] * T[0];
  } else {
    constexpr int a = DIR == 0 ? 1 : 2;  // momentum along DIR
    const double ir = 1.0 / U[0], u = U[1] * ir, v = U[2] * ir;
    const double p = gm1 * (U[3] - 0.5 * (U[1] * u + U[2] * v)), Ep = U[3] + p;
    const double un = DIR == 0 ? u : v;
    double aU[4] = {0.0, 0.0, 0.0, 0.0};
    double au = 0.0, av = 0.0, ap = 0.0, aEp = 0.0, air = 0.0;
    // F = (U_a, U_a u + [a=1] p, U_a v + [a=2] p, Ep un)
    aU[a] += gF[0] + gF[1] * u + gF[2] * v;
    au += gF[1] * U[a];
    av += gF[2] * U[a];
    ap += gF[a];
    aEp += gF[3] * un;
    (DIR == 0 ? au : av) += gF[3] * Ep;
    // A D = (D_a, D_a u + U_a du + [a=1] dp, D_a v + U_a dv + [a=2] dp,
    // (D_3 + dp) un + Ep dun) with du = (D1 - u D0)/rho, dv = (D2 - v D0)/rho,
    // dp = gm1 (D3 - u D1 - v D2 + q D0)
    auto jvp_rev = [&](const double* D, const double* g) {
      const double du = (D[1] - u * D[0]) * ir, dv = (D[2] - v * D[0]) * ir;
      const double dp = gm1 * (D[3] - (u * D[1] + v * D[2]) + 0.5 * (u * u + v * v) * D[0]);
      au += g[1] * D[a];
      av += g[2] * D[a];
      (DIR == 0 ? au : av) += g[3] * (D[3] + dp);
      aU[a] += g[1] * du + g[2] * dv;
      aEp += g[3] * (DIR == 0 ? du : dv);
      const double adu = g[1] * U[a] + (DIR == 0 ? g[3] * Ep : 0.0);
      const double adv = g[2] * U[a] + (DIR == 1 ? g[3] * Ep : 0.0);
      const double adp = g[a] + g[3] * un;
      au += adp * gm1 * (u * D[0] - D[1]) - adu * D[0] * ir;
      av += adp * gm1 * (v * D[0] - D[2]) - adv * D[0] * ir;
      air += adu * (D[1] - u * D[0]) + adv * (D[2] - v * D[0]);
    };
    jvp_rev(N, gH);
    jvp_rev(T, gE);
    // Ep = U3 + p, p = gm1 (U3 - (U1 u + U2 v)/2), u = U1 ir, v = U2 ir, ir = 1/U0
    ap += aEp;
    aU[3] += aEp + gm1 * ap;
    aU[1] -= 0.5 * gm1 * ap * u;
    aU[2] -= 0.5 * gm1 * ap * v;
    au -= 0.5 * gm1 * ap * U[1];
    av -= 0.5 * gm1 * ap * U[2];
    aU[1] += au * ir;
    aU[2] += av * ir;
    air += au * U[1] + av * U[2];
    aU[0] -= air * ir * ir;
#pragma unroll
    for (int k = 0; k < 4; ++k) gu[k] += aU[k];
  }
}

// A^T g for the Jacobian A of the direction-DIR flux at U (a reverse pass
// through jvp2, which is linear in its derivative argument): adds to out.
template <int EQ, int DIR>
__device__ __forceinline__ void jac2_t(const double* U, const double* g, double gm1, double* out) {
  if constexpr (EQ == HWENO_BURGERS) {
    out[0] += U[0] * g[0];
  } else {
    constexpr int a = DIR == 0 ? 1 : 2;
    const double ir = 1.0 / U[0], u = U[1] * ir, v = U[2] * ir;
    const double p = gm1 * (U[3] - 0.5 * (U[1] * u + U[2] * v)), Ep = U[3] + p;
    const double un = DIR == 0 ? u : v;
    const double adu = g[1] * U[a] + (DIR == 0 ? g[3] * Ep : 0.0);
    const double adv = g[2] * U[a] + (DIR == 1 ? g[3] * Ep : 0.0);
    const double adp = g[a] + g[3] * un;
    double aD[4] = {0.0, 0.0, 0.0, 0.0};
    aD[a] += g[0] + g[1] * u + g[2] * v;
    aD[3] += g[3] * un + gm1 * adp;
    aD[1] += adu * ir - gm1 * adp * u;
    aD[2] += adv * ir - gm1 * adp * v;
    aD[0] += 0.5 * gm1 * adp * (u * u + v * v) - (adu * u + adv * v) * ir;
#pragma unroll
    for (int k = 0; k < 4; ++k) out[k] += aD[k];
  }
}

template <int EQ, int DIR>
__global__ void __launch_bounds__(NT, 256 / NT) k_adjoint_sweep_2d(const __grid_constant__ AdjArgs2D a) {
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
  double* sG = &sLm[5 * M][0];  // [32][NH] (Euler)
  double* sP = sG + 32 * NH;    // [20][NH] (Euler)

  const int nx = a.nx, ny = a.ny;
  const long long Ntot = (long long)nx * ny;
  const int n = DIR == 0 ? nx : ny;
  // block -> (tile, line): the full tiles of every line first, the ragged
  // last tiles (shorter work) at the end of the dispatch order
  int tile = blockIdx.x, line = blockIdx.y;
  {
    const int T = gridDim.x, F = T - 1;
    if (F > 0 && n % P != 0) {
      const long long b = (long long)blockIdx.y * T + blockIdx.x, full = (long long)gridDim.y * F;
      if (b < full) { tile = (int)(b % F); line = (int)(b / F); }
      else { tile = F; line = (int)(b - full); }
    }
  }
  const int s = tile * P;
  const int np = min(P, n - s);
  HWENO_CHECK(np >= 1 && line >= 0 && line < (DIR == 0 ? ny : nx), a.status);
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
  auto src_of = [&](int p) {
    return DIR == 0 ? map_x(p, nx, a.sp) : map_y(p, ny, line, a.x0, a.dx, a.y0, a.dy, ts, a.sp);
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
        HWENO_CHECK(sr.idx >= 0 && sr.idx < n, a.status);
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

  // The 256 threads work in pairs on one item: thread it of the first half
  // (warps 0-3, sd = 0) and thread it of the second half (warps 4-7, sd = 1),
  // so that two warps per sub-partition keep the FP64 pipe fed.
  const int it = threadIdx.x & (NH - 1), sd = threadIdx.x / NH;
  const bool frozen = a.sp.adj_frozen != 0;

  // B1a: interfaces j = s-2+jf (jf = it); stencil loaded jf..jf+3 (slots
  // 0..3). Side sd reverses the "+" reconstruction (sd = 0: f^+, H^+ in
  // slots 0..2) or the "-" one (sd = 1: f^-, H^- in slots 1..3) and owns
  // those fields of the four slots; the central flux's slots go two and two.
  const int jf = it;
  const int fF = sd * M, fH = 2 * M + sd * M;  // this side's F and H fields
  auto acc = [&](int kk, int f, double x) { sIt[kk * NS + f][jf] += x; };
  double mf[M];
  double UL[4], UR[4], uL = 0, vL = 0, HL = 0, uR = 0, vR = 0, HR = 0;
  double sL = 0, sR = 0, iS = 0, ub = 0, vb = 0, Hb = 0;
  if (jf < np + 3) {
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
#pragma unroll
      for (int c = 0; c < M; ++c) {
        sIt[kk * NS + fF + c][jf] = 0.0;
        sIt[kk * NS + fH + c][jf] = 0.0;
      }
#pragma unroll
    for (int kk = 0; kk < 2; ++kk)
#pragma unroll
      for (int c = 0; c < M; ++c) sIt[(2 * sd + kk) * NS + 4 * M + c][jf] = 0.0;
#pragma unroll
    for (int c = 0; c < M; ++c) {
      mf[c] = (m1[c][jf + 1] - m1[c][jf]) * ih;
      const double mD = (mn[c][jf + 1] - mn[c][jf]) * ih2;
      const double mc = (mt[c][jf + 1] - mt[c][jf]) * ih;
      double gp[6] = {0, 0, 0, 0, 0, 0}, gm[6] = {0, 0, 0, 0, 0, 0};
      dflux_vjp(mD, gp, gm);
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) {
        acc(kk + sd, fF + c, sd ? gm[kk] : gp[kk]);
        acc(kk + sd, fH + c, sd ? gm[3 + kk] : gp[3 + kk]);
      }
      // central flux (Eq. mixed): -1/12, 7/12, 7/12, -1/12
      acc(2 * sd, 4 * M + c, (sd ? 7.0 : -1.0) * mc / 12.0);
      acc(2 * sd + 1, 4 * M + c, (sd ? -1.0 : 7.0) * mc / 12.0);
    }
    const double (*SF)[NL] = sd ? sFm : sFp;
    const double (*SH)[NL] = sd ? sHm : sHp;
    const int b = jf + sd;  // first loaded point of this side's stencil
    if constexpr (!EUL) {
      double g6[6] = {0, 0, 0, 0, 0, 0};
      side_half(sd, SF[0][b], SF[0][b + 1], SF[0][b + 2], SH[0][b], SH[0][b + 1], SH[0][b + 2],
                mf[0], w, g6, frozen);
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) {
        acc(kk + sd, fF, g6[kk]);
        acc(kk + sd, fH, g6[3 + kk]);
      }
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) { UL[c] = su[c][jf + 1]; UR[c] = su[c][jf + 2]; }
      velh2(UL, gm1, uL, vL, HL);
      velh2(UR, gm1, uR, vR, HR);
      sL = ::sqrt(UL[0]); sR = ::sqrt(UR[0]); iS = 1.0 / (sL + sR);
      ub = (sL * uL + sR * uR) * iS; vb = (sL * vL + sR * vR) * iS;
      Hb = (sL * HL + sR * HR) * iS;
      Eigen<double, 4> e;
      eigen2<DIR>(ub, vb, Hb, gm1, e);
      // this side's share of gL (16) and its flux value per field (4)
      double* part = (sd ? sP : sG) + it;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        double gq = 0.0;
#pragma unroll
        for (int c = 0; c < 4; ++c) gq += e.R[c][q] * mf[c];
        double pF[3], pH[3];
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
          pF[kk] = pH[kk] = 0.0;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            pF[kk] += e.L[q][c] * SF[c][b + kk];
            pH[kk] += e.L[q][c] * SH[c][b + kk];
          }
        }
        double g6[6] = {0, 0, 0, 0, 0, 0};
        part[(16 + q) * NH] =
            side_half(sd, pF[0], pF[1], pF[2], pH[0], pH[1], pH[2], gq, w, g6, frozen);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          double sl = 0.0;
#pragma unroll
          for (int kk = 0; kk < 3; ++kk) {
            sl += g6[kk] * SF[c][b + kk] + g6[3 + kk] * SH[c][b + kk];
            acc(kk + sd, fF + c, e.L[q][c] * g6[kk]);
            acc(kk + sd, fH + c, e.L[q][c] * g6[3 + kk]);
          }
          part[(q * 4 + c) * NH] = sl;
        }
      }
    }
  }
  __syncthreads();

  // B1b (first half): the eigenvector cotangents of the pair, their pullback
  // through the Roe average, and per slot, in place: gF, gH, direct gu
  // (splitting, Roe), direct gN
  if (sd == 0 && jf < np + 3) {
    double gUL[4] = {0, 0, 0, 0}, gUR[4] = {0, 0, 0, 0};
    if constexpr (EUL) {
      double* gLR = sG + it;  // [32] stride NH: gL[q][c] at q*4+c, gR[c][q] at 16+c*4+q
      double fq[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) fq[q] = gLR[(16 + q) * NH] + sP[(16 + q) * NH + it];
#pragma unroll
      for (int r = 0; r < 16; ++r) gLR[r * NH] += sP[r * NH + it];
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int q = 0; q < 4; ++q) gLR[(16 + c * 4 + q) * NH] = mf[c] * fq[q];
      double g3[3];
      eigen2_vjp<DIR>(ub, vb, Hb, gm1, gLR, g3);
      // Roe average -> the two states (slots 1 and 2, direct u cotangents)
      const double gsL = (g3[0] * (uL - ub) + g3[1] * (vL - vb) + g3[2] * (HL - Hb)) * iS;
      const double gsR = (g3[0] * (uR - ub) + g3[1] * (vR - vb) + g3[2] * (HR - Hb)) * iS;
      gUL[0] = 0.5 * gsL / sL;
      gUR[0] = 0.5 * gsR / sR;
      velh2_vjp(UL, gm1, g3[0] * sL * iS, g3[1] * sL * iS, g3[2] * sL * iS, gUL);
      velh2_vjp(UR, gm1, g3[0] * sR * iS, g3[1] * sR * iS, g3[2] * sR * iS, gUR);
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
#pragma unroll
      for (int c = 0; c < M; ++c) {
        const double fp = sIt[kk * NS + c][jf], fm = sIt[kk * NS + M + c][jf];
        const double hp = sIt[kk * NS + 2 * M + c][jf], hm = sIt[kk * NS + 3 * M + c][jf];
        double du = 0.5 * alpha * (fp - fm);
        if constexpr (EUL) {
          if (kk == 1) du += gUL[c];
          if (kk == 2) du += gUR[c];
        }
        sIt[kk * NS + c][jf] = 0.5 * (fp + fm);
        sIt[kk * NS + M + c][jf] = hh * (hp + hm);
        sIt[kk * NS + 2 * M + c][jf] = du;
        sIt[kk * NS + 3 * M + c][jf] = hh * alpha * (hp - hm);
      }
  }
  __syncthreads();

  // B2a: limiter items j = s-1+jl (jl = it); points j-1, j, j+1 loaded
  // jl+1..jl+3. Component-wise: the components are split between the pair;
  // characteristic: the characteristic fields are (q = 2 sd, 2 sd + 1), the
  // first half accumulating into sLm and the second into sP.
  const int jl = it;
  const bool charlim = EUL && lim == 1;
  if (jl < np + 2) {
    if (lim == 2 || (lim == 1 && !EUL)) {  // component-wise
#pragma unroll
      for (int c = 0; c < M; ++c) {
        if ((M == 1 ? 0 : c / (M / 2)) != sd) continue;
        double g5[5] = {0, 0, 0, 0, 0};
        limiter_vjp(su[c][jl + 1], su[c][jl + 2], su[c][jl + 3], h * sN[c][jl + 1],
                    h * sN[c][jl + 3], ml[c][jl] * ih, w, g5, frozen);
        sLm[c][jl] = g5[0]; sLm[M + c][jl] = g5[1]; sLm[2 * M + c][jl] = g5[2];
        sLm[3 * M + c][jl] = h * g5[3]; sLm[4 * M + c][jl] = h * g5[4];
      }
    } else if (!charlim) {  // limiter off
      if (sd == 0)
#pragma unroll
        for (int f = 0; f < 5 * M; ++f) sLm[f][jl] = 0.0;
    } else if constexpr (EUL) {  // characteristic, eigenvectors of A_d at U_j
      auto lacc = [&](int f, double x) {
        if (sd) sP[f * NH + it] += x; else sLm[f][jl] += x;
      };
#pragma unroll
      for (int f = 0; f < 5 * M; ++f) {
        if (sd) sP[f * NH + it] = 0.0; else sLm[f][jl] = 0.0;
      }
      double U0[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) U0[c] = su[c][jl + 2];
      double u0, v0, H0;
      velh2(U0, gm1, u0, v0, H0);
      Eigen<double, 4> e;
      eigen2<DIR>(u0, v0, H0, gm1, e);
      double* gLR = sG + it;  // rows of this side's two fields only
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if ((q >> 1) != sd) continue;  // q stays a compile-time index
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
        const double z = limiter_vjp(x[0], x[1], x[2], h * x[3], h * x[4], gz, w, g5, frozen);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          gLR[(16 + c * 4 + q) * NH] = ml[c][jl] * ih * z;
          gLR[(q * 4 + c) * NH] = g5[0] * su[c][jl + 1] + g5[1] * su[c][jl + 2] +
                                  g5[2] * su[c][jl + 3] +
                                  h * (g5[3] * sN[c][jl + 1] + g5[4] * sN[c][jl + 3]);
          lacc(c, e.L[q][c] * g5[0]);
          lacc(M + c, e.L[q][c] * g5[1]);
          lacc(2 * M + c, e.L[q][c] * g5[2]);
          lacc(3 * M + c, h * e.L[q][c] * g5[3]);
          lacc(4 * M + c, h * e.L[q][c] * g5[4]);
        }
      }
    }
  }
  __syncthreads();

  // B2b (first half, characteristic limiter): the pair's sums and the
  // eigenvector pullback onto U_j
  if constexpr (EUL) {
    if (charlim && sd == 0 && jl < np + 2) {
#pragma unroll
      for (int f = 0; f < 5 * M; ++f) sLm[f][jl] += sP[f * NH + it];
      double U0[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) U0[c] = su[c][jl + 2];
      double u0, v0, H0;
      velh2(U0, gm1, u0, v0, H0);
      double g3[3], gc[4] = {0, 0, 0, 0};
      eigen2_vjp<DIR>(u0, v0, H0, gm1, sG + it, g3);
      velh2_vjp(U0, gm1, g3[0], g3[1], g3[2], gc);
#pragma unroll
      for (int c = 0; c < 4; ++c) sLm[M + c][jl] += gc[c];
    }
  }
  __syncthreads();

  // C: per loaded point, gather the slots (fixed order) and pull the point
  // flux cotangents back: the first half of the pair to u, the second to N
  // and T
  for (int g = it; g < np + 6; g += NH) {
    double gF[M], gH[M], gE[M], gd[M];  // gd: direct part of gu (sd = 0) or gN (sd = 1)
#pragma unroll
    for (int c = 0; c < M; ++c) { gF[c] = gH[c] = gE[c] = gd[c] = 0.0; }
    const int fd = sd ? 3 * M : 2 * M;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const int jf = g - kk;
      if (jf < 0 || jf >= np + 3) continue;
#pragma unroll
      for (int c = 0; c < M; ++c) {
        if (sd == 0) gF[c] += sIt[kk * NS + c][jf];
        gH[c] += sIt[kk * NS + M + c][jf];
        gd[c] += sIt[kk * NS + fd + c][jf];
        gE[c] += sIt[kk * NS + 4 * M + c][jf];
      }
    }
    double u[M];
#pragma unroll
    for (int c = 0; c < M; ++c) u[c] = su[c][g];
    if (sd == 0) {
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) {
        const int jl = g - 1 - kk;
        if (jl < 0 || jl >= np + 2) continue;
#pragma unroll
        for (int c = 0; c < M; ++c) gd[c] += sLm[kk * M + c][jl];
      }
      double N[M], T[M];
#pragma unroll
      for (int c = 0; c < M; ++c) { N[c] = sN[c][g]; T[c] = sT[c][g]; }
      point2_vjp_u<EQ, DIR>(u, N, T, gF, gH, gE, gm1, gd);
#pragma unroll
      for (int c = 0; c < M; ++c) tU[c][g] = gd[c];
    } else {
      if (g - 1 >= 0 && g - 1 < np + 2)
#pragma unroll
        for (int c = 0; c < M; ++c) gd[c] += sLm[3 * M + c][g - 1];
      if (g - 3 >= 0 && g - 3 < np + 2)
#pragma unroll
        for (int c = 0; c < M; ++c) gd[c] += sLm[4 * M + c][g - 3];
      double gT[M];
#pragma unroll
      for (int c = 0; c < M; ++c) gT[c] = 0.0;
      jac2_t<EQ, DIR>(u, gH, gm1, gd);
      jac2_t<EQ, DIR>(u, gE, gm1, gT);
#pragma unroll
      for (int c = 0; c < M; ++c) { tN[c][g] = gd[c]; tT[c][g] = gT[c]; }
    }
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
