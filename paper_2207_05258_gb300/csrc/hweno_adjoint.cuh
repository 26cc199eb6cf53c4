// Reverse-mode derivatives (vector-Jacobian products) of the scalar building
// blocks of the L-HWENO stage (Zhang & Zhao, arXiv:2207.05258, Sec. 2.1-2.2),
// written by hand from the forward formulas. They differentiate the functions
// themselves (the per-weight form of the nonlinear weights), not the folded
// arrangement used by the forward kernels; beta_0 of the reconstruction is
// taken in the forward kernels' rewritten form (equal in exact arithmetic to
// Eq. GHYZP, with e1 = H_i and the square weights in the coefficients of the
// squared sums), which also keeps the cotangents of a1, a3 and e1 from
// cancelling in floating point; the |.| in tau keeps the sign of
// its argument at the point of evaluation (the branch of the forward run).
// With `frozen` the nonlinear weights count as constants: only the
// candidates' (linear) dependence on the data is propagated.
#pragma once

#include "hweno_math.cuh"

namespace hweno {

namespace adj {
constexpr double K6 = 63.0 / 130.0, K8 = 13.0 / 3.0, K9 = 781.0 / 20.0;
constexpr double K10 = 1421461.0 / 2275.0, K11 = 21520059541.0 / 1377684.0;
constexpr double C11 = 11.0 / 60.0, C19 = 19.0 / 30.0;
// beta_0 of the reconstruction as H_i^2 + E2^2 + E3^2 + A4^2 + K11 a5^2 (the
// forward kernels' form; e1 = a1 + a3/4 + a5/16 reduces to H_i): E2 =
// sqrt(13/3) e2, E3 = sqrt(781/20) e3, A4 = sqrt(1421461/2275) a4 in the
// stencil sums (square roots times the exact coefficients, to 20 digits)
constexpr double E2d = 0.52842290755678754049, E2l = 2.0976788148466414486;
constexpr double E3s = -1.6032089149031235916, E3h = -12.661835579599691806,
                 E3d = -7.9341267047029694945;
constexpr double A4d = -6.2490900436484649542, A4l = -12.498180087296929908;
}  // namespace adj

// Source of point p of an instance with n points (maybe a ghost): kind 0
// copy, 1 mirror (reflective wall), 2 imposed state (no dependence on the
// instance's values). Same mapping as the forward stage's loads.
__device__ __forceinline__ int ghost_src(int p, int n, int bclo, int bchi, int& kind) {
  kind = 0;
  if (p >= 0 && p < n) return p;
  const int b = p < 0 ? bclo : bchi;
  if (b == HWENO_BC_PERIODIC) return p < 0 ? p + n : p - n;
  if (b == HWENO_BC_OUTFLOW) return p < 0 ? 0 : n - 1;
  if (b == HWENO_BC_REFLECTIVE) { kind = 1; return p < 0 ? -p - 1 : 2 * n - 1 - p; }
  kind = 2;
  return 0;
}

__device__ __forceinline__ double sgn(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0); }

// One side of the nonlinear flux, f-hat^+ from (f, H = dx h) on {i-1, i, i+1}
// (Sec. 2.1): returns the value and adds mu * d f-hat / d input to g[6]
// (order fm, f0, fp, Hm, H0, Hp).
__device__ __forceinline__ double side_vjp(double fm, double f0, double fp, double Hm, double H0,
                                           double Hp, double mu, const Weights<double>& w,
                                           double* g, bool frozen = false) {
  using namespace adj;
  const double sHp = Hm + Hp, dHp = Hm - Hp, lap = fm - 2.0 * f0 + fp, dif = fm - fp;
  const double p0 = C11 * (fm + fp) + C19 * f0 + 0.05 * dHp + 0.5 * H0;
  const double p1 = fm / 6.0 + 5.0 * f0 / 6.0 + 2.0 * H0 / 3.0;
  const double p2 = 5.0 * f0 / 6.0 + fp / 6.0 + H0 / 3.0;
  const double E2 = E2d * dHp + E2l * lap;
  const double E3 = E3s * sHp + E3h * H0 + E3d * dif;
  const double A4 = A4d * dHp + A4l * lap;
  const double a5 = 0.25 * sHp + H0 + 0.75 * dif;
  const double h2 = H0 * H0;
  const double be0 = h2 + E2 * E2 + E3 * E3 + A4 * A4 + K11 * a5 * a5;
  const double s1 = H0 - f0 + fm, s2 = H0 + f0 - fp;
  const double be1 = h2 + K8 * s1 * s1, be2 = h2 + K8 * s2 * s2;
  const double d1 = be0 - be1, d2 = be0 - be2;
  const double t = fabs(d1) + fabs(d2), tau = 0.25 * t * t;
  const double b0 = be0 + w.eps, b1 = be1 + w.eps, b2 = be2 + w.eps;
  // 1/b0, 1/b1, 1/b2 from one division: b0 b1 b2 stays inside the FP64
  // range while beta < 1e100 (split-flux jumps below about 1e48)
  const double b12 = b1 * b2, inv = 1.0 / (b0 * b12);
  const double ib0 = b12 * inv, ib1 = b0 * b2 * inv, ib2 = b0 * b1 * inv;
  const double r0 = tau * ib0, r1 = tau * ib1, r2 = tau * ib2;
  const double o0 = w.g0 * (1.0 + r0), o1 = w.g1 * (1.0 + r1), o2 = w.g2 * (1.0 + r2);
  const double iS = 1.0 / (o0 + o1 + o2);
  const double Q0 = (p0 - w.g1 * p1 - w.g2 * p2) * w.ig0;
  const double fh = (o0 * Q0 + o1 * p1 + o2 * p2) * iS;
  // reverse
  const double gN = mu * iS, gS = -gN * fh;
  const double go0 = gN * Q0 + gS, go1 = gN * p1 + gS, go2 = gN * p2 + gS;
  const double gQ0 = gN * o0;
  const double gp0 = gQ0 * w.ig0;
  const double gp1 = gN * o1 - gQ0 * w.ig0 * w.g1;
  const double gp2 = gN * o2 - gQ0 * w.ig0 * w.g2;
  const double fz = frozen ? 0.0 : 1.0;  // weights held: no tau / beta terms
  const double c0 = fz * go0 * w.g0 * ib0, c1 = fz * go1 * w.g1 * ib1, c2 = fz * go2 * w.g2 * ib2;
  const double gtau = c0 + c1 + c2;
  const double gb0 = -c0 * r0, gb1 = -c1 * r1, gb2 = -c2 * r2;
  const double gt = 0.5 * t * gtau;
  const double gd1 = gt * sgn(d1), gd2 = gt * sgn(d2);
  const double gbe0 = gb0 + gd1 + gd2, gbe1 = gb1 - gd1, gbe2 = gb2 - gd2;
  const double gs1 = 2.0 * K8 * s1 * gbe1, gs2 = 2.0 * K8 * s2 * gbe2;
  const double tg = 2.0 * gbe0;
  const double gE2 = tg * E2, gE3 = tg * E3, gA4 = tg * A4, ga5 = K11 * a5 * tg;
  const double gsHp = E3s * gE3 + 0.25 * ga5;
  const double gdHp = E2d * gE2 + A4d * gA4 + 0.05 * gp0;
  const double glap = E2l * gE2 + A4l * gA4;
  const double gdif = E3d * gE3 + 0.75 * ga5;
  const double gH0 = 2.0 * H0 * (gbe0 + gbe1 + gbe2) + E3h * gE3 + ga5 + 0.5 * gp0 +
                     2.0 / 3.0 * gp1 + 1.0 / 3.0 * gp2 + gs1 + gs2;
  g[0] += C11 * gp0 + gp1 / 6.0 + glap + gdif + gs1;
  g[1] += C19 * gp0 + 5.0 / 6.0 * (gp1 + gp2) - 2.0 * glap - gs1 + gs2;
  g[2] += C11 * gp0 + gp2 / 6.0 + glap - gdif - gs2;
  g[3] += gsHp + gdHp;
  g[4] += gH0;
  g[5] += gsHp - gdHp;
  return fh;
}

// Both sides of one field's flux at x_{i+1/2}: returns f-hat = f-hat^+ +
// f-hat^-; gp (6: f^+ at i-1..i+1, H^+ at i-1..i+1) and gm (6: f^- at i..i+2,
// H^- at i..i+2) receive mu times the partial derivatives. The "-" side is
// the mirror image (reversed stencil, negated H).
__device__ __forceinline__ double flux_vjp(const double* fp_, const double* Hp_, const double* fm_,
                                         const double* Hm_, double mu, const Weights<double>& w,
                                         double* gp, double* gm, bool frozen = false) {
  const double fp = side_vjp(fp_[0], fp_[1], fp_[2], Hp_[0], Hp_[1], Hp_[2], mu, w, gp, frozen);
  double r[6] = {0, 0, 0, 0, 0, 0};
  const double fm =
      side_vjp(fm_[2], fm_[1], fm_[0], -Hm_[2], -Hm_[1], -Hm_[0], mu, w, r, frozen);
  gm[0] += r[2]; gm[1] += r[1]; gm[2] += r[0];
  gm[3] -= r[5]; gm[4] -= r[4]; gm[5] -= r[3];
  return fp + fm;
}

// One side of flux_vjp: sd = 0 the "+" side from (f0, f1, f2, H0, H1, H2) =
// f^+, H^+ at i-1..i+1; sd = 1 the "-" side from f^-, H^- at i..i+2 (its
// mirror image). Returns the side's value and adds mu times its partial
// derivatives to g (f then H, in stencil order).
__device__ __forceinline__ double side_half(int sd, double f0, double f1, double f2, double H0,
                                          double H1, double H2, double mu,
                                          const Weights<double>& w, double* g,
                                          bool frozen = false) {
  double r[6] = {0, 0, 0, 0, 0, 0};
  const double v = side_vjp(sd ? f2 : f0, f1, sd ? f0 : f2, sd ? -H2 : H0, sd ? -H1 : H1,
                            sd ? -H0 : H2, mu, w, r, frozen);
  if (sd) {
    g[0] += r[2]; g[1] += r[1]; g[2] += r[0];
    g[3] -= r[5]; g[4] -= r[4]; g[5] -= r[3];
  } else {
#pragma unroll
    for (int k = 0; k < 6; ++k) g[k] += r[k];
  }
  return v;
}

// Linear derivative flux D = dx (h-hat^+ + h-hat^-) (Sec. 2.1, p_0'):
// adds mu * dD/d input to gp, gm (same layout as flux_vjp).
__device__ __forceinline__ void dflux_vjp(double mu, double* gp, double* gm) {
  gp[0] += 0.25 * mu; gp[1] += -2.0 * mu; gp[2] += 1.75 * mu;
  gp[3] += mu / 12.0; gp[4] += -mu / 6.0; gp[5] += -5.0 * mu / 12.0;
  gm[0] += -1.75 * mu; gm[1] += 2.0 * mu; gm[2] += -0.25 * mu;
  gm[3] += -5.0 * mu / 12.0; gm[4] += -mu / 6.0; gm[5] += mu / 12.0;
}

// HWENO limiter (Sec. 2.2) in scaled form, out = dx v-tilde from point values
// um, u0, up and Vm = dx v_{i-1}, Vp = dx v_{i+1}: returns out and adds
// mu * d out / d input to g[5] (order um, u0, up, Vm, Vp).
__device__ __forceinline__ double limiter_vjp(double um, double u0, double up, double Vm, double Vp,
                                            double mu, const Weights<double>& w, double* g,
                                            bool frozen = false) {
  using namespace adj;
  const double sV = Vm + Vp, dV = Vm - Vp, lap = um - 2.0 * u0 + up, dup = up - um;
  const double q0 = 0.75 * dup - 0.25 * sV, q1 = u0 - um, q2 = up - u0;
  const double a2 = 0.25 * dV + lap, a3 = 0.25 * sV - 0.25 * dup, a4 = -0.25 * dV - 0.5 * lap;
  const double e1 = q0 + 0.25 * a3, e2 = a2 + K6 * a4;
  const double be0 = e1 * e1 + K8 * e2 * e2 + K9 * a3 * a3 + K10 * a4 * a4;
  const double be1 = q1 * q1, be2 = q2 * q2;
  const double d1 = be0 - be1, d2 = be0 - be2;
  const double t = fabs(d1) + fabs(d2), tau = 0.25 * t * t;
  const double b0 = be0 + w.eps, b1 = be1 + w.eps, b2 = be2 + w.eps;
  const double b12 = b1 * b2, inv = 1.0 / (b0 * b12);
  const double ib0 = b12 * inv, ib1 = b0 * b2 * inv, ib2 = b0 * b1 * inv;
  const double r0 = tau * ib0, r1 = tau * ib1, r2 = tau * ib2;
  const double l0 = w.d0 * (1.0 + r0), l1 = w.d1 * (1.0 + r1), l2 = w.d2 * (1.0 + r2);
  const double iS = 1.0 / (l0 + l1 + l2);
  const double Q0 = (q0 - w.d1 * q1 - w.d2 * q2) * w.id0;
  const double out = (l0 * Q0 + l1 * q1 + l2 * q2) * iS;
  const double gN = mu * iS, gS = -gN * out;
  const double gl0 = gN * Q0 + gS, gl1 = gN * q1 + gS, gl2 = gN * q2 + gS;
  const double gQ0 = gN * l0;
  double gq0 = gQ0 * w.id0;
  double gq1 = gN * l1 - gQ0 * w.id0 * w.d1;
  double gq2 = gN * l2 - gQ0 * w.id0 * w.d2;
  const double fz = frozen ? 0.0 : 1.0;
  const double c0 = fz * gl0 * w.d0 * ib0, c1 = fz * gl1 * w.d1 * ib1, c2 = fz * gl2 * w.d2 * ib2;
  const double gt = 0.5 * t * (c0 + c1 + c2);
  const double gd1 = gt * sgn(d1), gd2 = gt * sgn(d2);
  const double gbe0 = -c0 * r0 + gd1 + gd2;
  const double gbe1 = -c1 * r1 - gd1;
  const double gbe2 = -c2 * r2 - gd2;
  gq1 += 2.0 * q1 * gbe1;
  gq2 += 2.0 * q2 * gbe2;
  const double ge1 = 2.0 * e1 * gbe0, ge2 = 2.0 * K8 * e2 * gbe0;
  double ga3 = 2.0 * K9 * a3 * gbe0 + 0.25 * ge1;
  double ga4 = 2.0 * K10 * a4 * gbe0 + K6 * ge2;
  const double ga2 = ge2;
  gq0 += ge1;
  // a2, a3, a4, q0 -> (sV, dV, lap, dup)
  const double gsV = -0.25 * gq0 + 0.25 * ga3;
  const double gdV = 0.25 * ga2 - 0.25 * ga4;
  const double glap = ga2 - 0.5 * ga4;
  const double gdup = 0.75 * gq0 - 0.25 * ga3;
  g[0] += glap - gdup - gq1;
  g[1] += -2.0 * glap + gq1 - gq2;
  g[2] += glap + gdup + gq2;
  g[3] += gsV + gdV;
  g[4] += gsV - gdV;
  return out;
}

}  // namespace hweno
