// Device arithmetic of the L-HWENO scheme (Zhang & Zhao, arXiv:2207.05258).
//
// Formulation used on the GPU (same mathematics as the paper, arranged for an
// FP64 pipe that is the bottleneck on sm_103a):
//  * Derivative data enter pre-scaled by the mesh width: H = dx * h, so the
//    reconstruction formulas of Sec. 2.1 and the limiter of Sec. 2.2 carry no
//    dx; the derivative flux is returned as D = dx * p_0'(x_{i+1/2}).
//  * The nonlinear weights w_l = g_l (1 + tau / (beta_l + eps)) / S are never
//    formed one by one. In FP64 both sides of an interface are brought over
//    the common denominator b_0 b_1 b_2 (b_l = beta_l + eps), which leaves one
//    division per interface and field; in FP32 the per-side form with three
//    divisions is kept because the products can exceed the float range.
//  * The "-" flux at x_{i+1/2} is the mirror image of the "+" one: the "+"
//    procedure applied to the stencil {i+2, i+1, i} with the derivative data
//    negated, and the derivative flux negated back (Sec. 2.1).
#pragma once

#include <cuda_runtime.h>
#include <type_traits>

namespace hweno {

template <class Real>
struct Weights {
  Real g0, g1, g2;       // linear weights gamma_l (Sec. 2.1)
  Real d0, d1, d2;       // limiter linear weights d_l (Sec. 2.2)
  Real eps;
  Real ig0, id0;         // 1/gamma_0, 1/d_0
  Real rm, r0, rp, rH;   // p0 - g1 p1 - g2 p2 in f_{i-1}, f_i, f_{i+1}, H_i
};

// Largest finite value of the state precision.
template <class Real>
__device__ __forceinline__ constexpr Real real_max() {
  if constexpr (std::is_same<Real, double>::value) return 1.7976931348623157e308;
  else return 3.40282347e38f;
}

// Pick the FP64 or FP32 copy of a host-converted constant table.
template <class Real>
__device__ __forceinline__ const Real* pick(const double* d, const float* f) {
  if constexpr (std::is_same<Real, double>::value) return d;
  else return f;
}

template <class Real>
__device__ __forceinline__ Weights<Real> weights_from(const Real* v) {
  Weights<Real> w;
  w.g0 = v[0]; w.g1 = v[1]; w.g2 = v[2];
  w.d0 = v[3]; w.d1 = v[4]; w.d2 = v[5];
  w.eps = v[6];
  w.ig0 = v[7];
  w.id0 = v[8];
  w.rm = v[11]; w.r0 = v[12]; w.rp = v[13]; w.rH = v[14];
  return w;
}

// Maximum over the CTA (red: one slot per warp); the result is valid in
// warp 0. Contains barriers: call from every thread.
template <class T>
__device__ __forceinline__ T block_max_t(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : T(0);
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;
}

// Quantities of one "+" reconstruction (Sec. 2.1) from f^+ and H = dx h^+ on
// the stencil {i-1, i, i+1}: the candidate values at x_{i+1/2} (p0 only
// through r = p0 - g1 p1 - g2 p2, its share of the nonlinear combination),
// the smoothness indicators and tau.
template <class Real>
struct Cand {
  Real r, p1, p2;
  Real b0, b1, b2;  // beta_l + eps
  Real tau;
};

template <class Real>
__device__ __forceinline__ Cand<Real> candidates(Real fm, Real f0, Real fp, Real Hm, Real H0,
                                                 Real Hp, const Weights<Real>& w) {
  const Real eps = w.eps;
  Cand<Real> c;
  const Real sHp = Hm + Hp, dHp = Hm - Hp;
  const Real d1 = fm - f0, d2 = f0 - fp;  // the two one-sided differences
  const Real lap = d1 - d2;               // f_{i-1} - 2 f_i + f_{i+1}
  const Real dif = d1 + d2;               // f_{i-1} - f_{i+1}
  // p1 = 1/6 f_{i-1} + 5/6 f_i + 2/3 H_i, p2 = 5/6 f_i + 1/6 f_{i+1} + 1/3 H_i
  c.p1 = f0 + Real(1.0 / 6.0) * d1 + Real(2.0 / 3.0) * H0;
  c.p2 = f0 - Real(1.0 / 6.0) * d2 + Real(1.0 / 3.0) * H0;
  // p0 = 11/60 (f_{i-1} + f_{i+1}) + 19/30 f_i + (H_{i-1} - H_{i+1})/20 + H_i/2
  //    = f_i + 11/60 lap + dHp/20 + H_i/2
  if constexpr (std::is_same<Real, double>::value) {  // r as one linear form
    c.r = w.rm * fm + w.r0 * f0 + w.rp * fp + Real(0.05) * dHp + w.rH * H0;
  } else {  // FP32: no further constants held (the kernels are register capped)
    const Real p0 = f0 + Real(11.0 / 60.0) * lap + Real(0.05) * dHp + Real(0.5) * H0;
    c.r = p0 - w.g1 * c.p1 - w.g2 * c.p2;
  }
  // beta_0 of Eq. GHYZP as a sum of squares of the quintic's coefficients
  // a_1..a_5 (dx absorbed into H): e1^2 + 13/3 e2^2 + 781/20 e3^2 +
  // 1421461/2275 a4^2 + 21520059541/1377684 a5^2 with e1 = a1 + a3/4 + a5/16,
  // e2 = a2 + 63/130 a4, e3 = a3 + 8825/10934 a5. In the stencil values a1 and
  // a3 enter only e1 and e3, and e1 reduces to H_i exactly (the sHp and dif
  // terms cancel, the H_i coefficients sum to 1); e2 and e3 are taken
  // straight from sHp, dHp, H_i, lap, dif:
  //   a2 = 3/8 dHp + 5/4 lap, a3 = -11/24 sHp - 17/6 H_i - 15/8 dif,
  //   e2 = 33/130 dHp + 131/130 lap,
  //   e3 = -16831/65604 sHp - 33232/16401 H_i - 27765/21868 dif,
  //   a4 = -1/4 dHp - 1/2 lap, a5 = 1/4 sHp + H_i + 3/4 dif.
  // The weights of the first three squares ride on the coefficients (their
  // square roots times the coefficients above, to 20 digits):
  // E2 = sqrt(13/3) e2, E3 = sqrt(781/20) e3, A4 = sqrt(1421461/2275) a4.
  const Real E2 = Real(0.52842290755678754049) * dHp + Real(2.0976788148466414486) * lap;
  const Real E3 = Real(-1.6032089149031235916) * sHp + Real(-12.661835579599691806) * H0 +
                  Real(-7.9341267047029694945) * dif;
  const Real A4 = Real(-6.2490900436484649542) * dHp + Real(-12.498180087296929908) * lap;
  const Real a5 = Real(0.25) * sHp + H0 + Real(0.75) * dif;
  // beta_l + eps accumulated directly (eps enters each sum once, so no
  // separate addition; e1^2 + eps = H_i^2 + eps is shared with beta_1 and
  // beta_2); tau from the differences, where eps cancels
  const Real h2e = H0 * H0 + eps;
  c.b0 = h2e + E2 * E2 + E3 * E3 + A4 * A4 + Real(21520059541.0 / 1377684.0) * a5 * a5;
  // beta_1 = H_i^2 + 13/3 (H_i + d1)^2, beta_2 = H_i^2 + 13/3 (H_i + d2)^2,
  // with sqrt(13/3) on the inner sums (S_l = sqrt(13/3) (H_i + d_l))
  const Real kH = Real(2.0816659994661327353) * H0;
  const Real S1 = kH + Real(2.0816659994661327353) * d1;
  const Real S2 = kH + Real(2.0816659994661327353) * d2;
  c.b1 = h2e + S1 * S1;
  c.b2 = h2e + S2 * S2;
  const Real t = fabs(c.b0 - c.b1) + fabs(c.b0 - c.b2);
  c.tau = Real(0.25) * t * t;
  return c;
}

// Numerator and denominator of f-hat over the common factor b0 b1 b2:
// f-hat = num / den, num = (b0+tau) b1 b2 (p0 - g1 p1 - g2 p2)
//   + g1 (b1+tau) b0 b2 p1 + g2 (b2+tau) b0 b1 p2, den = g0 (b0+tau) b1 b2 + ...
// Each (b_l + tau) prod_{m != l} b_m is formed as P + tau prod_{m != l} b_m,
// P = b0 b1 b2.
template <class Real>
__device__ __forceinline__ void combine_nd(const Cand<Real>& c, const Weights<Real>& w, Real& num,
                                           Real& den) {
  const Real b12 = c.b1 * c.b2, b02 = c.b0 * c.b2, b01 = c.b0 * c.b1;
  const Real P = c.b0 * b12;
  const Real W0 = P + c.tau * b12;
  const Real W1 = w.g1 * (P + c.tau * b02);
  const Real W2 = w.g2 * (P + c.tau * b01);
  num = W0 * c.r + W1 * c.p1 + W2 * c.p2;
  den = w.g0 * W0 + W1 + W2;
}

// Quotient used where the FP32 path divides: the fast approximate division
// (a few ulp) in single precision; the IEEE division in double precision.
template <class Real>
__device__ __forceinline__ Real qdiv(Real a, Real b) {
  if constexpr (std::is_same<Real, float>::value) return __fdividef(a, b);
  else return a / b;
}

// f-hat of one side in the per-weight form (used for FP32).
template <class Real>
__device__ __forceinline__ Real combine_direct(const Cand<Real>& c, const Weights<Real>& w) {
  const Real o0 = w.g0 + w.g0 * qdiv(c.tau, c.b0);
  const Real o1 = w.g1 + w.g1 * qdiv(c.tau, c.b1);
  const Real o2 = w.g2 + w.g2 * qdiv(c.tau, c.b2);
  const Real num = o0 * w.ig0 * c.r + o1 * c.p1 + o2 * c.p2;
  return qdiv(num, o0 + o1 + o2);
}

// ---------------------------------------------------------------------------
// FP32: the "+" side and the mirrored "-" side of an interface carry the same
// arithmetic on different data, so they travel as the two lanes of packed
// FP32 pairs (one instruction for both sides: fma / add / mul .f32x2, sm_100
// and later). Each lane rounds exactly as a scalar FP32 operation would.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 pair(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// fast reciprocal of each lane (the approximate division of the FP32 path)
__device__ __forceinline__ float2 rcp2(float2 a) {
  return make_float2(__fdividef(1.f, a.x), __fdividef(1.f, a.y));
}

// f-hat^+ + f-hat^- of one (characteristic) field in FP32: lane x holds the
// "+" stencil (f^+, H^+ at i-1, i, i+1), lane y the mirrored "-" stencil
// (f^-, -H^- at i+2, i+1, i). The same formulas as candidates() and
// combine_direct(), lane by lane.
__device__ __forceinline__ float interface_flux_pair(float2 fm, float2 f0, float2 fp, float2 Hm,
                                                     float2 H0, float2 Hp,
                                                     const Weights<float>& w) {
  const float2 sHp = add2(Hm, Hp), dHp = sub2(Hm, Hp);
  const float2 d1 = sub2(fm, f0), d2 = sub2(f0, fp);
  const float2 lap = sub2(d1, d2), dif = add2(d1, d2);
  const float2 p1 = fma2(pair(1.0f / 6.0f), d1, fma2(pair(2.0f / 3.0f), H0, f0));
  const float2 p2 = fma2(pair(-1.0f / 6.0f), d2, fma2(pair(1.0f / 3.0f), H0, f0));
  const float2 p0 = fma2(pair(11.0f / 60.0f), lap, fma2(pair(0.05f), dHp, fma2(pair(0.5f), H0, f0)));
  const float2 r = fma2(pair(-w.g2), p2, fma2(pair(-w.g1), p1, p0));
  // smoothness indicators as in candidates() (square weights in the
  // coefficients), beta_l + eps accumulated directly
  const float2 E2 = fma2(pair(2.0976788148466414486f), lap, mul2(pair(0.52842290755678754049f), dHp));
  const float2 E3 = fma2(pair(-7.9341267047029694945f), dif,
                         fma2(pair(-12.661835579599691806f), H0,
                              mul2(pair(-1.6032089149031235916f), sHp)));
  const float2 A4 = fma2(pair(-12.498180087296929908f), lap, mul2(pair(-6.2490900436484649542f), dHp));
  const float2 a5 = fma2(pair(0.75f), dif, fma2(pair(0.25f), sHp, H0));
  const float2 h2e = fma2(H0, H0, pair(w.eps));
  const float2 b0 = fma2(mul2(pair(21520059541.0f / 1377684.0f), a5), a5,
                         fma2(A4, A4, fma2(E3, E3, fma2(E2, E2, h2e))));
  const float2 kH = mul2(pair(2.0816659994661327353f), H0);
  const float2 S1 = fma2(pair(2.0816659994661327353f), d1, kH);
  const float2 S2 = fma2(pair(2.0816659994661327353f), d2, kH);
  const float2 b1 = fma2(S1, S1, h2e), b2 = fma2(S2, S2, h2e);
  const float2 e1 = sub2(b0, b1), e2 = sub2(b0, b2);
  const float2 t = make_float2(fabsf(e1.x) + fabsf(e2.x), fabsf(e1.y) + fabsf(e2.y));
  const float2 tau = mul2(pair(0.25f), mul2(t, t));
  // per-weight form: o_l = g_l (1 + tau / b_l), f-hat = (o0 r / g0 + o1 p1 + o2 p2) / sum o_l
  const float2 o0 = fma2(pair(w.g0), mul2(tau, rcp2(b0)), pair(w.g0));
  const float2 o1 = fma2(pair(w.g1), mul2(tau, rcp2(b1)), pair(w.g1));
  const float2 o2 = fma2(pair(w.g2), mul2(tau, rcp2(b2)), pair(w.g2));
  const float2 num = fma2(mul2(o0, pair(w.ig0)), r, fma2(o1, p1, mul2(o2, p2)));
  const float2 q = mul2(num, rcp2(add2(add2(o0, o1), o2)));
  return q.x + q.y;
}

// Global Lax-Friedrichs splitting of one component (Sec. 2.1): the flux
// halves f^{+-} = (f +- alpha u) / 2 and the scaled derivative-flux halves
// (d / 2)(h +- alpha v), d the grid spacing. ha = alpha / 2 and
// hda = (d / 2) alpha are the caller's factors, formed once per thread.
// f / 2 and alpha / 2 are exact, so each flux half is one FMA with the bits
// of (f +- alpha u) rounded once and halved; the derivative halves round
// (d / 2) h first.
template <class Real>
__device__ __forceinline__ void split_pm(Real f, Real u, Real h, Real v, Real ha, Real hda,
                                         Real hd, Real& fp, Real& fm, Real& hp, Real& hm) {
  const Real hf = Real(0.5) * f;
  fp = ha * u + hf;
  fm = hf - ha * u;
  const Real hh = hd * h;
  hp = hda * v + hh;
  hm = hh - hda * v;
}

// A quotient n / d whose division is deferred, so that the quotients of
// several fields can share one reciprocal (resolve2). In FP32 the value is
// already final (d = 1).
template <class Real>
struct Frac {
  Real n, d;
};

// Scaling of the deferred quotients. A denominator is a product of factors
// of the size of beta + eps (beta grows like the square of the split-flux
// jumps): one side of an interface is of degree four in them, a pair of
// sides eight, a pair of fields sixteen, which leaves the FP64 range for
// split-flux jumps near 1e8. So each side's numerator and denominator are
// multiplied by one power of two that brings the denominator into [1, 2),
// by integer arithmetic on the exponent fields (off the FP64 pipe, no
// branches). Scaling by a power of two is exact, so the quotients keep the
// bits they have without it wherever that form stays in range.

// x 2^k by adding k to the exponent field: exact while x and the result are
// normal; a zero or subnormal x, or a result below the normal range, gives a
// zero of x's sign. Callers keep x 2^k below the overflow limit.
__device__ __forceinline__ double scale_pow2(double x, int k) {
  const int hi = __double2hiint(x), lo = __double2loint(x);
  const int e = ((hi >> 20) & 0x7ff) + k;
  const bool keep = ((hi & 0x7ff00000) != 0) & (e > 0);
  return __hiloint2double(keep ? ((hi & 0x800fffff) | (e << 20)) : (hi & 0x80000000),
                          keep ? lo : 0);
}

// n / d (d > 0, normal) as n', d' with d' in [1, 2) and n' / d' = n / d.
__device__ __forceinline__ void normalize(double& n, double& d) {
  const int hi = __double2hiint(d);
  const int k = 1023 - ((hi >> 20) & 0x7ff);
  d = __hiloint2double((hi & 0x800fffff) | 0x3ff00000, __double2loint(d));
  n = scale_pow2(n, k);
}

// n0/d0 and n1/d1 with one division: r = 1/(d0 d1) (the denominators are
// normalized, so the product lies in [1, 4)).
template <class Real>
__device__ __forceinline__ void resolve2(const Frac<Real>& a, const Frac<Real>& b, Real& qa,
                                         Real& qb) {
  if constexpr (std::is_same<Real, double>::value) {
    const Real r = Real(1) / (a.d * b.d);
    qa = a.n * b.d * r;
    qb = b.n * a.d * r;
  } else {
    qa = a.n;
    qb = b.n;
  }
}

// Three or four quotients with one division (all the characteristic fields
// of an interface or a limiter item): the denominators are normalized, so
// their product lies in [1, 64) (three) or [1, 256) (four).
template <class Real>
__device__ __forceinline__ void resolve3(const Frac<Real>& a, const Frac<Real>& b,
                                         const Frac<Real>& c, Real& qa, Real& qb, Real& qc) {
  if constexpr (std::is_same<Real, double>::value) {
    const Real dbc = b.d * c.d;
    const Real r = Real(1) / (a.d * dbc);
    qa = a.n * dbc * r;
    qb = b.n * (a.d * c.d) * r;
    qc = c.n * (a.d * b.d) * r;
  } else {
    qa = a.n;
    qb = b.n;
    qc = c.n;
  }
}
template <class Real>
__device__ __forceinline__ void resolve4(const Frac<Real>* f, Real* q) {
  if constexpr (std::is_same<Real, double>::value) {
    const Real d01 = f[0].d * f[1].d, d23 = f[2].d * f[3].d;
    const Real r = Real(1) / (d01 * d23);
    const Real r01 = d23 * r, r23 = d01 * r;  // 1/(d0 d1), 1/(d2 d3)
    q[0] = f[0].n * f[1].d * r01;
    q[1] = f[1].n * f[0].d * r01;
    q[2] = f[2].n * f[3].d * r23;
    q[3] = f[3].n * f[2].d * r23;
  } else {
    for (int i = 0; i < 4; ++i) q[i] = f[i].n;
  }
}

// The sum of two deferred quotients na/da + nb/db as one deferred quotient
// (each side normalized first).
template <class Real>
__device__ __forceinline__ Frac<Real> sum_frac(Real na, Real da, Real nb, Real db) {
  if constexpr (std::is_same<Real, double>::value) {
    normalize(na, da);
    normalize(nb, db);
    return Frac<Real>{na * db + nb * da, da * db};
  } else {
    return Frac<Real>{na + nb, Real(1)};
  }
}

template <class Real>
__device__ __forceinline__ Real resolve1(const Frac<Real>& a) {
  if constexpr (std::is_same<Real, double>::value) return a.n / a.d;
  else return a.n;
}

// Full interface flux of one (characteristic) field: f-hat = f-hat^+ + f-hat^-
// from f^+ at i-1..i+1, f^- at i..i+2 and the scaled derivative data, as a
// deferred quotient (FP64: both sides over the common denominator).
// Pairs (FP32 only): both sides in packed pairs. Measured: +5.6% for the 2D
// sweeps (96 registers allowed); in the 1D stage kernels, capped at 64
// registers for 8 CTAs per SM, the pairs spill and lose 5%, so they keep the
// scalar form.
template <class Real, bool Pairs = false>
__device__ __forceinline__ Frac<Real> interface_flux_frac(Real fpm, Real fp0, Real fpp, Real Hpm,
                                                          Real Hp0, Real Hpp, Real fm0, Real fm1,
                                                          Real fm2, Real Hm0, Real Hm1, Real Hm2,
                                                          const Weights<Real>& w) {
  if constexpr (std::is_same<Real, double>::value) {
    const Cand<Real> a = candidates(fpm, fp0, fpp, Hpm, Hp0, Hpp, w);
    const Cand<Real> b = candidates(fm2, fm1, fm0, -Hm2, -Hm1, -Hm0, w);  // mirror
    Real na, da, nb, db;
    combine_nd(a, w, na, da);
    combine_nd(b, w, nb, db);
    return sum_frac(na, da, nb, db);
  } else if constexpr (Pairs) {  // both sides at once, the mirror in lane y
    return Frac<Real>{interface_flux_pair(make_float2(fpm, fm2), make_float2(fp0, fm1),
                                          make_float2(fpp, fm0), make_float2(Hpm, -Hm2),
                                          make_float2(Hp0, -Hm1), make_float2(Hpp, -Hm0), w),
                      Real(1)};
  } else {
    const Cand<Real> a = candidates(fpm, fp0, fpp, Hpm, Hp0, Hpp, w);
    const Cand<Real> b = candidates(fm2, fm1, fm0, -Hm2, -Hm1, -Hm0, w);  // mirror
    return Frac<Real>{combine_direct(a, w) + combine_direct(b, w), Real(1)};
  }
}

template <class Real, bool Pairs = false>
__device__ __forceinline__ Real interface_flux(Real fpm, Real fp0, Real fpp, Real Hpm, Real Hp0,
                                               Real Hpp, Real fm0, Real fm1, Real fm2, Real Hm0,
                                               Real Hm1, Real Hm2, const Weights<Real>& w) {
  return resolve1(interface_flux_frac<Real, Pairs>(fpm, fp0, fpp, Hpm, Hp0, Hpp, fm0, fm1, fm2,
                                                   Hm0, Hm1, Hm2, w));
}

// Scaled derivative flux D = dx (h-hat^+ + h-hat^-) = dx (p_0'^+ + p_0'^-),
// linear (Sec. 2.1, h-hat = p_0'(x_{i+1/2}); the "-" side mirrored).
template <class Real>
__device__ __forceinline__ Real derivative_flux(Real fpm, Real fp0, Real fpp, Real Hpm, Real Hp0,
                                                Real Hpp, Real fm0, Real fm1, Real fm2, Real Hm0,
                                                Real Hm1, Real Hm2) {
  // "+" side: 0.25 (f_{i-1} - 8 f_i + 7 f_{i+1}) + (H_{i-1} - 2 H_i - 5 H_{i+1})/12;
  // "-" side (mirror): -(0.25 (f2 - 8 f1 + 7 f0) + (-H2 + 2 H1 + 5 H0)/12);
  // their sum as one linear form of the twelve values
  return Real(0.25) * fpm - Real(2) * fp0 + Real(1.75) * fpp - Real(1.75) * fm0 +
         Real(2) * fm1 - Real(0.25) * fm2 + Real(1.0 / 12.0) * Hpm - Real(1.0 / 6.0) * Hp0 -
         Real(5.0 / 12.0) * Hpp - Real(5.0 / 12.0) * Hm0 - Real(1.0 / 6.0) * Hm1 +
         Real(1.0 / 12.0) * Hm2;
}

// HWENO limiter (Sec. 2.2) in scaled form: point values um, u0, up and
// Vm = dx v_{i-1}, Vp = dx v_{i+1}; dx * v-tilde_i as a deferred quotient.
template <class Real>
__device__ __forceinline__ Frac<Real> limited_derivative_frac(Real um, Real u0, Real up, Real Vm,
                                                              Real Vp, const Weights<Real>& w) {
  const Real sV = Vm + Vp, dV = Vm - Vp;
  const Real q1 = u0 - um;                                    // dx q_1'
  const Real q2 = up - u0;                                    // dx q_2'
  const Real lap = q2 - q1;                                   // um - 2 u0 + up
  const Real du = q1 + q2;                                    // up - um
  const Real q0 = Real(0.75) * du - Real(0.25) * sV;          // dx q_0'(x_i) = a_1
  // beta_0 = e1^2 + 13/3 e2^2 + 781/20 a3^2 + 1421461/2275 a4^2 with
  // a2 = dV/4 + lap, a3 = (sV - du)/4, a4 = -dV/4 - lap/2, e1 = a1 + a3/4,
  // e2 = a2 + 63/130 a4 = 67/520 dV + 197/260 lap; the weights of the last
  // three squares ride on the coefficients (square roots, to 20 digits):
  // E2 = sqrt(13/3) e2, A3 = sqrt(781/20) a3, A4 = sqrt(1421461/2275) a4.
  const Real E2 = Real(0.26821465762352094858) * dV + Real(1.5772623149801082648) * lap;
  const Real A3 = Real(1.5622499799967993599) * (sV - du);
  const Real A4 = Real(-6.2490900436484649542) * dV + Real(-12.498180087296929908) * lap;
  const Real e1 = q0 + Real(0.040006401536409714721) * A3;  // a3 / 4 = A3 / (4 sqrt(781/20))
  // beta_l + eps accumulated directly, as in candidates()
  const Real b0 = e1 * e1 + w.eps + E2 * E2 + A3 * A3 + A4 * A4;
  const Real b1 = q1 * q1 + w.eps, b2 = q2 * q2 + w.eps;
  const Real t = fabs(b0 - b1) + fabs(b0 - b2);
  const Real tau = Real(0.25) * t * t;
  if constexpr (std::is_same<Real, double>::value) {
    const Real b12 = b1 * b2, b02 = b0 * b2, b01 = b0 * b1;
    const Real P = b0 * b12;  // as in combine_nd
    const Real L0 = P + tau * b12;
    const Real L1 = w.d1 * (P + tau * b02);
    const Real L2 = w.d2 * (P + tau * b01);
    const Real num = L0 * (q0 - w.d1 * q1 - w.d2 * q2) + L1 * q1 + L2 * q2;
    Real n = num, d = w.d0 * L0 + L1 + L2;
    normalize(n, d);
    return Frac<Real>{n, d};
  } else {
    const Real l0 = w.d0 + w.d0 * qdiv(tau, b0);
    const Real l1 = w.d1 + w.d1 * qdiv(tau, b1);
    const Real l2 = w.d2 + w.d2 * qdiv(tau, b2);
    const Real num = l0 * w.id0 * (q0 - w.d1 * q1 - w.d2 * q2) + l1 * q1 + l2 * q2;
    return Frac<Real>{qdiv(num, l0 + l1 + l2), Real(1)};
  }
}

// Two FP32 limited derivatives at once (lanes: two characteristic fields),
// the per-weight form of limited_derivative_frac lane by lane.
__device__ __forceinline__ float2 limited_derivative_pair(float2 um, float2 u0, float2 up,
                                                          float2 Vm, float2 Vp,
                                                          const Weights<float>& w) {
  const float2 sV = add2(Vm, Vp), dV = sub2(Vm, Vp);
  const float2 q1 = sub2(u0, um), q2 = sub2(up, u0);
  const float2 lap = sub2(q2, q1), du = add2(q1, q2);
  const float2 q0 = fma2(pair(0.75f), du, mul2(pair(-0.25f), sV));
  const float2 E2 = fma2(pair(1.5772623149801082648f), lap, mul2(pair(0.26821465762352094858f), dV));
  const float2 A3 = mul2(pair(1.5622499799967993599f), sub2(sV, du));
  const float2 A4 = fma2(pair(-12.498180087296929908f), lap, mul2(pair(-6.2490900436484649542f), dV));
  const float2 e1 = fma2(pair(0.040006401536409714721f), A3, q0);
  const float2 b0 = fma2(A4, A4, fma2(A3, A3, fma2(E2, E2, fma2(e1, e1, pair(w.eps)))));
  const float2 b1 = fma2(q1, q1, pair(w.eps)), b2 = fma2(q2, q2, pair(w.eps));
  const float2 e01 = sub2(b0, b1), e02 = sub2(b0, b2);
  const float2 t = make_float2(fabsf(e01.x) + fabsf(e02.x), fabsf(e01.y) + fabsf(e02.y));
  const float2 tau = mul2(pair(0.25f), mul2(t, t));
  const float2 l0 = fma2(pair(w.d0), mul2(tau, rcp2(b0)), pair(w.d0));
  const float2 l1 = fma2(pair(w.d1), mul2(tau, rcp2(b1)), pair(w.d1));
  const float2 l2 = fma2(pair(w.d2), mul2(tau, rcp2(b2)), pair(w.d2));
  const float2 c0 = fma2(pair(-w.d2), q2, fma2(pair(-w.d1), q1, q0));
  const float2 num = fma2(mul2(l0, pair(w.id0)), c0, fma2(l1, q1, mul2(l2, q2)));
  return mul2(num, rcp2(add2(add2(l0, l1), l2)));
}

template <class Real>
__device__ __forceinline__ Real limited_derivative(Real um, Real u0, Real up, Real Vm, Real Vp,
                                                   const Weights<Real>& w) {
  return resolve1(limited_derivative_frac(um, u0, up, Vm, Vp, w));
}

// 1/x: the IEEE division in FP64, the fast approximate reciprocal in FP32
// (as qdiv).
template <class Real>
__device__ __forceinline__ Real recip(Real x) {
  if constexpr (std::is_same<Real, float>::value) return __fdividef(1.f, x);
  else return Real(1) / x;
}

// sqrt(x): IEEE in FP64; in FP32 the approximate square root of PTX
// (sqrt.approx.f32: NaN for x < 0 or NaN, so a bad state still shows in the
// wave speed; +0 for +0).
template <class Real>
__device__ __forceinline__ Real fast_sqrt(Real x) {
  if constexpr (std::is_same<Real, float>::value) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
  } else {
    return sqrt(x);
  }
}

// Reciprocal square root (FP64: CUDA's rsqrt, within one ulp; FP32: the
// hardware approximation).
template <class Real>
__device__ __forceinline__ Real rsq(Real x) {
  if constexpr (std::is_same<Real, double>::value) return rsqrt(x);
  else return rsqrtf(x);
}

// c from c^2 for a wave speed: FP32 the approximate square root; FP64
// c^2 rsqrt(c^2) (one reciprocal square root instead of the longer IEEE
// square root), 0 at c^2 = 0, NaN for a negative or NaN c^2 as the square
// root would give.
template <class Real>
__device__ __forceinline__ Real speed_from_sq(Real c2) {
  if constexpr (std::is_same<Real, float>::value) return fast_sqrt(c2);
  else return c2 * rsq(c2 == Real(0) ? Real(1) : c2);
}

// c and 1/c from c^2 with one reciprocal square root.
template <class Real>
__device__ __forceinline__ void sound_speed(Real c2, Real& c, Real& ic) {
  ic = rsq(c2);
  c = c2 * ic;
}

// ---------------------------------------------------------------------------
// Euler eigen-systems in direction `dir` at a state given by velocity (u, v),
// enthalpy H and sound speed c (standard right/left eigenvectors of the flux
// Jacobian; eigenvalue order u-c, u, [shear], u+c). m = 3 (1D) or 4 (2D).
// Only what the projections need is formed: the left matrix row by row and
// the right matrix column by column.
// ---------------------------------------------------------------------------
// The characteristic system of the 1D Euler flux Jacobian at velocity u,
// enthalpy H and sound speed c (eigenvalue order u - c, u, u + c), with the
// left matrix in factored form. With b1 = (gamma - 1) / c^2, b2 = b1 u^2 / 2,
// A = (b2 x0 - b1 u x1 + b1 x2) / 2 and B = (u x0 - x1) / (2 c), the three
// rows of L applied to x are A + B, x0 - 2 A and A - B: eight operations per
// projected vector instead of nine for the rows applied one by one, and no
// 3 x 3 matrix held. Equal to euler_eigen's L and R in exact arithmetic.
template <class Real>
struct Char1 {
  Real u, c, H, q, hb1, hb2, hb1u, hic, huc;
  Char1() = default;
  __device__ __forceinline__ Char1(Real u_, Real H_, Real c_, Real ic, Real gm1)
      : u(u_), c(c_), H(H_) {
    q = Real(0.5) * u * u;
    hb1 = Real(0.5) * gm1 * ic * ic;
    hb2 = hb1 * q;
    hb1u = hb1 * u;
    hic = Real(0.5) * ic;
    huc = hic * u;
  }
  // the factors (A, B) of the vector x
  __device__ __forceinline__ void factors(Real x0, Real x1, Real x2, Real& A, Real& B) const {
    A = hb2 * x0 - hb1u * x1 + hb1 * x2;
    B = huc * x0 - hic * x1;
  }
  // row r of L applied to the vector with first component x0 and factors (A, B)
  __device__ __forceinline__ Real row(int r, Real x0, Real A, Real B) const {
    return r == 0 ? A + B : r == 1 ? x0 - Real(2) * A : A - B;
  }
  // R s (columns (1, u - c, H - u c), (1, u, q), (1, u + c, H + u c))
  __device__ __forceinline__ void right(const Real* s, Real* out) const {
    const Real uc = u * c;
    out[0] = s[0] + s[1] + s[2];
    out[1] = (u - c) * s[0] + u * s[1] + (u + c) * s[2];
    out[2] = (H - uc) * s[0] + q * s[1] + (H + uc) * s[2];
  }
};

template <class Real, int M>
struct Eigen {
  Real L[M][M];
  Real R[M][M];
};

template <class Real, int M>
__device__ __forceinline__ void euler_eigen(int dir, Real u, Real v, Real H, Real c, Real ic,
                                            Real gm1, Eigen<Real, M>& e) {
  const Real b1 = gm1 * ic * ic;
  if constexpr (M == 3) {
    const Real q = Real(0.5) * u * u;
    const Real b2 = b1 * q;
    const Real uc = u * ic;
    e.L[0][0] = Real(0.5) * (b2 + uc); e.L[0][1] = Real(-0.5) * (b1 * u + ic); e.L[0][2] = Real(0.5) * b1;
    e.L[1][0] = Real(1) - b2;          e.L[1][1] = b1 * u;                     e.L[1][2] = -b1;
    e.L[2][0] = Real(0.5) * (b2 - uc); e.L[2][1] = Real(-0.5) * (b1 * u - ic); e.L[2][2] = Real(0.5) * b1;
    e.R[0][0] = Real(1); e.R[0][1] = Real(1); e.R[0][2] = Real(1);
    e.R[1][0] = u - c;   e.R[1][1] = u;       e.R[1][2] = u + c;
    e.R[2][0] = H - u * c; e.R[2][1] = q;     e.R[2][2] = H + u * c;
  } else {
    const Real q = Real(0.5) * (u * u + v * v);
    const Real b2 = b1 * q;
    // normal / tangential velocity and their component slots
    const Real un = dir == 0 ? u : v, ut = dir == 0 ? v : u;
    const int kn = dir == 0 ? 1 : 2, kt = dir == 0 ? 2 : 1;
    const Real unc = un * ic;
    for (int r = 0; r < 4; ++r)
      for (int k = 0; k < 4; ++k) { e.L[r][k] = Real(0); e.R[r][k] = Real(0); }
    e.L[0][0] = Real(0.5) * (b2 + unc); e.L[0][kn] = Real(-0.5) * (b1 * un + ic);
    e.L[0][kt] = Real(-0.5) * b1 * ut;  e.L[0][3] = Real(0.5) * b1;
    e.L[1][0] = Real(1) - b2; e.L[1][kn] = b1 * un; e.L[1][kt] = b1 * ut; e.L[1][3] = -b1;
    e.L[2][0] = -ut; e.L[2][kt] = Real(1);
    e.L[3][0] = Real(0.5) * (b2 - unc); e.L[3][kn] = Real(-0.5) * (b1 * un - ic);
    e.L[3][kt] = Real(-0.5) * b1 * ut;  e.L[3][3] = Real(0.5) * b1;
    // columns: (1, un-c, ut, H - un c), (1, un, ut, q), (0, 0, 1, ut), (1, un+c, ut, H + un c)
    e.R[0][0] = Real(1); e.R[kn][0] = un - c; e.R[kt][0] = ut; e.R[3][0] = H - un * c;
    e.R[0][1] = Real(1); e.R[kn][1] = un;     e.R[kt][1] = ut; e.R[3][1] = q;
    e.R[kt][2] = Real(1); e.R[3][2] = ut;
    e.R[0][3] = Real(1); e.R[kn][3] = un + c; e.R[kt][3] = ut; e.R[3][3] = H + un * c;
  }
}

}  // namespace hweno
