// Oracle for the fifth-order finite-difference L-HWENO scheme of
// Zhang & Zhao, "A fifth-order finite difference HWENO scheme combined with
// limiter for hyperbolic conservation laws" (arXiv:2207.05258).
//
// TEST INFRASTRUCTURE. This file is a plain, slow, step-by-step CPU statement
// of the scheme in FP64. Only the tests, the smoke check and the CPU baseline
// of the benchmark call it; the library never does. It shares no code, header
// or table with the CUDA implementation.
//
// Every function follows the paper's order of operations and notation; where
// the paper is silent, garbled or inconsistent, the reading taken is stated
// here and named (R1, R2, ...) at the point of use:
//   R1  beta_2 of the reconstruction uses f_{i+1} (Sec. 2.1, Eq. GHYZP prints
//       f_{i-1}; the defining integral Eq. GHYZ gives f_{i+1}).
//   R2  every f, h in p_0, p_1, p_2, p_0' is the split value f^+, h^+.
//   R3  the "-" fluxes are the mirror image about x_{i+1/2} of the "+" ones:
//       stencil {i, i+1, i+2}, derivative data change sign.
//   R4  the mixed-derivative differences of Eq. md-app divide by dy for xi
//       and by dx for eta (the printed 1/dx, 1/dy are swapped).
//   R5  dt = CFL*dx/alpha (1D) or CFL/(alpha_x/dx + alpha_y/dy) (2D); the
//       accuracy tests use dx^{5/3} in place of dx; the last step lands on T.
//   R6  alpha = max over the grid of |f'(u)| (Euler: |u|+c per direction),
//       recomputed from the input state of every Runge-Kutta stage.
//   R7  characteristic decomposition at x_{i+1/2} uses the Roe average of
//       U_i and U_{i+1} (arithmetic mean as an option).
//   R8  the limiter of a system acts on characteristic variables with the
//       eigenvectors at U_i of the sweep direction (component-wise option).
//   R9  ghost values: periodic wrap; outflow copies U and its derivatives;
//       reflective mirrors U (normal momentum odd) with the normal
//       derivative of opposite parity and the tangential derivative of the
//       same parity; imposed states carry zero derivatives.
//   R10 double Mach reflection: Woodward-Colella setup, the incident shock
//       passes (x_foot, 0) at 60 degrees to the x axis.
//   R15 Buckley-Leverett (Example 3.4, non-convex f): alpha = max |f'(u)| over
//       the admissible states u in [0, 1], and over any grid value outside
//       [0, 1]; the maximum over [0, 1] is found by golden-section search.
//   R17 the forward-mode tangent (Dual) freezes alpha of every stage and dt of
//       every step, and keeps the |.| in tau on the branch of the forward
//       state; weights, eigenvectors and the limiter are differentiated
//       (freeze_weights also holds the nonlinear weights at their values).
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared (no FMA
// contraction, no fast-math).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Scalar types. `double` is the oracle proper. `Flop` is a double that counts
// every +, -, *, /, sqrt (fabs, comparisons and max count zero); it measures
// the algorithmic operation count of the scheme as written here.
// ---------------------------------------------------------------------------
long long g_flops = 0;

struct Flop {
  double v;
  Flop() : v(0.0) {}
  Flop(double x) : v(x) {}  // NOLINT: implicit, so constants mix in
};
inline Flop operator+(Flop a, Flop b) { ++g_flops; return Flop(a.v + b.v); }
inline Flop operator-(Flop a, Flop b) { ++g_flops; return Flop(a.v - b.v); }
inline Flop operator*(Flop a, Flop b) { ++g_flops; return Flop(a.v * b.v); }
inline Flop operator/(Flop a, Flop b) { ++g_flops; return Flop(a.v / b.v); }
inline Flop operator-(Flop a) { return Flop(-a.v); }
inline Flop& operator+=(Flop& a, Flop b) { a = a + b; return a; }
inline bool operator<(Flop a, Flop b) { return a.v < b.v; }
inline bool operator>(Flop a, Flop b) { return a.v > b.v; }
inline Flop sqrt(Flop a) { ++g_flops; return Flop(std::sqrt(a.v)); }
inline Flop fabs(Flop a) { return Flop(std::fabs(a.v)); }
inline double val(Flop a) { return a.v; }
inline double val(double a) { return a; }

// Dual: a value with one tangent (forward-mode differentiation). Used to
// differentiate a run with respect to its initial state; fabs takes the sign
// of the value (the branch taken by the forward run). DualT<Flop> counts the
// operations of the value and of the tangent together (the work of one
// Jacobian-vector product of the step).
inline double scalar_sqrt(double x) { return std::sqrt(x); }
inline Flop scalar_sqrt(Flop x) { return sqrt(x); }

template <class S>
struct DualT {
  S v, d;
  DualT() : v(0.0), d(0.0) {}
  DualT(double x) : v(x), d(0.0) {}  // NOLINT: implicit, so constants mix in
  DualT(S x, S t) : v(x), d(t) {}
  // hidden friends: found by argument-dependent lookup, and they let a double
  // operand convert to DualT implicitly
  friend DualT operator+(DualT a, DualT b) { return DualT(a.v + b.v, a.d + b.d); }
  friend DualT operator-(DualT a, DualT b) { return DualT(a.v - b.v, a.d - b.d); }
  friend DualT operator*(DualT a, DualT b) { return DualT(a.v * b.v, a.d * b.v + a.v * b.d); }
  friend DualT operator/(DualT a, DualT b) {
    const S q = a.v / b.v;
    return DualT(q, (a.d - q * b.d) / b.v);
  }
  friend DualT operator-(DualT a) { return DualT(-a.v, -a.d); }
  friend bool operator<(DualT a, DualT b) { return a.v < b.v; }
  friend bool operator>(DualT a, DualT b) { return a.v > b.v; }
  friend DualT sqrt(DualT a) {
    const S r = scalar_sqrt(a.v);
    return DualT(r, a.d / (S(2.0) * r));
  }
  friend DualT fabs(DualT a) { return a.v < S(0.0) ? DualT(-a.v, -a.d) : a; }
  friend double val(DualT a) { return val(a.v); }
};
using Dual = DualT<double>;
using DualFlop = DualT<Flop>;

// The global Lax-Friedrichs coefficient is a constant of each stage when a
// run is differentiated (its dependence on the state is frozen).
inline void freeze(double&) {}
inline void freeze(Flop&) {}
template <class S> inline void freeze(DualT<S>& a) { a.d = S(0.0); }

using std::fabs;
using std::sqrt;

template <class R> inline R sq(R a) { return a * a; }
template <class R> inline R rmax(R a, R b) { return (a < b) ? b : a; }

// ---------------------------------------------------------------------------
// Problem description (mirrored by a ctypes Structure in oracle/__init__.py).
// ---------------------------------------------------------------------------
enum { EQ_BURGERS = 0, EQ_EULER = 1, EQ_BUCKLEY = 2 };
enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_REFLECTIVE = 2, BC_INFLOW = 3,
       BC_DMR_BOTTOM = 4, BC_DMR_TOP = 5 };

}  // namespace

extern "C" {
struct or_problem {
  int eq;           // EQ_BURGERS, EQ_EULER or EQ_BUCKLEY (1D)
  int dim;          // 1 or 2
  int nx, ny;       // points per direction (ny = 1 in 1D)
  double x0, x1, y0, y1;
  double gas_gamma; // ratio of specific heats (Euler)
  int bc[4];        // x-low, x-high, y-low, y-high
  double inflow[4]; // imposed conserved state (inflow; DMR post-shock)
  double pre[4];    // DMR pre-shock conserved state
  double dmr_x0;    // DMR: x where the shock meets y = 0 at t = 0
  double dmr_speed; // DMR: normal shock speed
  double dmr_angle; // DMR: angle between shock and x axis (radians)
  double lin_w[3];  // gamma_0..2, reconstruction linear weights (Sec. 2.1)
  double lim_d[3];  // d_0..2, limiter linear weights (Sec. 2.2)
  double eps;       // epsilon of the nonlinear weights
  double cfl;
  int dt_mode;      // 0: CFL dx/alpha; 1: CFL dx^{5/3}/alpha; 2: fixed
  double dt_fixed;
  int limiter;      // 0 off, 1 characteristic, 2 component-wise
  int eig_avg;      // 0 Roe average, 1 arithmetic mean
  double alpha_fixed;  // > 0: use this alpha in every stage and direction
  int freeze_weights;  // tangent runs: nonlinear weights held constant
};
}

namespace {

inline int ncomp(const or_problem& P) {
  return P.eq == EQ_EULER ? (P.dim == 1 ? 3 : 4) : 1;
}

// Buckley-Leverett flux of Example 3.4, f(u) = 4u^2 / (4u^2 + (1 - u)^2), and
// its derivative by the quotient rule: with D = 4u^2 + (1 - u)^2,
// f' = (8u D - 4u^2 (8u - 2(1 - u))) / D^2 = 8u(1 - u) / D^2.
template <class R>
R bl_flux(R u) {
  const R D = 4.0 * u * u + (1.0 - u) * (1.0 - u);
  return 4.0 * u * u / D;
}
template <class R>
R bl_dflux(R u) {
  const R D = 4.0 * u * u + (1.0 - u) * (1.0 - u);
  return 8.0 * u * (1.0 - u) / (D * D);
}

// max of |f'| over [0, 1] (reading R15): f' vanishes at both ends and has a
// single interior maximum; golden-section search on the bracket.
double bl_alpha01() {
  static double cached = -1.0;
  if (cached >= 0.0) return cached;
  const double r = (std::sqrt(5.0) - 1.0) / 2.0;
  double a = 0.0, b = 1.0;
  for (int it = 0; it < 200 && b - a > 1e-15; ++it) {
    const double c = b - r * (b - a), d = a + r * (b - a);
    if (bl_dflux(c) > bl_dflux(d)) b = d;
    else a = c;
  }
  cached = bl_dflux(0.5 * (a + b));
  return cached;
}

// ---------------------------------------------------------------------------
// Sec. 2.1: HWENO reconstruction of f^+_{i+1/2} and h^+_{i+1/2} on the big
// stencil T0 = {i-1, i, i+1} and the small stencils T1 = {i-1, i},
// T2 = {i, i+1}. Inputs are the split point values f^+_{i-1..i+1},
// h^+_{i-1..i+1} (reading R2).
// ---------------------------------------------------------------------------
template <class R>
struct Face {
  R fhat, hhat;      // f^+_{i+1/2}, h^+_{i+1/2}
  R p[3], dp0;       // p_l(x_{i+1/2}), p_0'(x_{i+1/2})
  R beta[3], tau, omega[3];
};

// p_0'(x_{i+1/2}) of the quintic on T0 (Sec. 2.1): the linear flux of the
// derivative equation.
template <class R>
R p0_prime(const R f[3], const R h[3], double dx) {
  return (f[0] - 8.0 * f[1] + 7.0 * f[2]) / (4.0 * dx) + (h[0] - 2.0 * h[1] - 5.0 * h[2]) / 12.0;
}

// freeze_w: the nonlinear weights enter as constants (their tangent is
// dropped), for the frozen-weights derivative of the scheme. with_dp0 = false
// skips p_0' (hhat, dp0 stay 0): the characteristic-wise Euler flux uses only
// fhat of each characteristic field, its derivative flux being taken
// component by component (remarks after the 1D and 2D schemes).
template <class R>
Face<R> hweno_plus(const R f[3], const R h[3], double dx, const double g[3],
                   double eps, bool freeze_w = false, bool with_dp0 = true) {
  Face<R> o;
  const R fm = f[0], f0 = f[1], fp = f[2];
  const R hm = h[0], h0 = h[1], hp = h[2];

  // p_0, p_1, p_2 and p_0' at x_{i+1/2} (Sec. 2.1, values after Eq. HWEp12).
  o.p[0] = (11.0 / 60.0) * fm + (19.0 / 30.0) * f0 + (11.0 / 60.0) * fp +
           (dx / 20.0) * (hm + 10.0 * h0 - hp);
  o.p[1] = (1.0 / 6.0) * fm + (5.0 / 6.0) * f0 + (2.0 / 3.0) * dx * h0;
  o.p[2] = (5.0 / 6.0) * f0 + (1.0 / 6.0) * fp + (1.0 / 3.0) * dx * h0;
  o.dp0 = with_dp0 ? p0_prime(f, h, dx) : R(0.0);

  // a_1..a_5 and the smoothness indicators (Eq. GHYZP).
  const R a1 = dx * ((19.0 / 192.0) * hm + (79.0 / 48.0) * h0 + (19.0 / 192.0) * hp) +
               (27.0 / 64.0) * (fm - fp);
  const R a2 = dx * ((3.0 / 8.0) * hm - (3.0 / 8.0) * hp) +
               (5.0 / 4.0) * (fm - 2.0 * f0 + fp);
  const R a3 = -(dx * ((11.0 / 24.0) * hm + (17.0 / 6.0) * h0 + (11.0 / 24.0) * hp)) +
               (15.0 / 8.0) * (fp - fm);
  const R a4 = dx * ((1.0 / 4.0) * hp - (1.0 / 4.0) * hm) -
               (1.0 / 2.0) * (fm - 2.0 * f0 + fp);
  const R a5 = dx * ((1.0 / 4.0) * hm + h0 + (1.0 / 4.0) * hp) + (3.0 / 4.0) * (fm - fp);

  o.beta[0] = sq(a1 + (1.0 / 4.0) * a3 + (1.0 / 16.0) * a5) +
              (13.0 / 3.0) * sq(a2 + (63.0 / 130.0) * a4) +
              (781.0 / 20.0) * sq(a3 + (8825.0 / 10934.0) * a5) +
              (1421461.0 / 2275.0) * sq(a4) +
              (21520059541.0 / 1377684.0) * sq(a5);
  o.beta[1] = sq(h0 * dx) + (13.0 / 3.0) * sq(dx * h0 - f0 + fm);
  o.beta[2] = sq(h0 * dx) + (13.0 / 3.0) * sq(dx * h0 + f0 - fp);  // R1

  // tau (Eq. tau-fh) and the nonlinear weights.
  o.tau = 0.25 * sq(fabs(o.beta[0] - o.beta[1]) + fabs(o.beta[0] - o.beta[2]));
  R wbar[3];
  for (int l = 0; l < 3; ++l) wbar[l] = g[l] * (1.0 + o.tau / (o.beta[l] + eps));
  const R wsum = wbar[0] + wbar[1] + wbar[2];
  for (int l = 0; l < 3; ++l) o.omega[l] = wbar[l] / wsum;
  if (freeze_w)
    for (int l = 0; l < 3; ++l) freeze(o.omega[l]);

  // Final combination and the linear derivative flux.
  o.fhat = o.omega[0] * (o.p[0] / g[0] - (g[1] / g[0]) * o.p[1] - (g[2] / g[0]) * o.p[2]) +
           o.omega[1] * o.p[1] + o.omega[2] * o.p[2];
  o.hhat = o.dp0;
  return o;
}

// Mirror procedure for f^-_{i+1/2}, h^-_{i+1/2} (reading R3). Inputs are the
// split values f^-, h^- at i, i+1, i+2. The reflection x -> 2 x_{i+1/2} - x
// maps cell I_{i+1+k} onto I_{i-k}, keeps cell averages and flips the sign of
// derivative data; the reflected problem is the "+" problem, and the
// derivative flux reflects back with a sign change.
template <class R>
Face<R> hweno_minus(const R f[3], const R h[3], double dx, const double g[3],
                    double eps, bool freeze_w = false, bool with_dp0 = true) {
  const R fr[3] = {f[2], f[1], f[0]};
  const R hr[3] = {-h[2], -h[1], -h[0]};
  Face<R> o = hweno_plus(fr, hr, dx, g, eps, freeze_w, with_dp0);
  o.hhat = -o.hhat;
  o.dp0 = -o.dp0;
  return o;
}

// ---------------------------------------------------------------------------
// Sec. 2.2: HWENO limiter for the derivative at x_i from the point values
// u_{i-1}, u_i, u_{i+1} and the derivatives v_{i-1}, v_{i+1}.
// ---------------------------------------------------------------------------
template <class R>
struct Lim {
  R vt;
  R dq[3];
  R beta[3], tau, lambda[3];
};

template <class R>
Lim<R> hweno_limiter(R um, R u0, R up, R vm, R vp, double dx, const double d[3],
                     double eps, bool freeze_w = false) {
  Lim<R> o;
  o.dq[0] = (3.0 / (4.0 * dx)) * (up - um) - (1.0 / 4.0) * (vm + vp);
  o.dq[1] = (u0 - um) / dx;
  o.dq[2] = (up - u0) / dx;

  const R a1 = -(dx / 4.0) * (vm + vp) + (3.0 / 4.0) * (up - um);
  const R a2 = (dx / 4.0) * (vm - vp) + um - 2.0 * u0 + up;
  const R a3 = (dx / 4.0) * (vm + vp) + (1.0 / 4.0) * (um - up);
  const R a4 = (dx / 4.0) * (vp - vm) - (1.0 / 2.0) * (um - 2.0 * u0 + up);
  o.beta[0] = sq(a1 + (1.0 / 4.0) * a3) + (13.0 / 3.0) * sq(a2 + (63.0 / 130.0) * a4) +
              (781.0 / 20.0) * sq(a3) + (1421461.0 / 2275.0) * sq(a4);
  o.beta[1] = sq(u0 - um);
  o.beta[2] = sq(u0 - up);

  o.tau = 0.25 * sq(fabs(o.beta[0] - o.beta[1]) + fabs(o.beta[0] - o.beta[2]));
  R lbar[3];
  for (int l = 0; l < 3; ++l) lbar[l] = d[l] * (1.0 + o.tau / (o.beta[l] + eps));
  const R lsum = lbar[0] + lbar[1] + lbar[2];
  for (int l = 0; l < 3; ++l) o.lambda[l] = lbar[l] / lsum;
  if (freeze_w)
    for (int l = 0; l < 3; ++l) freeze(o.lambda[l]);

  o.vt = o.lambda[0] * (o.dq[0] / d[0] - (d[1] / d[0]) * o.dq[1] - (d[2] / d[0]) * o.dq[2]) +
         o.lambda[1] * o.dq[1] + o.lambda[2] * o.dq[2];
  return o;
}

// ---------------------------------------------------------------------------
// Physics. Burgers: f = g = u^2/2. Euler: Eq. euler1 (1D), Eq. euler2 (2D),
// E = p/(gamma-1) + rho |u|^2 / 2. `dir` is 0 for x and 1 for y. The
// derivative-equation fluxes h, xi, eta, theta of Eq. EQ3 are Jacobian-vector
// products A(U) D with D = U_x or U_y.
// ---------------------------------------------------------------------------
template <class R>
void flux(const or_problem& P, int dir, const R* U, R* F) {
  if (P.eq == EQ_BURGERS) { F[0] = 0.5 * U[0] * U[0]; return; }
  if (P.eq == EQ_BUCKLEY) { F[0] = bl_flux(U[0]); return; }
  const double gm = P.gas_gamma - 1.0;
  if (P.dim == 1) {
    const R rho = U[0], m = U[1], E = U[2];
    const R u = m / rho;
    const R p = gm * (E - 0.5 * m * u);
    F[0] = m; F[1] = m * u + p; F[2] = (E + p) * u;
    return;
  }
  const R rho = U[0], m = U[1], n = U[2], E = U[3];
  const R u = m / rho, v = n / rho;
  const R p = gm * (E - 0.5 * (m * u + n * v));
  if (dir == 0) { F[0] = m; F[1] = m * u + p; F[2] = m * v; F[3] = (E + p) * u; }
  else          { F[0] = n; F[1] = n * u; F[2] = n * v + p; F[3] = (E + p) * v; }
}

template <class R>
void jvp(const or_problem& P, int dir, const R* U, const R* D, R* out) {
  if (P.eq == EQ_BURGERS) { out[0] = U[0] * D[0]; return; }
  if (P.eq == EQ_BUCKLEY) { out[0] = bl_dflux(U[0]) * D[0]; return; }
  const double gm = P.gas_gamma - 1.0;
  if (P.dim == 1) {
    const R rho = U[0], m = U[1], E = U[2];
    const R u = m / rho;
    const R p = gm * (E - 0.5 * m * u);
    const R du = (D[1] - u * D[0]) / rho;
    const R dp = gm * (D[2] - u * D[1] + 0.5 * u * u * D[0]);
    out[0] = D[1];
    out[1] = D[1] * u + m * du + dp;
    out[2] = (D[2] + dp) * u + (E + p) * du;
    return;
  }
  const R rho = U[0], m = U[1], n = U[2], E = U[3];
  const R u = m / rho, v = n / rho;
  const R p = gm * (E - 0.5 * (m * u + n * v));
  const R du = (D[1] - u * D[0]) / rho;
  const R dv = (D[2] - v * D[0]) / rho;
  const R dp = gm * (D[3] - (u * D[1] + v * D[2]) + 0.5 * (u * u + v * v) * D[0]);
  if (dir == 0) {
    out[0] = D[1];
    out[1] = D[1] * u + m * du + dp;
    out[2] = D[1] * v + m * dv;
    out[3] = (D[3] + dp) * u + (E + p) * du;
  } else {
    out[0] = D[2];
    out[1] = D[2] * u + n * du;
    out[2] = D[2] * v + n * dv + dp;
    out[3] = (D[3] + dp) * v + (E + p) * dv;
  }
}

// max |f'(u)| contribution of one point (reading R6).
template <class R>
R wave_speed(const or_problem& P, int dir, const R* U) {
  if (P.eq == EQ_BURGERS) return fabs(U[0]);
  if (P.eq == EQ_BUCKLEY) return rmax(R(bl_alpha01()), fabs(bl_dflux(U[0])));  // R15
  const double gam = P.gas_gamma;
  if (P.dim == 1) {
    const R u = U[1] / U[0];
    const R p = (gam - 1.0) * (U[2] - 0.5 * U[1] * u);
    return fabs(u) + sqrt(gam * p / U[0]);
  }
  const R u = U[1] / U[0], v = U[2] / U[0];
  const R p = (gam - 1.0) * (U[3] - 0.5 * (U[1] * u + U[2] * v));
  const R c = sqrt(gam * p / U[0]);
  return (dir == 0 ? fabs(u) : fabs(v)) + c;
}

// Velocity, enthalpy and sound speed of the state used for the eigenvectors:
// Roe average of UL, UR (mode 0, reading R7), arithmetic mean (mode 1), or the
// state UL itself (UR == nullptr; used by the limiter, reading R8).
template <class R>
void eigen_state(const or_problem& P, const R* UL, const R* UR, int mode, R& u,
                 R& v, R& H, R& c) {
  const double gam = P.gas_gamma, gm = gam - 1.0;
  const int m = ncomp(P);
  const int iE = m - 1;
  auto prim = [&](const R* U, R& uu, R& vv, R& HH) {
    uu = U[1] / U[0];
    vv = (m == 4) ? U[2] / U[0] : R(0.0);
    const R ke = (m == 4) ? 0.5 * (U[1] * uu + U[2] * vv) : 0.5 * U[1] * uu;
    const R p = gm * (U[iE] - ke);
    HH = (U[iE] + p) / U[0];
  };
  if (UR == nullptr) {
    prim(UL, u, v, H);
  } else if (mode == 0) {
    R uL, vL, HL, uR, vR, HR;
    prim(UL, uL, vL, HL);
    prim(UR, uR, vR, HR);
    const R sL = sqrt(UL[0]), sR = sqrt(UR[0]);
    const R s = sL + sR;
    u = (sL * uL + sR * uR) / s;
    v = (m == 4) ? (sL * vL + sR * vR) / s : R(0.0);
    H = (sL * HL + sR * HR) / s;
  } else {
    R Um[4];
    for (int k = 0; k < m; ++k) Um[k] = 0.5 * (UL[k] + UR[k]);
    prim(Um, u, v, H);
  }
  const R q2 = (m == 4) ? u * u + v * v : u * u;
  c = sqrt(gm * (H - 0.5 * q2));
}

// Eigenvectors of the Euler flux Jacobian in direction `dir` (standard forms).
// Rm holds right eigenvectors as columns, Lm = Rm^{-1}; both m x m row-major.
// Eigenvalue order: u-c, u, (u: shear, 2D), u+c (u -> v for dir = 1).
template <class R>
void eigenvectors(const or_problem& P, int dir, R u, R v, R H, R c, R* Rm, R* Lm,
                  R* lam) {
  const double gm = P.gas_gamma - 1.0;
  const int m = ncomp(P);
  const R b1 = gm / (c * c);
  if (m == 3) {
    const R b2 = 0.5 * b1 * u * u;
    const R Rv[9] = {1.0, 1.0, 1.0,
                     u - c, u, u + c,
                     H - u * c, 0.5 * u * u, H + u * c};
    const R Lv[9] = {0.5 * (b2 + u / c), -0.5 * (b1 * u + 1.0 / c), 0.5 * b1,
                     1.0 - b2, b1 * u, -b1,
                     0.5 * (b2 - u / c), -0.5 * (b1 * u - 1.0 / c), 0.5 * b1};
    for (int k = 0; k < 9; ++k) { Rm[k] = Rv[k]; Lm[k] = Lv[k]; }
    if (lam) { lam[0] = u - c; lam[1] = u; lam[2] = u + c; }
    return;
  }
  const R b2 = 0.5 * b1 * (u * u + v * v);
  const R q2h = 0.5 * (u * u + v * v);
  if (dir == 0) {
    const R Rv[16] = {1.0, 1.0, 0.0, 1.0,
                      u - c, u, 0.0, u + c,
                      v, v, 1.0, v,
                      H - u * c, q2h, v, H + u * c};
    const R Lv[16] = {0.5 * (b2 + u / c), -0.5 * (b1 * u + 1.0 / c), -0.5 * b1 * v, 0.5 * b1,
                      1.0 - b2, b1 * u, b1 * v, -b1,
                      -v, 0.0, 1.0, 0.0,
                      0.5 * (b2 - u / c), -0.5 * (b1 * u - 1.0 / c), -0.5 * b1 * v, 0.5 * b1};
    for (int k = 0; k < 16; ++k) { Rm[k] = Rv[k]; Lm[k] = Lv[k]; }
    if (lam) { lam[0] = u - c; lam[1] = u; lam[2] = u; lam[3] = u + c; }
  } else {
    const R Rv[16] = {1.0, 1.0, 0.0, 1.0,
                      u, u, 1.0, u,
                      v - c, v, 0.0, v + c,
                      H - v * c, q2h, u, H + v * c};
    const R Lv[16] = {0.5 * (b2 + v / c), -0.5 * b1 * u, -0.5 * (b1 * v + 1.0 / c), 0.5 * b1,
                      1.0 - b2, b1 * u, b1 * v, -b1,
                      -u, 1.0, 0.0, 0.0,
                      0.5 * (b2 - v / c), -0.5 * b1 * u, -0.5 * (b1 * v - 1.0 / c), 0.5 * b1};
    for (int k = 0; k < 16; ++k) { Rm[k] = Rv[k]; Lm[k] = Lv[k]; }
    if (lam) { lam[0] = v - c; lam[1] = v; lam[2] = v; lam[3] = v + c; }
  }
}

template <class R>
void matvec(int m, const R* A, const R* x, R* y) {
  for (int r = 0; r < m; ++r) {
    R s = A[r * m] * x[0];
    for (int k = 1; k < m; ++k) s = s + A[r * m + k] * x[k];
    y[r] = s;
  }
}

// ---------------------------------------------------------------------------
// One sweep line: numerical fluxes at the n+1 interfaces x_{i-1/2}, i = 0..n,
// of a line of n interior points, from a ghosted line (index g = i + 2) of
// states U, split-flux inputs (f, hd) and the derivative data for the mixed
// term. Outputs per interface: fhat (HWENO, Sec. 2.1, characteristic-wise for
// Euler per the remarks of Sec. 2.1 and 2.2-2D), hhat (p_0', component-wise),
// mixed (Eq. mixed, central, no splitting; nullable).
// ---------------------------------------------------------------------------
template <class R>
void sweep_line(const or_problem& P, int dir, int n, double dx, R alpha,
                const std::vector<const R*>& Ug,   // [m] ghosted lines
                const std::vector<const R*>& Dg,   // [m] derivative along dir
                const std::vector<const R*>& Fg,   // [m] flux along dir
                const std::vector<const R*>& Hg,   // [m] A_dir D
                const std::vector<const R*>& Xg,   // [m] mixed flux or empty
                std::vector<R*>& fhat, std::vector<R*>& hhat,
                std::vector<R*>& mixed) {
  const int m = ncomp(P);
  const double* gw = P.lin_w;
  // Global Lax-Friedrichs splitting of f and h (Sec. 2.1).
  const int ng = n + 4;
  std::vector<std::vector<R>> fp(m, std::vector<R>(ng)), fmn(m, std::vector<R>(ng)),
      hp(m, std::vector<R>(ng)), hmn(m, std::vector<R>(ng));
  for (int c = 0; c < m; ++c)
    for (int g = 0; g < ng; ++g) {
      fp[c][g] = 0.5 * (Fg[c][g] + alpha * Ug[c][g]);
      fmn[c][g] = 0.5 * (Fg[c][g] - alpha * Ug[c][g]);
      hp[c][g] = 0.5 * (Hg[c][g] + alpha * Dg[c][g]);
      hmn[c][g] = 0.5 * (Hg[c][g] - alpha * Dg[c][g]);
    }

  for (int j = 0; j <= n; ++j) {
    // interface x_{i+1/2} with i = j - 1, ghosted index gi = i + 2 = j + 1
    const int gi = j + 1;
    R fh[4], hh[4];
    if (m == 1) {
      const R f3p[3] = {fp[0][gi - 1], fp[0][gi], fp[0][gi + 1]};
      const R h3p[3] = {hp[0][gi - 1], hp[0][gi], hp[0][gi + 1]};
      const R f3m[3] = {fmn[0][gi], fmn[0][gi + 1], fmn[0][gi + 2]};
      const R h3m[3] = {hmn[0][gi], hmn[0][gi + 1], hmn[0][gi + 2]};
      const Face<R> a = hweno_plus(f3p, h3p, dx, gw, P.eps, P.freeze_weights != 0);
      const Face<R> b = hweno_minus(f3m, h3m, dx, gw, P.eps, P.freeze_weights != 0);
      fh[0] = a.fhat + b.fhat;
      hh[0] = a.hhat + b.hhat;
    } else {
      // Local characteristic decomposition at x_{i+1/2} (remarks after the
      // 1D and 2D schemes): project f^{+-} and h^{+-} on the stencil with the
      // left eigenvectors, reconstruct each field, back-project.
      R UL[4], UR[4];
      for (int c = 0; c < m; ++c) { UL[c] = Ug[c][gi]; UR[c] = Ug[c][gi + 1]; }
      R u, v, H, cs, Rm[16], Lm[16];
      eigen_state(P, UL, UR, P.eig_avg, u, v, H, cs);
      eigenvectors(P, dir, u, v, H, cs, Rm, Lm, (R*)nullptr);
      R wfp[3][4], whp[3][4], wfm[3][4], whm[3][4];
      for (int k = 0; k < 3; ++k) {
        R x1[4], x2[4], x3[4], x4[4];
        for (int c = 0; c < m; ++c) {
          x1[c] = fp[c][gi - 1 + k]; x2[c] = hp[c][gi - 1 + k];
          x3[c] = fmn[c][gi + k];    x4[c] = hmn[c][gi + k];
        }
        matvec(m, Lm, x1, wfp[k]); matvec(m, Lm, x2, whp[k]);
        matvec(m, Lm, x3, wfm[k]); matvec(m, Lm, x4, whm[k]);
      }
      R fchar[4];
      for (int s = 0; s < m; ++s) {
        const R f3p[3] = {wfp[0][s], wfp[1][s], wfp[2][s]};
        const R h3p[3] = {whp[0][s], whp[1][s], whp[2][s]};
        const R f3m[3] = {wfm[0][s], wfm[1][s], wfm[2][s]};
        const R h3m[3] = {whm[0][s], whm[1][s], whm[2][s]};
        const Face<R> a = hweno_plus(f3p, h3p, dx, gw, P.eps, P.freeze_weights != 0, false);
        const Face<R> b = hweno_minus(f3m, h3m, dx, gw, P.eps, P.freeze_weights != 0, false);
        fchar[s] = a.fhat + b.fhat;
      }
      matvec(m, Rm, fchar, fh);
      // derivative flux: linear p_0', component by component; the "-" side
      // is the mirror image (reversed stencil, negated h, negated result)
      for (int c = 0; c < m; ++c) {
        const R f3p[3] = {fp[c][gi - 1], fp[c][gi], fp[c][gi + 1]};
        const R h3p[3] = {hp[c][gi - 1], hp[c][gi], hp[c][gi + 1]};
        const R f3r[3] = {fmn[c][gi + 2], fmn[c][gi + 1], fmn[c][gi]};
        const R h3r[3] = {-hmn[c][gi + 2], -hmn[c][gi + 1], -hmn[c][gi]};
        hh[c] = p0_prime(f3p, h3p, dx) + (-p0_prime(f3r, h3r, dx));
      }
    }
    for (int c = 0; c < m; ++c) { fhat[c][j] = fh[c]; hhat[c][j] = hh[c]; }
    if (!Xg.empty()) {
      // Eq. mixed: -1/12 x_{i-1} + 7/12 x_i + 7/12 x_{i+1} - 1/12 x_{i+2}
      for (int c = 0; c < m; ++c)
        mixed[c][j] = -(1.0 / 12.0) * Xg[c][gi - 1] + (7.0 / 12.0) * Xg[c][gi] +
                      (7.0 / 12.0) * Xg[c][gi + 1] - (1.0 / 12.0) * Xg[c][gi + 2];
    }
  }
}

// Limited derivative along a line (Sec. 2.2), n interior points; U and D are
// ghosted (g = i + 2). Characteristic-wise with eigenvectors at U_i (R8) or
// component-wise; limiter = 0 copies D.
template <class R>
void limit_line(const or_problem& P, int dir, int n, double dx,
                const std::vector<const R*>& Ug, const std::vector<const R*>& Dg,
                std::vector<R*>& Dt) {
  const int m = ncomp(P);
  for (int i = 0; i < n; ++i) {
    const int g = i + 2;
    if (P.limiter == 0) {
      for (int c = 0; c < m; ++c) Dt[c][i] = Dg[c][g];
      continue;
    }
    if (m == 1 || P.limiter == 2) {
      for (int c = 0; c < m; ++c)
        Dt[c][i] = hweno_limiter(Ug[c][g - 1], Ug[c][g], Ug[c][g + 1], Dg[c][g - 1],
                                 Dg[c][g + 1], dx, P.lim_d, P.eps, P.freeze_weights != 0).vt;
      continue;
    }
    R U0[4];
    for (int c = 0; c < m; ++c) U0[c] = Ug[c][g];
    R u, v, H, cs, Rm[16], Lm[16];
    eigen_state(P, U0, (const R*)nullptr, 0, u, v, H, cs);
    eigenvectors(P, dir, u, v, H, cs, Rm, Lm, (R*)nullptr);
    R xm[4], x0[4], xp[4], dm[4], dp[4];
    R wm[4], w0[4], wp[4], zm[4], zp[4], zt[4], out[4];
    for (int c = 0; c < m; ++c) {
      xm[c] = Ug[c][g - 1]; x0[c] = Ug[c][g]; xp[c] = Ug[c][g + 1];
      dm[c] = Dg[c][g - 1]; dp[c] = Dg[c][g + 1];
    }
    matvec(m, Lm, xm, wm); matvec(m, Lm, x0, w0); matvec(m, Lm, xp, wp);
    matvec(m, Lm, dm, zm); matvec(m, Lm, dp, zp);
    for (int s = 0; s < m; ++s)
      zt[s] = hweno_limiter(wm[s], w0[s], wp[s], zm[s], zp[s], dx, P.lim_d, P.eps,
                            P.freeze_weights != 0).vt;
    matvec(m, Rm, zt, out);
    for (int c = 0; c < m; ++c) Dt[c][i] = out[c];
  }
}

// ---------------------------------------------------------------------------
// Ghost values (reading R9; double Mach reflection R10).
// ---------------------------------------------------------------------------
// Sign of component c under reflection through a wall normal to `dir`.
inline double refl_sign(const or_problem& P, int dir, int c) {
  if (P.eq == EQ_BURGERS) return -1.0;  // Burgers: (x, u) -> (-x, -u)
  if (P.eq == EQ_BUCKLEY) return 1.0;   // a saturation: even
  return (c == 1 + dir) ? -1.0 : 1.0;   // normal momentum is odd
}

inline double dmr_shock_x(const or_problem& P, double y, double t) {
  return P.dmr_x0 + y / std::tan(P.dmr_angle) + P.dmr_speed * t / std::sin(P.dmr_angle);
}

// 1D line ghost fill along `dir` for one line; `pos` is the fixed coordinate
// of the line in the other direction (2D), used by the DMR conditions.
// Ug, Vg, Wg are ghosted lines (n + 4); V is the derivative along dir, W the
// other derivative (nullable in 1D).
template <class R>
void fill_line(const or_problem& P, int dir, int n, double lo, double h, double pos,
               double t, R** Ug, R** Vg, R** Wg) {
  const int m = ncomp(P);
  for (int side = 0; side < 2; ++side) {
    const int kind = P.bc[2 * dir + side];
    for (int k = 1; k <= 2; ++k) {
      const int i = side == 0 ? -k : n - 1 + k;  // ghost point index
      const int g = i + 2;
      int src = -1;
      bool mirror = false, imposed = false;
      const double* state = nullptr;
      switch (kind) {
        case BC_PERIODIC: src = (i + n) % n; break;
        case BC_OUTFLOW: src = side == 0 ? 0 : n - 1; break;
        case BC_REFLECTIVE: src = side == 0 ? -i - 1 : 2 * n - 1 - i; mirror = true; break;
        case BC_INFLOW: imposed = true; state = P.inflow; break;
        case BC_DMR_BOTTOM:
          if (pos < P.dmr_x0) { imposed = true; state = P.inflow; }
          else { src = side == 0 ? -i - 1 : 2 * n - 1 - i; mirror = true; }
          break;
        case BC_DMR_TOP: {
          const double yg = lo + (i + 0.5) * h;
          imposed = true;
          state = (pos < dmr_shock_x(P, yg, t)) ? P.inflow : P.pre;
          break;
        }
      }
      for (int c = 0; c < m; ++c) {
        if (imposed) {
          Ug[c][g] = state[c];
          Vg[c][g] = 0.0;
          if (Wg) Wg[c][g] = 0.0;
        } else if (mirror) {
          const int s = src + 2;
          const double su = refl_sign(P, dir, c);
          Ug[c][g] = su * Ug[c][s];
          Vg[c][g] = -su * Vg[c][s];         // normal derivative: opposite parity
          if (Wg) Wg[c][g] = su * Wg[c][s];  // tangential derivative: same parity
        } else {
          const int s = src + 2;
          Ug[c][g] = Ug[c][s];
          Vg[c][g] = Vg[c][s];
          if (Wg) Wg[c][g] = Wg[c][s];
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Spatial operator, 1D (Eq. odeH and the operators L^1, L^2 of Sec. 2.2).
// U, V: [m][n]. Outputs L1, L2 [m][n], Vt (limited V, nullable), alpha.
// ---------------------------------------------------------------------------
template <class R>
void rhs_1d(const or_problem& P, const R* U, const R* V, double t, R* L1, R* L2,
            R* Vt, R* alpha_out) {
  const int m = ncomp(P), n = P.nx, ng = n + 4;
  const double dx = (P.x1 - P.x0) / n;
  std::vector<R> Ug(m * ng), Vg(m * ng), Fg(m * ng), Hg(m * ng);
  for (int c = 0; c < m; ++c)
    for (int i = 0; i < n; ++i) { Ug[c * ng + i + 2] = U[c * n + i]; Vg[c * ng + i + 2] = V[c * n + i]; }
  std::vector<R*> up(m), vp(m);
  for (int c = 0; c < m; ++c) { up[c] = &Ug[c * ng]; vp[c] = &Vg[c * ng]; }
  fill_line(P, 0, n, P.x0, dx, 0.0, t, up.data(), vp.data(), (R**)nullptr);

  // alpha = max |f'(u)| over the grid (R6)
  R alpha = 0.0;
  for (int i = 0; i < n; ++i) {
    R Ui[4];
    for (int c = 0; c < m; ++c) Ui[c] = U[c * n + i];
    alpha = rmax(alpha, wave_speed(P, 0, Ui));
  }
  if (P.alpha_fixed > 0.0) alpha = P.alpha_fixed;
  freeze(alpha);
  if (alpha_out) *alpha_out = alpha;

  // point fluxes f and h = f'(u) v on the ghosted line
  for (int g = 0; g < ng; ++g) {
    R Ui[4], Vi[4], Fi[4], Hi[4];
    for (int c = 0; c < m; ++c) { Ui[c] = Ug[c * ng + g]; Vi[c] = Vg[c * ng + g]; }
    flux(P, 0, Ui, Fi);
    jvp(P, 0, Ui, Vi, Hi);
    for (int c = 0; c < m; ++c) { Fg[c * ng + g] = Fi[c]; Hg[c * ng + g] = Hi[c]; }
  }

  std::vector<R> fh(m * (n + 1)), hh(m * (n + 1));
  std::vector<const R*> cu(m), cv(m), cf(m), ch(m), cx;
  std::vector<R*> pfh(m), phh(m), pmx;
  for (int c = 0; c < m; ++c) {
    cu[c] = &Ug[c * ng]; cv[c] = &Vg[c * ng]; cf[c] = &Fg[c * ng]; ch[c] = &Hg[c * ng];
    pfh[c] = &fh[c * (n + 1)]; phh[c] = &hh[c * (n + 1)];
  }
  sweep_line(P, 0, n, dx, alpha, cu, cv, cf, ch, cx, pfh, phh, pmx);

  for (int c = 0; c < m; ++c)
    for (int i = 0; i < n; ++i) {
      L1[c * n + i] = -(fh[c * (n + 1) + i + 1] - fh[c * (n + 1) + i]) / dx;
      L2[c * n + i] = -(hh[c * (n + 1) + i + 1] - hh[c * (n + 1) + i]) / dx;
    }
  if (Vt) {
    std::vector<R*> pvt(m);
    for (int c = 0; c < m; ++c) pvt[c] = Vt + c * n;
    limit_line(P, 0, n, dx, cu, cv, pvt);
  }
}

// ---------------------------------------------------------------------------
// Spatial operator, 2D (Eq. ode2H, Eq. mixed, reading R4). U, V, W: [m][ny][nx].
// ---------------------------------------------------------------------------
template <class R>
void rhs_2d(const or_problem& P, const R* U, const R* V, const R* W, double t,
            R* L1, R* L2, R* L3, R* Vt, R* Wt, R* alpha_out) {
  const int m = ncomp(P), nx = P.nx, ny = P.ny;
  const double dx = (P.x1 - P.x0) / nx, dy = (P.y1 - P.y0) / ny;
  const size_t npt = (size_t)nx * ny;
  auto at = [&](const R* A, int c, int j, int i) { return A[(size_t)c * npt + (size_t)j * nx + i]; };

  // alpha_x, alpha_y (R6)
  R ax = 0.0, ay = 0.0;
  for (size_t q = 0; q < npt; ++q) {
    R Uq[4];
    for (int c = 0; c < m; ++c) Uq[c] = U[c * npt + q];
    ax = rmax(ax, wave_speed(P, 0, Uq));
    ay = rmax(ay, wave_speed(P, 1, Uq));
  }
  if (P.alpha_fixed > 0.0) ax = ay = P.alpha_fixed;
  freeze(ax);
  freeze(ay);
  if (alpha_out) { alpha_out[0] = ax; alpha_out[1] = ay; }

  std::vector<R> A1(m * npt, R(0.0)), A2(m * npt, R(0.0)), A3(m * npt, R(0.0));

  // x-sweep, row by row: f-hat (HWENO in x), h-hat (p_0'), eta-hat (mixed)
  {
    const int ng = nx + 4;
    std::vector<R> Ug(m * ng), Vg(m * ng), Wg(m * ng), Fg(m * ng), Hg(m * ng), Eg(m * ng);
    std::vector<R> fh(m * (nx + 1)), hh(m * (nx + 1)), eh(m * (nx + 1)), vt(m * nx);
    for (int j = 0; j < ny; ++j) {
      for (int c = 0; c < m; ++c)
        for (int i = 0; i < nx; ++i) {
          Ug[c * ng + i + 2] = at(U, c, j, i);
          Vg[c * ng + i + 2] = at(V, c, j, i);
          Wg[c * ng + i + 2] = at(W, c, j, i);
        }
      std::vector<R*> up(m), vp(m), wp(m);
      for (int c = 0; c < m; ++c) { up[c] = &Ug[c * ng]; vp[c] = &Vg[c * ng]; wp[c] = &Wg[c * ng]; }
      const double ypos = P.y0 + (j + 0.5) * dy;
      fill_line(P, 0, nx, P.x0, dx, ypos, t, up.data(), vp.data(), wp.data());
      for (int g = 0; g < ng; ++g) {
        R Ui[4], Vi[4], Wi[4], Fi[4], Hi[4], Ei[4];
        for (int c = 0; c < m; ++c) { Ui[c] = Ug[c * ng + g]; Vi[c] = Vg[c * ng + g]; Wi[c] = Wg[c * ng + g]; }
        flux(P, 0, Ui, Fi);
        jvp(P, 0, Ui, Vi, Hi);   // h   = f'(u) u_x
        jvp(P, 0, Ui, Wi, Ei);   // eta = f'(u) u_y
        for (int c = 0; c < m; ++c) { Fg[c * ng + g] = Fi[c]; Hg[c * ng + g] = Hi[c]; Eg[c * ng + g] = Ei[c]; }
      }
      std::vector<const R*> cu(m), cv(m), cf(m), ch(m), ce(m);
      std::vector<R*> pfh(m), phh(m), peh(m), pvt(m);
      for (int c = 0; c < m; ++c) {
        cu[c] = &Ug[c * ng]; cv[c] = &Vg[c * ng]; cf[c] = &Fg[c * ng]; ch[c] = &Hg[c * ng];
        ce[c] = &Eg[c * ng];
        pfh[c] = &fh[c * (nx + 1)]; phh[c] = &hh[c * (nx + 1)]; peh[c] = &eh[c * (nx + 1)];
        pvt[c] = &vt[c * nx];
      }
      sweep_line(P, 0, nx, dx, ax, cu, cv, cf, ch, ce, pfh, phh, peh);
      for (int c = 0; c < m; ++c)
        for (int i = 0; i < nx; ++i) {
          const size_t q = (size_t)c * npt + (size_t)j * nx + i;
          A1[q] = -(fh[c * (nx + 1) + i + 1] - fh[c * (nx + 1) + i]) / dx;
          A2[q] = -(hh[c * (nx + 1) + i + 1] - hh[c * (nx + 1) + i]) / dx;
          A3[q] = -(eh[c * (nx + 1) + i + 1] - eh[c * (nx + 1) + i]) / dx;  // R4
        }
      if (Vt) {
        limit_line(P, 0, nx, dx, cu, cv, pvt);
        for (int c = 0; c < m; ++c)
          for (int i = 0; i < nx; ++i) Vt[(size_t)c * npt + (size_t)j * nx + i] = vt[c * nx + i];
      }
    }
  }

  // y-sweep, column by column: g-hat (HWENO in y), theta-hat (p_0'), xi-hat
  {
    const int ng = ny + 4;
    std::vector<R> Ug(m * ng), Vg(m * ng), Wg(m * ng), Gg(m * ng), Tg(m * ng), Xg(m * ng);
    std::vector<R> gh(m * (ny + 1)), th(m * (ny + 1)), xh(m * (ny + 1)), wt(m * ny);
    for (int i = 0; i < nx; ++i) {
      for (int c = 0; c < m; ++c)
        for (int j = 0; j < ny; ++j) {
          Ug[c * ng + j + 2] = at(U, c, j, i);
          Vg[c * ng + j + 2] = at(V, c, j, i);
          Wg[c * ng + j + 2] = at(W, c, j, i);
        }
      std::vector<R*> up(m), vp(m), wp(m);
      for (int c = 0; c < m; ++c) { up[c] = &Ug[c * ng]; vp[c] = &Vg[c * ng]; wp[c] = &Wg[c * ng]; }
      const double xpos = P.x0 + (i + 0.5) * dx;
      // along y the normal derivative is W and the tangential one is V
      fill_line(P, 1, ny, P.y0, dy, xpos, t, up.data(), wp.data(), vp.data());
      for (int g = 0; g < ng; ++g) {
        R Ui[4], Vi[4], Wi[4], Gi[4], Ti[4], Xi[4];
        for (int c = 0; c < m; ++c) { Ui[c] = Ug[c * ng + g]; Vi[c] = Vg[c * ng + g]; Wi[c] = Wg[c * ng + g]; }
        flux(P, 1, Ui, Gi);
        jvp(P, 1, Ui, Wi, Ti);   // theta = g'(u) u_y
        jvp(P, 1, Ui, Vi, Xi);   // xi    = g'(u) u_x
        for (int c = 0; c < m; ++c) { Gg[c * ng + g] = Gi[c]; Tg[c * ng + g] = Ti[c]; Xg[c * ng + g] = Xi[c]; }
      }
      std::vector<const R*> cu(m), cw(m), cg(m), ct(m), cx(m);
      std::vector<R*> pgh(m), pth(m), pxh(m), pwt(m);
      for (int c = 0; c < m; ++c) {
        cu[c] = &Ug[c * ng]; cw[c] = &Wg[c * ng]; cg[c] = &Gg[c * ng]; ct[c] = &Tg[c * ng];
        cx[c] = &Xg[c * ng];
        pgh[c] = &gh[c * (ny + 1)]; pth[c] = &th[c * (ny + 1)]; pxh[c] = &xh[c * (ny + 1)];
        pwt[c] = &wt[c * ny];
      }
      sweep_line(P, 1, ny, dy, ay, cu, cw, cg, ct, cx, pgh, pth, pxh);
      for (int c = 0; c < m; ++c)
        for (int j = 0; j < ny; ++j) {
          const size_t q = (size_t)c * npt + (size_t)j * nx + i;
          A1[q] = A1[q] - (gh[c * (ny + 1) + j + 1] - gh[c * (ny + 1) + j]) / dy;
          A2[q] = A2[q] - (xh[c * (ny + 1) + j + 1] - xh[c * (ny + 1) + j]) / dy;  // R4
          A3[q] = A3[q] - (th[c * (ny + 1) + j + 1] - th[c * (ny + 1) + j]) / dy;
        }
      if (Wt) {
        limit_line(P, 1, ny, dy, cu, cw, pwt);
        for (int c = 0; c < m; ++c)
          for (int j = 0; j < ny; ++j) Wt[(size_t)c * npt + (size_t)j * nx + i] = wt[c * ny + j];
      }
    }
  }
  for (size_t q = 0; q < m * npt; ++q) { L1[q] = A1[q]; L2[q] = A2[q]; L3[q] = A3[q]; }
}

// ---------------------------------------------------------------------------
// Time step (reading R5) and SSP-RK3 with the limited derivative (Sec. 2.2,
// the fully discrete scheme).
// ---------------------------------------------------------------------------
double time_step(const or_problem& P, double ax, double ay, double t, double t_end,
                 bool* lands) {
  const double dx = (P.x1 - P.x0) / P.nx;
  const double dy = P.dim == 2 ? (P.y1 - P.y0) / P.ny : 1.0;
  double dt;
  if (P.dt_mode == 2) {
    dt = P.dt_fixed;
  } else {
    const double hx = P.dt_mode == 1 ? std::pow(dx, 5.0 / 3.0) : dx;
    const double hy = P.dt_mode == 1 ? std::pow(dy, 5.0 / 3.0) : dy;
    const double rate = P.dim == 1 ? ax / hx : ax / hx + ay / hy;
    dt = rate > 0.0 ? P.cfl / rate : std::numeric_limits<double>::infinity();
  }
  const double rest = t_end - t;
  *lands = dt >= rest;
  return *lands ? rest : dt;
}

template <class R>
void step_generic(const or_problem& P, R* U, R* V, R* W, double* t, double t_end,
                  double* dt_out) {
  const int m = ncomp(P);
  const size_t n = (size_t)m * P.nx * (P.dim == 2 ? P.ny : 1);
  const bool two = P.dim == 2;
  if (*t >= t_end) { if (dt_out) *dt_out = 0.0; return; }

  auto rhs = [&](const R* u, const R* v, const R* w, double ts, R* l1, R* l2, R* l3,
                 R* vt, R* wt, R* al) {
    if (two) rhs_2d(P, u, v, w, ts, l1, l2, l3, vt, wt, al);
    else rhs_1d(P, u, v, ts, l1, l2, vt, al);
  };
  // dt from alpha of u^n
  R al[2] = {R(0.0), R(0.0)};
  {
    const size_t npt = (size_t)P.nx * (two ? P.ny : 1);
    for (size_t q = 0; q < npt; ++q) {
      R Uq[4];
      for (int c = 0; c < m; ++c) Uq[c] = U[c * npt + q];
      al[0] = rmax(al[0], wave_speed(P, 0, Uq));
      if (two) al[1] = rmax(al[1], wave_speed(P, 1, Uq));
    }
  }
  bool lands = false;
  const double dt = time_step(P, val(al[0]), val(al[1]), *t, t_end, &lands);

  std::vector<R> L1(n), L2(n), L3(two ? n : 0), Vt0(n), Wt0(two ? n : 0);
  std::vector<R> U1(n), V1(n), W1(two ? n : 0), U2(n), V2(n), W2(two ? n : 0);
  std::vector<R> Vtk(n), Wtk(two ? n : 0);
  R dum[2];
  // stage 1
  rhs(U, V, W, *t, L1.data(), L2.data(), L3.data(), Vt0.data(), Wt0.data(), dum);
  for (size_t q = 0; q < n; ++q) {
    U1[q] = U[q] + dt * L1[q];
    V1[q] = Vt0[q] + dt * L2[q];
    if (two) W1[q] = Wt0[q] + dt * L3[q];
  }
  // stage 2
  rhs(U1.data(), V1.data(), W1.data(), *t + dt, L1.data(), L2.data(), L3.data(),
      Vtk.data(), Wtk.data(), dum);
  for (size_t q = 0; q < n; ++q) {
    U2[q] = 0.75 * U[q] + 0.25 * (U1[q] + dt * L1[q]);
    V2[q] = 0.75 * Vt0[q] + 0.25 * (Vtk[q] + dt * L2[q]);
    if (two) W2[q] = 0.75 * Wt0[q] + 0.25 * (Wtk[q] + dt * L3[q]);
  }
  // stage 3
  rhs(U2.data(), V2.data(), W2.data(), *t + 0.5 * dt, L1.data(), L2.data(), L3.data(),
      Vtk.data(), Wtk.data(), dum);
  for (size_t q = 0; q < n; ++q) {
    U[q] = (1.0 / 3.0) * U[q] + (2.0 / 3.0) * (U2[q] + dt * L1[q]);
    V[q] = (1.0 / 3.0) * Vt0[q] + (2.0 / 3.0) * (Vtk[q] + dt * L2[q]);
    if (two) W[q] = (1.0 / 3.0) * Wt0[q] + (2.0 / 3.0) * (Wtk[q] + dt * L3[q]);
  }
  *t = lands ? t_end : *t + dt;
  if (dt_out) *dt_out = dt;
}

}  // namespace

// ---------------------------------------------------------------------------
// C entry points (ctypes). All arrays are host FP64, [m][ny][nx] per field.
// ---------------------------------------------------------------------------
extern "C" {

int or_ncomp(const or_problem* P) { return ncomp(*P); }

// out: fhat, hhat, p0, p1, p2, dp0, beta0..2, tau, omega0..2 (13 values)
void or_hweno_face(int side, const double* f, const double* h, double dx,
                   const double* g, double eps, double* out) {
  const Face<double> o = side == 0 ? hweno_plus(f, h, dx, g, eps) : hweno_minus(f, h, dx, g, eps);
  const double v[13] = {o.fhat, o.hhat, o.p[0], o.p[1], o.p[2], o.dp0, o.beta[0],
                        o.beta[1], o.beta[2], o.tau, o.omega[0], o.omega[1], o.omega[2]};
  std::memcpy(out, v, sizeof v);
}

// Tangent of one face (Dual): out = (d fhat, d hhat) along (df, dh), with
// the nonlinear weights frozen or not.
void or_hweno_face_tangent(int side, const double* f, const double* h, const double* df,
                           const double* dh, double dx, const double* g, double eps, int frozen,
                           double* out) {
  Dual fd[3], hd[3];
  for (int k = 0; k < 3; ++k) { fd[k] = Dual(f[k], df[k]); hd[k] = Dual(h[k], dh[k]); }
  const Face<Dual> o = side == 0 ? hweno_plus(fd, hd, dx, g, eps, frozen != 0)
                                 : hweno_minus(fd, hd, dx, g, eps, frozen != 0);
  out[0] = o.fhat.d;
  out[1] = o.hhat.d;
}

// Tangent of the limiter (Dual): d vt along (dum, du0, dup, dvm, dvp).
double or_limiter_tangent(double um, double u0, double up, double vm, double vp,
                          const double* dir, double dx, const double* d, double eps,
                          int frozen) {
  const Lim<Dual> o = hweno_limiter(Dual(um, dir[0]), Dual(u0, dir[1]), Dual(up, dir[2]),
                                    Dual(vm, dir[3]), Dual(vp, dir[4]), dx, d, eps, frozen != 0);
  return o.vt.d;
}

// out: vt, dq0..2, beta0..2, tau, lambda0..2 (11 values)
void or_limiter(double um, double u0, double up, double vm, double vp, double dx,
                const double* d, double eps, double* out) {
  const Lim<double> o = hweno_limiter(um, u0, up, vm, vp, dx, d, eps);
  const double v[11] = {o.vt, o.dq[0], o.dq[1], o.dq[2], o.beta[0], o.beta[1],
                        o.beta[2], o.tau, o.lambda[0], o.lambda[1], o.lambda[2]};
  std::memcpy(out, v, sizeof v);
}

void or_flux(const or_problem* P, int dir, const double* U, double* F) { flux(*P, dir, U, F); }
double or_bl_alpha01() { return bl_alpha01(); }
void or_jvp(const or_problem* P, int dir, const double* U, const double* D, double* out) {
  jvp(*P, dir, U, D, out);
}
double or_wave_speed(const or_problem* P, int dir, const double* U) {
  return wave_speed(*P, dir, U);
}
// Eigenvectors at the average of UL, UR (UR null: at UL). Rm, Lm: m x m.
void or_eigen(const or_problem* P, int dir, const double* UL, const double* UR,
              double* Rm, double* Lm, double* lam) {
  double u, v, H, c;
  eigen_state(*P, UL, UR, P->eig_avg, u, v, H, c);
  eigenvectors(*P, dir, u, v, H, c, Rm, Lm, lam);
}

void or_rhs_1d(const or_problem* P, const double* U, const double* V, double t, double* L1,
               double* L2, double* Vt, double* alpha) {
  rhs_1d(*P, U, V, t, L1, L2, Vt, alpha);
}
void or_rhs_2d(const or_problem* P, const double* U, const double* V, const double* W,
               double t, double* L1, double* L2, double* L3, double* Vt, double* Wt,
               double* alpha) {
  rhs_2d(*P, U, V, W, t, L1, L2, L3, Vt, Wt, alpha);
}

void or_step(const or_problem* P, double* U, double* V, double* W, double* t, double t_end,
             double* dt) {
  step_generic(*P, U, V, W, t, t_end, dt);
}

// Steps until t reaches t_end or max_steps steps were taken; returns steps.
long or_run(const or_problem* P, double* U, double* V, double* W, double* t, double t_end,
            long max_steps) {
  long k = 0;
  while (*t < t_end && k < max_steps) {
    double dt;
    step_generic(*P, U, V, W, t, t_end, &dt);
    ++k;
  }
  return k;
}

// Forward-mode derivative of a run: advances (U, V, W) and their tangents
// (dU, dV, dW) until t_end or max_steps, with alpha frozen in every stage and
// the time steps those of the run itself. Returns the steps taken.
long or_run_tangent(const or_problem* P, double* U, double* V, double* W, double* dU,
                    double* dV, double* dW, double* t, double t_end, long max_steps) {
  const int m = ncomp(*P);
  const size_t n = (size_t)m * P->nx * (P->dim == 2 ? P->ny : 1);
  const bool two = P->dim == 2;
  std::vector<Dual> u(n), v(n), w(two ? n : 0);
  for (size_t q = 0; q < n; ++q) {
    u[q] = Dual(U[q], dU[q]);
    v[q] = Dual(V[q], dV[q]);
    if (two) w[q] = Dual(W[q], dW[q]);
  }
  long k = 0;
  while (*t < t_end && k < max_steps) {
    double dt;
    step_generic(*P, u.data(), v.data(), w.data(), t, t_end, &dt);
    ++k;
  }
  for (size_t q = 0; q < n; ++q) {
    U[q] = u[q].v; dU[q] = u[q].d;
    V[q] = v[q].v; dV[q] = v[q].d;
    if (two) { W[q] = w[q].v; dW[q] = w[q].d; }
  }
  return k;
}

// Algorithmic operations of one SSP-RK3 step per grid point, counted by the
// Flop scalar on the given problem and state (one step, all three stages,
// the time-step reduction and the stage combinations).
double or_flops_per_point_step(const or_problem* P, const double* U, const double* V,
                               const double* W) {
  const int m = ncomp(*P);
  const size_t npt = (size_t)P->nx * (P->dim == 2 ? P->ny : 1);
  const size_t n = (size_t)m * npt;
  std::vector<Flop> u(n), v(n), w(P->dim == 2 ? n : 0);
  for (size_t q = 0; q < n; ++q) { u[q] = U[q]; v[q] = V[q]; if (P->dim == 2) w[q] = W[q]; }
  double t = 0.0;
  g_flops = 0;
  step_generic(*P, u.data(), v.data(), w.data(), &t, 1e300, (double*)nullptr);
  return (double)g_flops / (double)npt;
}

// Operations of one forward-mode (dual-number) step per grid point: the
// values and the tangents together, with the wave speeds frozen as in
// or_run_tangent (tangent seeds dU, dV, dW).
double or_tangent_flops_per_point_step(const or_problem* P, const double* U, const double* V,
                                       const double* W, const double* dU, const double* dV,
                                       const double* dW) {
  const int m = ncomp(*P);
  const size_t npt = (size_t)P->nx * (P->dim == 2 ? P->ny : 1);
  const size_t n = (size_t)m * npt;
  const bool two = P->dim == 2;
  std::vector<DualFlop> u(n), v(n), w(two ? n : 0);
  for (size_t q = 0; q < n; ++q) {
    u[q] = DualFlop(Flop(U[q]), Flop(dU[q]));
    v[q] = DualFlop(Flop(V[q]), Flop(dV[q]));
    if (two) w[q] = DualFlop(Flop(W[q]), Flop(dW[q]));
  }
  double t = 0.0;
  g_flops = 0;
  step_generic(*P, u.data(), v.data(), w.data(), &t, 1e300, (double*)nullptr);
  return (double)g_flops / (double)npt;
}

}  // extern "C"
