// Fused 2D L-HWENO stage (Zhang & Zhao, arXiv:2207.05258, Eq. ode2H with the
// mixed-derivative fluxes of Eq. mixed and the dimension-by-dimension
// limiter): one CTA per block of kColsY2D x kRowsY2D points does both
// directions of one SSP-RK3 stage.
//
//  x part  the block's rows with two x-ghost columns on each side: point
//          fluxes f, h = A_x V, eta = A_x W and the split f^{+-}, dx h^{+-};
//          the characteristic HWENO f-hat, the linear h-hat and the central
//          eta-hat at the block's x-interfaces; per point the x parts of
//          L^1, L^2, L^3 and the x-limited v~, kept in shared memory;
//  y part  as the y-sweep of the split form (stage2d.cu), its epilogue
//          taking the x parts from shared memory instead of global scratch.
//
// Against the split form (an x-sweep and a y-sweep launch per stage) it
// halves the launches of a step and removes the x parts' round trip through
// global memory, at the price of the x-interfaces on the block edges, which
// both neighbouring blocks compute (17 interfaces per 16 points of a row).
// Results agree with the split form to rounding.
#include <cfloat>

#include <cuda_pipeline.h>

#include "hweno.h"
#include "flux2d.cuh"
#include "hweno_math.cuh"
#include "internal.h"
#include "stage2d_common.cuh"

namespace hweno {
namespace {

constexpr int kC = kColsY2D, kR = kRowsY2D;  // block: kC columns x kR rows
constexpr int kXL = kC + 4;                  // x part: loaded points per row
constexpr int kXF = kC + 1;                  // x part: interfaces per row

template <int EQ, class Real>
struct FLayout {
  static constexpr int M = Dim2<EQ>::M;
  static constexpr bool EUL = EQ == HWENO_EULER;
  static constexpr int NE = EUL ? 5 : 0;        // sqrt(rho), u, v, H, c^2
  static constexpr int XP = kR * kXL;           // x part: loaded points
  static constexpr int XF = kR * kXF;           // x part: interfaces
  static constexpr int YP = (kR + 4) * kC;      // y part: loaded points
  static constexpr int YF = (kR + 1) * kC;      // y part: interfaces
  static constexpr int PE = kR * kC;            // points of the block
  // FP32 stages 2-3: U^n, v~^n, w~^n of the block's points, prefetched
  static constexpr int NPRE = std::is_same<Real, float>::value ? 3 * M : 0;
  static constexpr size_t xwords = (size_t)(7 * M + NE) * XP + (size_t)3 * M * XF;
  static constexpr size_t ywords = (size_t)(7 * M + NE) * YP + (size_t)3 * M * YF +
                                   (size_t)NPRE * PE;
  static constexpr size_t awords = xwords > ywords ? xwords : ywords;  // phases share it
  static constexpr size_t bytes = sizeof(Real) * (awords + (size_t)4 * M * PE) + 64;
};

template <int EQ, class Real, int MODE>
__global__ void __launch_bounds__(kThreads2D, (MinBlocks<Real, HWENO_MINB_Y_F64, HWENO_MINB_Y_F32>::value))
k_stage_2d(const __grid_constant__ Args2D a) {
  using Lay = FLayout<EQ, Real>;
  constexpr int M = Lay::M;
  constexpr bool EUL = Lay::EUL;
  constexpr int C = kC, P = Lay::YP;
  static_assert(Lay::XF <= kThreads2D && Lay::YF <= kThreads2D && Lay::PE <= kThreads2D,
                "one interface or point per thread in each phase");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  unsigned* const st = a.status;
  // B: the x parts of L^1, L^2, L^3 and v~ of the block's points (both phases)
  const auto sXpart = tile_view<Lay::PE>(sm + Lay::awords, 4 * M, st);
  __shared__ Real red[kThreads2D / 32];
  __shared__ double s_dt, s_ts;

  if (a.skip_done && !(a.t[0] < a.t_end)) return;
  const int nx = a.nx, ny = a.ny;
  const long long N = (long long)nx * ny;
  const int i0 = blockIdx.x * C, j0 = blockIdx.y * kR;
  const int ncol = min(C, nx - i0), nrow = min(kR, ny - j0);
  HWENO_CHECK(ncol >= 1 && nrow >= 1, st);
  const Real* geo = pick<Real>(a.geod, a.geof);
  const Real dx = geo[0], idx = geo[1], idx2 = geo[2];
  const Real dy = geo[3], idy = geo[4], idy2 = geo[5];
  const Real gam = pick<Real>(a.sp.wd, a.sp.wf)[9], gm1 = gam - Real(1);
  const Weights<Real> w = weights_from(pick<Real>(a.sp.wd, a.sp.wf));
  const Real* U = static_cast<const Real*>(a.U);
  const Real* V = static_cast<const Real*>(a.V);
  const Real* W = static_cast<const Real*>(a.W);
  // time step and boundary time of the stage, once per CTA
  if (threadIdx.x == 0) {
    double dt = 0.0;
    if constexpr (MODE == MODE_STAGE1) {
      int lands;
      dt = time_step2(a, lands);
      if (blockIdx.x == 0 && blockIdx.y == 0) {
        a.dt[0] = dt;
        a.lands[0] = lands;
      }
    } else {
      dt = a.dt[0];
    }
    s_dt = dt;
    s_ts = __dadd_rn(a.t[0], __dmul_rn(a.stage_c, dt));
  }

  // ---------------- x part ----------------
  {
    const auto sU = tile_view<Lay::XP>(sm, M, st);
    const auto sV = tile_view<Lay::XP>(sm + 1 * M * Lay::XP, M, st);
    const auto sFp = tile_view<Lay::XP>(sm + 2 * M * Lay::XP, M, st);
    const auto sFm = tile_view<Lay::XP>(sm + 3 * M * Lay::XP, M, st);
    const auto sHp = tile_view<Lay::XP>(sm + 4 * M * Lay::XP, M, st);
    const auto sHm = tile_view<Lay::XP>(sm + 5 * M * Lay::XP, M, st);
    const auto sEta = tile_view<Lay::XP>(sm + 6 * M * Lay::XP, M, st);
    const auto sE = tile_view<Lay::XP>(sm + 7 * M * Lay::XP, Lay::NE, st);
    Real* const xi = sm + (size_t)(7 * M + Lay::NE) * Lay::XP;
    const auto sF = tile_view<Lay::XF>(xi, M, st);
    const auto sD = tile_view<Lay::XF>(xi + 1 * M * Lay::XF, M, st);
    const auto sN = tile_view<Lay::XF>(xi + 2 * M * Lay::XF, M, st);
    const Real alpha = Real(a.alpha_in[0]);
    const Real hdx = Real(0.5) * dx;
    const Real ha = Real(0.5) * alpha, hda = hdx * alpha;
    // loaded points: row r, column g (point i0 - 2 + g)
    for (int k = threadIdx.x; k < Lay::XP; k += blockDim.x) {
      const int r = k / kXL, g = k % kXL;
      if (r >= nrow || g >= ncol + 4) continue;
      const int j = j0 + r;
      const Src s = map_x(i0 - 2 + g, nx, a.sp);
      HWENO_CHECK(s.kind == 2 || (s.idx >= 0 && s.idx < nx), st);
      Real u[M], v[M], ww[M];
#pragma unroll
      for (int c = 0; c < M; ++c) {
        if (s.kind == 2) {
          u[c] = Real(imposed(a.sp, s, c)); v[c] = Real(0); ww[c] = Real(0);
        } else {
          const long long q = c * N + (long long)j * nx + s.idx;
          u[c] = U[q]; v[c] = V[q]; ww[c] = W[q];
          if (s.kind == 1) {
            const Real sg = Real(refl2<EQ, 0>(c));
            u[c] *= sg; v[c] *= -sg; ww[c] *= sg;
          }
        }
        sU[c][k] = u[c];
        sV[c][k] = v[c];
      }
      Prim2<Real> pq{};
      Real rr = Real(0);  // 1/sqrt(rho)
      if constexpr (EUL) pq = prim2_rr(u, gm1, rr);
      Real F[M], H[M], E[M];
      flux2<EQ, 0>(u, pq, F);
      jvp2<EQ, 0>(u, pq, v, gm1, H);
      jvp2<EQ, 0>(u, pq, ww, gm1, E);
#pragma unroll
      for (int c = 0; c < M; ++c) {
        split_pm(F[c], u[c], H[c], v[c], ha, hda, hdx, sFp[c][k], sFm[c][k], sHp[c][k],
                 sHm[c][k]);
        sEta[c][k] = E[c];
      }
      if constexpr (EUL) {
        sE[0][k] = u[0] * rr;
        sE[1][k] = pq.u;
        sE[2][k] = pq.v;
        sE[3][k] = pq.Ep * pq.ir;
        sE[4][k] = gam * pq.p * pq.ir;
      }
    }
    __syncthreads();

    // x-interfaces x_{i0+jf-1/2} of row r; the left point is loaded column jf + 1
    for (int k = threadIdx.x; k < Lay::XF; k += blockDim.x) {
      const int r = k / kXF, jf = k % kXF;
      if (r >= nrow || jf > ncol) continue;
      const int b = r * kXL + jf + 1;  // loaded index of the left point
      if constexpr (!EUL) {
        sF[0][k] = interface_flux<Real, true>(sFp[0][b - 1], sFp[0][b], sFp[0][b + 1],
                                              sHp[0][b - 1], sHp[0][b], sHp[0][b + 1],
                                              sFm[0][b], sFm[0][b + 1], sFm[0][b + 2],
                                              sHm[0][b], sHm[0][b + 1], sHm[0][b + 2], w);
      } else {
        Real uu, vv, HH;
        if (a.sp.eig_avg == 0) {
          const Real sl = sE[0][b], sr = sE[0][b + 1];
          const Real is = recip(sl + sr);
          uu = (sl * sE[1][b] + sr * sE[1][b + 1]) * is;
          vv = (sl * sE[2][b] + sr * sE[2][b + 1]) * is;
          HH = (sl * sE[3][b] + sr * sE[3][b + 1]) * is;
        } else {
          Real Um[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) Um[c] = Real(0.5) * (sU[c][b] + sU[c][b + 1]);
          const Prim2<Real> pm = prim2(Um, gm1);
          uu = pm.u; vv = pm.v; HH = pm.Ep * pm.ir;
        }
        Char2<Real, 0> e;
        e.init(uu, vv, HH, gm1 * (HH - Real(0.5) * (uu * uu + vv * vv)), gm1);
        Frac<Real> fr[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          auto pj = [&](const auto& A, int g) { return e.left(q, A[0][g], A[1][g], A[2][g], A[3][g]); };
          fr[q] = interface_flux_frac<Real, true>(pj(sFp, b - 1), pj(sFp, b), pj(sFp, b + 1),
                                                  pj(sHp, b - 1), pj(sHp, b), pj(sHp, b + 1),
                                                  pj(sFm, b), pj(sFm, b + 1), pj(sFm, b + 2),
                                                  pj(sHm, b), pj(sHm, b + 1), pj(sHm, b + 2), w);
        }
        Real fch[4], out[4];
        resolve4(fr, fch);
        e.right(fch, out);
#pragma unroll
        for (int c = 0; c < 4; ++c) sF[c][k] = out[c];
      }
#pragma unroll
      for (int c = 0; c < M; ++c) {
        sD[c][k] = derivative_flux(sFp[c][b - 1], sFp[c][b], sFp[c][b + 1], sHp[c][b - 1],
                                   sHp[c][b], sHp[c][b + 1], sFm[c][b], sFm[c][b + 1],
                                   sFm[c][b + 2], sHm[c][b], sHm[c][b + 1], sHm[c][b + 2]);
        sN[c][k] = Real(7.0 / 12.0) * (sEta[c][b] + sEta[c][b + 1]) -
                   Real(1.0 / 12.0) * (sEta[c][b - 1] + sEta[c][b + 2]);
      }
    }
    __syncthreads();

    // points: x parts of L and the x-limited v~
    for (int k = threadIdx.x; k < Lay::PE; k += blockDim.x) {
      const int r = k / C, col = k % C;
      if (r >= nrow || col >= ncol) continue;
      const int g = r * kXL + col + 2;  // loaded index
      const int f = r * kXF + col;      // left interface
      Real vt[M];
      if (a.sp.limiter == 0) {
#pragma unroll
        for (int c = 0; c < M; ++c) vt[c] = sV[c][g];
      } else if (!EUL || a.sp.limiter == 2) {
#pragma unroll
        for (int c = 0; c < M; ++c)
          vt[c] = limited_derivative(sU[c][g - 1], sU[c][g], sU[c][g + 1], dx * sV[c][g - 1],
                                     dx * sV[c][g + 1], w) * idx;
      } else if constexpr (EUL) {
        Char2<Real, 0> e;
        e.init(sE[1][g], sE[2][g], sE[3][g], sE[4][g], gm1);
        Real z[4];
        auto pj = [&](int q, const auto& A, int gg) {
          return e.left(q, A[0][gg], A[1][gg], A[2][gg], A[3][gg]);
        };
        if constexpr (std::is_same<Real, float>::value) {  // two fields per packed pair
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int q0 = 2 * h, q1 = 2 * h + 1;
            auto p2 = [&](const auto& A, int gg) { return make_float2(pj(q0, A, gg), pj(q1, A, gg)); };
            const float2 o = limited_derivative_pair(p2(sU, g - 1), p2(sU, g), p2(sU, g + 1),
                                                     mul2(pair(dx), p2(sV, g - 1)),
                                                     mul2(pair(dx), p2(sV, g + 1)), w);
            z[q0] = o.x;
            z[q1] = o.y;
          }
        } else {
          Frac<Real> zr[4];
#pragma unroll
          for (int q = 0; q < 4; ++q)
            zr[q] = limited_derivative_frac(pj(q, sU, g - 1), pj(q, sU, g), pj(q, sU, g + 1),
                                            dx * pj(q, sV, g - 1), dx * pj(q, sV, g + 1), w);
          resolve4(zr, z);
        }
        e.right(z, vt);
#pragma unroll
        for (int c = 0; c < 4; ++c) vt[c] *= idx;
      }
#pragma unroll
      for (int c = 0; c < M; ++c) {
        sXpart[c][k] = -(sF[c][f + 1] - sF[c][f]) * idx;
        sXpart[M + c][k] = -(sD[c][f + 1] - sD[c][f]) * idx2;
        sXpart[2 * M + c][k] = -(sN[c][f + 1] - sN[c][f]) * idx;
        sXpart[3 * M + c][k] = vt[c];
      }
    }
    __syncthreads();  // the y part reuses the x part's shared memory
  }

  // ---------------- y part ----------------
  const auto sPts = tile_view<P>(sm, 7 * M, st);
  auto PT = [&](int qty, int c) { return sPts[qty * M + c]; };
  const auto sEig = tile_view<P>(sm + (size_t)7 * M * P, Lay::NE, st);
  Real* const sI = sm + (size_t)(7 * M + Lay::NE) * P;
  const auto sIf = tile_view<Lay::YF>(sI, 3 * M, st);
  auto IF = [&](int kind, int c) { return sIf[kind * M + c]; };
  const auto sPre = tile_view<Lay::PE>(sI + (size_t)3 * M * Lay::YF, Lay::NPRE, st);
  const double ts = s_ts;
  {
    const Real alpha = Real(a.alpha_in[1]);
    const Real hdy = Real(0.5) * dy;
    const Real ha = Real(0.5) * alpha, hda = hdy * alpha;
    // FP32: all of the tile's loads as asynchronous copies first (U and W in
    // quantities 0 and 1, V in quantity 6, which the same thread overwrites
    // with xi), then the prefetch of the stage's U^n, v~^n, w~^n
    constexpr int ITER = (P + kThreads2D - 1) / kThreads2D;
    Src src[ITER];
    if constexpr (Lay::NPRE > 0) {
#pragma unroll
      for (int it = 0; it < ITER; ++it) {
        const int k = threadIdx.x + it * kThreads2D;
        const int r = k / C, col = k % C;
        if (k >= P || col >= ncol || r >= nrow + 4) continue;
        const int i = i0 + col;
        src[it] = map_y(j0 - 2 + r, ny, i, a.x0, a.dx, a.y0, a.dy, ts, a.sp);
        HWENO_CHECK(src[it].kind == 2 || (src[it].idx >= 0 && src[it].idx < ny), st);
        if (src[it].kind != 2) {
#pragma unroll
          for (int c = 0; c < M; ++c) {
            const long long q = c * N + (long long)src[it].idx * nx + i;
            __pipeline_memcpy_async(&PT(0, c)[k], U + q, sizeof(Real));
            __pipeline_memcpy_async(&PT(1, c)[k], W + q, sizeof(Real));
            __pipeline_memcpy_async(&PT(6, c)[k], V + q, sizeof(Real));
          }
        }
      }
      __pipeline_commit();
      if constexpr (MODE == MODE_STAGE2 || MODE == MODE_STAGE3) {
        const int k = threadIdx.x, r = k / C, col = k % C;
        if (k < Lay::PE && col < ncol && r < nrow) {
          const long long q = (long long)(j0 + r) * nx + i0 + col;
#pragma unroll
          for (int c = 0; c < M; ++c) {
            __pipeline_memcpy_async(&sPre[c][k], static_cast<const Real*>(a.U0) + c * N + q,
                                    sizeof(Real));
            __pipeline_memcpy_async(&sPre[M + c][k], static_cast<const Real*>(a.Vt0) + c * N + q,
                                    sizeof(Real));
            __pipeline_memcpy_async(&sPre[2 * M + c][k],
                                    static_cast<const Real*>(a.Wt0) + c * N + q, sizeof(Real));
          }
        }
      }
      __pipeline_commit();
      __pipeline_wait_prior(1);  // this thread's tile copies
    }
#pragma unroll
    for (int it = 0; it < ITER; ++it) {
      const int k = threadIdx.x + it * kThreads2D;
      const int r = k / C, col = k % C;
      if (k >= P || col >= ncol || r >= nrow + 4) continue;
      const int i = i0 + col;
      Src s;
      if constexpr (Lay::NPRE > 0) {
        s = src[it];
      } else {
        s = map_y(j0 - 2 + r, ny, i, a.x0, a.dx, a.y0, a.dy, ts, a.sp);
        HWENO_CHECK(s.kind == 2 || (s.idx >= 0 && s.idx < ny), st);
      }
      Real u[M], v[M], ww[M];
#pragma unroll
      for (int c = 0; c < M; ++c) {
        if (s.kind == 2) {
          u[c] = Real(imposed(a.sp, s, c)); v[c] = Real(0); ww[c] = Real(0);
        } else {
          if constexpr (Lay::NPRE > 0) {
            u[c] = PT(0, c)[k]; v[c] = PT(6, c)[k]; ww[c] = PT(1, c)[k];
          } else {
            const long long q = c * N + (long long)s.idx * nx + i;
            u[c] = U[q]; v[c] = V[q]; ww[c] = W[q];
          }
          if (s.kind == 1) {
            const Real sg = Real(refl2<EQ, 1>(c));
            u[c] *= sg; ww[c] *= -sg; v[c] *= sg;
          }
        }
        PT(0, c)[k] = u[c];
        PT(1, c)[k] = ww[c];
      }
      Prim2<Real> pq{};
      Real rr = Real(0);  // 1/sqrt(rho)
      if constexpr (EUL) pq = prim2_rr(u, gm1, rr);
      Real G[M], T[M], X[M];
      flux2<EQ, 1>(u, pq, G);
      jvp2<EQ, 1>(u, pq, ww, gm1, T);
      jvp2<EQ, 1>(u, pq, v, gm1, X);
#pragma unroll
      for (int c = 0; c < M; ++c) {
        split_pm(G[c], u[c], T[c], ww[c], ha, hda, hdy, PT(2, c)[k], PT(3, c)[k], PT(4, c)[k],
                 PT(5, c)[k]);
        PT(6, c)[k] = X[c];
      }
      if constexpr (EUL) {
        sEig[0][k] = u[0] * rr;
        sEig[1][k] = pq.u;
        sEig[2][k] = pq.v;
        sEig[3][k] = pq.Ep * pq.ir;
        sEig[4][k] = gam * pq.p * pq.ir;
      }
    }
  }
  __syncthreads();

  // y-interfaces y_{j0+r-1/2}, r = 0..nrow; lower point at loaded row r + 1
  for (int k = threadIdx.x; k < Lay::YF; k += blockDim.x) {
    const int r = k / C, col = k % C;
    if (col >= ncol || r > nrow) continue;
    const int gl = r + 1;
    auto at = [&](const auto& A, int rr) { return A[rr * C + col]; };
    if constexpr (!EUL) {
      IF(0, 0)[k] = interface_flux<Real, true>(at(PT(2, 0), gl - 1), at(PT(2, 0), gl),
                                               at(PT(2, 0), gl + 1), at(PT(4, 0), gl - 1),
                                               at(PT(4, 0), gl), at(PT(4, 0), gl + 1),
                                               at(PT(3, 0), gl), at(PT(3, 0), gl + 1),
                                               at(PT(3, 0), gl + 2), at(PT(5, 0), gl),
                                               at(PT(5, 0), gl + 1), at(PT(5, 0), gl + 2), w);
    } else {
      Real uu, vv, HH;
      const int kl = gl * C + col, kr = (gl + 1) * C + col;
      if (a.sp.eig_avg == 0) {
        const Real sl = sEig[0][kl], sr = sEig[0][kr];
        const Real is = recip(sl + sr);
        uu = (sl * sEig[1][kl] + sr * sEig[1][kr]) * is;
        vv = (sl * sEig[2][kl] + sr * sEig[2][kr]) * is;
        HH = (sl * sEig[3][kl] + sr * sEig[3][kr]) * is;
      } else {
        Real Um[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) Um[c] = Real(0.5) * (PT(0, c)[kl] + PT(0, c)[kr]);
        const Prim2<Real> pm = prim2(Um, gm1);
        uu = pm.u; vv = pm.v; HH = pm.Ep * pm.ir;
      }
      Char2<Real, 1> e;
      e.init(uu, vv, HH, gm1 * (HH - Real(0.5) * (uu * uu + vv * vv)), gm1);
      Frac<Real> fr[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        auto pj = [&](int qty, int g) {
          const int kk = g * C + col;
          return e.left(q, PT(qty, 0)[kk], PT(qty, 1)[kk], PT(qty, 2)[kk], PT(qty, 3)[kk]);
        };
        fr[q] = interface_flux_frac<Real, true>(pj(2, gl - 1), pj(2, gl), pj(2, gl + 1),
                                                pj(4, gl - 1), pj(4, gl), pj(4, gl + 1),
                                                pj(3, gl), pj(3, gl + 1), pj(3, gl + 2),
                                                pj(5, gl), pj(5, gl + 1), pj(5, gl + 2), w);
      }
      Real fch[4], out[4];
      resolve4(fr, fch);
      e.right(fch, out);
#pragma unroll
      for (int c = 0; c < 4; ++c) IF(0, c)[k] = out[c];
    }
#pragma unroll
    for (int c = 0; c < M; ++c) {
      IF(1, c)[k] = derivative_flux(at(PT(2, c), gl - 1), at(PT(2, c), gl), at(PT(2, c), gl + 1),
                                    at(PT(4, c), gl - 1), at(PT(4, c), gl), at(PT(4, c), gl + 1),
                                    at(PT(3, c), gl), at(PT(3, c), gl + 1), at(PT(3, c), gl + 2),
                                    at(PT(5, c), gl), at(PT(5, c), gl + 1), at(PT(5, c), gl + 2));
      IF(2, c)[k] = Real(7.0 / 12.0) * (at(PT(6, c), gl) + at(PT(6, c), gl + 1)) -
                    Real(1.0 / 12.0) * (at(PT(6, c), gl - 1) + at(PT(6, c), gl + 2));
    }
  }
  __syncthreads();

  // points: the y parts, the y-limited w~, the SSP-RK3 combination and the
  // wave speeds of the new state
  const Real rdt = Real(s_dt);
  Real ax = Real(0), ay = Real(0);
  bool bad = false;
  if constexpr (Lay::NPRE > 0) __pipeline_wait_prior(0);  // this thread's prefetch
  for (int k = threadIdx.x; k < Lay::PE; k += blockDim.x) {
    const int r = k / C, col = k % C;
    if (col >= ncol || r >= nrow) continue;
    const int kc = (r + 2) * C + col;
    HWENO_CHECK(j0 + r < ny && i0 + col < nx, st);
    const long long q = (long long)(j0 + r) * nx + i0 + col;
    Real l1[M], l2[M], l3[M], vt[M], wt[M], u[M];
#pragma unroll
    for (int c = 0; c < M; ++c) {
      const int ka = r * C + col, kb = (r + 1) * C + col;
      l1[c] = sXpart[c][k] - (IF(0, c)[kb] - IF(0, c)[ka]) * idy;
      l2[c] = sXpart[M + c][k] - (IF(2, c)[kb] - IF(2, c)[ka]) * idy;
      l3[c] = sXpart[2 * M + c][k] - (IF(1, c)[kb] - IF(1, c)[ka]) * idy2;
      vt[c] = sXpart[3 * M + c][k];
      u[c] = PT(0, c)[kc];
    }
    if (a.sp.limiter == 0) {
#pragma unroll
      for (int c = 0; c < M; ++c) wt[c] = PT(1, c)[kc];
    } else if (!EUL || a.sp.limiter == 2) {
#pragma unroll
      for (int c = 0; c < M; ++c)
        wt[c] = limited_derivative(PT(0, c)[kc - C], u[c], PT(0, c)[kc + C],
                                   dy * PT(1, c)[kc - C], dy * PT(1, c)[kc + C], w) * idy;
    } else if constexpr (EUL) {
      Char2<Real, 1> e;
      e.init(sEig[1][kc], sEig[2][kc], sEig[3][kc], sEig[4][kc], gm1);
      Real z[4];
      auto pj = [&](int q, int qty, int kk) {
        return e.left(q, PT(qty, 0)[kk], PT(qty, 1)[kk], PT(qty, 2)[kk], PT(qty, 3)[kk]);
      };
      if constexpr (std::is_same<Real, float>::value) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int q0 = 2 * h, q1 = 2 * h + 1;
          auto p2 = [&](int qty, int kk) { return make_float2(pj(q0, qty, kk), pj(q1, qty, kk)); };
          const float2 o = limited_derivative_pair(p2(0, kc - C), p2(0, kc), p2(0, kc + C),
                                                   mul2(pair(dy), p2(1, kc - C)),
                                                   mul2(pair(dy), p2(1, kc + C)), w);
          z[q0] = o.x;
          z[q1] = o.y;
        }
      } else {
        Frac<Real> zr[4];
#pragma unroll
        for (int qq = 0; qq < 4; ++qq)
          zr[qq] = limited_derivative_frac(pj(qq, 0, kc - C), pj(qq, 0, kc), pj(qq, 0, kc + C),
                                           dy * pj(qq, 1, kc - C), dy * pj(qq, 1, kc + C), w);
        resolve4(zr, z);
      }
      e.right(z, wt);
#pragma unroll
      for (int c = 0; c < 4; ++c) wt[c] *= idy;
    }
    Real un[M];
#pragma unroll
    for (int c = 0; c < M; ++c) {
      const long long qc = c * N + q;
      Real vn, wn;
      if constexpr (MODE == MODE_STAGE1) {
        un[c] = u[c] + rdt * l1[c];
        vn = vt[c] + rdt * l2[c];
        wn = wt[c] + rdt * l3[c];
        static_cast<Real*>(a.VT)[qc] = vt[c];  // v~^n (stage 1: VT is the stored v~^n)
        static_cast<Real*>(a.Wt0out)[qc] = wt[c];
      } else {
        Real u0, v0, w0;
        if constexpr (Lay::NPRE > 0) {
          u0 = sPre[c][k]; v0 = sPre[M + c][k]; w0 = sPre[2 * M + c][k];
        } else {
          u0 = static_cast<const Real*>(a.U0)[qc];
          v0 = static_cast<const Real*>(a.Vt0)[qc];
          w0 = static_cast<const Real*>(a.Wt0)[qc];
        }
        const Real c0 = MODE == MODE_STAGE2 ? Real(0.75) : Real(1.0 / 3.0);
        const Real c1 = MODE == MODE_STAGE2 ? Real(0.25) : Real(2.0 / 3.0);
        un[c] = c0 * u0 + c1 * (u[c] + rdt * l1[c]);
        vn = c0 * v0 + c1 * (vt[c] + rdt * l2[c]);
        wn = c0 * w0 + c1 * (wt[c] + rdt * l3[c]);
      }
      static_cast<Real*>(a.Uout)[qc] = un[c];
      static_cast<Real*>(a.Vout)[qc] = vn;
      static_cast<Real*>(a.Wout)[qc] = wn;
    }
    if constexpr (MODE == MODE_STAGE1 || MODE == MODE_STAGE2) {
      Real sx, sy;
      speeds2<EQ>(un, gam, sx, sy);
      bad |= !(sx <= real_max<Real>()) || !(sy <= real_max<Real>());
      ax = fmax(ax, sx);
      ay = fmax(ay, sy);
    }
  }
  if constexpr (MODE == MODE_STAGE1 || MODE == MODE_STAGE2) {
    if (bad) atomicOr(a.status, STATUS_NONFINITE);
    ax = block_max_t(ax, red);
    if (threadIdx.x == 0)
      atomicMax(&a.alpha_out[0], (unsigned long long)__double_as_longlong((double)ax));
    ay = block_max_t(ay, red);
    if (threadIdx.x == 0)
      atomicMax(&a.alpha_out[1], (unsigned long long)__double_as_longlong((double)ay));
  }
}

template <int EQ, class Real, int MODE>
cudaError_t fused_launch(const Args2D& a, cudaStream_t s) {
  constexpr size_t bytes = FLayout<EQ, Real>::bytes;
  static unsigned configured = 0;  // devices whose limit is raised
  if (const cudaError_t e = ensure_smem_limit(k_stage_2d<EQ, Real, MODE>, bytes, configured)) return e;
  const dim3 grid((a.nx + kC - 1) / kC, (a.ny + kR - 1) / kR);
  k_stage_2d<EQ, Real, MODE><<<grid, kThreads2D, bytes, s>>>(a);
  return cudaGetLastError();
}

template <int EQ, class Real>
cudaError_t fused_mode(int mode, const Args2D& a, cudaStream_t s) {
  switch (mode) {
    case MODE_STAGE1: return fused_launch<EQ, Real, MODE_STAGE1>(a, s);
    case MODE_STAGE2: return fused_launch<EQ, Real, MODE_STAGE2>(a, s);
    default: return fused_launch<EQ, Real, MODE_STAGE3>(a, s);
  }
}

}  // namespace

cudaError_t launch_stage_fused_2d(int eq, bool fp32, int mode, const Args2D& a, cudaStream_t s) {
  if (mode == MODE_RHS) return cudaErrorInvalidValue;
  if (eq == HWENO_BURGERS)
    return fp32 ? fused_mode<HWENO_BURGERS, float>(mode, a, s)
                : fused_mode<HWENO_BURGERS, double>(mode, a, s);
  return fp32 ? fused_mode<HWENO_EULER, float>(mode, a, s)
              : fused_mode<HWENO_EULER, double>(mode, a, s);
}

}  // namespace hweno
