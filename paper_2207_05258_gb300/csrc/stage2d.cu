// Two-dimensional L-HWENO stage (Zhang & Zhao, arXiv:2207.05258, Eq. ode2H
// with the mixed-derivative fluxes of Eq. mixed and the dimension-by-
// dimension limiter), as two kernels per Runge-Kutta stage:
//
//  x-sweep  one CTA per row segment (kTileX2D points): loads U, V, W with
//           x-ghosts, forms f, h = A_x V, eta = A_x W and the split f^{+-},
//           dx h^{+-}; per x-interface the characteristic HWENO f-hat
//           (eigenvectors of A_x at the Roe average), the linear h-hat and
//           the central eta-hat; per point the x parts of L^1, L^2, L^3 and
//           the x-limited derivative v~. Writes them to scratch.
//  y-sweep  one CTA per kColsY2D x kRowsY2D block: the same in y with
//           g, theta = A_y W, xi = A_y V (ghosts from the y boundary
//           conditions, including the double-Mach wall and the exact shock
//           motion), adds the x parts, forms the y-limited w~, combines the
//           SSP-RK3 stage and reduces the wave speeds of the new state.
//
// The FP64 pipe bounds both kernels; the scratch round trip between them is
// a few percent of the HBM time budget and keeps each tile's shared memory
// small enough for several CTAs per SM.
#include <algorithm>
#include <cfloat>

#include <cuda_pipeline.h>

#include "hweno.h"
#include "flux2d.cuh"
#include "stage2d_common.cuh"
#include "hweno_math.cuh"
#include "internal.h"

namespace hweno {
namespace {

// ---------------------------------------------------------------------------
template <int EQ, class Real>
__global__ void __launch_bounds__(256) k_alpha_2d(const __grid_constant__ Args2D a) {
  constexpr int M = Dim2<EQ>::M;
  __shared__ Real red[8];
  if (a.skip_done && !(a.t[0] < a.t_end)) return;
  const long long N = (long long)a.nx * a.ny;
  const Real* U = static_cast<const Real*>(a.U);
  const Real gam = pick<Real>(a.sp.wd, a.sp.wf)[9];
  Real ax = Real(0), ay = Real(0);
  bool bad = false;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N;
       q += (long long)gridDim.x * blockDim.x) {
    Real u[M];
#pragma unroll
    for (int c = 0; c < M; ++c) u[c] = U[c * N + q];
    Real sx, sy;
    speeds2<EQ>(u, gam, sx, sy);
    bad |= !(sx <= real_max<Real>()) || !(sy <= real_max<Real>());
    ax = fmax(ax, sx);
    ay = fmax(ay, sy);
  }
  if (bad) atomicOr(a.status, STATUS_NONFINITE);
  ax = block_max_t(ax, red);
  if (threadIdx.x == 0)
    atomicMax(&a.alpha_out[0], (unsigned long long)__double_as_longlong((double)ax));
  ay = block_max_t(ay, red);
  if (threadIdx.x == 0)
    atomicMax(&a.alpha_out[1], (unsigned long long)__double_as_longlong((double)ay));
}

// ---------------------------------------------------------------------------
// x-sweep
// ---------------------------------------------------------------------------
template <int EQ, class Real, int MODE>
__global__ void __launch_bounds__(kThreads2D, (MinBlocks<Real, HWENO_MINB_X_F64, HWENO_MINB_X_F32>::value)) k_xsweep_2d(const __grid_constant__ Args2D a) {
  constexpr int M = Dim2<EQ>::M;
  constexpr bool EUL = EQ == HWENO_EULER;
  constexpr int NP = kTileX2D + 4, NF = kTileX2D + 1;
  __shared__ Real sU_[M][NP], sV_[M][NP];
  __shared__ Real sFp_[M][NP], sFm_[M][NP], sHp_[M][NP], sHm_[M][NP], sEta_[M][NP];
  __shared__ Real sE_[EUL ? 5 : 1][EUL ? NP : 1];  // sqrt(rho), u, v, H, c^2
  __shared__ Real sF_[M][NF], sD_[M][NF], sN_[M][NF];
  unsigned* const st = a.status;
  const auto sU = tile_view(sU_, st), sV = tile_view(sV_, st);
  const auto sFp = tile_view(sFp_, st), sFm = tile_view(sFm_, st);
  const auto sHp = tile_view(sHp_, st), sHm = tile_view(sHm_, st);
  const auto sEta = tile_view(sEta_, st);
  const auto sE = tile_view(sE_, st);
  const auto sF = tile_view(sF_, st), sD = tile_view(sD_, st), sN = tile_view(sN_, st);

  if (a.skip_done && !(a.t[0] < a.t_end)) return;
  const int nx = a.nx;
  const long long N = (long long)nx * a.ny;
  // block -> (row segment, row): the full segments of every row first, the
  // ragged last segments (shorter work) at the end of the dispatch order
  int tile = blockIdx.x, j = blockIdx.y;
  {
    const int T = gridDim.x, F = T - 1;
    if (F > 0 && nx % kTileX2D != 0) {
      const long long b = (long long)blockIdx.y * T + blockIdx.x, full = (long long)a.ny * F;
      if (b < full) { tile = (int)(b % F); j = (int)(b / F); }
      else { tile = F; j = (int)(b - full); }
    }
  }
  const int i0 = tile * kTileX2D;
  const int np = min(kTileX2D, nx - i0);
  HWENO_CHECK(np >= 1 && j >= 0 && j < a.ny, st);
  const long long row = (long long)j * nx;
  const Real* geo = pick<Real>(a.geod, a.geof);
  const Real dx = geo[0], idx = geo[1], idx2 = geo[2];
  const Real alpha = Real(a.alpha_in[0]);
  const Real gam = pick<Real>(a.sp.wd, a.sp.wf)[9], gm1 = gam - Real(1);
  const Weights<Real> w = weights_from(pick<Real>(a.sp.wd, a.sp.wf));
  if constexpr (MODE == MODE_STAGE1) {
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
      int lands;
      const double dt = time_step2(a, lands);
      a.dt[0] = dt;
      a.lands[0] = lands;
    }
  }

  {
    const Real* U = static_cast<const Real*>(a.U);
    const Real* V = static_cast<const Real*>(a.V);
    const Real* W = static_cast<const Real*>(a.W);
    const Real hdx = Real(0.5) * dx;
    const Real ha = Real(0.5) * alpha, hda = hdx * alpha;
    for (int g = threadIdx.x; g < np + 4; g += blockDim.x) {
      const Src s = map_x(i0 - 2 + g, nx, a.sp);
      HWENO_CHECK(s.kind == 2 || (s.idx >= 0 && s.idx < nx), st);
      Real u[M], v[M], ww[M];
#pragma unroll
      for (int c = 0; c < M; ++c) {
        if (s.kind == 2) {
          u[c] = Real(imposed(a.sp, s, c)); v[c] = Real(0); ww[c] = Real(0);
        } else {
          const long long q = c * N + row + s.idx;
          u[c] = U[q]; v[c] = V[q]; ww[c] = W[q];
          if (s.kind == 1) {
            const Real sg = Real(refl2<EQ, 0>(c));
            u[c] *= sg; v[c] *= -sg; ww[c] *= sg;
          }
        }
        sU[c][g] = u[c];
        sV[c][g] = v[c];
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
        split_pm(F[c], u[c], H[c], v[c], ha, hda, hdx, sFp[c][g], sFm[c][g], sHp[c][g],
                 sHm[c][g]);
        sEta[c][g] = E[c];
      }
      if constexpr (EUL) {
        sE[0][g] = u[0] * rr;
        sE[1][g] = pq.u;
        sE[2][g] = pq.v;
        sE[3][g] = pq.Ep * pq.ir;
        sE[4][g] = gam * pq.p * pq.ir;
      }
    }
  }
  __syncthreads();

  for (int jf = threadIdx.x; jf <= np; jf += blockDim.x) {
    const int gl = jf + 1;
    if constexpr (!EUL) {
      sF[0][jf] = interface_flux<Real, true>(sFp[0][gl - 1], sFp[0][gl], sFp[0][gl + 1], sHp[0][gl - 1],
                                 sHp[0][gl], sHp[0][gl + 1], sFm[0][gl], sFm[0][gl + 1],
                                 sFm[0][gl + 2], sHm[0][gl], sHm[0][gl + 1], sHm[0][gl + 2], w);
    } else {
      Real uu, vv, HH;
      if (a.sp.eig_avg == 0) {
        const Real sl = sE[0][gl], sr = sE[0][gl + 1];
        const Real is = recip(sl + sr);
        uu = (sl * sE[1][gl] + sr * sE[1][gl + 1]) * is;
        vv = (sl * sE[2][gl] + sr * sE[2][gl + 1]) * is;
        HH = (sl * sE[3][gl] + sr * sE[3][gl + 1]) * is;
      } else {
        Real Um[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) Um[c] = Real(0.5) * (sU[c][gl] + sU[c][gl + 1]);
        const Prim2<Real> pm = prim2(Um, gm1);
        uu = pm.u; vv = pm.v; HH = pm.Ep * pm.ir;
      }
      Char2<Real, 0> e;
      e.init(uu, vv, HH, gm1 * (HH - Real(0.5) * (uu * uu + vv * vv)), gm1);
      Frac<Real> fr[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        auto pj = [&](const auto& A, int g) { return e.left(r, A[0][g], A[1][g], A[2][g], A[3][g]); };
        fr[r] = interface_flux_frac<Real, true>(pj(sFp, gl - 1), pj(sFp, gl), pj(sFp, gl + 1),
                                    pj(sHp, gl - 1), pj(sHp, gl), pj(sHp, gl + 1), pj(sFm, gl),
                                    pj(sFm, gl + 1), pj(sFm, gl + 2), pj(sHm, gl),
                                    pj(sHm, gl + 1), pj(sHm, gl + 2), w);
      }
      Real fch[4];
      resolve4(fr, fch);
      Real out[4];
      e.right(fch, out);
#pragma unroll
      for (int c = 0; c < 4; ++c) sF[c][jf] = out[c];
    }
#pragma unroll
    for (int c = 0; c < M; ++c) {
      sD[c][jf] = derivative_flux(sFp[c][gl - 1], sFp[c][gl], sFp[c][gl + 1], sHp[c][gl - 1],
                                  sHp[c][gl], sHp[c][gl + 1], sFm[c][gl], sFm[c][gl + 1],
                                  sFm[c][gl + 2], sHm[c][gl], sHm[c][gl + 1], sHm[c][gl + 2]);
      // Eq. mixed: -1/12 eta_{i-1} + 7/12 eta_i + 7/12 eta_{i+1} - 1/12 eta_{i+2}
      sN[c][jf] = Real(7.0 / 12.0) * (sEta[c][gl] + sEta[c][gl + 1]) -
                  Real(1.0 / 12.0) * (sEta[c][gl - 1] + sEta[c][gl + 2]);
    }
  }
  __syncthreads();

  Real* LX = static_cast<Real*>(a.LX);
  Real* VT = static_cast<Real*>(a.VT);
  for (int ip = threadIdx.x; ip < np; ip += blockDim.x) {
    const int g = ip + 2;
    HWENO_CHECK(i0 + ip < nx, st);
    const long long q = row + i0 + ip;
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
      auto pj = [&](int r, const auto& A, int gg) {
        return e.left(r, A[0][gg], A[1][gg], A[2][gg], A[3][gg]);
      };
      if constexpr (std::is_same<Real, float>::value) {  // two fields per packed pair
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r0 = 2 * h, r1 = 2 * h + 1;
          auto p2 = [&](const auto& A, int gg) { return make_float2(pj(r0, A, gg), pj(r1, A, gg)); };
          const float2 o = limited_derivative_pair(p2(sU, g - 1), p2(sU, g), p2(sU, g + 1),
                                                   mul2(pair(dx), p2(sV, g - 1)),
                                                   mul2(pair(dx), p2(sV, g + 1)), w);
          z[r0] = o.x;
          z[r1] = o.y;
        }
      } else {
        Frac<Real> zr[4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
          zr[r] = limited_derivative_frac(pj(r, sU, g - 1), pj(r, sU, g), pj(r, sU, g + 1),
                                          dx * pj(r, sV, g - 1), dx * pj(r, sV, g + 1), w);
        resolve4(zr, z);
      }
      e.right(z, vt);
#pragma unroll
      for (int c = 0; c < 4; ++c) vt[c] *= idx;
    }
#pragma unroll
    for (int c = 0; c < M; ++c) {
      LX[c * N + q] = -(sF[c][ip + 1] - sF[c][ip]) * idx;
      LX[(M + c) * N + q] = -(sD[c][ip + 1] - sD[c][ip]) * idx2;
      LX[(2 * M + c) * N + q] = -(sN[c][ip + 1] - sN[c][ip]) * idx;
      VT[c * N + q] = vt[c];
    }
  }
}

// ---------------------------------------------------------------------------
// y-sweep + stage combination
// ---------------------------------------------------------------------------
template <int EQ, class Real>
struct YLayout {
  static constexpr int M = Dim2<EQ>::M;
  static constexpr bool EUL = EQ == HWENO_EULER;
  static constexpr int R = kRowsY2D + 4, C = kColsY2D, P = R * C;  // loaded points
  static constexpr int RF = kRowsY2D + 1;                          // interface rows
  // per-point arrays: U, W, G+, G-, T+, T-, xi (M each), eigen data (5, Euler)
  static constexpr int NQ = 7 * M + (EUL ? 5 : 0);
  static constexpr int NI = 3 * M;                                  // g-hat, theta-hat, xi-hat
  // FP32: the epilogue's global inputs (x parts of L, v~, U^n, v~^n, w~^n),
  // fetched asynchronously at the start, one row of kRowsY2D x C per field
  static constexpr int NPRE = std::is_same<Real, float>::value ? 7 * M : 0;
  static constexpr int PE = kRowsY2D * C;
  static constexpr size_t bytes =
      sizeof(Real) * ((size_t)NQ * P + (size_t)NI * RF * C + (size_t)NPRE * PE) + 64;
};

template <int EQ, class Real, int MODE>
__global__ void __launch_bounds__(kThreads2D, (MinBlocks<Real, HWENO_MINB_Y_F64, HWENO_MINB_Y_F32>::value)) k_ysweep_2d(const __grid_constant__ Args2D a) {
  using Lay = YLayout<EQ, Real>;
  constexpr int M = Lay::M;
  constexpr bool EUL = Lay::EUL;
  constexpr int C = Lay::C, P = Lay::P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  unsigned* const st = a.status;
  // point arrays [7M][P]: quantity qty of component c at loaded point r * C + col
  const auto sPts = tile_view<P>(sm, 7 * M, st);
  auto PT = [&](int qty, int c) { return sPts[qty * M + c]; };
  const auto sEig = tile_view<P>(sm + (size_t)7 * M * P, EUL ? 5 : 0, st);  // Euler: 5 x P
  Real* sI = sm + (size_t)Lay::NQ * P;  // interface arrays [3M][RF * C]
  const auto sIf = tile_view<Lay::RF * C>(sI, 3 * M, st);
  auto IF = [&](int kind, int c) { return sIf[kind * M + c]; };
  __shared__ Real red[kThreads2D / 32];
  __shared__ double s_dt, s_ts;

  if (a.skip_done && !(a.t[0] < a.t_end)) return;
  const int nx = a.nx, ny = a.ny;
  const long long N = (long long)nx * ny;
  const int i0 = blockIdx.x * C, j0 = blockIdx.y * kRowsY2D;
  const int ncol = min(C, nx - i0), nrow = min(kRowsY2D, ny - j0);
  static_assert(kRowsY2D * C <= kThreads2D, "one epilogue point per thread");
  // FP32: copies of this thread's epilogue inputs, started asynchronously
  // after the tile's own loads (below), so that their latency hides behind
  // the point and interface phases
  const auto sPre = tile_view<Lay::PE>(sI + (size_t)Lay::NI * Lay::RF * C, Lay::NPRE, st);
  auto prefetch_epilogue = [&]() {
    const int k = threadIdx.x, r = k / C, col = k % C;
    if (k < Lay::PE && col < ncol && r < nrow) {
      const long long q = (long long)(j0 + r) * nx + i0 + col;
      const Real* LX = static_cast<const Real*>(a.LX);
      const Real* VT = static_cast<const Real*>(a.VT);
      auto cp = [&](int f, const Real* src) {
        __pipeline_memcpy_async(&sPre[f][k], src, sizeof(Real));
      };
#pragma unroll
      for (int c = 0; c < M; ++c) {
        cp(c, LX + c * N + q);
        cp(M + c, LX + (M + c) * N + q);
        cp(2 * M + c, LX + (2 * M + c) * N + q);
        cp(3 * M + c, VT + c * N + q);
        if constexpr (MODE == MODE_STAGE2 || MODE == MODE_STAGE3) {
          cp(4 * M + c, static_cast<const Real*>(a.U0) + c * N + q);
          cp(5 * M + c, static_cast<const Real*>(a.Vt0) + c * N + q);
          cp(6 * M + c, static_cast<const Real*>(a.Wt0) + c * N + q);
        }
      }
    }
    __pipeline_commit();
  };
  const Real* geo = pick<Real>(a.geod, a.geof);
  const Real dy = geo[3], idy = geo[4], idy2 = geo[5];
  const Real alpha = Real(a.alpha_in[1]);
  const Real gam = pick<Real>(a.sp.wd, a.sp.wf)[9], gm1 = gam - Real(1);
  const Weights<Real> w = weights_from(pick<Real>(a.sp.wd, a.sp.wf));
  // time step and boundary time of the stage, once per CTA
  if (threadIdx.x == 0) {
    double dt = 0.0;
    if constexpr (MODE == MODE_STAGE1) {
      int lands;
      dt = time_step2(a, lands);
    } else if constexpr (MODE != MODE_RHS) {
      dt = a.dt[0];
    }
    s_dt = dt;
    s_ts = __dadd_rn(a.t[0], __dmul_rn(a.stage_c, dt));
  }
  __syncthreads();
  const double ts = s_ts;

  {
    const Real* U = static_cast<const Real*>(a.U);
    const Real* V = static_cast<const Real*>(a.V);
    const Real* W = static_cast<const Real*>(a.W);
    const Real hdy = Real(0.5) * dy;
    const Real ha = Real(0.5) * alpha, hda = hdy * alpha;
    // FP32: every load of the tile is issued first, as asynchronous copies
    // into the slots the values occupy anyway (U and W in quantities 0 and
    // 1; V in quantity 6, which this thread overwrites with xi = A_y V of
    // the same point), so that their latencies overlap; the epilogue inputs
    // follow. Each thread then reads only the points it copied itself.
    constexpr int ITER = (P + kThreads2D - 1) / kThreads2D;
    Src src[ITER];
    if constexpr (Lay::NPRE > 0) {
#pragma unroll
      for (int it = 0; it < ITER; ++it) {
        const int k = threadIdx.x + it * kThreads2D;
        const int r = k / C, col = k % C;
        if (k >= P || col >= ncol || r >= nrow + 4) continue;
        const int i = i0 + col, jj = j0 - 2 + r;
        src[it] = map_y(jj, ny, i, a.x0, a.dx, a.y0, a.dy, ts, a.sp);
        HWENO_CHECK(src[it].kind == 2 || (src[it].idx >= 0 && src[it].idx < ny && i < nx), st);
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
      prefetch_epilogue();
      __pipeline_wait_prior(1);  // this thread's tile copies (the epilogue's may still run)
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
        HWENO_CHECK(s.kind == 2 || (s.idx >= 0 && s.idx < ny && i < nx), st);
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

  // interfaces y_{j0+r-1/2}, r = 0..nrow; lower point at loaded row r + 1
  for (int k = threadIdx.x; k < Lay::RF * C; k += blockDim.x) {
    const int r = k / C, col = k % C;
    if (col >= ncol || r > nrow) continue;
    const int gl = r + 1;
    auto at = [&](const auto& A, int rr) { return A[rr * C + col]; };
    if constexpr (!EUL) {
      IF(0, 0)[k] = interface_flux<Real, true>(at(PT(2, 0), gl - 1), at(PT(2, 0), gl), at(PT(2, 0), gl + 1),
                                   at(PT(4, 0), gl - 1), at(PT(4, 0), gl), at(PT(4, 0), gl + 1),
                                   at(PT(3, 0), gl), at(PT(3, 0), gl + 1), at(PT(3, 0), gl + 2),
                                   at(PT(5, 0), gl), at(PT(5, 0), gl + 1), at(PT(5, 0), gl + 2), w);
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
      for (int rr = 0; rr < 4; ++rr) {
        auto pj = [&](int qty, int g) {
          const int kk = g * C + col;
          return e.left(rr, PT(qty, 0)[kk], PT(qty, 1)[kk], PT(qty, 2)[kk], PT(qty, 3)[kk]);
        };
        fr[rr] = interface_flux_frac<Real, true>(pj(2, gl - 1), pj(2, gl), pj(2, gl + 1), pj(4, gl - 1),
                                     pj(4, gl), pj(4, gl + 1), pj(3, gl), pj(3, gl + 1),
                                     pj(3, gl + 2), pj(5, gl), pj(5, gl + 1), pj(5, gl + 2), w);
      }
      Real fch[4];
      resolve4(fr, fch);
      Real out[4];
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

  const Real rdt = Real(s_dt);
  Real ax = Real(0), ay = Real(0);
  bool bad = false;
  const Real* LX = static_cast<const Real*>(a.LX);
  const Real* VT = static_cast<const Real*>(a.VT);
  if constexpr (Lay::NPRE > 0) __pipeline_wait_prior(0);  // this thread's copies
  for (int k = threadIdx.x; k < kRowsY2D * C; k += blockDim.x) {
    const int r = k / C, col = k % C;
    if (col >= ncol || r >= nrow) continue;
    const int g = r + 2;
    const int kc = g * C + col;
    HWENO_CHECK(j0 + r < ny && i0 + col < nx, st);
    const long long q = (long long)(j0 + r) * nx + i0 + col;
    // an epilogue input: prefetched (FP32) or read here
    auto in = [&](int f, const Real* src) -> Real {
      if constexpr (Lay::NPRE > 0) return sPre[f][k];
      else return *src;
    };
    Real l1[M], l2[M], l3[M], vt[M], wt[M], u[M];
#pragma unroll
    for (int c = 0; c < M; ++c) {
      const int ka = r * C + col, kb = (r + 1) * C + col;
      l1[c] = in(c, LX + c * N + q) - (IF(0, c)[kb] - IF(0, c)[ka]) * idy;
      l2[c] = in(M + c, LX + (M + c) * N + q) - (IF(2, c)[kb] - IF(2, c)[ka]) * idy;
      l3[c] = in(2 * M + c, LX + (2 * M + c) * N + q) - (IF(1, c)[kb] - IF(1, c)[ka]) * idy2;
      vt[c] = in(3 * M + c, VT + c * N + q);
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
      auto pj = [&](int rr, int qty, int kk) {
        return e.left(rr, PT(qty, 0)[kk], PT(qty, 1)[kk], PT(qty, 2)[kk], PT(qty, 3)[kk]);
      };
      if constexpr (std::is_same<Real, float>::value) {  // two fields per packed pair
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r0 = 2 * h, r1 = 2 * h + 1;
          auto p2 = [&](int qty, int kk) { return make_float2(pj(r0, qty, kk), pj(r1, qty, kk)); };
          const float2 o = limited_derivative_pair(p2(0, kc - C), p2(0, kc), p2(0, kc + C),
                                                   mul2(pair(dy), p2(1, kc - C)),
                                                   mul2(pair(dy), p2(1, kc + C)), w);
          z[r0] = o.x;
          z[r1] = o.y;
        }
      } else {
        Frac<Real> zr[4];
#pragma unroll
        for (int rr = 0; rr < 4; ++rr)
          zr[rr] = limited_derivative_frac(pj(rr, 0, kc - C), pj(rr, 0, kc), pj(rr, 0, kc + C),
                                           dy * pj(rr, 1, kc - C), dy * pj(rr, 1, kc + C), w);
        resolve4(zr, z);
      }
      e.right(z, wt);
#pragma unroll
      for (int c = 0; c < 4; ++c) wt[c] *= idy;
    }
    if constexpr (MODE == MODE_RHS) {
#pragma unroll
      for (int c = 0; c < M; ++c) {
        static_cast<Real*>(a.L1)[c * N + q] = l1[c];
        static_cast<Real*>(a.L2)[c * N + q] = l2[c];
        static_cast<Real*>(a.L3)[c * N + q] = l3[c];
        if (a.Wlim) static_cast<Real*>(a.Wlim)[c * N + q] = wt[c];
      }
    } else {
      Real un[M];
#pragma unroll
      for (int c = 0; c < M; ++c) {
        const long long qc = c * N + q;
        Real vn, wn;
        if constexpr (MODE == MODE_STAGE1) {
          un[c] = u[c] + rdt * l1[c];
          vn = vt[c] + rdt * l2[c];
          wn = wt[c] + rdt * l3[c];
          static_cast<Real*>(a.Wt0out)[qc] = wt[c];
        } else {
          const Real u0 = in(4 * M + c, static_cast<const Real*>(a.U0) + qc);
          const Real v0 = in(5 * M + c, static_cast<const Real*>(a.Vt0) + qc);
          const Real w0 = in(6 * M + c, static_cast<const Real*>(a.Wt0) + qc);
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
cudaError_t ysweep_launch(const Args2D& a, cudaStream_t s) {
  constexpr size_t bytes = YLayout<EQ, Real>::bytes;
  static unsigned configured = 0;  // devices whose limit is raised
  if (const cudaError_t e = ensure_smem_limit(k_ysweep_2d<EQ, Real, MODE>, bytes, configured)) return e;
  const dim3 grid((a.nx + kColsY2D - 1) / kColsY2D, (a.ny + kRowsY2D - 1) / kRowsY2D);
  k_ysweep_2d<EQ, Real, MODE><<<grid, kThreads2D, bytes, s>>>(a);
  return cudaGetLastError();
}

template <int EQ, class Real>
cudaError_t ysweep_mode(int mode, const Args2D& a, cudaStream_t s) {
  switch (mode) {
    case MODE_RHS: return ysweep_launch<EQ, Real, MODE_RHS>(a, s);
    case MODE_STAGE1: return ysweep_launch<EQ, Real, MODE_STAGE1>(a, s);
    case MODE_STAGE2: return ysweep_launch<EQ, Real, MODE_STAGE2>(a, s);
    default: return ysweep_launch<EQ, Real, MODE_STAGE3>(a, s);
  }
}

template <int EQ, class Real>
cudaError_t xsweep_mode(int mode, const Args2D& a, cudaStream_t s) {
  const dim3 grid((a.nx + kTileX2D - 1) / kTileX2D, a.ny);
  if (mode == MODE_STAGE1) k_xsweep_2d<EQ, Real, MODE_STAGE1><<<grid, kThreads2D, 0, s>>>(a);
  else k_xsweep_2d<EQ, Real, MODE_RHS><<<grid, kThreads2D, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_alpha_2d(int eq, bool fp32, const Args2D& a, cudaStream_t s) {
  const long long N = (long long)a.nx * a.ny;
  const int blocks = (int)std::min<long long>((N + 255) / 256, 152LL * 8);
  if (eq == HWENO_BURGERS) {
    if (fp32) k_alpha_2d<HWENO_BURGERS, float><<<blocks, 256, 0, s>>>(a);
    else k_alpha_2d<HWENO_BURGERS, double><<<blocks, 256, 0, s>>>(a);
  } else {
    if (fp32) k_alpha_2d<HWENO_EULER, float><<<blocks, 256, 0, s>>>(a);
    else k_alpha_2d<HWENO_EULER, double><<<blocks, 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// The x-sweep only distinguishes stage 1 (which records dt) from the rest.
cudaError_t launch_xsweep_2d(int eq, bool fp32, int mode, const Args2D& a, cudaStream_t s) {
  if (eq == HWENO_BURGERS)
    return fp32 ? xsweep_mode<HWENO_BURGERS, float>(mode, a, s)
                : xsweep_mode<HWENO_BURGERS, double>(mode, a, s);
  return fp32 ? xsweep_mode<HWENO_EULER, float>(mode, a, s)
              : xsweep_mode<HWENO_EULER, double>(mode, a, s);
}

cudaError_t launch_ysweep_2d(int eq, bool fp32, int mode, const Args2D& a, cudaStream_t s) {
  if (eq == HWENO_BURGERS)
    return fp32 ? ysweep_mode<HWENO_BURGERS, float>(mode, a, s)
                : ysweep_mode<HWENO_BURGERS, double>(mode, a, s);
  return fp32 ? ysweep_mode<HWENO_EULER, float>(mode, a, s)
              : ysweep_mode<HWENO_EULER, double>(mode, a, s);
}

}  // namespace hweno
