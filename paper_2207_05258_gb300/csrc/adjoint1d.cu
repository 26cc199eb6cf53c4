// Discrete adjoint of one SSP-RK3 stage of the 1D L-HWENO scheme (Zhang &
// Zhao, arXiv:2207.05258, Sec. 2.1-2.2) in FP64, with the wave speed alpha and
// the time step of the forward run frozen and the |.| branches of tau taken at
// the forward state.
//
// One CTA owns a tile of points [s, s + P). Every quantity of the forward
// stage that depends on an owned point is differentiated inside the tile: the
// interfaces x_{j+1/2}, j = s-2 .. s+P (each stencil touches points j-1..j+2)
// and the limited derivatives at j = s-1 .. s+P. Each such item stores its
// contributions to its stencil slots in shared memory; every owned point then
// gathers, in a fixed order, the slots that refer to it (directly, or through
// a mirrored or copied ghost at a wall). Periodic images need no mapping: the
// items are indexed locally, so an owned point reads exactly the items around
// it. No atomics: the result is the same bit for bit on every run.
#include "hweno.h"
#include "hweno_adjoint.cuh"
#include "internal.h"

namespace hweno {
namespace {

constexpr int P = kTile1D;     // owned points per tile
constexpr int NL = P + 6;      // loaded points s-3 .. s+P+2
constexpr int NI = P + 3;      // interfaces j = s-2 .. s+P
constexpr int NV = P + 2;      // limited derivatives j = s-1 .. s+P

__global__ void __launch_bounds__(128) k_adjoint_burgers_1d(const __grid_constant__ AdjArgs1D a) {
  __shared__ double su[NL], sv[NL], sFp[NL], sFm[NL], sHp[NL], sHm[NL];
  __shared__ double mL1[P + 4], mL2[P + 4], mVt[NV];
  __shared__ double gu[NI][4], gv[NI][4];
  __shared__ double lu[NV][3], lv[NV][2];

  const int b = blockIdx.x;
  const int k = a.tile_inst[b], s = a.tile_start[b], n = a.inst_n[k];
  const int np = min(P, n - s);
  HWENO_CHECK(s >= 0 && np >= 1, a.status);
  const long long off = a.inst_off[k];
  const double dt = a.dt[k];
  if (dt == 0.0) {  // the instance did not step: the stage is the identity
    for (int ip = threadIdx.x; ip < np; ip += blockDim.x) {
      const long long q = off + s + ip;
      a.outU[q] = a.lamU[q];
      a.outV[q] = a.lamV[q];
      if (a.accOutU) { a.accOutU[q] = 0.0; a.accOutVt[q] = 0.0; }
    }
    return;
  }
  const double* geo = a.inst_geo + 3 * k;
  const double dx = geo[0], idx = geo[1], idx2 = geo[2];
  const double alpha = a.alpha[k];
  const Weights<double> w = weights_from(a.sp.wd);
  const bool periodic = a.sp.bc[0] == HWENO_BC_PERIODIC;
  const double hdx = 0.5 * dx;

  // forward point data on s-3 .. s+np+2
  for (int g = threadIdx.x; g < np + 6; g += blockDim.x) {
    int kind;
    const int src = ghost_src(s - 3 + g, n, a.sp.bc[0], a.sp.bc[1], kind);
    HWENO_CHECK(kind == 2 || (src >= 0 && src < n), a.status);
    double u, v;
    if (kind == 2) { u = a.sp.inflow[0]; v = 0.0; }
    else {
      u = a.U[off + src];
      v = a.V[off + src];
      if (kind == 1) { u = -u; }  // Burgers wall: u odd, u_x even
    }
    su[g] = u;
    sv[g] = v;
    const double F = 0.5 * u * u, H = u * v;
    sFp[g] = 0.5 * (F + alpha * u);
    sFm[g] = 0.5 * (F - alpha * u);
    sHp[g] = hdx * (H + alpha * v);
    sHm[g] = hdx * (H - alpha * v);
  }
  // cotangents of L^1, L^2 at s-2 .. s+np+1 and of v~ at s-1 .. s+np
  auto pt = [&](int p) { return periodic ? (p % n + n) % n : p; };
  for (int g = threadIdx.x; g < np + 4; g += blockDim.x) {
    const int p = pt(s - 2 + g);
    const bool in = p >= 0 && p < n;
    const double lu_ = in ? a.lamU[off + p] : 0.0, lv_ = in ? a.lamV[off + p] : 0.0;
    mL1[g] = a.b * dt * lu_;
    mL2[g] = a.b * dt * lv_;
  }
  for (int g = threadIdx.x; g < np + 2; g += blockDim.x) {
    const int p = pt(s - 1 + g);
    const bool in = p >= 0 && p < n;
    mVt[g] = in ? a.b * a.lamV[off + p] + (a.accVt ? a.accVt[off + p] : 0.0) : 0.0;
  }
  __syncthreads();

  // interfaces j = s-2+jf: stencil points j-1..j+2 are loaded indices jf..jf+3
  for (int jf = threadIdx.x; jf < np + 3; jf += blockDim.x) {
    const double mf = (mL1[jf + 1] - mL1[jf]) * idx;    // d J / d f-hat_{j+1/2}
    const double mD = (mL2[jf + 1] - mL2[jf]) * idx2;   // d J / d (dx h-hat_{j+1/2})
    double gp[6] = {0, 0, 0, 0, 0, 0}, gm[6] = {0, 0, 0, 0, 0, 0};
    flux_vjp(&sFp[jf], &sHp[jf], &sFm[jf + 1], &sHm[jf + 1], mf, w, gp, gm,
             a.sp.adj_frozen != 0);
    dflux_vjp(mD, gp, gm);
    // chain to (u, v) of the four stencil points
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const int g = jf + kk;
      const double u = su[g], v = sv[g];
      const double gFp = kk < 3 ? gp[kk] : 0.0, gHp = kk < 3 ? gp[3 + kk] : 0.0;
      const double gFm = kk > 0 ? gm[kk - 1] : 0.0, gHm = kk > 0 ? gm[3 + kk - 1] : 0.0;
      gu[jf][kk] = 0.5 * (u + alpha) * gFp + 0.5 * (u - alpha) * gFm + hdx * v * (gHp + gHm);
      gv[jf][kk] = hdx * (u + alpha) * gHp + hdx * (u - alpha) * gHm;
    }
  }
  // limited derivatives j = s-1+jl: points j-1, j, j+1 are loaded jl+1..jl+3
  const bool limited = a.sp.limiter != 0;  // 0: v-tilde = v
  for (int jl = threadIdx.x; jl < np + 2; jl += blockDim.x) {
    double g[5] = {0, 0, 0, 0, 0};
    if (limited)
      limiter_vjp(su[jl + 1], su[jl + 2], su[jl + 3], dx * sv[jl + 1], dx * sv[jl + 3],
                  mVt[jl] * idx, w, g, a.sp.adj_frozen != 0);
    lu[jl][0] = g[0]; lu[jl][1] = g[1]; lu[jl][2] = g[2];
    lv[jl][0] = dx * g[3]; lv[jl][1] = dx * g[4];
  }
  __syncthreads();

  for (int ip = threadIdx.x; ip < np; ip += blockDim.x) {
    const int i = s + ip;
    const long long q = off + i;
    double ru = a.b * a.lamU[q] + (a.accU ? a.accU[q] : 0.0), rv = 0.0;
#pragma unroll
    for (int d = 0; d < 4; ++d) { ru += gu[ip + d][3 - d]; rv += gv[ip + d][3 - d]; }
#pragma unroll
    for (int d = 0; d < 3; ++d) ru += lu[ip + d][2 - d];
    rv += lv[ip][1] + lv[ip + 2][0];  // v_{i} enters v~_{i+1} (slot j-1) and v~_{i-1} (slot j+1)
    if (!limited) rv += mVt[ip + 1];
    if (!periodic) {
      // ghosts at walls refer to owned points 0, 1 (left) and n-1, n-2 (right)
      auto add = [&](int jf, int kk, int p) {  // interface item jf, slot kk, point p
        HWENO_CHECK_RETURN(jf >= 0 && jf < NI, a.status);
        int kind;
        const int src = ghost_src(p, n, a.sp.bc[0], a.sp.bc[1], kind);
        if (kind == 2 || src != i) return;
        const double sg = kind == 1 ? -1.0 : 1.0;
        ru += sg * gu[jf][kk];
        rv += gv[jf][kk];
      };
      auto addl = [&](int jl, int kk, int p) {  // limiter item jl, slot kk (0 or 2)
        HWENO_CHECK_RETURN(jl >= 0 && jl < NV, a.status);
        int kind;
        const int src = ghost_src(p, n, a.sp.bc[0], a.sp.bc[1], kind);
        if (kind == 2 || src != i) return;
        const double sg = kind == 1 ? -1.0 : 1.0;
        ru += sg * lu[jl][kk];
        rv += lv[jl][kk == 0 ? 0 : 1];
      };
      if (i <= 1) {  // left wall: items j = -1, 0 (local jf = j - s + 2, jl = j - s + 1)
        add(1 - s, 0, -2);
        add(1 - s, 1, -1);
        add(2 - s, 0, -1);
        addl(1 - s, 0, -1);
      }
      if (i >= n - 2) {  // right wall: items j = n-2, n-1
        add(n - s, 3, n);          // j = n-2
        add(n + 1 - s, 2, n);      // j = n-1
        add(n + 1 - s, 3, n + 1);
        addl(n - s, 2, n);         // j = n-1
      }
    }
    a.outU[q] = ru;
    a.outV[q] = rv;
    if (a.accOutU) {
      a.accOutU[q] = a.cN * a.lamNU[q] + a.c2 * a.lamU[q];
      a.accOutVt[q] = a.cN * a.lamNV[q] + a.c2 * a.lamV[q];
    }
  }
}

}  // namespace

cudaError_t launch_adjoint_1d(int eq, const AdjArgs1D& a, int ntiles, cudaStream_t s) {
  if (eq != HWENO_BURGERS) return launch_adjoint_1d_euler(a, ntiles, s);
  k_adjoint_burgers_1d<<<ntiles, 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace hweno
