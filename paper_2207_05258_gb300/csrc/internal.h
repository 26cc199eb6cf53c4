// Internal interface between the host side of the library (hweno_api.cu) and
// its kernels (stage1d.cu, stage2d.cu). Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include "hweno.h"
#include <stdint.h>

namespace hweno {

// Raise kernel f's dynamic shared-memory limit to `bytes` once per device
// (the attribute belongs to the function on the current device); `done`
// holds one bit per device already configured.
template <class K>
inline cudaError_t ensure_smem_limit(K* f, size_t bytes, unsigned& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned bit = dev < 32 ? (1u << dev) : 0u;
  if (bit && (done & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done |= bit;
  return e;
}

// Status-word bits written by kernels (read by hweno_sync_status).
// STATUS_BOUNDS: a device-side index check of a checked build failed.
enum : unsigned { STATUS_NONFINITE = 1u, STATUS_TIMEOUT = 2u, STATUS_BOUNDS = 4u };

// ---------------------------------------------------------------------------
// Checked builds (compiled with -DHWENO_CHECKS=1; a stand-in for a memory
// checker). Shared-memory tiles are reached through views whose rows and
// columns are checked against their extents, and global indices through
// HWENO_CHECK at the points where they are formed. A failed check sets
// STATUS_BOUNDS in the context's status word (no trap: the context stays
// usable) and the access goes to element 0 of the array instead, so nothing
// outside it is touched. In a normal build the views are the plain arrays
// and the checks vanish.
// ---------------------------------------------------------------------------
#if defined(HWENO_CHECKS) && HWENO_CHECKS
#define HWENO_CHECK(cond, status)                                     \
  do {                                                                \
    if (!(cond)) atomicOr((status), STATUS_BOUNDS);                   \
  } while (0)
// the same, leaving the enclosing function (a lambda) when the check fails
#define HWENO_CHECK_RETURN(cond, status)                              \
  do {                                                                \
    if (!(cond)) {                                                    \
      atomicOr((status), STATUS_BOUNDS);                              \
      return;                                                         \
    }                                                                 \
  } while (0)

template <class T, int C>
struct CheckedRow {
  T* p;
  unsigned* st;
  __device__ __forceinline__ T& operator[](int i) const {
    if ((unsigned)i >= (unsigned)C) {
      atomicOr(st, STATUS_BOUNDS);
      i = 0;
    }
    return p[i];
  }
};
template <class T, int C>
struct CheckedTile {
  T* base;
  int rows;
  unsigned* st;
  __device__ __forceinline__ CheckedRow<T, C> operator[](int r) const {
    if ((unsigned)r >= (unsigned)rows) {
      atomicOr(st, STATUS_BOUNDS);
      r = 0;
    }
    return CheckedRow<T, C>{base + (size_t)r * C, st};
  }
};
// view of a [rows][C] tile at p (dynamic shared memory)
template <int C, class T>
__device__ __forceinline__ CheckedTile<T, C> tile_view(T* p, int rows, unsigned* st) {
  return CheckedTile<T, C>{p, rows, st};
}
// view of a static [R][C] shared array
template <class T, int R, int C>
__device__ __forceinline__ CheckedTile<T, C> tile_view(T (&a)[R][C], unsigned* st) {
  return CheckedTile<T, C>{&a[0][0], R, st};
}
#else
#define HWENO_CHECK(cond, status) ((void)0)
#define HWENO_CHECK_RETURN(cond, status) ((void)0)
template <int C, class T>
__device__ __forceinline__ T (*tile_view(T* p, int, unsigned*))[C] {
  return reinterpret_cast<T(*)[C]>(p);
}
template <class T, int R, int C>
__device__ __forceinline__ T (*tile_view(T (&a)[R][C], unsigned*))[C] {
  return a;
}
#endif

enum Mode { MODE_RHS = 0, MODE_STAGE1 = 1, MODE_STAGE2 = 2, MODE_STAGE3 = 3 };

// 1D tiles: one CTA of `threads` threads handles up to threads * ppt - 4
// consecutive points of one instance, so that each phase takes ppt passes:
// the tile plus four ghosts, its interfaces and its updates all fit in
// threads * ppt slots. Variant 0 (128 threads, one point each) is the
// default; hweno_autotune measures the others. kThreads1D is the CTA size of
// the wave-speed kernel.
struct TileVariant {
  int threads, ppt;
};
constexpr TileVariant kVariants1D[] = {{128, 1}, {64, 1}, {256, 1}, {128, 2}, {64, 2}};
constexpr int kNumVariants1D = HWENO_TILE_VARIANTS;
static_assert(sizeof(kVariants1D) / sizeof(kVariants1D[0]) == kNumVariants1D, "variant table");
constexpr int tile_points(int v) { return kVariants1D[v].threads * kVariants1D[v].ppt - 4; }
constexpr int kThreads1D = 128;
constexpr int kTile1D = tile_points(0);
constexpr int kMinTile1D = 60;  // smallest tile of any variant

constexpr int kConstTable = 15;

// Bounds of the options that enter the deferred quotients. The kernels
// resolve quotients whose denominators are products of factors of the size
// of beta + eps (the nonlinear weights of two sides of two fields over a
// common denominator) times powers of the linear weights. Within these
// bounds those products stay above the FP64 underflow limit: where beta = 0
// (constant data, where tau = 0 too) they are eps^12 g^4 >= 1e-264. Large
// beta (large data) is handled in the kernels, which rescale each side's
// numerator and denominator by an exact power of two (hweno_math.cuh,
// normalize).
constexpr double kEpsMin = 1e-20, kEpsMax = 1e6, kWeightMin = 1e-6;

struct SchemeParams {
  double lin_w[3], lim_d[3], eps, cfl, dt_fixed;
  int dt_mode, limiter, eig_avg;
  int adj_frozen;  // adjoint: nonlinear weights held at their forward values
  double gas_gamma;
  int bc[4];
  double inflow[4], pre[4];
  float inflowf[4], pref[4];  // the same in FP32 (the 1D loads read these)
  double dmr_x0, dmr_speed, dmr_angle;
  double dmr_tan, dmr_sin;  // tan and sin of dmr_angle, evaluated on the host
  // constants in both precisions, converted once on the host
  // (fill_constant_table): g0, g1, g2, d0, d1, d2, eps, 1/g0, 1/d0, gas
  // gamma, (Buckley-Leverett) max |f'| over [0, 1], and the coefficients of
  // p0 - g1 p1 - g2 p2 in f_{i-1}, f_i, f_{i+1}, H_i
  double wd[kConstTable];
  float wf[kConstTable];
};

// The constant table of SchemeParams. p0 - g1 p1 - g2 p2 (the quintic's
// share of the nonlinear combination, Sec. 2.1) is a fixed linear form in
// the stencil values once the linear weights are known: with p0, p1, p2 of
// Sec. 2.1 its coefficients are 11/60 - g1/6 (f_{i-1}), 19/30 - 5 (g1 + g2)/6
// (f_i), 11/60 - g2/6 (f_{i+1}), 1/2 - 2 g1/3 - g2/3 (H_i) and 1/20
// (H_{i-1} - H_{i+1}, a literal in the kernels).
inline void fill_constant_table(SchemeParams& sp, const double g[3], const double d[3],
                                double eps, double gas_gamma, double bl_alpha) {
  const double tab[kConstTable] = {g[0], g[1], g[2], d[0], d[1], d[2], eps, 1.0 / g[0],
                                   1.0 / d[0], gas_gamma, bl_alpha,
                                   11.0 / 60.0 - g[1] / 6.0,
                                   19.0 / 30.0 - 5.0 * (g[1] + g[2]) / 6.0,
                                   11.0 / 60.0 - g[2] / 6.0,
                                   0.5 - 2.0 * g[1] / 3.0 - g[2] / 3.0};
  for (int i = 0; i < kConstTable; ++i) { sp.wd[i] = tab[i]; sp.wf[i] = (float)tab[i]; }
}

// Arguments of one 1D launch (all instances of the batch).
struct Args1D {
  // stage input state (u^{(k-1)}, v^{(k-1)}) and, for stages 2-3, u^n, v~^n
  const void* U;
  const void* V;
  const void* U0;
  const void* Vt0;
  // outputs: stage state, the stored v~^n (stage 1) or L^1, L^2, v~ (rhs)
  void* Uout;
  void* Vout;
  void* Vt0out;
  void* L1;
  void* L2;
  void* Vlim;
  // batch tables (device)
  const int* tile_inst;
  const int* tile_start;
  const int* inst_n;
  const long long* inst_off;  // first point of each instance
  const double* inst_dx;
  const double* inst_hx;      // dx or dx^{5/3} per dt_mode
  const double* inst_geo;     // per instance dx, 1/dx, 1/dx^2 (FP64)
  const float* inst_geof;     // the same in FP32
  // per-instance scalars (device)
  const double* t;
  double t_end;
  int skip_done;              // instances with t >= t_end do nothing
  const double* alpha_in;     // wave speed of the stage input
  unsigned long long* alpha_out;  // max wave speed of the stage output (bits)
  double* dt;                 // per-instance time step (written in stage 1)
  const double* dt_in;        // stage 1 takes dt from here when not null (replay)
  int* lands;                 // dt was clipped to t_end (stage 1)
  unsigned* status;
  SchemeParams sp;
};

// Minimum resident CTAs per SM requested from the compiler for the stage
// kernels, per precision (register budget = 64K / (threads x this)); chosen
// by measurement: the FP64 kernels are FP64-pipe bound at any occupancy
// (1..4 CTAs gave the same throughput), the FP32 ones gain from more warps
// (1D: 8 CTAs, 64 registers, +12%; 2D: 5 CTAs).
#ifndef HWENO_MINB_1D_F64
#define HWENO_MINB_1D_F64 1
#endif
#ifndef HWENO_MINB_1D_F32
#define HWENO_MINB_1D_F32 8
#endif
#ifndef HWENO_MINB_X_F64
#define HWENO_MINB_X_F64 1
#endif
#ifndef HWENO_MINB_X_F32
#define HWENO_MINB_X_F32 5
#endif
#ifndef HWENO_MINB_Y_F64
#define HWENO_MINB_Y_F64 1
#endif
#ifndef HWENO_MINB_Y_F32
#define HWENO_MINB_Y_F32 5
#endif
template <class Real, int F64, int F32>
struct MinBlocks { static constexpr int value = sizeof(Real) == 8 ? F64 : F32; };

// 2D tiles. x-sweep: one CTA per row segment of kTileX2D points (like 1D).
// y-sweep: one CTA per block of kColsY2D columns x kRowsY2D rows, so that
// (kRowsY2D + 1) x kColsY2D interfaces = kThreads2D.
constexpr int kThreads2D = 128;
constexpr int kTileX2D = kThreads2D - 4;
constexpr int kColsY2D = 16;
constexpr int kRowsY2D = kThreads2D / kColsY2D - 1;

// Arguments of the 2D launches (one instance).
struct Args2D {
  const void* U;  // stage input
  const void* V;
  const void* W;
  const void* U0;  // u^n, v~^n, w~^n (stages 2-3)
  const void* Vt0;
  const void* Wt0;
  void* Uout;
  void* Vout;
  void* Wout;
  void* Wt0out;  // stage 1: w~^n
  void* LX;      // x-sweep result [3m][ny][nx]: x parts of L^1, L^2, L^3
  void* VT;      // x-sweep limited derivative v~ [m][ny][nx]
  void* L1;      // rhs outputs
  void* L2;
  void* L3;
  void* Wlim;
  int nx, ny;
  double dx, dy, hx, hy;  // mesh widths; h of the time-step rule
  double geod[6];         // dx, 1/dx, 1/dx^2, dy, 1/dy, 1/dy^2
  float geof[6];
  double x0, y0;
  const double* t;
  double t_end;
  int skip_done;
  double stage_c;  // boundary time of the stage: t + stage_c * dt
  const double* alpha_in;          // [2]: alpha_x, alpha_y of the stage input
  unsigned long long* alpha_out;   // [2]: of the stage output (bits)
  double* dt;
  int* lands;
  unsigned* status;
  const double* dt_in;  // replay (adjoint): time step given per step, else null
  SchemeParams sp;
};

cudaError_t launch_alpha_2d(int eq, bool fp32, const Args2D& a, cudaStream_t s);
cudaError_t launch_xsweep_2d(int eq, bool fp32, int mode, const Args2D& a, cudaStream_t s);
// Fused stage (stage2d_fused.cu): the x- and y-parts of one SSP-RK3 stage in
// one launch, one CTA per kColsY2D x kRowsY2D block (modes STAGE1..3).
cudaError_t launch_stage_fused_2d(int eq, bool fp32, int mode, const Args2D& a, cudaStream_t s);
cudaError_t launch_ysweep_2d(int eq, bool fp32, int mode, const Args2D& a, cudaStream_t s);

// Adjoint of one stage of a 1D step (adjoint1d.cu), FP64. With x_k =
// a_k B(x^n) + b G(x_{k-1}), G(x) = (U + dt L^1(x), v~(x) + dt L^2(x)), it
// writes out = G'(x_{k-1})^T (b lam) [+ acc], i.e. the adjoint of the stage
// input. Optionally (stage 2) also acc = cN lamN + c2 lam, the cotangent of
// the base term (U^n, v~(x^n)).
struct AdjArgs1D {
  const double* U;       // stage input state x_{k-1}
  const double* V;
  const double* lamU;    // adjoint of the stage output
  const double* lamV;
  const double* accU;    // added to the U result (stage 1), nullable
  const double* accVt;   // added to the cotangent of v~ (stage 1), nullable
  const double* lamNU;   // lambda^{n+1} for acc (stage 2), nullable
  const double* lamNV;
  double* outU;
  double* outV;
  double* accOutU;       // acc (stage 2), nullable
  double* accOutVt;
  double b, cN, c2;
  const int* tile_inst;
  const int* tile_start;
  const int* inst_n;
  const long long* inst_off;
  const double* inst_geo;
  const double* alpha;   // frozen wave speed of the stage input, per instance
  const double* dt;      // time step per instance (0: the instance did not step)
  unsigned* status;      // checked builds: STATUS_BOUNDS
  SchemeParams sp;
};

cudaError_t launch_adjoint_1d(int eq, const AdjArgs1D& a, int ntiles, cudaStream_t s);
cudaError_t launch_adjoint_1d_euler(const AdjArgs1D& a, int ntiles, cudaStream_t s);

// Adjoint of one stage of a 2D step (adjoint2d.cu), FP64, as two sweeps over
// lines (rows, then columns). With G(x) = (U + dt L^1, v~ + dt L^2, w~ + dt
// L^3): the x sweep writes the cotangents that flow through the x-direction
// terms (f-hat, h-hat, eta-hat, v~) to `part` [3m][ny][nx]; the y sweep adds
// those of the y-direction terms (g-hat, theta-hat, xi-hat, w~), the stage's
// direct term b lamU (+ accU) and `part`, and writes out (and, stage 2, acc).
struct AdjArgs2D {
  const double* U;  // stage input state
  const double* V;
  const double* W;
  const double* lamU;  // adjoint of the stage output
  const double* lamV;
  const double* lamW;
  const double* accU;   // stage 1: cotangents of the base term, nullable
  const double* accVt;
  const double* accWt;
  const double* lamNU;  // stage 2: lambda^{n+1} for acc, nullable
  const double* lamNV;
  const double* lamNW;
  double* part;         // x-sweep result [3m][ny][nx]
  double* outU;
  double* outV;
  double* outW;
  double* accOutU;      // stage 2: acc = cN lamN + c2 lam, nullable
  double* accOutVt;
  double* accOutWt;
  double b, cN, c2;
  int nx, ny;
  double dx, dy;
  double geod[6];       // dx, 1/dx, 1/dx^2, dy, 1/dy, 1/dy^2
  double x0, y0;
  const double* t;      // time at the start of the step (boundary time)
  double stage_c;       // boundary time of the stage: t + stage_c * dt
  const double* alpha;  // [2] frozen alpha_x, alpha_y of the stage input
  const double* dt;     // [1] (0: the step did not happen)
  unsigned* status;     // checked builds: STATUS_BOUNDS
  SchemeParams sp;
};

cudaError_t launch_adjoint_2d(int eq, int dir, const AdjArgs2D& a, cudaStream_t s);

// Conserved totals (totals.cu): per-tile FP64 partial sums, then a
// fixed-order sum per instance. Tiles: the 1D tile table, or row segments of
// kTileX2D points in 2D (instance 0).
cudaError_t launch_totals(int m, bool fp32, int dim, const void* U, int ntiles, int tile,
                          const int* tile_inst, const int* tile_start, const int* inst_n,
                          const long long* inst_off, int batch, int nx, int ny, double cell,
                          const double* inst_dx, double* partial, double* totals,
                          cudaStream_t s);

// Launchers (stage1d.cu, stage1d_f32.cu). eq: 0 Burgers, 1 Euler; variant:
// index into kVariants1D (the tile table must match its tile_points).
cudaError_t launch_alpha_1d_f64(int eq, int variant, const Args1D& a, int ntiles, cudaStream_t s);
cudaError_t launch_alpha_1d_f32(int eq, int variant, const Args1D& a, int ntiles, cudaStream_t s);
cudaError_t launch_stage_1d_f64(int eq, int variant, int mode, const Args1D& a, int ntiles,
                                cudaStream_t s);
cudaError_t launch_stage_1d_f32(int eq, int variant, int mode, const Args1D& a, int ntiles,
                                cudaStream_t s);
// Persistent run of a 1D batch (stage1d_impl.cuh, k_run_1d): `steps` whole
// SSP-RK3 steps in one launch. CTAs take tickets (step, stage, tile) in that
// lexicographic order from `next`; a tile waits (bounded) until its instance
// has completed every tile of the previous stage, counted in done[k]; the
// last stage-3 tile of an instance does the time update and releases the
// next step. alpha slots: [parity][stage][batch], zeroed by the host before
// the launch, slot [0][0] holding alpha(U^n) of the first step.
struct PersistArgs {
  unsigned long long* next;   // ticket counter (zero at launch)
  unsigned* done;             // per instance: completed tiles (zero at launch)
  unsigned* done3;            // per instance: completed stage-3 tiles of the step
  const int* inst_tiles;      // tiles per instance in the launch's tile table
  unsigned long long* alpha;  // 2 x 3 x batch
  void* U1; void* V1; void* U2; void* V2; void* Vt0;  // stage buffers
  int* active;                // instances with t < t_end after the last step
  unsigned long long* pu;     // point-updates of stepping instances (nullable)
  int steps, ntiles, batch;
  unsigned wait_extra;        // test hook: tiles of instance 0 wait for this many more
};

// Fused step of small instances (stage1d_impl.cuh, k_step_small_1d): one CTA
// per instance of at most kFusedPoints points runs the wave speed, the three
// stages and the time update of one step. Stage buffers as in a plain step;
// alpha slots [3][batch].
constexpr int kFusedThreads = 128, kFusedPPT = 4;
constexpr int kFusedPoints = kFusedThreads * kFusedPPT - 4;
static_assert(kFusedPoints == HWENO_FUSED_MAX_POINTS, "fused tile");
struct FusedArgs {
  void* U1; void* V1; void* U2; void* V2; void* Vt0;
  unsigned long long* alpha;  // 3 x batch
  double* dt_used;            // nullable
  int* active;
  unsigned long long* pu;     // nullable
  int batch;
  int steps = 1;              // cluster step: steps per launch
};
cudaError_t launch_step_small_1d_f64(int eq, const Args1D& a, const FusedArgs& f, cudaStream_t s);
cudaError_t launch_step_small_1d_f32(int eq, const Args1D& a, const FusedArgs& f, cudaStream_t s);
cudaError_t launch_step_small_1d_bl(bool fp32, const Args1D& a, const FusedArgs& f,
                                    cudaStream_t s);
inline cudaError_t launch_step_small_1d(int eq, bool fp32, const Args1D& a, const FusedArgs& f,
                                        cudaStream_t s) {
  if (eq == HWENO_BUCKLEY) return launch_step_small_1d_bl(fp32, a, f, s);
  return fp32 ? launch_step_small_1d_f32(eq, a, f, s) : launch_step_small_1d_f64(eq, a, f, s);
}

// Fused step on thread-block clusters (stage1d_impl.cuh, k_step_cluster_1d):
// one cluster per instance of at most kClusterMax * kTile1D points, one tile
// per CTA, each CTA alone on its SM (kClusterSmem of shared memory); max_n is
// the largest instance of the batch.
constexpr int kClusterMax = 8;
constexpr size_t kClusterSmem = 116 * 1024;
// Latency form of the cluster step: 28-point tiles, up to 16 CTAs per cluster
constexpr int kSplitTile = 28, kSplitMax = 16;
static_assert(kSplitMax <= 32 && kClusterMax <= 32, "one lane per CTA in the cluster's alpha");
static_assert(kClusterMax * kTile1D == HWENO_CLUSTER_MAX_POINTS, "cluster step size");
cudaError_t launch_step_cluster_1d_f64(int eq, const Args1D& a, const FusedArgs& f, int max_n,
                                       cudaStream_t s);
cudaError_t launch_step_cluster_1d_f32(int eq, const Args1D& a, const FusedArgs& f, int max_n,
                                       cudaStream_t s);
cudaError_t launch_step_cluster_1d_bl(bool fp32, const Args1D& a, const FusedArgs& f, int max_n,
                                      cudaStream_t s);
inline cudaError_t launch_step_cluster_1d(int eq, bool fp32, const Args1D& a, const FusedArgs& f,
                                          int max_n, cudaStream_t s) {
  if (eq == HWENO_BUCKLEY) return launch_step_cluster_1d_bl(fp32, a, f, max_n, s);
  return fp32 ? launch_step_cluster_1d_f32(eq, a, f, max_n, s)
              : launch_step_cluster_1d_f64(eq, a, f, max_n, s);
}

cudaError_t launch_run_1d_f64(int eq, int variant, const Args1D& a, const PersistArgs& p,
                              int ctas, cudaStream_t s);
cudaError_t launch_run_1d_f32(int eq, int variant, const Args1D& a, const PersistArgs& p,
                              int ctas, cudaStream_t s);
cudaError_t launch_run_1d_bl(bool fp32, int variant, const Args1D& a, const PersistArgs& p,
                             int ctas, cudaStream_t s);
// Resident CTAs of the persistent kernel per SM (occupancy), for the grid size.
int run_1d_ctas_per_sm(int eq, bool fp32, int variant);
int run_1d_ctas_per_sm_f64(int eq, int variant);
int run_1d_ctas_per_sm_f32(int eq, int variant);
int run_1d_ctas_per_sm_bl(bool fp32, int variant);

// Buckley-Leverett kernels, both precisions (stage1d_bl.cu).
cudaError_t launch_alpha_1d_bl(bool fp32, int variant, const Args1D& a, int ntiles,
                               cudaStream_t s);
cudaError_t launch_stage_1d_bl(bool fp32, int variant, int mode, const Args1D& a, int ntiles,
                               cudaStream_t s);
inline cudaError_t launch_run_1d(int eq, bool fp32, int variant, const Args1D& a,
                                 const PersistArgs& p, int ctas, cudaStream_t s) {
  if (eq == HWENO_BUCKLEY) return launch_run_1d_bl(fp32, variant, a, p, ctas, s);
  return fp32 ? launch_run_1d_f32(eq, variant, a, p, ctas, s)
              : launch_run_1d_f64(eq, variant, a, p, ctas, s);
}
inline int run_1d_ctas_per_sm(int eq, bool fp32, int variant) {
  if (eq == HWENO_BUCKLEY) return run_1d_ctas_per_sm_bl(fp32, variant);
  return fp32 ? run_1d_ctas_per_sm_f32(eq, variant) : run_1d_ctas_per_sm_f64(eq, variant);
}
inline cudaError_t launch_alpha_1d(int eq, bool fp32, int variant, const Args1D& a, int ntiles,
                                   cudaStream_t s) {
  if (eq == HWENO_BUCKLEY) return launch_alpha_1d_bl(fp32, variant, a, ntiles, s);
  return fp32 ? launch_alpha_1d_f32(eq, variant, a, ntiles, s)
              : launch_alpha_1d_f64(eq, variant, a, ntiles, s);
}
inline cudaError_t launch_stage_1d(int eq, bool fp32, int variant, int mode, const Args1D& a,
                                   int ntiles, cudaStream_t s) {
  if (eq == HWENO_BUCKLEY) return launch_stage_1d_bl(fp32, variant, mode, a, ntiles, s);
  return fp32 ? launch_stage_1d_f32(eq, variant, mode, a, ntiles, s)
              : launch_stage_1d_f64(eq, variant, mode, a, ntiles, s);
}
// Time update after stage 3; counts the instances still active and, when
// pu is not null, adds inst_n[k] * rows (the instance's points; rows = ny in
// 2D, 1 in 1D) of every instance that took the step.
// Number of instances with t < t_end (one CTA; written, not added).
cudaError_t launch_count_active(int batch, const double* t, double t_end, int* active,
                                cudaStream_t s);
cudaError_t launch_finalize(int batch, const double* dt, const int* lands, double* t,
                            double t_end, double* dt_used, const double* alpha,
                            int* active_count, unsigned* status, const int* inst_n, int rows,
                            unsigned long long* pu, cudaStream_t s);

}  // namespace hweno
