// Host side of the C ABI declared in include/hweno.h: argument checking,
// ownership of all device scratch, the tile tables of ragged batches, and the
// launch sequence of one SSP-RK3 step (Sec. 2.2 of Zhang & Zhao,
// arXiv:2207.05258):
//
//   memset(alpha slots, active counter)
//   alpha(U^n)                         -> slot 0            (per instance)
//   stage 1: U^n, V^n    -> U1, V1, V~^n;  alpha(U1) -> slot 1; dt from slot 0
//   stage 2: U1, V1      -> U2, V2;        alpha(U2) -> slot 2
//   stage 3: U2, V2      -> U^{n+1}, V^{n+1} (in place; reads U^n, V~^n pointwise)
//   finalize: t += dt (landing exactly on t_end), active count, status
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "hweno.h"
#include "internal.h"

using namespace hweno;

struct hweno_ctx {
  int eq = 0, dim = 1, m = 1, batch = 1;
  bool fp32 = false;
  std::vector<int> nx;
  int ny = 1;
  double x0 = 0, x1 = 1, y0 = 0, y1 = 1, gamma = 1.4;
  hweno_bc bc{};
  hweno_options opt{};
  long long npts = 0;
  size_t elems = 0, esize = 8;
  // 1D batch tables of every tile variant, made in create: (instance, first
  // point) per tile and tiles per instance. Choosing a variant only switches
  // the pointers below, so it never writes device memory that kernels still
  // in flight on a caller's stream may read. 2D: one entry in variant 0.
  int* d_vt_inst[kNumVariants1D] = {};
  int* d_vt_start[kNumVariants1D] = {};
  int* d_vt_tiles[kNumVariants1D] = {};
  int vt_ntiles[kNumVariants1D] = {};
  // instance-size classes (1D batches): class of each instance, and per
  // variant a tile table ordered by class with each class's tile range, so
  // that the stages can run each class with its own tile variant
  // (hweno_autotune_classes); made in create
  int nclasses = 0;
  std::vector<int> inst_class;
  std::vector<int> class_lo, class_hi;  // smallest / largest instance of a class
  int* d_ct_inst[kNumVariants1D] = {};
  int* d_ct_start[kNumVariants1D] = {};
  int ct_first[kNumVariants1D][HWENO_MAX_SIZE_CLASSES + 1] = {};
  int class_variant[HWENO_MAX_SIZE_CLASSES] = {};
  bool mixed = false;  // stages launched per class (set by hweno_autotune_classes)
  // the current variant (aliases of the arrays above)
  int ntiles = 0;
  int variant = 0;
  int tile = kTile1D;
  int tiles_cap = 0;  // largest table (smallest tile)
  int* d_tile0_inst = nullptr;   // variant 0, used by the adjoint
  int* d_tile0_start = nullptr;
  int ntiles0 = 0;
  int* d_tile_inst = nullptr;
  int* d_tile_start = nullptr;
  int* d_inst_n = nullptr;
  long long* d_inst_off = nullptr;
  double* d_inst_dx = nullptr;
  double* d_hx[2] = {};            // h of the time-step rule: dx, dx^{5/3} (made in create)
  double* d_inst_hx = nullptr;     // the one dt_mode selects (alias)
  double* d_inst_geo = nullptr;   // per instance dx, 1/dx, 1/dx^2
  float* d_inst_geof = nullptr;   // the same in FP32
  std::vector<double> inst_dx;
  // per-instance scalars
  unsigned long long* d_alpha = nullptr;  // 3 slots x batch (x 2 directions in 2D)
  double* d_dt = nullptr;
  int* d_lands = nullptr;
  int* d_active = nullptr;
  unsigned* d_status = nullptr;
  // stage scratch
  void* d_U1 = nullptr; void* d_V1 = nullptr; void* d_W1 = nullptr;
  void* d_U2 = nullptr; void* d_V2 = nullptr; void* d_W2 = nullptr;
  void* d_Vt0 = nullptr; void* d_Wt0 = nullptr;
  void* d_LX = nullptr; void* d_VT = nullptr;  // 2D: x-sweep results
  // adjoint scratch (FP64 Burgers / Euler contexts, allocated in create): the
  // adjoints of the stage-2 and stage-1 outputs, the base-term cotangents and
  // (2D) the x-sweep part, each m x points doubles per field
  double* d_adj = nullptr;
  // persistent run (1D, allocated in create)
  unsigned long long* d_next = nullptr;  // ticket counter, then done[batch], done3[batch]
  unsigned* d_done = nullptr;
  unsigned* d_done3 = nullptr;
  unsigned long long* d_palpha = nullptr;  // 2 x 3 x batch alpha slots
  int* d_inst_tiles = nullptr;  // tiles per instance of the current variant (alias)
  int persist_ctas = 0;          // resident CTAs of the current variant's persistent kernel
  int max_n = 0;  // largest instance (1D)
  int inject = 0;  // hweno_test_inject: 1 = the next persistent run waits in vain
  // pipelined host-buffer steps (1D batches, created in create): streams,
  // events and per-chunk counters
  static constexpr int kChunks = 8;
  cudaStream_t cs[kChunks] = {};
  cudaEvent_t ce[kChunks] = {};
  cudaEvent_t ce0 = nullptr;
  int* d_chunk_active = nullptr;
  // device copies for the host-buffer entry point
  void* d_hU = nullptr; void* d_hV = nullptr; void* d_hW = nullptr;
  double* d_ht = nullptr;
  int launches = 0;
  int step_launches = 0;  // kernels per step of this context
  // point-update counter of hweno_run (device) and its recorded graph
  unsigned long long* d_pu = nullptr;
  double* d_partial = nullptr;  // per-tile partial sums of hweno_totals
  int ntiles_tot = 0;
  cudaGraphExec_t graph = nullptr;
  void* g_U = nullptr; void* g_V = nullptr; void* g_W = nullptr;
  double* g_t = nullptr;
  double g_tend = 0.0;
  int g_k = 0;
  bool capturing = false;
  cudaEvent_t tune_ev[2] = {};  // hweno_autotune's timing events
  // kernel timing (hweno_profile_start / hweno_profile_read)
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_kind;
  int ev_used = 0;
  std::string err;
};

namespace {

int fail(hweno_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(hweno_ctx* c, cudaError_t e, const char* what) {
  return fail(c, HWENO_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool weights_ok(const double* w) {
  return w[0] >= kWeightMin && w[1] >= kWeightMin && w[2] >= kWeightMin &&
         std::fabs(w[0] + w[1] + w[2] - 1.0) <= 1e-12;
}

int check_options(const hweno_options* o, std::string& why) {
  if (!weights_ok(o->lin_w)) { why = "lin_w must be >= 1e-6 each and sum to 1"; return HWENO_EINVAL; }
  if (!weights_ok(o->lim_d)) { why = "lim_d must be >= 1e-6 each and sum to 1"; return HWENO_EINVAL; }
  if (!(o->eps >= kEpsMin && o->eps <= kEpsMax)) { why = "eps must lie in [1e-20, 1e6]"; return HWENO_EINVAL; }
  if (!(o->cfl > 0)) { why = "cfl must be > 0"; return HWENO_EINVAL; }
  if (o->dt_mode < 0 || o->dt_mode > 2) { why = "dt_mode must be 0, 1 or 2"; return HWENO_EINVAL; }
  if (o->dt_mode == 2 && !(o->dt_fixed > 0)) { why = "dt_fixed must be > 0"; return HWENO_EINVAL; }
  if (o->limiter < 0 || o->limiter > 2) { why = "limiter must be 0, 1 or 2"; return HWENO_EINVAL; }
  if (o->eig_avg < 0 || o->eig_avg > 1) { why = "eig_avg must be 0 or 1"; return HWENO_EINVAL; }
  if (o->fused_small < 0 || o->fused_small > 2) { why = "fused_small must be 0, 1 or 2"; return HWENO_EINVAL; }
  if (o->adj_frozen_weights < 0 || o->adj_frozen_weights > 1) {
    why = "adj_frozen_weights must be 0 or 1";
    return HWENO_EINVAL;
  }
  if (o->fused_2d < 0 || o->fused_2d > 1) {
    why = "fused_2d must be 0 or 1";
    return HWENO_EINVAL;
  }
  if (o->tile_variant < 0 || o->tile_variant >= kNumVariants1D) {
    why = "tile_variant out of range";
    return HWENO_EINVAL;
  }
  return HWENO_OK;
}

bool bc_ok_1d(int b) { return b >= HWENO_BC_PERIODIC && b <= HWENO_BC_INFLOW; }

// Adjoint scratch (hweno_adjoint_step), allocated in create for the contexts
// the adjoint is built for (FP64 Burgers and Euler). Fields: 0-2 lambda of
// the stage-2 output (U, V, W), 3-5 of the stage-1 output, 6-8 the base-term
// cotangents, 9-11 the 2D x-sweep part (of U, V and W); each m x points
// doubles. 1D has no W fields and no x-sweep part, so its six fields are
// stored back to back.
bool adjoint_applies(const hweno_ctx* c) { return !c->fp32 && c->eq != HWENO_BUCKLEY; }
int adjoint_fields(const hweno_ctx* c) { return c->dim == 2 ? 12 : 6; }
size_t adjoint_scratch_bytes(const hweno_ctx* c) {
  return sizeof(double) * (size_t)c->m * (size_t)c->npts * (size_t)adjoint_fields(c);
}

template <class T>
int dalloc(hweno_ctx* c, T** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(c, e == cudaErrorMemoryAllocation ? HWENO_ENOMEM : HWENO_ECUDA,
                std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return HWENO_OK;
}

void free_all(hweno_ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  void* ptrs[] = {c->d_pu, c->d_partial, c->d_inst_n, c->d_inst_off, c->d_inst_dx,
                  c->d_hx[0], c->d_hx[1], c->d_inst_geo, c->d_inst_geof, c->d_alpha, c->d_dt,
                  c->d_lands, c->d_active, c->d_status,
                  c->d_U1, c->d_V1, c->d_W1, c->d_U2, c->d_V2, c->d_W2, c->d_Vt0, c->d_Wt0,
                  c->d_LX, c->d_VT, c->d_hU, c->d_hV, c->d_hW, c->d_ht,
                  c->d_adj, c->d_next, c->d_palpha, c->d_chunk_active};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int v = 0; v < kNumVariants1D; ++v) {
    void* vp[] = {c->d_vt_inst[v], c->d_vt_start[v], c->d_vt_tiles[v], c->d_ct_inst[v],
                  c->d_ct_start[v]};
    for (void* p : vp)
      if (p) cudaFree(p);
    c->d_vt_inst[v] = c->d_vt_start[v] = c->d_vt_tiles[v] = nullptr;
    c->d_ct_inst[v] = c->d_ct_start[v] = nullptr;
  }
  for (int i = 0; i < hweno_ctx::kChunks; ++i) {
    if (c->cs[i]) cudaStreamDestroy(c->cs[i]);
    if (c->ce[i]) cudaEventDestroy(c->ce[i]);
    c->cs[i] = nullptr;
    c->ce[i] = nullptr;
  }
  if (c->ce0) cudaEventDestroy(c->ce0);
  c->ce0 = nullptr;
  for (cudaEvent_t& ev : c->tune_ev) {
    if (ev) cudaEventDestroy(ev);
    ev = nullptr;
  }
}

// Buckley-Leverett alpha over the admissible states (Example 3.4): with
// D = 5u^2 - 2u + 1, f'(u) = 8u(1 - u)/D^2 vanishes at u = 0 and u = 1 and
// peaks where its derivative, proportional to 10u^3 - 15u^2 + 1, vanishes in
// (0, 1/2); the root is bracketed by the sign change and bisected.
double buckley_alpha01() {
  static const double value = [] {
    double lo = 0.0, hi = 0.5;  // cubic: +1 at 0, -1.5 at 1/2
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (10.0 * mid * mid * mid - 15.0 * mid * mid + 1.0 > 0.0) lo = mid;
      else hi = mid;
    }
    const double u = 0.5 * (lo + hi), D = 5.0 * u * u - 2.0 * u + 1.0;
    return 8.0 * u * (1.0 - u) / (D * D);
  }();
  return value;
}

SchemeParams scheme_params(const hweno_ctx* c) {
  SchemeParams sp{};
  for (int i = 0; i < 3; ++i) { sp.lin_w[i] = c->opt.lin_w[i]; sp.lim_d[i] = c->opt.lim_d[i]; }
  sp.eps = c->opt.eps;
  sp.cfl = c->opt.cfl;
  sp.dt_fixed = c->opt.dt_fixed;
  sp.dt_mode = c->opt.dt_mode;
  sp.limiter = c->opt.limiter;
  sp.eig_avg = c->opt.eig_avg;
  sp.adj_frozen = c->opt.adj_frozen_weights;
  sp.gas_gamma = c->gamma;
  sp.bc[0] = c->bc.xlo; sp.bc[1] = c->bc.xhi; sp.bc[2] = c->bc.ylo; sp.bc[3] = c->bc.yhi;
  for (int i = 0; i < 4; ++i) {
    sp.inflow[i] = c->bc.inflow[i];
    sp.pre[i] = c->bc.pre[i];
    sp.inflowf[i] = (float)c->bc.inflow[i];
    sp.pref[i] = (float)c->bc.pre[i];
  }
  sp.dmr_x0 = c->bc.dmr_x0;
  sp.dmr_speed = c->bc.dmr_speed;
  sp.dmr_angle = c->bc.dmr_angle;
  sp.dmr_tan = std::tan(c->bc.dmr_angle);
  sp.dmr_sin = std::sin(c->bc.dmr_angle);
  fill_constant_table(sp, c->opt.lin_w, c->opt.lim_d, c->opt.eps, c->gamma,
                      c->eq == HWENO_BUCKLEY ? buckley_alpha01() : 0.0);
  return sp;
}

// Tile table of a 1D batch for tiles of `tile` points: (instance, first point)
// per CTA, instances in order.
void tile_table(const std::vector<int>& nx, int tile, std::vector<int>& tinst,
                std::vector<int>& tstart) {
  tinst.clear();
  tstart.clear();
  for (size_t k = 0; k < nx.size(); ++k)
    for (int s = 0; s < nx[k]; s += tile) { tinst.push_back((int)k); tstart.push_back(s); }
}

// Make the tables of variant v (1D, made in create) current and size the
// persistent grid for it. A graph recorded by hweno_run for another variant
// is dropped (it holds the old launch shapes). No device memory is written.
int use_variant(hweno_ctx* c, int v) {
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) ||
      (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
    return cuda_fail(c, e, "device attributes");
  const int per_sm = run_1d_ctas_per_sm(c->eq, c->fp32, v);
  if (per_sm < 1) return fail(c, HWENO_ECUDA, "persistent kernel does not fit on an SM");
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  c->mixed = false;
  c->variant = v;
  c->tile = tile_points(v);
  c->d_tile_inst = c->d_vt_inst[v];
  c->d_tile_start = c->d_vt_start[v];
  c->d_inst_tiles = c->d_vt_tiles[v];
  c->ntiles = c->vt_ntiles[v];
  c->persist_ctas = sms * per_sm;
  return HWENO_OK;
}

// Size classes of a 1D batch: the distinct instance sizes when there are at
// most HWENO_MAX_SIZE_CLASSES of them, else octaves of the size (log2
// buckets above the smallest instance, the last bucket open-ended).
void size_classes(hweno_ctx* c) {
  std::vector<int> d(c->nx);
  std::sort(d.begin(), d.end());
  d.erase(std::unique(d.begin(), d.end()), d.end());
  c->inst_class.assign(c->batch, 0);
  if ((int)d.size() <= HWENO_MAX_SIZE_CLASSES) {
    c->nclasses = (int)d.size();
    for (int k = 0; k < c->batch; ++k)
      c->inst_class[k] = (int)(std::lower_bound(d.begin(), d.end(), c->nx[k]) - d.begin());
  } else {
    const int lo = d.front();
    int top = 0;
    for (int k = 0; k < c->batch; ++k) {
      int q = 0;
      while (q + 1 < HWENO_MAX_SIZE_CLASSES && (long long)lo << (q + 1) <= c->nx[k]) ++q;
      c->inst_class[k] = q;
      top = std::max(top, q);
    }
    c->nclasses = top + 1;
  }
  c->class_lo.assign(c->nclasses, 1 << 30);
  c->class_hi.assign(c->nclasses, 0);
  for (int k = 0; k < c->batch; ++k) {
    const int q = c->inst_class[k];
    c->class_lo[q] = std::min(c->class_lo[q], c->nx[k]);
    c->class_hi[q] = std::max(c->class_hi[q], c->nx[k]);
  }
}

// Tile table of variant-size tiles ordered by size class (instances in
// order within a class); first[q] = first tile of class q.
void class_tile_table(const hweno_ctx* c, int tile, std::vector<int>& tinst,
                      std::vector<int>& tstart, int* first) {
  tinst.clear();
  tstart.clear();
  for (int q = 0; q < c->nclasses; ++q) {
    first[q] = (int)tinst.size();
    for (int k = 0; k < c->batch; ++k)
      if (c->inst_class[k] == q)
        for (int s = 0; s < c->nx[k]; s += tile) { tinst.push_back(k); tstart.push_back(s); }
  }
  first[c->nclasses] = (int)tinst.size();
}

// One stage of every instance: one launch of the current variant, or (after
// hweno_autotune_classes) one launch per run of size classes that chose the
// same variant, over that run's tiles of the class-ordered table.
cudaError_t launch_stage_all(hweno_ctx* c, int mode, const Args1D& a, cudaStream_t s,
                             int* launches) {
  if (!c->mixed) {
    ++*launches;
    return launch_stage_1d(c->eq, c->fp32, c->variant, mode, a, c->ntiles, s);
  }
  for (int q = 0; q < c->nclasses;) {
    const int v = c->class_variant[q];
    int q1 = q + 1;
    while (q1 < c->nclasses && c->class_variant[q1] == v) ++q1;
    const int t0 = c->ct_first[v][q], t1 = c->ct_first[v][q1];
    if (t1 > t0) {
      Args1D b = a;
      b.tile_inst = c->d_ct_inst[v] + t0;
      b.tile_start = c->d_ct_start[v] + t0;
      ++*launches;
      if (const cudaError_t e = launch_stage_1d(c->eq, c->fp32, v, mode, b, t1 - t0, s)) return e;
    }
    q = q1;
  }
  return cudaSuccess;
}

// Per-instance h of the time-step rule: dx (dt_mode 0, 2) or dx^{5/3}
// (dt_mode 1), both made in create.
void select_hx(hweno_ctx* c) { c->d_inst_hx = c->d_hx[c->opt.dt_mode == 1 ? 1 : 0]; }

Args1D base_args_1d(const hweno_ctx* c) {
  Args1D a{};
  a.tile_inst = c->d_tile_inst;
  a.tile_start = c->d_tile_start;
  a.inst_n = c->d_inst_n;
  a.inst_off = c->d_inst_off;
  a.inst_dx = c->d_inst_dx;
  a.inst_hx = c->d_inst_hx;
  a.inst_geo = c->d_inst_geo;
  a.inst_geof = c->d_inst_geof;
  a.status = c->d_status;
  a.sp = scheme_params(c);
  return a;
}

// Event bracket around one launch when profiling is on (kind 0 alpha, 1 stage,
// 2 finalize).
void prof_begin(hweno_ctx* c, cudaStream_t s) {
  if (!c->capturing && c->ev_used + 2 <= (int)c->ev.size()) cudaEventRecord(c->ev[c->ev_used], s);
}
void prof_end(hweno_ctx* c, cudaStream_t s, int kind) {
  if (!c->capturing && c->ev_used + 2 <= (int)c->ev.size()) {
    cudaEventRecord(c->ev[c->ev_used + 1], s);
    c->ev_kind[c->ev_used / 2] = kind;
    c->ev_used += 2;
  }
}

void destroy_events(hweno_ctx* c) {
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  c->ev.clear();
  c->ev_kind.clear();
  c->ev_used = 0;
}

unsigned long long* slot(hweno_ctx* c, int k) { return c->d_alpha + (size_t)k * c->batch; }
const double* slotd(hweno_ctx* c, int k) {
  return reinterpret_cast<const double*>(c->d_alpha + (size_t)k * c->batch);
}

// One step of the instances [k0, k1) (tiles [t0, t1) of the current tile
// table), counting the instances still active into *active. Instances
// outside the range are not touched.
int step_1d_range(hweno_ctx* c, void* U, void* V, double* t, double t_end, double* dt_used,
                  cudaStream_t s, int k0, int k1, int t0, int t1, int* active) {
  cudaError_t e;
  const size_t nk = (size_t)(k1 - k0);
  for (int j = 0; j < 3; ++j)
    if ((e = cudaMemsetAsync(slot(c, j) + k0, 0, sizeof(unsigned long long) * nk, s)))
      return cuda_fail(c, e, "memset");
  Args1D a = base_args_1d(c);
  a.tile_inst += t0;
  a.tile_start += t0;
  const int nt = t1 - t0;
  a.t = t;
  a.t_end = t_end;
  a.skip_done = 1;
  a.dt = c->d_dt;
  a.lands = c->d_lands;
  a.U = U;
  a.alpha_out = slot(c, 0);
  if ((e = launch_alpha_1d(c->eq, c->fp32, c->variant, a, nt, s))) return cuda_fail(c, e, "alpha");
  a.V = V; a.Uout = c->d_U1; a.Vout = c->d_V1; a.Vt0out = c->d_Vt0;
  a.alpha_in = slotd(c, 0); a.alpha_out = slot(c, 1);
  if ((e = launch_stage_1d(c->eq, c->fp32, c->variant, MODE_STAGE1, a, nt, s)))
    return cuda_fail(c, e, "stage 1");
  a.U = c->d_U1; a.V = c->d_V1; a.U0 = U; a.Vt0 = c->d_Vt0; a.Uout = c->d_U2; a.Vout = c->d_V2;
  a.Vt0out = nullptr;
  a.alpha_in = slotd(c, 1); a.alpha_out = slot(c, 2);
  if ((e = launch_stage_1d(c->eq, c->fp32, c->variant, MODE_STAGE2, a, nt, s)))
    return cuda_fail(c, e, "stage 2");
  a.U = c->d_U2; a.V = c->d_V2; a.U0 = U; a.Vt0 = c->d_Vt0; a.Uout = U; a.Vout = V;
  a.alpha_in = slotd(c, 2); a.alpha_out = nullptr;
  if ((e = launch_stage_1d(c->eq, c->fp32, c->variant, MODE_STAGE3, a, nt, s)))
    return cuda_fail(c, e, "stage 3");
  if ((e = launch_finalize((int)nk, c->d_dt + k0, c->d_lands + k0, t + k0, t_end,
                           dt_used ? dt_used + k0 : nullptr, slotd(c, 0) + k0, active,
                           c->d_status, c->d_inst_n + k0, 1, c->d_pu, s)))
    return cuda_fail(c, e, "finalize");
  return HWENO_OK;
}

int step_1d(hweno_ctx* c, void* U, void* V, double* t, double t_end, double* dt_used,
            cudaStream_t s) {
  cudaError_t e;
  const bool cluster = c->opt.fused_small == 2 && c->max_n <= kClusterMax * kTile1D;
  if ((c->opt.fused_small == 1 && c->max_n <= kFusedPoints) || cluster) {  // one launch per step
    if ((e = cudaMemsetAsync(c->d_active, 0, sizeof(int), s))) return cuda_fail(c, e, "memset");
    Args1D a = base_args_1d(c);
    a.t = t;
    a.t_end = t_end;
    a.skip_done = 1;
    a.dt = c->d_dt;
    a.lands = c->d_lands;
    a.U = U;
    a.V = V;
    FusedArgs f{};
    f.U1 = c->d_U1; f.V1 = c->d_V1; f.U2 = c->d_U2; f.V2 = c->d_V2; f.Vt0 = c->d_Vt0;
    f.alpha = c->d_alpha; f.dt_used = dt_used; f.active = c->d_active; f.pu = c->d_pu;
    f.batch = c->batch;
    prof_begin(c, s);
    bool launched = true;
    if (cluster) {
      e = launch_step_cluster_1d(c->eq, c->fp32, a, f, (int)c->max_n, s);
      if (e == cudaErrorNotSupported) launched = false;  // no such cluster here: tiled kernels
      else if (e) return cuda_fail(c, e, "cluster step");
    } else if ((e = launch_step_small_1d(c->eq, c->fp32, a, f, s))) {
      return cuda_fail(c, e, "fused step");
    }
    if (launched) {
      prof_end(c, s, 1);
      c->launches = c->step_launches = 1;
      return HWENO_OK;
    }
  }
  if ((e = cudaMemsetAsync(c->d_alpha, 0, sizeof(unsigned long long) * 3 * c->batch, s)) ||
      (e = cudaMemsetAsync(c->d_active, 0, sizeof(int), s)))
    return cuda_fail(c, e, "memset");
  Args1D a = base_args_1d(c);
  a.t = t;
  a.t_end = t_end;
  a.skip_done = 1;
  a.dt = c->d_dt;
  a.lands = c->d_lands;
  // alpha(U^n)
  a.U = U;
  a.alpha_out = slot(c, 0);
  prof_begin(c, s);
  if ((e = launch_alpha_1d(c->eq, c->fp32, c->variant, a, c->ntiles, s)))
    return cuda_fail(c, e, "alpha");
  prof_end(c, s, 0);
  int nl = 2;  // alpha and finalize
  // stage 1
  a.U = U; a.V = V; a.Uout = c->d_U1; a.Vout = c->d_V1; a.Vt0out = c->d_Vt0;
  a.alpha_in = slotd(c, 0); a.alpha_out = slot(c, 1);
  prof_begin(c, s);
  if ((e = launch_stage_all(c, MODE_STAGE1, a, s, &nl))) return cuda_fail(c, e, "stage 1");
  prof_end(c, s, 1);
  // stage 2
  a.U = c->d_U1; a.V = c->d_V1; a.U0 = U; a.Vt0 = c->d_Vt0; a.Uout = c->d_U2; a.Vout = c->d_V2;
  a.Vt0out = nullptr;
  a.alpha_in = slotd(c, 1); a.alpha_out = slot(c, 2);
  prof_begin(c, s);
  if ((e = launch_stage_all(c, MODE_STAGE2, a, s, &nl))) return cuda_fail(c, e, "stage 2");
  prof_end(c, s, 1);
  // stage 3 (in place)
  a.U = c->d_U2; a.V = c->d_V2; a.U0 = U; a.Vt0 = c->d_Vt0; a.Uout = U; a.Vout = V;
  a.alpha_in = slotd(c, 2); a.alpha_out = nullptr;
  prof_begin(c, s);
  if ((e = launch_stage_all(c, MODE_STAGE3, a, s, &nl))) return cuda_fail(c, e, "stage 3");
  prof_end(c, s, 1);
  prof_begin(c, s);
  if ((e = launch_finalize(c->batch, c->d_dt, c->d_lands, t, t_end, dt_used, slotd(c, 0),
                           c->d_active, c->d_status, c->d_inst_n, 1, c->d_pu, s)))
    return cuda_fail(c, e, "finalize");
  prof_end(c, s, 2);
  c->launches = c->step_launches = nl;
  return HWENO_OK;
}

double step_h(const hweno_ctx* c, double h) {
  return c->opt.dt_mode == 1 ? std::pow(h, 5.0 / 3.0) : h;
}

Args2D base_args_2d(const hweno_ctx* c) {
  Args2D a{};
  a.nx = c->nx[0];
  a.ny = c->ny;
  a.dx = (c->x1 - c->x0) / c->nx[0];
  a.dy = (c->y1 - c->y0) / c->ny;
  a.hx = step_h(c, a.dx);
  a.hy = step_h(c, a.dy);
  const double geo[6] = {a.dx, 1.0 / a.dx, 1.0 / (a.dx * a.dx), a.dy, 1.0 / a.dy,
                         1.0 / (a.dy * a.dy)};
  for (int i = 0; i < 6; ++i) { a.geod[i] = geo[i]; a.geof[i] = (float)geo[i]; }
  a.x0 = c->x0;
  a.y0 = c->y0;
  a.status = c->d_status;
  a.dt = c->d_dt;
  a.lands = c->d_lands;
  a.LX = c->d_LX;
  a.sp = scheme_params(c);
  return a;
}

// One stage of a 2D step: an x-sweep (x parts of L and v~ into scratch) and
// a y-sweep (y parts, w~, RK combination, next alpha), or the fused stage
// kernel (fused_2d); each launch bracketed for hweno_profile_*.
cudaError_t stage_2d(hweno_ctx* c, int mode, const Args2D& a, cudaStream_t s) {
  cudaError_t e;
  if (c->opt.fused_2d) {
    prof_begin(c, s);
    if ((e = launch_stage_fused_2d(c->eq, c->fp32, mode, a, s))) return e;
    prof_end(c, s, 1);
    return cudaSuccess;
  }
  prof_begin(c, s);
  if ((e = launch_xsweep_2d(c->eq, c->fp32, mode, a, s))) return e;
  prof_end(c, s, 1);
  prof_begin(c, s);
  if ((e = launch_ysweep_2d(c->eq, c->fp32, mode, a, s))) return e;
  prof_end(c, s, 1);
  return cudaSuccess;
}

// One SSP-RK3 step in 2D: alpha(U^n); per stage the x and y parts.
int step_2d(hweno_ctx* c, void* U, void* V, void* W, double* t, double t_end, double* dt_used,
            cudaStream_t s) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(c->d_alpha, 0, sizeof(unsigned long long) * 6, s)) ||
      (e = cudaMemsetAsync(c->d_active, 0, sizeof(int), s)))
    return cuda_fail(c, e, "memset");
  Args2D a = base_args_2d(c);
  a.t = t;
  a.t_end = t_end;
  a.skip_done = 1;
  a.U = U;
  a.alpha_out = c->d_alpha;
  prof_begin(c, s);
  if ((e = launch_alpha_2d(c->eq, c->fp32, a, s))) return cuda_fail(c, e, "alpha");
  prof_end(c, s, 0);
  struct Stage { const void *u, *v, *w; void *uo, *vo, *wo, *vt; int slot_in; double sc; };
  const Stage st[3] = {
      {U, V, W, c->d_U1, c->d_V1, c->d_W1, c->d_Vt0, 0, 0.0},
      {c->d_U1, c->d_V1, c->d_W1, c->d_U2, c->d_V2, c->d_W2, c->d_VT, 1, 1.0},
      {c->d_U2, c->d_V2, c->d_W2, U, V, W, c->d_VT, 2, 0.5}};
  for (int k = 0; k < 3; ++k) {
    const int mode = MODE_STAGE1 + k;
    a.U = st[k].u; a.V = st[k].v; a.W = st[k].w;
    a.U0 = U; a.Vt0 = c->d_Vt0; a.Wt0 = c->d_Wt0;
    a.Uout = st[k].uo; a.Vout = st[k].vo; a.Wout = st[k].wo;
    a.Wt0out = k == 0 ? c->d_Wt0 : nullptr;
    a.VT = st[k].vt;
    a.stage_c = st[k].sc;
    a.alpha_in = reinterpret_cast<const double*>(c->d_alpha + 2 * st[k].slot_in);
    a.alpha_out = k < 2 ? c->d_alpha + 2 * (k + 1) : nullptr;
    if ((e = stage_2d(c, mode, a, s))) return cuda_fail(c, e, "stage");
  }
  prof_begin(c, s);
  if ((e = launch_finalize(1, c->d_dt, c->d_lands, t, t_end, dt_used,
                           reinterpret_cast<const double*>(c->d_alpha), c->d_active,
                           c->d_status, c->d_inst_n, c->ny, c->d_pu, s)))
    return cuda_fail(c, e, "finalize");
  prof_end(c, s, 2);
  c->launches = c->step_launches = c->opt.fused_2d ? 5 : 8;
  return HWENO_OK;
}

int rhs_2d(hweno_ctx* c, const void* U, const void* V, const void* W, void* dU, void* dV,
           void* dW, void* Vlim, void* Wlim, const double* t, cudaStream_t s) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(c->d_alpha, 0, sizeof(unsigned long long) * 2, s)))
    return cuda_fail(c, e, "memset");
  Args2D a = base_args_2d(c);
  a.t = t;
  a.t_end = 0.0;
  a.skip_done = 0;
  a.U = U; a.V = V; a.W = W;
  a.alpha_out = c->d_alpha;
  prof_begin(c, s);
  if ((e = launch_alpha_2d(c->eq, c->fp32, a, s))) return cuda_fail(c, e, "alpha");
  prof_end(c, s, 0);
  a.alpha_in = reinterpret_cast<const double*>(c->d_alpha);
  a.alpha_out = nullptr;
  a.VT = Vlim ? Vlim : c->d_VT;
  a.L1 = dU; a.L2 = dV; a.L3 = dW; a.Wlim = Wlim;
  a.stage_c = 0.0;
  prof_begin(c, s);
  if ((e = launch_xsweep_2d(c->eq, c->fp32, MODE_RHS, a, s))) return cuda_fail(c, e, "x-sweep");
  prof_end(c, s, 1);
  prof_begin(c, s);
  if ((e = launch_ysweep_2d(c->eq, c->fp32, MODE_RHS, a, s))) return cuda_fail(c, e, "y-sweep");
  prof_end(c, s, 1);
  c->launches = 3;
  return HWENO_OK;
}

int rhs_1d(hweno_ctx* c, const void* U, const void* V, void* dU, void* dV, void* Vlim,
           const double* t, cudaStream_t s) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(c->d_alpha, 0, sizeof(unsigned long long) * c->batch, s)))
    return cuda_fail(c, e, "memset");
  Args1D a = base_args_1d(c);
  a.t = t;
  a.t_end = 0.0;
  a.skip_done = 0;
  a.U = U;
  a.alpha_out = slot(c, 0);
  prof_begin(c, s);
  if ((e = launch_alpha_1d(c->eq, c->fp32, c->variant, a, c->ntiles, s)))
    return cuda_fail(c, e, "alpha");
  prof_end(c, s, 0);
  a.V = V; a.L1 = dU; a.L2 = dV; a.Vlim = Vlim;
  a.alpha_in = slotd(c, 0); a.alpha_out = nullptr;
  prof_begin(c, s);
  if ((e = launch_stage_1d(c->eq, c->fp32, c->variant, MODE_RHS, a, c->ntiles, s)))
    return cuda_fail(c, e, "rhs");
  prof_end(c, s, 1);
  c->launches = 2;
  return HWENO_OK;
}

}  // namespace

extern "C" {

int hweno_default_options(hweno_options* o) {
  if (!o) return HWENO_EINVAL;
  std::memset(o, 0, sizeof *o);
  o->lin_w[0] = 0.98; o->lin_w[1] = 0.01; o->lin_w[2] = 0.01;
  o->lim_d[0] = 0.98; o->lim_d[1] = 0.01; o->lim_d[2] = 0.01;
  o->eps = 1e-6;
  o->cfl = 0.6;
  o->dt_mode = 0;
  o->dt_fixed = 0.0;
  o->limiter = 1;
  o->eig_avg = 0;
  o->tile_variant = 0;
  o->fused_small = 0;
  return HWENO_OK;
}

int hweno_create(hweno_ctx** out, int equation, const hweno_grid* grid, double gamma,
                 const hweno_bc* bc) {
  if (!out) return HWENO_EINVAL;
  *out = nullptr;
  if (!grid || !bc) return HWENO_EINVAL;
  hweno_ctx* c = new (std::nothrow) hweno_ctx();
  if (!c) return HWENO_ENOMEM;
  auto bad = [&](const char* why) {
    delete c;
    (void)why;
    return HWENO_EINVAL;
  };
  if (equation != HWENO_BURGERS && equation != HWENO_EULER && equation != HWENO_BUCKLEY)
    return bad("equation");
  if (equation == HWENO_BUCKLEY &&
      (grid->dim != 1 || bc->xlo == HWENO_BC_REFLECTIVE || bc->xhi == HWENO_BC_REFLECTIVE))
    return bad("Buckley-Leverett: 1D, no reflective walls");
  if (grid->dim != 1 && grid->dim != 2) return bad("dim");
  if (grid->precision != HWENO_FP64 && grid->precision != HWENO_FP32) return bad("precision");
  if (!(grid->x1 > grid->x0)) return bad("x range");
  if (grid->batch < 1) return bad("batch");
  if (grid->dim == 2 && (grid->batch != 1 || !(grid->y1 > grid->y0) || grid->ny < 4))
    return bad("2D grid");
  if (equation == HWENO_EULER && !(gamma > 1.0)) return bad("gamma");
  c->eq = equation;
  c->dim = grid->dim;
  c->m = equation == HWENO_EULER ? (grid->dim == 1 ? 3 : 4) : 1;
  c->batch = grid->batch;
  c->fp32 = grid->precision == HWENO_FP32;
  c->esize = c->fp32 ? 4 : 8;
  c->ny = grid->dim == 2 ? grid->ny : 1;
  c->x0 = grid->x0; c->x1 = grid->x1; c->y0 = grid->y0; c->y1 = grid->y1;
  c->gamma = gamma;
  c->bc = *bc;
  hweno_default_options(&c->opt);
  c->nx.resize(c->batch);
  for (int k = 0; k < c->batch; ++k) {
    c->nx[k] = grid->nx_per_instance ? grid->nx_per_instance[k] : grid->nx;
    if (c->nx[k] < 4) return bad("nx < 4");
    c->max_n = std::max(c->max_n, c->nx[k]);
  }
  // boundary conditions
  const int sides[4] = {bc->xlo, bc->xhi, bc->ylo, bc->yhi};
  if (grid->dim == 1) {
    if (!bc_ok_1d(bc->xlo) || !bc_ok_1d(bc->xhi)) return bad("bc");
    if ((bc->xlo == HWENO_BC_PERIODIC) != (bc->xhi == HWENO_BC_PERIODIC)) return bad("periodic");
  } else {
    for (int i = 0; i < 4; ++i)
      if (sides[i] < HWENO_BC_PERIODIC || sides[i] > HWENO_BC_DMR_TOP) return bad("bc");
    if (bc->xlo >= HWENO_BC_DMR_BOTTOM || bc->xhi >= HWENO_BC_DMR_BOTTOM) return bad("bc x");
    if (bc->ylo == HWENO_BC_DMR_TOP || bc->yhi == HWENO_BC_DMR_BOTTOM) return bad("bc dmr side");
    if ((bc->xlo == HWENO_BC_PERIODIC) != (bc->xhi == HWENO_BC_PERIODIC)) return bad("periodic x");
    if ((bc->ylo == HWENO_BC_PERIODIC) != (bc->yhi == HWENO_BC_PERIODIC)) return bad("periodic y");
    if ((bc->ylo == HWENO_BC_DMR_BOTTOM || bc->yhi == HWENO_BC_DMR_TOP) &&
        (equation != HWENO_EULER || !(std::sin(bc->dmr_angle) > 0) || !(std::tan(bc->dmr_angle) > 0)))
      return bad("dmr");
  }
  // sizes and tile tables: every 1D variant's table; 2D one entry
  std::vector<long long> off(c->batch);
  c->inst_dx.resize(c->batch);
  long long acc = 0;
  for (int k = 0; k < c->batch; ++k) {
    off[k] = acc;
    acc += c->nx[k];
    c->inst_dx[k] = (c->x1 - c->x0) / c->nx[k];
  }
  const int nvar = grid->dim == 1 ? kNumVariants1D : 1;
  std::vector<int> tinst[kNumVariants1D], tstart[kNumVariants1D], ntk[kNumVariants1D];
  std::vector<int> cinst[kNumVariants1D], cstart[kNumVariants1D];
  if (grid->dim == 1) size_classes(c);
  for (int v = 0; v < nvar; ++v) {
    if (grid->dim == 1) {
      const int tp = tile_points(v);
      tile_table(c->nx, tp, tinst[v], tstart[v]);
      for (int k = 0; k < c->batch; ++k) ntk[v].push_back((c->nx[k] + tp - 1) / tp);
      class_tile_table(c, tp, cinst[v], cstart[v], c->ct_first[v]);
    } else {
      tinst[v] = {0};
      tstart[v] = {0};
      ntk[v] = {1};
    }
    c->vt_ntiles[v] = (int)tinst[v].size();
    c->tiles_cap = std::max(c->tiles_cap, c->vt_ntiles[v]);
  }
  if (grid->dim == 2) acc = (long long)c->nx[0] * c->ny;
  c->npts = acc;
  c->elems = (size_t)c->m * (size_t)acc;
  c->ntiles_tot = grid->dim == 1 ? c->tiles_cap
                                 : ((c->nx[0] + kTileX2D - 1) / kTileX2D) * c->ny;

  int rc = HWENO_OK;
  const size_t fb = c->elems * c->esize;
  const size_t B = (size_t)c->batch;
  for (int v = 0; v < nvar && rc == HWENO_OK; ++v)
    if ((rc = dalloc(c, &c->d_vt_inst[v], sizeof(int) * tinst[v].size())) ||
        (rc = dalloc(c, &c->d_vt_start[v], sizeof(int) * tstart[v].size())) ||
        (rc = dalloc(c, &c->d_vt_tiles[v], sizeof(int) * ntk[v].size())) ||
        (grid->dim == 1 &&
         ((rc = dalloc(c, &c->d_ct_inst[v], sizeof(int) * cinst[v].size())) ||
          (rc = dalloc(c, &c->d_ct_start[v], sizeof(int) * cstart[v].size())))))
      break;
  if (rc != HWENO_OK ||
      (rc = dalloc(c, &c->d_inst_n, sizeof(int) * B)) ||
      (rc = dalloc(c, &c->d_inst_off, sizeof(long long) * B)) ||
      (rc = dalloc(c, &c->d_inst_dx, sizeof(double) * B)) ||
      (rc = dalloc(c, &c->d_hx[0], sizeof(double) * B)) ||
      (rc = dalloc(c, &c->d_hx[1], sizeof(double) * B)) ||
      (rc = dalloc(c, &c->d_inst_geo, sizeof(double) * 3 * B)) ||
      (rc = dalloc(c, &c->d_inst_geof, sizeof(float) * 3 * B)) ||
      (rc = dalloc(c, &c->d_alpha, sizeof(unsigned long long) * 3 * B * 2)) ||
      (rc = dalloc(c, &c->d_dt, sizeof(double) * B)) ||
      (rc = dalloc(c, &c->d_lands, sizeof(int) * B)) ||
      (rc = dalloc(c, &c->d_active, sizeof(int))) ||
      (rc = dalloc(c, &c->d_status, sizeof(unsigned))) ||
      (rc = dalloc(c, &c->d_pu, sizeof(unsigned long long))) ||
      (rc = dalloc(c, &c->d_partial, sizeof(double) * 4 * (size_t)c->ntiles_tot)) ||
      (rc = dalloc(c, &c->d_U1, fb)) || (rc = dalloc(c, &c->d_V1, fb)) ||
      (rc = dalloc(c, &c->d_U2, fb)) || (rc = dalloc(c, &c->d_V2, fb)) ||
      (rc = dalloc(c, &c->d_Vt0, fb)) || (rc = dalloc(c, &c->d_hU, fb)) ||
      (rc = dalloc(c, &c->d_hV, fb)) || (rc = dalloc(c, &c->d_ht, sizeof(double) * B)) ||
      (c->dim == 2 &&
       ((rc = dalloc(c, &c->d_W1, fb)) || (rc = dalloc(c, &c->d_W2, fb)) ||
        (rc = dalloc(c, &c->d_Wt0, fb)) || (rc = dalloc(c, &c->d_LX, 3 * fb)) ||
        (rc = dalloc(c, &c->d_VT, fb)) || (rc = dalloc(c, &c->d_hW, fb)))) ||
      (c->dim == 1 &&
       ((rc = dalloc(c, &c->d_next, sizeof(unsigned long long) + 2 * sizeof(unsigned) * B)) ||
        (rc = dalloc(c, &c->d_palpha, sizeof(unsigned long long) * 6 * B)) ||
        (rc = dalloc(c, &c->d_chunk_active, sizeof(int) * hweno_ctx::kChunks)))) ||
      (adjoint_applies(c) && (rc = dalloc(c, &c->d_adj, adjoint_scratch_bytes(c))))) {
    free_all(c);
    delete c;
    return rc;
  }
  if (c->dim == 1) {
    c->d_done = reinterpret_cast<unsigned*>(c->d_next + 1);
    c->d_done3 = c->d_done + B;
  }
#if defined(HWENO_CHECKS) && HWENO_CHECKS
  {  // checked builds: stage scratch starts as NaN, so that a read before a write shows
    struct Buf { void* p; size_t bytes; };
    const Buf bufs[] = {{c->d_U1, fb}, {c->d_V1, fb}, {c->d_U2, fb}, {c->d_V2, fb},
                        {c->d_Vt0, fb}, {c->d_hU, fb}, {c->d_hV, fb}, {c->d_W1, fb},
                        {c->d_W2, fb}, {c->d_Wt0, fb}, {c->d_LX, 3 * fb}, {c->d_VT, fb},
                        {c->d_hW, fb}, {c->d_dt, sizeof(double) * B},
                        {c->d_palpha, sizeof(unsigned long long) * 6 * B},
                        {c->d_alpha, sizeof(unsigned long long) * 6 * B},
                        {c->d_adj, c->d_adj ? adjoint_scratch_bytes(c) : 0}};
    for (const Buf& b : bufs)
      if (b.p && cudaMemset(b.p, 0xff, b.bytes) != cudaSuccess) {
        free_all(c);
        delete c;
        return HWENO_ECUDA;
      }
  }
#endif
  // events and (1D batches) the streams of the pipelined host-buffer step
  bool made = cudaEventCreate(&c->tune_ev[0]) == cudaSuccess &&
              cudaEventCreate(&c->tune_ev[1]) == cudaSuccess;
  if (made && c->dim == 1 && c->batch > 1) {
    made = cudaEventCreateWithFlags(&c->ce0, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < hweno_ctx::kChunks && made; ++i)
      made = cudaStreamCreateWithFlags(&c->cs[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&c->ce[i], cudaEventDisableTiming) == cudaSuccess;
  }
  if (!made) {
    free_all(c);
    delete c;
    return HWENO_ECUDA;
  }
  std::vector<double> geo(3 * B), hx53(B);
  std::vector<float> geof(3 * B);
  for (size_t k = 0; k < B; ++k) {
    const double d = c->inst_dx[k];
    const double g3[3] = {d, 1.0 / d, 1.0 / (d * d)};
    for (int i = 0; i < 3; ++i) { geo[3 * k + i] = g3[i]; geof[3 * k + i] = (float)g3[i]; }
    hx53[k] = std::pow(d, 5.0 / 3.0);
  }
  bool copy_failed = false;
  for (int v = 0; v < nvar && !copy_failed; ++v)
    copy_failed =
        cudaMemcpy(c->d_vt_inst[v], tinst[v].data(), sizeof(int) * tinst[v].size(),
                   cudaMemcpyHostToDevice) ||
        cudaMemcpy(c->d_vt_start[v], tstart[v].data(), sizeof(int) * tstart[v].size(),
                   cudaMemcpyHostToDevice) ||
        cudaMemcpy(c->d_vt_tiles[v], ntk[v].data(), sizeof(int) * ntk[v].size(),
                   cudaMemcpyHostToDevice) ||
        (grid->dim == 1 &&
         (cudaMemcpy(c->d_ct_inst[v], cinst[v].data(), sizeof(int) * cinst[v].size(),
                     cudaMemcpyHostToDevice) ||
          cudaMemcpy(c->d_ct_start[v], cstart[v].data(), sizeof(int) * cstart[v].size(),
                     cudaMemcpyHostToDevice)));
  copy_failed = copy_failed ||
      cudaMemcpy(c->d_inst_geo, geo.data(), sizeof(double) * 3 * B, cudaMemcpyHostToDevice) ||
      cudaMemcpy(c->d_inst_geof, geof.data(), sizeof(float) * 3 * B, cudaMemcpyHostToDevice) ||
      cudaMemcpy(c->d_inst_n, c->nx.data(), sizeof(int) * B, cudaMemcpyHostToDevice) ||
      cudaMemcpy(c->d_inst_off, off.data(), sizeof(long long) * B, cudaMemcpyHostToDevice) ||
      cudaMemcpy(c->d_inst_dx, c->inst_dx.data(), sizeof(double) * B, cudaMemcpyHostToDevice) ||
      cudaMemcpy(c->d_hx[0], c->inst_dx.data(), sizeof(double) * B, cudaMemcpyHostToDevice) ||
      cudaMemcpy(c->d_hx[1], hx53.data(), sizeof(double) * B, cudaMemcpyHostToDevice) ||
      cudaMemset(c->d_status, 0, sizeof(unsigned)) ||
      cudaMemset(c->d_pu, 0, sizeof(unsigned long long));
  if (copy_failed) {
    free_all(c);
    delete c;
    return HWENO_ECUDA;
  }
  // variant 0 (also the adjoint's table) and the paper's dt rule
  c->d_tile0_inst = c->d_tile_inst = c->d_vt_inst[0];
  c->d_tile0_start = c->d_tile_start = c->d_vt_start[0];
  c->d_inst_tiles = c->d_vt_tiles[0];
  c->ntiles0 = c->ntiles = c->vt_ntiles[0];
  select_hx(c);
  if (c->dim == 1 && (rc = use_variant(c, 0)) != HWENO_OK) {
    free_all(c);
    delete c;
    return rc;
  }
  *out = c;
  return HWENO_OK;
}

int hweno_set_options(hweno_ctx* c, const hweno_options* o) {
  if (!c || !o) return HWENO_EINVAL;
  std::string why;
  if (check_options(o, why) != HWENO_OK) return fail(c, HWENO_EINVAL, why);
  const hweno_options old = c->opt;
  c->opt = *o;
  int rc = HWENO_OK;
  if (c->dim == 1 && o->tile_variant != c->variant) rc = use_variant(c, o->tile_variant);
  if (rc != HWENO_OK) c->opt = old;
  select_hx(c);
  // a graph recorded by hweno_run holds the old scheme parameters
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  return rc;
}

int hweno_get_options(const hweno_ctx* c, hweno_options* out) {
  if (!c || !out) return HWENO_EINVAL;
  *out = c->opt;
  return HWENO_OK;
}

int hweno_rhs(hweno_ctx* c, const void* U, const void* V, const void* W, void* dU, void* dV,
              void* dW, void* Vlim, void* Wlim, const double* t, void* stream) {
  if (!c) return HWENO_EINVAL;
  if (!U || !V || !dU || !dV || !t) return fail(c, HWENO_EINVAL, "null array");
  if (c->dim == 1 && (W || dW || Wlim)) return fail(c, HWENO_EINVAL, "W given in 1D");
  if (c->dim == 2 && (!W || !dW)) return fail(c, HWENO_EINVAL, "W and dW required in 2D");
  c->err.clear();
  if (c->dim == 2)
    return rhs_2d(c, U, V, W, dU, dV, dW, Vlim, Wlim, t, static_cast<cudaStream_t>(stream));
  return rhs_1d(c, U, V, dU, dV, Vlim, t, static_cast<cudaStream_t>(stream));
}

int hweno_step(hweno_ctx* c, void* U, void* V, void* W, double* t, double t_end,
               double* dt_used, void* stream) {
  if (!c) return HWENO_EINVAL;
  if (!U || !V || !t) return fail(c, HWENO_EINVAL, "null array");
  if (c->dim == 1 && W) return fail(c, HWENO_EINVAL, "W given in 1D");
  if (c->dim == 2 && !W) return fail(c, HWENO_EINVAL, "W required in 2D");
  if (!std::isfinite(t_end)) return fail(c, HWENO_EINVAL, "t_end not finite");
  c->err.clear();
  if (c->dim == 2) return step_2d(c, U, V, W, t, t_end, dt_used, static_cast<cudaStream_t>(stream));
  return step_1d(c, U, V, t, t_end, dt_used, static_cast<cudaStream_t>(stream));
}

int hweno_run(hweno_ctx* c, void* U, void* V, void* W, double* t, double t_end,
              long long max_steps, int k, long long* steps_taken, long long* point_updates,
              void* stream) {
  if (!c) return HWENO_EINVAL;
  if (!stream) return fail(c, HWENO_EINVAL, "hweno_run needs a non-NULL stream");
  if (!U || !V || !t || k < 1 || max_steps < 0) return fail(c, HWENO_EINVAL, "bad argument");
  if ((c->dim == 1) != (W == nullptr)) return fail(c, HWENO_EINVAL, "W must be given iff 2D");
  if (!std::isfinite(t_end)) return fail(c, HWENO_EINVAL, "t_end not finite");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (!c->graph || c->g_U != U || c->g_V != V || c->g_W != W || c->g_t != t ||
      c->g_tend != t_end || c->g_k != k) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)))
      return cuda_fail(c, e, "cudaStreamBeginCapture");
    c->capturing = true;
    int rc = HWENO_OK;
    for (int i = 0; i < k && rc == HWENO_OK; ++i) rc = hweno_step(c, U, V, W, t, t_end, nullptr, stream);
    c->capturing = false;
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    if (rc != HWENO_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      c->graph = nullptr;
      return cuda_fail(c, e, "cudaGraphInstantiate");
    }
    c->g_U = U; c->g_V = V; c->g_W = W; c->g_t = t; c->g_tend = t_end; c->g_k = k;
  }
  if ((e = cudaMemsetAsync(c->d_pu, 0, sizeof(unsigned long long), s)))
    return cuda_fail(c, e, "memset");
  long long taken = 0;
  while (taken < max_steps) {
    if ((e = cudaGraphLaunch(c->graph, s))) return cuda_fail(c, e, "cudaGraphLaunch");
    taken += k;
    const int active = hweno_active_instances(c, stream);
    if (active < 0) return active;
    if (active == 0) break;
  }
  unsigned long long pu = 0;
  if ((e = cudaMemcpyAsync(&pu, c->d_pu, sizeof pu, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaStreamSynchronize(s)))
    return cuda_fail(c, e, "read point updates");
  if (steps_taken) *steps_taken = taken;
  if (point_updates) *point_updates = (long long)pu;
  c->launches = (int)std::min<long long>(2147483647LL, (long long)c->step_launches * taken);
  return hweno_sync_status(c, stream);
}

int hweno_run_persistent(hweno_ctx* c, void* U, void* V, double* t, double t_end, int steps,
                         long long* point_updates, void* stream) {
  if (!c) return HWENO_EINVAL;
  if (c->dim != 1) return fail(c, HWENO_ENOTSUP, "persistent run built for 1D batches");
  if (!U || !V || !t || steps < 1) return fail(c, HWENO_EINVAL, "bad argument");
  if (!std::isfinite(t_end)) return fail(c, HWENO_EINVAL, "t_end not finite");
  if ((long long)steps * 3LL * c->ntiles >= (1LL << 31))
    return fail(c, HWENO_EINVAL, "too many steps for one launch");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (c->opt.fused_small == 2 && c->max_n <= kClusterMax * kTile1D) {
    // small instances: the K steps as one launch of the cluster step
    if ((e = cudaMemsetAsync(c->d_active, 0, sizeof(int), s)) ||
        (e = cudaMemsetAsync(c->d_pu, 0, sizeof(unsigned long long), s)))
      return cuda_fail(c, e, "memset");
    Args1D a = base_args_1d(c);
    a.t = t;
    a.t_end = t_end;
    a.skip_done = 1;
    a.dt = c->d_dt;
    a.lands = c->d_lands;
    a.U = U;
    a.V = V;
    FusedArgs f{};
    f.U1 = c->d_U1; f.V1 = c->d_V1; f.U2 = c->d_U2; f.V2 = c->d_V2; f.Vt0 = c->d_Vt0;
    f.alpha = c->d_alpha; f.dt_used = nullptr; f.active = c->d_active; f.pu = c->d_pu;
    f.batch = c->batch;
    f.steps = steps;
    prof_begin(c, s);
    e = launch_step_cluster_1d(c->eq, c->fp32, a, f, (int)c->max_n, s);
    if (e == cudaSuccess) {
      prof_end(c, s, 1);
      c->launches = 1;
      if (!point_updates) return HWENO_OK;
      unsigned long long pu = 0;
      if ((e = cudaMemcpyAsync(&pu, c->d_pu, sizeof pu, cudaMemcpyDeviceToHost, s)) ||
          (e = cudaStreamSynchronize(s)))
        return cuda_fail(c, e, "read point updates");
      *point_updates = (long long)pu;
      return hweno_sync_status(c, stream);
    }
    if (e != cudaErrorNotSupported) return cuda_fail(c, e, "cluster run");
    // no such cluster here: the tiled persistent kernel below
  }
  const size_t B = c->batch;
  const unsigned wait_extra = c->inject == 1 ? 1u : 0u;  // hweno_test_inject
  c->inject = 0;
  if ((e = cudaMemsetAsync(c->d_next, 0, sizeof(unsigned long long) + 2 * sizeof(unsigned) * B, s)) ||
      (e = cudaMemsetAsync(c->d_palpha, 0, sizeof(unsigned long long) * 6 * B, s)) ||
      (e = cudaMemsetAsync(c->d_active, 0, sizeof(int), s)) ||
      (e = cudaMemsetAsync(c->d_pu, 0, sizeof(unsigned long long), s)))
    return cuda_fail(c, e, "memset");
  Args1D a = base_args_1d(c);
  a.t = t;
  a.t_end = t_end;
  a.skip_done = 1;
  a.dt = c->d_dt;
  a.lands = c->d_lands;
  a.U = U;
  a.V = V;
  a.alpha_out = c->d_palpha;  // alpha(U^n) of the first step: slot [0][0]
  prof_begin(c, s);
  if ((e = launch_alpha_1d(c->eq, c->fp32, c->variant, a, c->ntiles, s)))
    return cuda_fail(c, e, "alpha");
  prof_end(c, s, 0);
  a.alpha_out = nullptr;
  PersistArgs p{};
  p.next = c->d_next; p.done = c->d_done; p.done3 = c->d_done3;
  p.inst_tiles = c->d_inst_tiles; p.alpha = c->d_palpha;
  p.U1 = c->d_U1; p.V1 = c->d_V1; p.U2 = c->d_U2; p.V2 = c->d_V2; p.Vt0 = c->d_Vt0;
  p.active = c->d_active; p.pu = c->d_pu;
  p.steps = steps; p.ntiles = c->ntiles; p.batch = c->batch;
  p.wait_extra = wait_extra;
  prof_begin(c, s);
  if ((e = launch_run_1d(c->eq, c->fp32, c->variant, a, p, c->persist_ctas, s)))
    return cuda_fail(c, e, "persistent run");
  prof_end(c, s, 1);
  c->launches = 2;
  if (point_updates) {
    unsigned long long pu = 0;
    if ((e = cudaMemcpyAsync(&pu, c->d_pu, sizeof pu, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s)))
      return cuda_fail(c, e, "read point updates");
    *point_updates = (long long)pu;
    return hweno_sync_status(c, stream);
  }
  return HWENO_OK;
}

namespace {

// hweno_step_host for 1D: the batch is cut into up to kChunks ranges of
// whole instances with about equal points; each range is copied in, stepped
// and copied out on its own stream, so that copies of one range overlap the
// kernels of the others. Ordered after the work on `s` and before what
// follows on it.
int step_host_1d_pipelined(hweno_ctx* c, void* U, void* V, double* t, double t_end, int nsteps,
                           cudaStream_t s) {
  cudaError_t e;
  const int C = std::min(hweno_ctx::kChunks, c->batch);
  // ranges of instances and of tiles
  const int tp = tile_points(c->variant);
  std::vector<long long> first_tile(c->batch + 1, 0), first_pt(c->batch + 1, 0);
  for (int k = 0; k < c->batch; ++k) {
    first_tile[k + 1] = first_tile[k] + (c->nx[k] + tp - 1) / tp;
    first_pt[k + 1] = first_pt[k] + c->nx[k];
  }
  std::vector<int> cut(C + 1, 0);
  cut[C] = c->batch;
  for (int i = 1, k = 0; i < C; ++i) {
    const long long goal = first_pt[c->batch] * i / C;
    while (k < c->batch && first_pt[k] < goal) ++k;
    cut[i] = std::max(k, cut[i - 1]);
  }
  if ((e = cudaEventRecord(c->ce0, s))) return cuda_fail(c, e, "event record");
  const size_t es = (size_t)c->m * c->esize;
  char* dU = static_cast<char*>(c->d_hU);
  char* dV = static_cast<char*>(c->d_hV);
  char* hU = static_cast<char*>(U);
  char* hV = static_cast<char*>(V);
  for (int i = 0; i < C; ++i) {
    const int k0 = cut[i], k1 = cut[i + 1];
    cudaStream_t cs = c->cs[i];
    if ((e = cudaStreamWaitEvent(cs, c->ce0, 0))) return cuda_fail(c, e, "wait");
    if (k1 > k0) {
      const size_t o = es * (size_t)first_pt[k0], b = es * (size_t)(first_pt[k1] - first_pt[k0]);
      const size_t tb = sizeof(double) * (k1 - k0);
      if ((e = cudaMemcpyAsync(dU + o, hU + o, b, cudaMemcpyHostToDevice, cs)) ||
          (e = cudaMemcpyAsync(dV + o, hV + o, b, cudaMemcpyHostToDevice, cs)) ||
          (e = cudaMemcpyAsync(c->d_ht + k0, t + k0, tb, cudaMemcpyHostToDevice, cs)) ||
          (e = cudaMemsetAsync(c->d_chunk_active + i, 0, sizeof(int), cs)))
        return cuda_fail(c, e, "copy in");
      for (int j = 0; j < nsteps; ++j) {
        const int rc = step_1d_range(c, c->d_hU, c->d_hV, c->d_ht, t_end, nullptr, cs, k0, k1,
                                     (int)first_tile[k0], (int)first_tile[k1],
                                     c->d_chunk_active + i);
        if (rc != HWENO_OK) return rc;
      }
      if ((e = cudaMemcpyAsync(hU + o, dU + o, b, cudaMemcpyDeviceToHost, cs)) ||
          (e = cudaMemcpyAsync(hV + o, dV + o, b, cudaMemcpyDeviceToHost, cs)) ||
          (e = cudaMemcpyAsync(t + k0, c->d_ht + k0, tb, cudaMemcpyDeviceToHost, cs)))
        return cuda_fail(c, e, "copy out");
    }
    if ((e = cudaEventRecord(c->ce[i], cs)) || (e = cudaStreamWaitEvent(s, c->ce[i], 0)))
      return cuda_fail(c, e, "event");
  }
  // instances still active, counted after all ranges (their finalize counters
  // are per range and per step)
  if ((e = launch_count_active(c->batch, c->d_ht, t_end, c->d_active, s)))
    return cuda_fail(c, e, "count");
  c->launches = 5 * nsteps * C + 1;
  return HWENO_OK;
}

}  // namespace

#if defined(HWENO_CHECKS) && HWENO_CHECKS
namespace {
// Self-test of the device-side checks: one row and one column past the end of
// a checked shared-memory view. The views redirect both reads to element 0,
// so nothing outside the array is touched, and flag STATUS_BOUNDS.
__global__ void k_check_selftest(unsigned* status, double* sink) {
  __shared__ double buf[2][4];
  const auto v = tile_view(buf, status);
  buf[threadIdx.x / 4][threadIdx.x % 4] = 1.0;
  __syncthreads();
  if (threadIdx.x == 0) *sink = v[2][0] + v[0][4];
}
}  // namespace
#endif

int hweno_test_inject(hweno_ctx* c, int kind) {
  if (!c) return HWENO_EINVAL;
  if (kind < 0 || kind > 2) return fail(c, HWENO_EINVAL, "unknown injection");
  if (kind == 2) {
#if defined(HWENO_CHECKS) && HWENO_CHECKS
    k_check_selftest<<<1, 8>>>(c->d_status, c->d_dt);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HWENO_OK : cuda_fail(c, e, "check self-test");
#else
    return fail(c, HWENO_ENOTSUP, "device-side checks are compiled in checked builds only");
#endif
  }
  c->inject = kind;
  return HWENO_OK;
}

int hweno_step_host(hweno_ctx* c, void* U, void* V, void* W, double* t, double t_end,
                    int nsteps, void* stream) {
  if (!c) return HWENO_EINVAL;
  if (!U || !V || !t || nsteps < 0) return fail(c, HWENO_EINVAL, "bad argument");
  if (c->dim == 1 && W) return fail(c, HWENO_EINVAL, "W given in 1D");
  if (c->dim == 2 && !W) return fail(c, HWENO_EINVAL, "W required in 2D");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (c->dim == 1 && !c->opt.fused_small && c->batch > 1) {
    const int rc = step_host_1d_pipelined(c, U, V, t, t_end, nsteps, s);
    if (rc != HWENO_OK) return rc;
    return hweno_sync_status(c, stream);
  }
  const size_t fb = c->elems * c->esize, tb = sizeof(double) * c->batch;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(c->d_hU, U, fb, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(c->d_hV, V, fb, cudaMemcpyHostToDevice, s)) ||
      (c->dim == 2 && (e = cudaMemcpyAsync(c->d_hW, W, fb, cudaMemcpyHostToDevice, s))) ||
      (e = cudaMemcpyAsync(c->d_ht, t, tb, cudaMemcpyHostToDevice, s)))
    return cuda_fail(c, e, "copy in");
  for (int i = 0; i < nsteps; ++i) {
    const int rc = hweno_step(c, c->d_hU, c->d_hV, c->dim == 2 ? c->d_hW : nullptr, c->d_ht,
                              t_end, nullptr, stream);
    if (rc != HWENO_OK) return rc;
  }
  if ((e = cudaMemcpyAsync(U, c->d_hU, fb, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaMemcpyAsync(V, c->d_hV, fb, cudaMemcpyDeviceToHost, s)) ||
      (c->dim == 2 && (e = cudaMemcpyAsync(W, c->d_hW, fb, cudaMemcpyDeviceToHost, s))) ||
      (e = cudaMemcpyAsync(t, c->d_ht, tb, cudaMemcpyDeviceToHost, s)))
    return cuda_fail(c, e, "copy out");
  return hweno_sync_status(c, stream);
}

int hweno_autotune(hweno_ctx* c, const void* U, const void* V, const void* W, const double* t,
                   double t_end, int* chosen, double* ms, void* stream) {
  if (!c) return HWENO_EINVAL;
  if (!U || !V || !t) return fail(c, HWENO_EINVAL, "null array");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = c->tune_ev[0], e1 = c->tune_ev[1];
  if (c->dim == 2) {  // the split and the fused form of a stage
    if (!W) return fail(c, HWENO_EINVAL, "W required in 2D");
    Args2D a = base_args_2d(c);
    a.t = t; a.t_end = t_end; a.skip_done = 1;
    a.U = U; a.alpha_out = c->d_alpha;
    cudaError_t e;
    if ((e = cudaMemsetAsync(c->d_alpha, 0, sizeof(unsigned long long) * 6, s)) ||
        (e = launch_alpha_2d(c->eq, c->fp32, a, s)))
      return cuda_fail(c, e, "autotune");
    a.V = V; a.W = W; a.U0 = U; a.Vt0 = c->d_Vt0; a.Wt0 = c->d_Wt0;
    a.Uout = c->d_U1; a.Vout = c->d_V1; a.Wout = c->d_W1; a.Wt0out = c->d_Wt0; a.VT = c->d_Vt0;
    a.stage_c = 0.0;
    a.alpha_in = reinterpret_cast<const double*>(c->d_alpha);
    a.alpha_out = c->d_alpha + 2;
    const int keep = c->opt.fused_2d;
    float best_ms[2] = {1e30f, 1e30f};
    for (int f = 0; f < 2; ++f) {
      c->opt.fused_2d = f;
      for (int r = 0; r < 4; ++r) {  // first launch warms up, then the best of three
        cudaEventRecord(e0, s);
        if ((e = stage_2d(c, MODE_STAGE1, a, s))) {
          c->opt.fused_2d = keep;
          return cuda_fail(c, e, "autotune");
        }
        cudaEventRecord(e1, s);
        if ((e = cudaEventSynchronize(e1))) {
          c->opt.fused_2d = keep;
          return cuda_fail(c, e, "autotune");
        }
        float x = 0.f;
        cudaEventElapsedTime(&x, e0, e1);
        if (r > 0) best_ms[f] = std::min(best_ms[f], x);
      }
      if (ms) ms[f] = best_ms[f];
    }
    c->opt.fused_2d = best_ms[1] < best_ms[0] ? 1 : 0;
    if (c->graph) cudaGraphExecDestroy(c->graph);  // recorded for the other form
    c->graph = nullptr;
    if (chosen) *chosen = c->opt.fused_2d;
    return hweno_sync_status(c, stream);
  }
  int best = 0;
  float best_ms = 1e30f;
  int rc = HWENO_OK;
  for (int v = 0; v < kNumVariants1D && rc == HWENO_OK; ++v) {
    if ((rc = use_variant(c, v)) != HWENO_OK) break;
    Args1D a = base_args_1d(c);
    a.t = t; a.t_end = t_end; a.skip_done = 1; a.dt = c->d_dt; a.lands = c->d_lands;
    a.U = U; a.V = V; a.Uout = c->d_U1; a.Vout = c->d_V1; a.Vt0out = c->d_Vt0;
    a.alpha_in = slotd(c, 0); a.alpha_out = slot(c, 1);
    Args1D pre = a;  // wave speed of U into slot 0, read by the stage-1 launches
    pre.alpha_out = slot(c, 0);
    cudaError_t e;
    if ((e = cudaMemsetAsync(c->d_alpha, 0, sizeof(unsigned long long) * 3 * c->batch, s)) ||
        (e = launch_alpha_1d(c->eq, c->fp32, v, pre, c->ntiles, s))) {
      rc = cuda_fail(c, e, "autotune");
      break;
    }
    float tv = 1e30f;
    for (int r = 0; r < 4; ++r) {  // first launch warms up, then the best of three
      cudaEventRecord(e0, s);
      if ((e = launch_stage_1d(c->eq, c->fp32, v, MODE_STAGE1, a, c->ntiles, s))) {
        rc = cuda_fail(c, e, "autotune");
        break;
      }
      cudaEventRecord(e1, s);
      if ((e = cudaEventSynchronize(e1))) { rc = cuda_fail(c, e, "autotune"); break; }
      float x = 0.f;
      cudaEventElapsedTime(&x, e0, e1);
      if (r > 0) tv = std::min(tv, x);
    }
    if (ms) ms[v] = tv;
    if (tv < best_ms) { best_ms = tv; best = v; }
  }
  if (rc != HWENO_OK) {
    if (use_variant(c, 0) == HWENO_OK) c->opt.tile_variant = 0;
    return rc;
  }
  if ((rc = use_variant(c, best)) != HWENO_OK) return rc;
  c->opt.tile_variant = best;
  if (chosen) *chosen = best;
  return hweno_sync_status(c, stream);
}

int hweno_size_classes(const hweno_ctx* c, int* lo, int* hi) {
  if (!c) return HWENO_EINVAL;
  if (c->dim != 1) return 0;
  for (int q = 0; q < c->nclasses; ++q) {
    if (lo) lo[q] = c->class_lo[q];
    if (hi) hi[q] = c->class_hi[q];
  }
  return c->nclasses;
}

int hweno_autotune_classes(hweno_ctx* c, const void* U, const void* V, const double* t,
                           double t_end, int* chosen, double* ms, void* stream) {
  if (!c) return HWENO_EINVAL;
  if (c->dim != 1) return fail(c, HWENO_ENOTSUP, "size classes are built for 1D batches");
  if (!U || !V || !t) return fail(c, HWENO_EINVAL, "null array");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = c->tune_ev[0], e1 = c->tune_ev[1];
  const int keep = c->variant;
  int rc = HWENO_OK;
  cudaError_t e;
  // wave speed of U into slot 0 for every instance (current variant's table)
  {
    Args1D pre = base_args_1d(c);
    pre.t = t; pre.t_end = t_end; pre.skip_done = 1; pre.U = U; pre.alpha_out = slot(c, 0);
    if ((e = cudaMemsetAsync(c->d_alpha, 0, sizeof(unsigned long long) * 3 * c->batch, s)) ||
        (e = launch_alpha_1d(c->eq, c->fp32, c->variant, pre, c->ntiles, s)))
      return cuda_fail(c, e, "autotune classes");
  }
  int best[HWENO_MAX_SIZE_CLASSES];
  for (int q = 0; q < c->nclasses && rc == HWENO_OK; ++q) {
    float best_ms = 1e30f;
    best[q] = keep;
    for (int v = 0; v < kNumVariants1D && rc == HWENO_OK; ++v) {
      const int t0 = c->ct_first[v][q], t1 = c->ct_first[v][q + 1];
      Args1D a = base_args_1d(c);
      a.tile_inst = c->d_ct_inst[v] + t0;
      a.tile_start = c->d_ct_start[v] + t0;
      a.t = t; a.t_end = t_end; a.skip_done = 1; a.dt = c->d_dt; a.lands = c->d_lands;
      a.U = U; a.V = V; a.Uout = c->d_U1; a.Vout = c->d_V1; a.Vt0out = c->d_Vt0;
      a.alpha_in = slotd(c, 0); a.alpha_out = slot(c, 1);
      float tv = 1e30f;
      for (int r = 0; r < 4 && t1 > t0; ++r) {  // first launch warms up, then the best of three
        cudaEventRecord(e0, s);
        if ((e = launch_stage_1d(c->eq, c->fp32, v, MODE_STAGE1, a, t1 - t0, s))) {
          rc = cuda_fail(c, e, "autotune classes");
          break;
        }
        cudaEventRecord(e1, s);
        if ((e = cudaEventSynchronize(e1))) { rc = cuda_fail(c, e, "autotune classes"); break; }
        float x = 0.f;
        cudaEventElapsedTime(&x, e0, e1);
        if (r > 0) tv = std::min(tv, x);
      }
      if (ms) ms[q * kNumVariants1D + v] = tv;
      if (tv < best_ms) { best_ms = tv; best[q] = v; }
    }
  }
  if (rc != HWENO_OK) return rc;
  if (chosen)
    for (int q = 0; q < c->nclasses; ++q) chosen[q] = best[q];
  if ((rc = hweno_set_class_variants(c, best)) != HWENO_OK) return rc;
  return hweno_sync_status(c, stream);
}

int hweno_set_class_variants(hweno_ctx* c, const int* variants) {
  if (!c) return HWENO_EINVAL;
  if (c->dim != 1) return fail(c, HWENO_ENOTSUP, "size classes are built for 1D batches");
  if (!variants) return fail(c, HWENO_EINVAL, "null array");
  for (int q = 0; q < c->nclasses; ++q)
    if (variants[q] < 0 || variants[q] >= kNumVariants1D)
      return fail(c, HWENO_EINVAL, "tile variant out of range");
  bool same = true;
  for (int q = 0; q < c->nclasses; ++q) same = same && variants[q] == variants[0];
  if (same) {  // one variant for every class: as hweno_set_options' tile_variant
    const int rc = use_variant(c, variants[0]);
    if (rc == HWENO_OK) c->opt.tile_variant = variants[0];
    return rc;
  }
  for (int q = 0; q < c->nclasses; ++q) c->class_variant[q] = variants[q];
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  c->mixed = true;
  return HWENO_OK;
}

int hweno_totals(hweno_ctx* c, const void* U, double* totals, void* stream) {
  if (!c) return HWENO_EINVAL;
  if (!U || !totals) return fail(c, HWENO_EINVAL, "null array");
  const double cell = c->dim == 2 ? ((c->x1 - c->x0) / c->nx[0]) * ((c->y1 - c->y0) / c->ny) : 0.0;
  const int ntot = c->dim == 1 ? c->ntiles : c->ntiles_tot;
  const cudaError_t e = launch_totals(c->m, c->fp32, c->dim, U, ntot, c->tile, c->d_tile_inst,
                                      c->d_tile_start, c->d_inst_n, c->d_inst_off, c->batch,
                                      c->nx[0], c->ny, cell, c->dim == 1 ? c->d_inst_dx : nullptr,
                                      c->d_partial, totals, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(c, e, "totals");
  c->launches = 2;
  return HWENO_OK;
}

namespace {

double* adj_field(hweno_ctx* c, int f) {
  const int slot = c->dim == 2 ? f : (f / 3) * 2 + f % 3;  // 1D: 0 1 3 4 6 7 -> 0..5
  return c->d_adj + (size_t)slot * (size_t)c->m * (size_t)c->npts;
}

int adjoint_1d(hweno_ctx* c, const void* U, const void* V, const double* dt, double* lU,
               double* lV, bool replay, cudaStream_t s) {
  cudaError_t e;
  // 1. replay stages 1 and 2 of the forward step with its dt; alpha of each
  //    stage input lands in slots 0, 1, 2 (frozen in the adjoint). Without
  //    replay the stage states and slots come from a record.
  if (replay) {
    if ((e = cudaMemsetAsync(c->d_alpha, 0, sizeof(unsigned long long) * 3 * c->batch, s)))
      return cuda_fail(c, e, "memset");
    Args1D a = base_args_1d(c);
    a.t = c->d_ht;  // unused with skip_done = 0
    a.t_end = 0.0;
    a.skip_done = 0;
    a.dt = c->d_dt;
    a.lands = c->d_lands;
    a.dt_in = dt;
    a.U = U;
    a.alpha_out = slot(c, 0);
    if ((e = launch_alpha_1d(c->eq, false, c->variant, a, c->ntiles, s)))
      return cuda_fail(c, e, "alpha");
    a.V = V; a.Uout = c->d_U1; a.Vout = c->d_V1; a.Vt0out = c->d_Vt0;
    a.alpha_in = slotd(c, 0); a.alpha_out = slot(c, 1);
    if ((e = launch_stage_1d(c->eq, false, c->variant, MODE_STAGE1, a, c->ntiles, s)))
      return cuda_fail(c, e, "replay stage 1");
    a.U = c->d_U1; a.V = c->d_V1; a.U0 = U; a.Vt0 = c->d_Vt0; a.Uout = c->d_U2; a.Vout = c->d_V2;
    a.Vt0out = nullptr; a.alpha_in = slotd(c, 1); a.alpha_out = slot(c, 2);
    if ((e = launch_stage_1d(c->eq, false, c->variant, MODE_STAGE2, a, c->ntiles, s)))
      return cuda_fail(c, e, "replay stage 2");
  }
  // 2. reverse stages 3, 2, 1 (the adjoint kernels use the default tiles)
  double *aU2 = adj_field(c, 0), *aV2 = adj_field(c, 1), *aU1 = adj_field(c, 3),
         *aV1 = adj_field(c, 4), *acU = adj_field(c, 6), *acV = adj_field(c, 7);
  AdjArgs1D g{};
  g.tile_inst = c->d_tile0_inst; g.tile_start = c->d_tile0_start; g.inst_n = c->d_inst_n;
  g.inst_off = c->d_inst_off; g.inst_geo = c->d_inst_geo; g.dt = dt;
  g.status = c->d_status;
  g.sp = scheme_params(c);
  // stage 3: lambda2 = (2/3) G'(x2)^T lambda^{n+1}
  g.U = static_cast<const double*>(c->d_U2); g.V = static_cast<const double*>(c->d_V2);
  g.alpha = slotd(c, 2); g.lamU = lU; g.lamV = lV; g.b = 2.0 / 3.0;
  g.outU = aU2; g.outV = aV2;
  if ((e = launch_adjoint_1d(c->eq, g, c->ntiles0, s))) return cuda_fail(c, e, "adjoint 3");
  // stage 2: lambda1 = (1/4) G'(x1)^T lambda2; acc = lambda^{n+1}/3 + 3 lambda2/4
  g.U = static_cast<const double*>(c->d_U1); g.V = static_cast<const double*>(c->d_V1);
  g.alpha = slotd(c, 1); g.lamU = aU2; g.lamV = aV2; g.b = 0.25;
  g.outU = aU1; g.outV = aV1;
  g.lamNU = lU; g.lamNV = lV; g.accOutU = acU; g.accOutVt = acV;
  g.cN = 1.0 / 3.0; g.c2 = 0.75;
  if ((e = launch_adjoint_1d(c->eq, g, c->ntiles0, s))) return cuda_fail(c, e, "adjoint 2");
  // stage 1: lambda^n = G'(x^n)^T lambda1 + base-term cotangents
  g.U = static_cast<const double*>(U); g.V = static_cast<const double*>(V);
  g.alpha = slotd(c, 0); g.lamU = aU1; g.lamV = aV1; g.b = 1.0;
  g.accU = acU; g.accVt = acV; g.lamNU = nullptr; g.lamNV = nullptr;
  g.accOutU = nullptr; g.accOutVt = nullptr;
  g.outU = lU; g.outV = lV;
  if ((e = launch_adjoint_1d(c->eq, g, c->ntiles0, s))) return cuda_fail(c, e, "adjoint 1");
  c->launches = replay ? 6 : 3;
  return HWENO_OK;
}

int adjoint_2d(hweno_ctx* c, const void* U, const void* V, const void* W, const double* t,
               const double* dt, double* lU, double* lV, double* lW, bool replay,
               cudaStream_t s) {
  cudaError_t e;
  // 1. replay stages 1 and 2 with the recorded dt (alpha slots 0, 1, 2);
  //    without replay the stage states and slots come from a record
  Args2D a = base_args_2d(c);
  if (replay) {
    if ((e = cudaMemsetAsync(c->d_alpha, 0, sizeof(unsigned long long) * 6, s)))
      return cuda_fail(c, e, "memset");
    a.t = t;
    a.t_end = 0.0;
    a.skip_done = 0;
    a.dt_in = dt;
    a.U = U;
    a.alpha_out = c->d_alpha;
    if ((e = launch_alpha_2d(c->eq, false, a, s))) return cuda_fail(c, e, "alpha");
    struct Stage { const void *u, *v, *w; void *uo, *vo, *wo, *vt; double sc; };
    const Stage st[2] = {{U, V, W, c->d_U1, c->d_V1, c->d_W1, c->d_Vt0, 0.0},
                         {c->d_U1, c->d_V1, c->d_W1, c->d_U2, c->d_V2, c->d_W2, c->d_VT, 1.0}};
    for (int k = 0; k < 2; ++k) {
      const int mode = MODE_STAGE1 + k;
      a.U = st[k].u; a.V = st[k].v; a.W = st[k].w;
      a.U0 = U; a.Vt0 = c->d_Vt0; a.Wt0 = c->d_Wt0;
      a.Uout = st[k].uo; a.Vout = st[k].vo; a.Wout = st[k].wo;
      a.Wt0out = k == 0 ? c->d_Wt0 : nullptr;
      a.VT = st[k].vt;
      a.stage_c = st[k].sc;
      a.alpha_in = reinterpret_cast<const double*>(c->d_alpha + 2 * k);
      a.alpha_out = c->d_alpha + 2 * (k + 1);
      // the same form as the forward step, so that a replay gives a record's bits
      if ((e = stage_2d(c, mode, a, s))) return cuda_fail(c, e, "replay");
    }
  }
  // 2. reverse stages 3, 2, 1: an x sweep into `part`, then a y sweep
  AdjArgs2D g{};
  g.nx = c->nx[0]; g.ny = c->ny; g.dx = a.dx; g.dy = a.dy;
  for (int i = 0; i < 6; ++i) g.geod[i] = a.geod[i];
  g.x0 = c->x0; g.y0 = c->y0; g.t = t; g.dt = dt; g.sp = a.sp;
  g.status = c->d_status;
  g.part = adj_field(c, 9);
  double* f[9];
  for (int i = 0; i < 9; ++i) f[i] = adj_field(c, i);
  struct Rev {
    const void *u, *v, *w;
    int slot;
    double b, sc;
    const double *lu, *lv, *lw;
    double *ou, *ov, *ow;
  };
  const Rev rv[3] = {
      {c->d_U2, c->d_V2, c->d_W2, 2, 2.0 / 3.0, 0.5, lU, lV, lW, f[0], f[1], f[2]},
      {c->d_U1, c->d_V1, c->d_W1, 1, 0.25, 1.0, f[0], f[1], f[2], f[3], f[4], f[5]},
      {U, V, W, 0, 1.0, 0.0, f[3], f[4], f[5], lU, lV, lW}};
  for (int k = 0; k < 3; ++k) {
    g.U = static_cast<const double*>(rv[k].u);
    g.V = static_cast<const double*>(rv[k].v);
    g.W = static_cast<const double*>(rv[k].w);
    g.alpha = reinterpret_cast<const double*>(c->d_alpha + 2 * rv[k].slot);
    g.b = rv[k].b;
    g.stage_c = rv[k].sc;
    g.lamU = rv[k].lu; g.lamV = rv[k].lv; g.lamW = rv[k].lw;
    g.outU = rv[k].ou; g.outV = rv[k].ov; g.outW = rv[k].ow;
    const bool st2 = k == 1, st1 = k == 2;
    g.lamNU = st2 ? lU : nullptr; g.lamNV = st2 ? lV : nullptr; g.lamNW = st2 ? lW : nullptr;
    g.accOutU = st2 ? f[6] : nullptr; g.accOutVt = st2 ? f[7] : nullptr;
    g.accOutWt = st2 ? f[8] : nullptr;
    g.cN = 1.0 / 3.0; g.c2 = 0.75;
    g.accU = st1 ? f[6] : nullptr; g.accVt = st1 ? f[7] : nullptr; g.accWt = st1 ? f[8] : nullptr;
    if ((e = launch_adjoint_2d(c->eq, 0, g, s))) return cuda_fail(c, e, "adjoint x");
    if ((e = launch_adjoint_2d(c->eq, 1, g, s))) return cuda_fail(c, e, "adjoint y");
  }
  // replay: the wave speed and two stages of one (fused) or two launches each
  c->launches = replay ? 6 + 1 + 2 * (c->opt.fused_2d ? 1 : 2) : 6;
  return HWENO_OK;
}

// A step record: the stage states x1 = (U1, V1 [, W1]) and x2 = (U2, V2
// [, W2]) of one forward step and its wave-speed slots, so that the adjoint
// of that step needs no replay.
int record_fields(const hweno_ctx* c) { return c->dim == 2 ? 6 : 4; }
size_t record_alpha_bytes(const hweno_ctx* c) {
  return sizeof(unsigned long long) * (c->dim == 2 ? 6 : 3 * (size_t)c->batch);
}
size_t record_bytes(const hweno_ctx* c) {
  const size_t b = record_fields(c) * c->elems * sizeof(double) + record_alpha_bytes(c);
  return (b + 255) / 256 * 256;
}

// Copy the context's stage states and slots into a record, or back.
int record_copy(hweno_ctx* c, void* rec, bool to_record, cudaStream_t s) {
  void* bufs[6] = {c->d_U1, c->d_V1, c->d_U2, c->d_V2, c->d_W1, c->d_W2};
  const size_t fb = c->elems * sizeof(double);
  char* r = static_cast<char*>(rec);
  const int nf = record_fields(c);
  cudaError_t e;
  for (int i = 0; i < nf; ++i) {
    void* dst = to_record ? static_cast<void*>(r + i * fb) : bufs[i];
    const void* src = to_record ? bufs[i] : static_cast<const void*>(r + i * fb);
    if ((e = cudaMemcpyAsync(dst, src, fb, cudaMemcpyDeviceToDevice, s)))
      return cuda_fail(c, e, "record copy");
  }
  void* ra = r + nf * fb;
  if ((e = cudaMemcpyAsync(to_record ? ra : static_cast<void*>(c->d_alpha),
                           to_record ? static_cast<const void*>(c->d_alpha) : ra,
                           record_alpha_bytes(c), cudaMemcpyDeviceToDevice, s)))
    return cuda_fail(c, e, "record copy");
  return HWENO_OK;
}

// Checks shared by the adjoint entry points; HWENO_OK when the call may run.
int adjoint_check(hweno_ctx* c, const void* U, const void* V, const void* W, const double* dt,
                  const void* lamU, const void* lamV, const void* lamW) {
  if (c->fp32) return fail(c, HWENO_ENOTSUP, "adjoint built for FP64 states");
  if (c->eq == HWENO_BUCKLEY)
    return fail(c, HWENO_ENOTSUP, "adjoint built for Burgers and Euler");
  if (c->eq == HWENO_EULER && c->opt.eig_avg != 0)
    return fail(c, HWENO_ENOTSUP, "adjoint built for the Roe-averaged eigenvectors");
  const bool two = c->dim == 2;
  if (!U || !V || !dt || !lamU || !lamV || (two != (W != nullptr)) || (two != (lamW != nullptr)))
    return fail(c, HWENO_EINVAL, "bad argument");
  const int bcs[4] = {c->bc.xlo, c->bc.xhi, c->bc.ylo, c->bc.yhi};
  for (int d = 0; d < c->dim; ++d)
    if ((bcs[2 * d] == HWENO_BC_PERIODIC) != (bcs[2 * d + 1] == HWENO_BC_PERIODIC))
      return fail(c, HWENO_ENOTSUP, "adjoint needs both ends of a direction periodic or neither");
  if (!c->d_adj) return fail(c, HWENO_ENOTSUP, "no adjoint scratch in this context");
  return HWENO_OK;
}

// The adjoint of one step, with the stage states replayed (record null) or
// taken from a record.
int adjoint_any(hweno_ctx* c, const void* U, const void* V, const void* W, const double* t,
                const double* dt, void* lamU, void* lamV, void* lamW, const void* record,
                cudaStream_t s) {
  int rc;
  if ((rc = adjoint_check(c, U, V, W, dt, lamU, lamV, lamW)) != HWENO_OK) return rc;
  if (record && (rc = record_copy(c, const_cast<void*>(record), false, s)) != HWENO_OK)
    return rc;
  const bool replay = record == nullptr;
  if (c->dim == 1)
    return adjoint_1d(c, U, V, dt, static_cast<double*>(lamU), static_cast<double*>(lamV),
                      replay, s);
  const double* tt = t;
  if (!tt) {  // no boundary time given: the boundaries must not depend on it
    if (c->bc.yhi == HWENO_BC_DMR_TOP)
      return fail(c, HWENO_EINVAL, "the double-Mach top boundary needs the step's time t");
    cudaError_t e;
    if ((e = cudaMemsetAsync(c->d_ht, 0, sizeof(double), s))) return cuda_fail(c, e, "memset");
    tt = c->d_ht;
  }
  return adjoint_2d(c, U, V, W, tt, dt, static_cast<double*>(lamU), static_cast<double*>(lamV),
                    static_cast<double*>(lamW), replay, s);
}

}  // namespace

int hweno_adjoint_step(hweno_ctx* c, const void* U, const void* V, const void* W,
                       const double* t, const double* dt, void* lamU, void* lamV, void* lamW,
                       void* stream) {
  if (!c) return HWENO_EINVAL;
  return adjoint_any(c, U, V, W, t, dt, lamU, lamV, lamW, nullptr,
                     static_cast<cudaStream_t>(stream));
}

long long hweno_adjoint_record_bytes(const hweno_ctx* c) {
  if (!c) return -1;
  return (long long)record_bytes(c);
}

int hweno_step_record(hweno_ctx* c, void* U, void* V, void* W, double* t, double t_end,
                      double* dt_used, void* record, void* stream) {
  if (!c) return HWENO_EINVAL;
  if (!record) return fail(c, HWENO_EINVAL, "null record");
  if (c->fp32) return fail(c, HWENO_ENOTSUP, "records are built for FP64 states");
  int rc = hweno_step(c, U, V, W, t, t_end, dt_used, stream);
  if (rc != HWENO_OK) return rc;
  return record_copy(c, record, true, static_cast<cudaStream_t>(stream));
}

int hweno_adjoint_step_recorded(hweno_ctx* c, const void* U, const void* V, const void* W,
                                const void* record, const double* t, const double* dt,
                                void* lamU, void* lamV, void* lamW, void* stream) {
  if (!c) return HWENO_EINVAL;
  if (!record) return fail(c, HWENO_EINVAL, "null record");
  return adjoint_any(c, U, V, W, t, dt, lamU, lamV, lamW, record,
                     static_cast<cudaStream_t>(stream));
}

int hweno_sync_status(hweno_ctx* c, void* stream) {
  if (!c) return HWENO_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "synchronize");
  unsigned st = 0;
  if ((e = cudaMemcpy(&st, c->d_status, sizeof st, cudaMemcpyDeviceToHost)))
    return cuda_fail(c, e, "read status");
  if (st) {
    cudaMemset(c->d_status, 0, sizeof(unsigned));
    if (st & STATUS_TIMEOUT)
      return fail(c, HWENO_ETIMEOUT, "a persistent-run wait gave up (dependency not met in ~2 s)");
    if (st & STATUS_BOUNDS)
      return fail(c, HWENO_EBOUNDS, "a device-side index check failed (checked build)");
    if (st & STATUS_NONFINITE) return fail(c, HWENO_ENONFINITE, "non-finite wave speed");
  }
  return HWENO_OK;
}

long long hweno_num_points(const hweno_ctx* c) { return c ? c->npts : -1; }

int hweno_active_instances(hweno_ctx* c, void* stream) {
  if (!c) return HWENO_EINVAL;
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(c, e, "synchronize");
  int n = 0;
  if ((e = cudaMemcpy(&n, c->d_active, sizeof n, cudaMemcpyDeviceToHost)))
    return cuda_fail(c, e, "read active");
  return n;
}

int hweno_launches_last_call(const hweno_ctx* c) { return c ? c->launches : -1; }

int hweno_profile_start(hweno_ctx* c, int capacity) {
  if (!c || capacity < 0) return HWENO_EINVAL;
  destroy_events(c);
  c->ev.resize(2 * (size_t)capacity);
  c->ev_kind.assign(capacity, 0);
  for (size_t i = 0; i < c->ev.size(); ++i) {
    const cudaError_t e = cudaEventCreate(&c->ev[i]);
    if (e != cudaSuccess) {
      c->ev.resize(i);
      destroy_events(c);
      return cuda_fail(c, e, "cudaEventCreate");
    }
  }
  return HWENO_OK;
}

int hweno_profile_read(hweno_ctx* c, double* ms, int* n, void* stream) {
  if (!c || !ms || !n) return HWENO_EINVAL;
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(c, e, "synchronize");
  for (int k = 0; k < 3; ++k) { ms[k] = 0.0; n[k] = 0; }
  for (int i = 0; i + 1 < c->ev_used; i += 2) {
    float t = 0.f;
    if ((e = cudaEventElapsedTime(&t, c->ev[i], c->ev[i + 1])) != cudaSuccess)
      return cuda_fail(c, e, "cudaEventElapsedTime");
    const int kind = c->ev_kind[i / 2];
    ms[kind] += t;
    n[kind] += 1;
  }
  c->ev_used = 0;
  return HWENO_OK;
}

const char* hweno_last_error(const hweno_ctx* c) { return c ? c->err.c_str() : "null context"; }

int hweno_destroy(hweno_ctx* c) {
  if (!c) return HWENO_OK;
  destroy_events(c);
  free_all(c);
  delete c;
  return HWENO_OK;
}

}  // extern "C"
