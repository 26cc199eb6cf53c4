// Allocation-free variant of hweno_step for a single 1D instance in FP64.
//
// Some callers cannot allocate device memory: code that runs inside a host
// framework which owns every device allocation (its own pool or arena, where a
// stray cudaMalloc would be invisible to it or is forbidden by policy), code
// that must not trigger cudaMalloc's implicit device synchronisation on a
// latency-critical path, and plug-ins loaded into processes that only hand
// them pre-allocated buffers. Such callers cannot create a context, because
// hweno_create allocates the stage buffers. This entry point takes the same
// step with all of its scratch - the three stage states, the stored limited
// derivative, the per-stage wave speeds, the time step and the tile table -
// in one fixed array that is part of the library image (a file-scope
// __device__ array of kNoallocScratchBytes), so it calls no cudaMalloc,
// cudaFree or allocating library routine.
//
// The array is placed on every GPU that loads the library and stays there
// until the process exits. All calls share it, so two calls whose work
// overlaps on the GPU (different streams, or different host threads) race and
// corrupt each other; serialise them. Each call resets the parts that must
// start at zero (wave-speed maxima, the status word) before use.
#include <cmath>
#include <mutex>

#include "hweno.h"
#include "internal.h"

using namespace hweno;

namespace {

constexpr int kMaxComp = 3;  // Euler 1D
constexpr size_t kFieldBytes = sizeof(double) * kMaxComp * HWENO_NOALLOC_MAX_POINTS;
constexpr int kMaxTiles = (HWENO_NOALLOC_MAX_POINTS + kTile1D - 1) / kTile1D;

// Byte offsets inside the scratch array (each 256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffU1 = 0;
constexpr size_t kOffV1 = kOffU1 + align256(kFieldBytes);
constexpr size_t kOffU2 = kOffV1 + align256(kFieldBytes);
constexpr size_t kOffV2 = kOffU2 + align256(kFieldBytes);
constexpr size_t kOffVt0 = kOffV2 + align256(kFieldBytes);
constexpr size_t kOffAlpha = kOffVt0 + align256(kFieldBytes);           // 3 x u64
constexpr size_t kOffDt = kOffAlpha + 256;                              // double
constexpr size_t kOffLands = kOffDt + 256;                              // int
constexpr size_t kOffActive = kOffLands + 256;                          // int
constexpr size_t kOffStatus = kOffActive + 256;                         // unsigned
constexpr size_t kOffInstN = kOffStatus + 256;                          // int
constexpr size_t kOffInstOff = kOffInstN + 256;                         // long long
constexpr size_t kOffInstDx = kOffInstOff + 256;                        // double
constexpr size_t kOffInstHx = kOffInstDx + 256;                         // double
constexpr size_t kOffInstGeo = kOffInstHx + 256;                       // double[3]
constexpr size_t kOffInstGeof = kOffInstGeo + 256;                      // float[3]
constexpr size_t kOffTileInst = kOffInstGeof + 256;                     // int[kMaxTiles]
constexpr size_t kOffTileStart = kOffTileInst + align256(sizeof(int) * kMaxTiles);
constexpr size_t kNoallocScratchBytes = kOffTileStart + align256(sizeof(int) * kMaxTiles);

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of g_noalloc_scratch per device, looked up once per device
// (with that device current) on its first call.
std::mutex g_mutex;
void* g_addr[256] = {};

// Per-call metadata: the tile table of one instance, its size and mesh
// widths, and zeroed wave-speed maxima, active counter and status word.
__global__ void k_noalloc_setup(unsigned char* base, int ntiles, int n, double dx, double hx) {
  int* tile_inst = reinterpret_cast<int*>(base + kOffTileInst);
  int* tile_start = reinterpret_cast<int*>(base + kOffTileStart);
  for (int b = threadIdx.x; b < ntiles; b += blockDim.x) {
    tile_inst[b] = 0;
    tile_start[b] = b * kTile1D;
  }
  if (threadIdx.x == 0) {
    unsigned long long* alpha = reinterpret_cast<unsigned long long*>(base + kOffAlpha);
    alpha[0] = alpha[1] = alpha[2] = 0ull;
    *reinterpret_cast<int*>(base + kOffActive) = 0;
    *reinterpret_cast<unsigned*>(base + kOffStatus) = 0u;
    *reinterpret_cast<int*>(base + kOffInstN) = n;
    *reinterpret_cast<long long*>(base + kOffInstOff) = 0;
    *reinterpret_cast<double*>(base + kOffInstDx) = dx;
    *reinterpret_cast<double*>(base + kOffInstHx) = hx;
    double* geo = reinterpret_cast<double*>(base + kOffInstGeo);
    float* geof = reinterpret_cast<float*>(base + kOffInstGeof);
    geo[0] = dx;
    geo[1] = 1.0 / dx;
    geo[2] = 1.0 / (dx * dx);
    for (int i = 0; i < 3; ++i) geof[i] = (float)geo[i];
  }
}

bool weights_valid(const double* w) {
  return w[0] >= kWeightMin && w[1] >= kWeightMin && w[2] >= kWeightMin &&
         std::fabs(w[0] + w[1] + w[2] - 1.0) <= 1e-12;
}

bool options_valid(const hweno_options* o) {
  return weights_valid(o->lin_w) && weights_valid(o->lim_d) && o->eps >= kEpsMin &&
         o->eps <= kEpsMax && o->cfl > 0 &&
         o->dt_mode >= 0 && o->dt_mode <= 2 && (o->dt_mode != 2 || o->dt_fixed > 0) &&
         o->limiter >= 0 && o->limiter <= 2 && o->eig_avg >= 0 && o->eig_avg <= 1 &&
         o->tile_variant == 0;
}

bool bc_valid(int b) { return b >= HWENO_BC_PERIODIC && b <= HWENO_BC_INFLOW; }

}  // namespace

extern "C" int hweno_step_1d_noalloc(int equation, int nx, double x0, double x1, double gamma,
                                     const hweno_bc* bc, const hweno_options* opt, double* U,
                                     double* V, double* t, double t_end, double* dt_used,
                                     void* stream) {
  if (equation != HWENO_BURGERS && equation != HWENO_EULER) return HWENO_EINVAL;
  if (nx < 4 || nx > HWENO_NOALLOC_MAX_POINTS) return HWENO_EINVAL;
  if (!(x1 > x0) || !bc || !U || !V || !t || !std::isfinite(t_end)) return HWENO_EINVAL;
  if (equation == HWENO_EULER && !(gamma > 1.0)) return HWENO_EINVAL;
  if (!bc_valid(bc->xlo) || !bc_valid(bc->xhi)) return HWENO_EINVAL;
  if ((bc->xlo == HWENO_BC_PERIODIC) != (bc->xhi == HWENO_BC_PERIODIC)) return HWENO_EINVAL;
  hweno_options o;
  if (opt) {
    if (!options_valid(opt)) return HWENO_EINVAL;
    o = *opt;
  } else {
    hweno_default_options(&o);
  }

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return HWENO_ECUDA;
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return HWENO_ECUDA;
      g_addr[dev] = p;
    }
    base = static_cast<unsigned char*>(g_addr[dev]);
  }

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int ntiles = (nx + kTile1D - 1) / kTile1D;
  const double dx = (x1 - x0) / nx;
  const double hx = o.dt_mode == 1 ? std::pow(dx, 5.0 / 3.0) : dx;
  k_noalloc_setup<<<1, 256, 0, s>>>(base, ntiles, nx, dx, hx);
  if (cudaGetLastError() != cudaSuccess) return HWENO_ECUDA;

  Args1D a{};
  a.tile_inst = reinterpret_cast<const int*>(base + kOffTileInst);
  a.tile_start = reinterpret_cast<const int*>(base + kOffTileStart);
  a.inst_n = reinterpret_cast<const int*>(base + kOffInstN);
  a.inst_off = reinterpret_cast<const long long*>(base + kOffInstOff);
  a.inst_dx = reinterpret_cast<const double*>(base + kOffInstDx);
  a.inst_hx = reinterpret_cast<const double*>(base + kOffInstHx);
  a.inst_geo = reinterpret_cast<const double*>(base + kOffInstGeo);
  a.inst_geof = reinterpret_cast<const float*>(base + kOffInstGeof);
  a.status = reinterpret_cast<unsigned*>(base + kOffStatus);
  a.dt = reinterpret_cast<double*>(base + kOffDt);
  a.lands = reinterpret_cast<int*>(base + kOffLands);
  SchemeParams& sp = a.sp;
  for (int i = 0; i < 3; ++i) { sp.lin_w[i] = o.lin_w[i]; sp.lim_d[i] = o.lim_d[i]; }
  sp.eps = o.eps;
  sp.cfl = o.cfl;
  sp.dt_fixed = o.dt_fixed;
  sp.dt_mode = o.dt_mode;
  sp.limiter = o.limiter;
  sp.eig_avg = o.eig_avg;
  sp.gas_gamma = gamma;
  sp.bc[0] = bc->xlo; sp.bc[1] = bc->xhi; sp.bc[2] = bc->ylo; sp.bc[3] = bc->yhi;
  for (int i = 0; i < 4; ++i) {
    sp.inflow[i] = bc->inflow[i];
    sp.pre[i] = bc->pre[i];
    sp.inflowf[i] = (float)bc->inflow[i];
    sp.pref[i] = (float)bc->pre[i];
  }
  fill_constant_table(sp, o.lin_w, o.lim_d, o.eps, gamma, 0.0);
  a.t = t;
  a.t_end = t_end;
  a.skip_done = 1;

  unsigned long long* alpha = reinterpret_cast<unsigned long long*>(base + kOffAlpha);
  void* U1 = base + kOffU1;
  void* V1 = base + kOffV1;
  void* U2 = base + kOffU2;
  void* V2 = base + kOffV2;
  void* Vt0 = base + kOffVt0;
  const bool fp32 = false;

  a.U = U;
  a.alpha_out = alpha + 0;
  if (launch_alpha_1d(equation, fp32, 0, a, ntiles, s) != cudaSuccess) return HWENO_ECUDA;
  a.U = U; a.V = V; a.Uout = U1; a.Vout = V1; a.Vt0out = Vt0;
  a.alpha_in = reinterpret_cast<const double*>(alpha + 0); a.alpha_out = alpha + 1;
  if (launch_stage_1d(equation, fp32, 0, MODE_STAGE1, a, ntiles, s) != cudaSuccess) return HWENO_ECUDA;
  a.U = U1; a.V = V1; a.U0 = U; a.Vt0 = Vt0; a.Uout = U2; a.Vout = V2; a.Vt0out = nullptr;
  a.alpha_in = reinterpret_cast<const double*>(alpha + 1); a.alpha_out = alpha + 2;
  if (launch_stage_1d(equation, fp32, 0, MODE_STAGE2, a, ntiles, s) != cudaSuccess) return HWENO_ECUDA;
  a.U = U2; a.V = V2; a.U0 = U; a.Vt0 = Vt0; a.Uout = U; a.Vout = V;
  a.alpha_in = reinterpret_cast<const double*>(alpha + 2); a.alpha_out = nullptr;
  if (launch_stage_1d(equation, fp32, 0, MODE_STAGE3, a, ntiles, s) != cudaSuccess) return HWENO_ECUDA;
  if (launch_finalize(1, a.dt, a.lands, t, t_end, dt_used, reinterpret_cast<const double*>(alpha),
                      reinterpret_cast<int*>(base + kOffActive), a.status, nullptr, 1,
                      nullptr, s) != cudaSuccess)
    return HWENO_ECUDA;

  unsigned st = 0;
  if (cudaMemcpyAsync(&st, a.status, sizeof st, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return HWENO_ECUDA;
  return (st & STATUS_NONFINITE) ? HWENO_ENONFINITE : HWENO_OK;
}
