// One-dimensional L-HWENO stage kernels (Zhang & Zhao, arXiv:2207.05258,
// Sec. 2.1-2.2) for ragged batches of independent instances.
//
// One CTA owns a tile of up to kTile1D consecutive points of one instance and
// does the whole stage for it in one pass:
//   1. load U, V on the tile plus two ghost points per side into shared
//      memory, producing ghost values from the boundary conditions on the fly;
//   2. per point: f, h = f'(u) v, the global Lax-Friedrichs split f^{+-},
//      dx h^{+-} (alpha of the stage input, per instance) and, for Euler, the
//      quantities the eigenvectors need;
//   3. per interface (each interface once): the characteristic projection
//      (Euler, eigenvectors at the Roe average), the nonlinear HWENO flux of
//      every field and side, the back-projection, and the linear derivative
//      flux component by component;
//   4. per point: the flux differences L^1, L^2, the HWENO limiter
//      (characteristic-wise for Euler), the SSP-RK3 combination, the stores,
//      and the maximum wave speed of the new state for the next stage.
// The FP64 pipe bounds these kernels, so every point and interface quantity is
// computed once and divisions are folded (see hweno_math.cuh).
#include "stage1d_impl.cuh"

namespace hweno {
namespace {

__global__ void k_finalize(int batch, const double* dt, const int* lands, double* t, double t_end,
                           double* dt_used, const double* alpha, int* active, unsigned* status,
                           const int* inst_n, int rows, unsigned long long* pu) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= batch) return;
  double tk = t[k];
  double d = 0.0;
  if (tk < t_end) {
    d = dt[k];
    tk = lands[k] ? t_end : tk + d;
    t[k] = tk;
    if (!(alpha[k] <= DBL_MAX)) atomicOr(status, STATUS_NONFINITE);
    if (pu) atomicAdd(pu, (unsigned long long)inst_n[k] * (unsigned long long)rows);
  }
  if (dt_used) dt_used[k] = d;
  if (tk < t_end) atomicAdd(active, 1);
}

__global__ void k_count_active(int batch, const double* t, double t_end, int* active) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int mine = 0;
  for (int k = threadIdx.x; k < batch; k += blockDim.x) mine += t[k] < t_end;
  atomicAdd(&cnt, mine);
  __syncthreads();
  if (threadIdx.x == 0) *active = cnt;
}

}  // namespace

cudaError_t launch_count_active(int batch, const double* t, double t_end, int* active,
                                cudaStream_t s) {
  k_count_active<<<1, 256, 0, s>>>(batch, t, t_end, active);
  return cudaGetLastError();
}

cudaError_t launch_alpha_1d_f64(int eq, int variant, const Args1D& a, int ntiles, cudaStream_t s) {
  return alpha_prec<double>(eq, variant, a, ntiles, s);
}

cudaError_t launch_stage_1d_f64(int eq, int variant, int mode, const Args1D& a, int ntiles,
                                cudaStream_t s) {
  return stage_prec<double>(eq, variant, mode, a, ntiles, s);
}

cudaError_t launch_run_1d_f64(int eq, int variant, const Args1D& a, const PersistArgs& p,
                              int ctas, cudaStream_t s) {
  return run_prec<double>(eq, variant, a, p, ctas, s);
}

int run_1d_ctas_per_sm_f64(int eq, int variant) { return occupancy_prec<double>(eq, variant); }

cudaError_t launch_step_small_1d_f64(int eq, const Args1D& a, const FusedArgs& f, cudaStream_t s) {
  return step_small_prec<double>(eq, a, f, s);
}

cudaError_t launch_step_cluster_1d_f64(int eq, const Args1D& a, const FusedArgs& f, int max_n,
                                       cudaStream_t s) {
  return step_cluster_prec<double>(eq, a, f, max_n, s);
}

cudaError_t launch_finalize(int batch, const double* dt, const int* lands, double* t,
                            double t_end, double* dt_used, const double* alpha, int* active,
                            unsigned* status, const int* inst_n, int rows,
                            unsigned long long* pu, cudaStream_t s) {
  k_finalize<<<(batch + 127) / 128, 128, 0, s>>>(batch, dt, lands, t, t_end, dt_used, alpha,
                                                  active, status, inst_n, rows, pu);
  return cudaGetLastError();
}

}  // namespace hweno
