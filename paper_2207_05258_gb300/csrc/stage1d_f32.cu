// FP32 instantiations of the one-dimensional stage kernels (state and
// reconstruction in single precision; wave speeds, time steps and times stay
// FP64). Separate translation unit so that both precisions compile in
// parallel.
#include "stage1d_impl.cuh"

namespace hweno {

cudaError_t launch_alpha_1d_f32(int eq, int variant, const Args1D& a, int ntiles, cudaStream_t s) {
  return alpha_prec<float>(eq, variant, a, ntiles, s);
}

cudaError_t launch_stage_1d_f32(int eq, int variant, int mode, const Args1D& a, int ntiles,
                                cudaStream_t s) {
  return stage_prec<float>(eq, variant, mode, a, ntiles, s);
}

cudaError_t launch_run_1d_f32(int eq, int variant, const Args1D& a, const PersistArgs& p,
                              int ctas, cudaStream_t s) {
  return run_prec<float>(eq, variant, a, p, ctas, s);
}

int run_1d_ctas_per_sm_f32(int eq, int variant) { return occupancy_prec<float>(eq, variant); }

cudaError_t launch_step_small_1d_f32(int eq, const Args1D& a, const FusedArgs& f, cudaStream_t s) {
  return step_small_prec<float>(eq, a, f, s);
}

cudaError_t launch_step_cluster_1d_f32(int eq, const Args1D& a, const FusedArgs& f, int max_n,
                                       cudaStream_t s) {
  return step_cluster_prec<float>(eq, a, f, max_n, s);
}

}  // namespace hweno
