// The 1D stage and wave-speed kernels (stage1d_impl.cuh) for the
// Buckley-Leverett equation of Example 3.4 (Zhang & Zhao, arXiv:2207.05258,
// Sec. 3), in FP64 and FP32, in a translation unit of their own so that the
// three equations compile in parallel.
#include "stage1d_impl.cuh"

namespace hweno {

cudaError_t launch_alpha_1d_bl(bool fp32, int variant, const Args1D& a, int ntiles,
                               cudaStream_t s) {
  return fp32 ? alpha_variants<HWENO_BUCKLEY, float>(variant, a, ntiles, s)
              : alpha_variants<HWENO_BUCKLEY, double>(variant, a, ntiles, s);
}

cudaError_t launch_stage_1d_bl(bool fp32, int variant, int mode, const Args1D& a, int ntiles,
                               cudaStream_t s) {
  return fp32 ? stage_variants<HWENO_BUCKLEY, float>(variant, mode, a, ntiles, s)
              : stage_variants<HWENO_BUCKLEY, double>(variant, mode, a, ntiles, s);
}

cudaError_t launch_run_1d_bl(bool fp32, int variant, const Args1D& a, const PersistArgs& p,
                             int ctas, cudaStream_t s) {
  return fp32 ? run_variants<HWENO_BUCKLEY, float>(variant, a, p, ctas, s)
              : run_variants<HWENO_BUCKLEY, double>(variant, a, p, ctas, s);
}

cudaError_t launch_step_small_1d_bl(bool fp32, const Args1D& a, const FusedArgs& f,
                                    cudaStream_t s) {
  return fp32 ? step_small_launch<HWENO_BUCKLEY, float>(a, f, s)
              : step_small_launch<HWENO_BUCKLEY, double>(a, f, s);
}

cudaError_t launch_step_cluster_1d_bl(bool fp32, const Args1D& a, const FusedArgs& f, int max_n,
                                      cudaStream_t s) {
  return fp32 ? step_cluster_launch<HWENO_BUCKLEY, float>(a, f, max_n, s)
              : step_cluster_launch<HWENO_BUCKLEY, double>(a, f, max_n, s);
}

int run_1d_ctas_per_sm_bl(bool fp32, int variant) {
  return fp32 ? occupancy_variants<HWENO_BUCKLEY, float>(variant)
              : occupancy_variants<HWENO_BUCKLEY, double>(variant);
}

}  // namespace hweno
