// Instantiations of the fused step kernel (lbm_step_kernel.cuh) for one storage family.
#include "lbm_step_kernel.cuh"

namespace lbm {

cudaError_t launch_step_f64(int cfg, const StepArgs& a, bool reduce, cudaStream_t st) {
    return launch_step_cfg<double, true>(cfg, a, reduce, st);
}

}  // namespace lbm
